// Host side of the TMA loads: tensor-map descriptors for the population
// array and the density buffers of a lattice.  The encode function is taken
// from the driver through the runtime's entry-point query, so the library
// does not link the driver library directly.
#include <cstdio>
#include <cudaTypedefs.h>

#include "cplbm_internal.h"

namespace cplbm {

namespace {
PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}
}  // namespace

bool build_tma_maps(const Lattice &L, TmaMaps *m, char *err, size_t errlen)
{
    m->valid = 0;
    m->tx = L.tx;
    m->ty = L.ty;
    // populations in the storage type, density in the arithmetic type
    const size_t es = pop_bytes(L.precision), er = rho_bytes(L.precision);
    const CUtensorMapDataType dt = L.precision == P_F64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                   : L.precision == P_F16_OFF ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                              : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const CUtensorMapDataType dr = L.precision == P_F64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                                        : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    if (8LL * L.plane + 2LL * L.pitch >= 2147483647LL) {
        // the TMA path addresses the planes with 32-bit offsets
        snprintf(err, errlen, "lattice too large for 32-bit plane offsets");
        return false;
    }
    if ((L.pitch * es) % 16 || (L.plane * es) % 16 || (L.pitch * er) % 16 ||
        (L.tx != 32 && L.tx != 64)) {
        snprintf(err, errlen, "layout not TMA-aligned (pitch %d, tile %dx%d)",
                 L.pitch, L.tx, L.ty);
        return false;
    }
    auto encode = encode_fn();
    if (!encode) {
        snprintf(err, errlen, "cuTensorMapEncodeTiled unavailable");
        return false;
    }
    // density box from x = X0 - 4 (16-B aligned) covering the 2-node halo;
    // population boxes from X0 - 16 B or X0 covering a 1-node shift
    const cuuint32_t bx = (cuuint32_t)(L.tx + 8), bxp = (cuuint32_t)(L.tx + 16 / es);
    {
        cuuint64_t dims[3] = {(cuuint64_t)L.pitch, (cuuint64_t)L.nyf, 8};
        cuuint64_t strides[2] = {(cuuint64_t)L.pitch * es, (cuuint64_t)L.plane * es};
        cuuint32_t box[3] = {bxp, (cuuint32_t)L.ty, 1};
        cuuint32_t estr[3] = {1, 1, 1};
        CUresult r = encode(&m->pops, dt, 3, L.pops, dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            snprintf(err, errlen, "tensor map (populations): error %d", (int)r);
            return false;
        }
    }
    for (int k = 0; k < 2; ++k) {
        cuuint64_t dims[2] = {(cuuint64_t)L.pitch, (cuuint64_t)L.nyf};
        cuuint64_t strides[1] = {(cuuint64_t)L.pitch * er};
        cuuint32_t box[2] = {bx, (cuuint32_t)(L.ty + 4)};
        cuuint32_t estr[2] = {1, 1};
        CUresult r = encode(&m->rho[k], dr, 2, L.rho[k], dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            snprintf(err, errlen, "tensor map (density): error %d", (int)r);
            return false;
        }
    }
    m->valid = 1;
    return true;
}

}  // namespace cplbm
