// Allocation-free FP64 step (lbm_step_noalloc in include/cplbm.h).
//
// For callers that may not allocate device memory themselves or through a
// library: for example a host application whose allocator owns the whole
// GPU and forbids other code from calling cudaMalloc, or one that cannot
// afford the device-wide synchronisation that cudaMalloc and cudaFree can
// cause while other work shares the GPU.  The caller passes only its own
// population array; the density hand-over buffers that a context would
// allocate live in one fixed device array of this file instead.
//
// The array is file-scope and static, so every GPU that loads the library
// holds it until the process exits, and every call shares it: calls that
// overlap on the GPU (different streams, or different host threads) race on
// it.  Each call clears the parts that must start at zero.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include <cudaTypedefs.h>

#include "../../include/cplbm.h"
#include "device_common.cuh"

namespace cplbm {
namespace {

constexpr size_t kScratchDoubles = LBM_NOALLOC_SCRATCH_BYTES / sizeof(double);

// The shared scratch of every lbm_step_noalloc call on a device.
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

// In host code the name g_noalloc_scratch is only a stand-in for the device
// array, not its address.  The address is looked up with the device current
// and cached per device together with the unique ID of the CUDA context it
// belongs to: after a device reset the primary context is a new one, the
// module is loaded again at a new address, and the next call looks it up
// again.  Where the driver cannot report a context ID, every call looks the
// address up.
constexpr int kMaxDevices = 64;
struct ScratchAddr {
    bool valid;
    unsigned long long ctx_id;
    double *ptr;
};
std::mutex g_setup_mutex;
ScratchAddr g_scratch_addr[kMaxDevices] = {};

bool current_context_id(unsigned long long *id)
{
    static PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
    static PFN_cuCtxGetId_v12000 get_id = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(p);
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(p);
    }
    CUcontext ctx = nullptr;
    return get_current && get_id && get_current(&ctx) == CUDA_SUCCESS && ctx &&
           get_id(ctx, id) == CUDA_SUCCESS;
}

cudaError_t scratch_on_current_device(int device, double **out)
{
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    unsigned long long id = 0;
    const bool have_id = current_context_id(&id);
    ScratchAddr &a = g_scratch_addr[device];
    if (!(have_id && a.valid && a.ctx_id == id)) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        a.ptr = static_cast<double *>(p);
        a.ctx_id = id;
        a.valid = have_id;
    }
    *out = a.ptr;
    return cudaSuccess;
}

// Offsets of the parts carved from the scratch array, in doubles, each part
// starting on a 256-byte boundary: the two density generations, then both
// generations of the eight partial-sum classes at the sizes a context would
// allocate for them (ring_elems).
constexpr size_t kAlign = 256 / sizeof(double);
inline size_t round_up(size_t n) { return (n + kAlign - 1) / kAlign * kAlign; }
size_t scratch_layout(const Lattice &L, size_t *rho_off, size_t ring_off[2][R_COUNT],
                      size_t *ring_begin)
{
    const size_t field = round_up((size_t)L.nyf * L.nx);
    size_t off = 0;
    for (int k = 0; k < 2; ++k) {
        rho_off[k] = off;
        off += field;
    }
    *ring_begin = off;
    for (int k = 0; k < 2; ++k)
        for (int c = 0; c < R_COUNT; ++c) {
            ring_off[k][c] = off;
            off += round_up(ring_elems(L, c));
        }
    return off;
}

// rho = sum_i f_i at every fluid node, from natural-order populations.
__global__ void noalloc_density_kernel(const Lattice L, const double *f,
                                       double *rho)
{
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= (long long)L.nx * L.nyf) return;
    const int x = (int)(n % L.nx), r = (int)(n / L.nx);
    const long long N = (long long)L.nx * L.ny;
    const long long g = (long long)(r + L.walls) * L.nx + x;
    double s = 0.0;
    for (int i = 0; i < 9; ++i) s += f[i * N + g];
    rho[fidx(L, r, x)] = s;
}

// Rest population back into plane 0: f_0 = rho - sum_{i>0} f_i.
__global__ void noalloc_rest_kernel(const Lattice L, int cur, double *f)
{
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= (long long)L.nx * L.nyf) return;
    const int x = (int)(n % L.nx), r = (int)(n / L.nx);
    const long long N = (long long)L.nx * L.ny;
    const long long g = (long long)(r + L.walls) * L.nx + x;
    double s = 0.0;
    for (int i = 1; i < 9; ++i) s += f[i * N + g];
    f[g] = load_rho<SF64>(L, cur, r, x) - s;
}

lbm_status fail_msg(lbm_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    set_global_error(buf);
    return st;
}

}  // namespace
}  // namespace cplbm

using namespace cplbm;

extern "C" lbm_status lbm_step_noalloc(
    const lbm_config *cfg, int eos, double a, double b, double R,
    double T_over_Tc, double omega, double mu_bottom, int top_mode,
    double mu_top, double *f, int nsteps)
{
    if (!cfg || !f) return fail_msg(LBM_ERR_ARG, "null argument");
    if (cfg->precision != LBM_F64)
        return fail_msg(LBM_ERR_ARG, "lbm_step_noalloc supports LBM_F64 only");
    if (cfg->nx < 5 || cfg->ny < 5 || (cfg->walls && cfg->ny < 7))
        return fail_msg(LBM_ERR_ARG, "lattice too small (%d x %d)", cfg->nx,
                        cfg->ny);
    if (cfg->walls != 0 && cfg->walls != 1)
        return fail_msg(LBM_ERR_ARG, "walls must be 0 or 1");
    if (!(cfg->tau > 0.5) || !(cfg->kappa >= 0) || !std::isfinite(cfg->tau) ||
        !std::isfinite(cfg->kappa))
        return fail_msg(LBM_ERR_ARG, "need tau > 0.5 and kappa >= 0");
    if (nsteps < 0 || (nsteps & 1))
        return fail_msg(LBM_ERR_ARG, "nsteps must be even and >= 0 (got %d)",
                        nsteps);
    if (eos < LBM_EOS_VDW || eos > LBM_EOS_RKS || !(a > 0 && b > 0 && R > 0))
        return fail_msg(LBM_ERR_ARG, "invalid EOS parameters");
    if (!(T_over_Tc > 0) || top_mode < 0 || top_mode > 1)
        return fail_msg(LBM_ERR_ARG, "invalid temperature or top_mode");

    Lattice L{};
    L.nx = cfg->nx;
    L.ny = cfg->ny;
    L.walls = cfg->walls;
    L.nyf = cfg->walls ? cfg->ny - 2 : cfg->ny;
    L.pitch = cfg->nx;
    L.nyf_pad = (L.nyf + 31) / 32 * 32;
    // f is [9][ny][nx]: planes 1..8 act as the in-place population array,
    // starting at the first fluid row
    L.plane = (long long)cfg->nx * cfg->ny;
    const size_t field = (size_t)L.nyf * L.nx;
    size_t rho_off[2], ring_off[2][R_COUNT], ring_begin;
    const size_t need = scratch_layout(L, rho_off, ring_off, &ring_begin);
    if (need > kScratchDoubles)
        return fail_msg(LBM_ERR_ARG,
                        "lattice %d x %d needs %zu bytes of scratch; the "
                        "fixed array holds %zu (LBM_NOALLOC_SCRATCH_BYTES)",
                        cfg->nx, cfg->ny, need * sizeof(double),
                        (size_t)LBM_NOALLOC_SCRATCH_BYTES);

    double Tc, rhoc;
    if (!host_critical(eos, a, b, R, &Tc, &rhoc))
        return fail_msg(LBM_ERR_NUMERIC, "critical point not found");
    const double alpha = host_alpha(eos, T_over_Tc, omega);
    L.tau = cfg->tau;
    L.kappa = cfg->kappa;
    L.rho_ref = 0.0;
    L.eos.kind = eos;
    L.eos.a = a;
    L.eos.b = b;
    L.eos.RT = R * T_over_Tc * Tc;
    L.eos.aalpha = a * alpha;
    L.mu_bottom = mu_bottom;
    L.top_mode = top_mode;
    L.mu_top = mu_top;
    L.precision = P_F64;
    L.wait_cycles = WAIT_CYCLES_DEFAULT;  // no TMA path here; set for completeness
    set_consts(L);
    step_default_shape(P_F64, &L.tx, &L.ty);

    if (cfg->device < 0 || cfg->device >= kMaxDevices)
        return fail_msg(LBM_ERR_ARG, "device ordinal %d out of range",
                        cfg->device);
    cudaError_t e = cudaSetDevice(cfg->device);
    if (e != cudaSuccess)
        return fail_msg(LBM_ERR_CUDA, "cudaSetDevice(%d): %s", cfg->device,
                        cudaGetErrorString(e));
    double *scratch = nullptr;
    e = scratch_on_current_device(cfg->device, &scratch);
    if (e != cudaSuccess)
        return fail_msg(LBM_ERR_CUDA, "cudaGetSymbolAddress: %s",
                        cudaGetErrorString(e));
    L.pops = f + L.plane + (long long)L.walls * L.nx;
    for (int k = 0; k < 2; ++k) {
        L.rho[k] = scratch + rho_off[k];
        for (int c = 0; c < R_COUNT; ++c) L.ring[k][c] = scratch + ring_off[k][c];
    }
#ifdef CPLBM_CHECK_BOUNDS
    // f holds 9 planes of nx * ny values; no error flag here, so an access
    // outside its buffer is skipped without a report
    set_bounds(L, (8 * L.plane - (long long)L.walls * L.nx) * (long long)sizeof(double),
               (long long)field * (long long)sizeof(double));
#endif

    cudaStream_t s = (cudaStream_t)cfg->stream;
    // the partial sums are read for tile-edge nodes from the first step on
    // and must start at zero; the last call left its own values there
    e = cudaMemsetAsync(scratch + ring_begin, 0, (need - ring_begin) * sizeof(double), s);
    if (e != cudaSuccess)
        return fail_msg(LBM_ERR_CUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    const unsigned blocks = (unsigned)((field + 255) / 256);
    noalloc_density_kernel<<<blocks, 256, 0, s>>>(L, f, (double *)L.rho[0]);
    e = cudaGetLastError();
    for (int k = 0; k < nsteps && e == cudaSuccess; ++k)
        e = launch_step(L, k & 1, k & 1, s);
    if (e == cudaSuccess) {
        noalloc_rest_kernel<<<blocks, 256, 0, s>>>(L, 0, f);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess)
        return fail_msg(LBM_ERR_CUDA, "kernel launch: %s", cudaGetErrorString(e));
    return LBM_OK;
}
