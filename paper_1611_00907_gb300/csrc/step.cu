// Fused time step: dispatch to the per-precision kernels (step_<precision>.cu,
// templates in step_impl.cuh) and the table of compiled tile shapes.
#include "cplbm_internal.h"

namespace cplbm {

#define CPLBM_PREC_DECL(tag)                                                   \
    cudaError_t launch_step_##tag(const Lattice &L, int parity, int cur,       \
                                  cudaStream_t s, const TmaMaps *maps);        \
    cudaError_t launch_batch_##tag(const BatchList &w, int parity, int cur,   \
                                   int tx, int ty, cudaStream_t s);
CPLBM_PREC_DECL(f64)
CPLBM_PREC_DECL(f32)
CPLBM_PREC_DECL(f32off)
CPLBM_PREC_DECL(f16off)
#undef CPLBM_PREC_DECL
cudaError_t launch_pt_f64(const Lattice &L, int parity, int cur, cudaStream_t s,
                          const TmaMaps *maps);
cudaError_t launch_pt_f32(const Lattice &L, int parity, int cur, cudaStream_t s,
                          const TmaMaps *maps);

template <class T>
static void fill_consts(Consts<T> &k, const Lattice &L)
{
    const EosParams &e = L.eos;
    k.tau = T(L.tau);
    k.omega = T(1) / T(L.tau);
    k.kappa = T(L.kappa);
    k.rho_ref = T(L.rho_ref);
    k.mu_bottom = T(L.mu_bottom);
    k.mu_top = T(L.mu_top);
    k.eos.kind = e.kind;
    k.eos.a = T(e.a);
    k.eos.b = T(e.b);
    k.eos.RT = T(e.RT);
    k.eos.aalpha = T(e.aalpha);
    k.eos.quarter_b = T(0.25 * e.b);
    k.eos.pr_c = T(e.b > 0 ? e.aalpha / (2.0 * 1.4142135623730951 * e.b) : 0.0);
    k.eos.pr_s2m1 = T(0.41421356237309515);
    k.eos.pr_s2p1 = T(2.414213562373095);
    k.eos.rks_c = T(e.b > 0 ? e.aalpha / e.b : 0.0);
}

void set_consts(Lattice &L)
{
    fill_consts(L.cf, L);
    fill_consts(L.cd, L);
}

// Tile shapes with a compiled kernel (all precisions; same list in
// step_impl.cuh).
#define CPLBM_STEP_SHAPES(X) X(32, 16) X(32, 24) X(32, 32) X(64, 16) X(64, 32)

bool step_shape_supported(int prec, int tx, int ty)
{
    (void)prec;
#define CPLBM_CASE(a, b) if (tx == a && ty == b) return true;
    CPLBM_STEP_SHAPES(CPLBM_CASE)
#undef CPLBM_CASE
    return false;
}

int step_shapes(int *tx, int *ty, int max)
{
    int n = 0;
#define CPLBM_CASE(a, b)                    \
    if (n < max) { tx[n] = a; ty[n] = b; }  \
    ++n;
    CPLBM_STEP_SHAPES(CPLBM_CASE)
#undef CPLBM_CASE
    return n;
}

void step_default_shape(int prec, int *tx, int *ty)
{
    // fastest measured on GB300 for the 4096^2 workload (lbm_autotune picks
    // per lattice): the two-nodes-per-lane path's 64 x 16 for FP32
    // arithmetic (FP32, FP32-offset and FP16 storage), 32 x 32 for FP64
    *tx = prec == P_F64 ? 32 : 64;
    *ty = prec == P_F64 ? 32 : 16;
}

void pt_shape(int prec, int *tx, int *ty)
{
    // FP32: the step's default tile (two nodes per lane)
    *tx = prec == P_F64 ? 32 : 64;
    *ty = 16;
}

bool pt_shape_supported(int prec, int tx, int ty)
{
    if (prec == P_F64) return tx == 32 && ty == 16;
    if (prec == P_F32) return (tx == 64 && ty == 16) || (tx == 32 && ty == 32);
    return false;
}

cudaError_t launch_step_pt(const Lattice &L, int parity, int cur, cudaStream_t s,
                           const TmaMaps *maps)
{
    if (L.walls || !pt_shape_supported(L.precision, L.tx, L.ty)) return cudaErrorInvalidValue;
    if (L.precision == P_F64) return launch_pt_f64(L, parity, cur, s, maps);
    return launch_pt_f32(L, parity, cur, s, maps);
}

cudaError_t launch_step_batch(const BatchList &w, int parity, int cur, int precision,
                              int tx, int ty, cudaStream_t s)
{
    switch (precision) {
    case P_F64: return launch_batch_f64(w, parity, cur, tx, ty, s);
    case P_F32: return launch_batch_f32(w, parity, cur, tx, ty, s);
    case P_F32_OFF: return launch_batch_f32off(w, parity, cur, tx, ty, s);
    case P_F16_OFF: return launch_batch_f16off(w, parity, cur, tx, ty, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_step(const Lattice &L, int parity, int cur, cudaStream_t s,
                        const TmaMaps *maps)
{
    switch (L.precision) {
    case P_F64: return launch_step_f64(L, parity, cur, s, maps);
    case P_F32: return launch_step_f32(L, parity, cur, s, maps);
    case P_F32_OFF: return launch_step_f32off(L, parity, cur, s, maps);
    case P_F16_OFF: return launch_step_f16off(L, parity, cur, s, maps);
    }
    return cudaErrorInvalidValue;
}

}  // namespace cplbm
