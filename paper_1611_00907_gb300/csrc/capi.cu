// C ABI of the cplbm library (include/cplbm.h): context and device memory,
// argument checks, EOS set-up and the host side of every call.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <new>
#include <string>

#include "../../include/cplbm.h"
#include "cplbm_internal.h"
#include "trace.h"

using namespace cplbm;

#include "context.h"

static thread_local std::string g_err;

namespace cplbm {
namespace {
// Device allocations the library holds, and the countdown of the test hook
// lbm_test_fail_device_alloc (negative: disarmed).
std::atomic<long long> g_live_allocs{0};
std::atomic<int> g_fail_countdown{-1};
}  // namespace

cudaError_t dev_alloc(void **p, size_t bytes)
{
    *p = nullptr;
    int n = g_fail_countdown.load();
    while (n >= 0 && !g_fail_countdown.compare_exchange_weak(n, n - 1)) {
    }
    if (n == 0) return cudaErrorMemoryAllocation;  // the injected failure
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) ++g_live_allocs;
    else *p = nullptr;
    return e;
}

void dev_free(void *p)
{
    if (!p) return;
    if (cudaFree(p) == cudaSuccess) --g_live_allocs;
}
}  // namespace cplbm

namespace {

lbm_status fail(lbm_ctx *c, lbm_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    (c ? c->err : g_err) = buf;
    return s;
}

#define CUDA_TRY(c, call)                                                    \
    do {                                                                     \
        cudaError_t e_ = (call);                                             \
        if (e_ != cudaSuccess)                                               \
            return fail((c), e_ == cudaErrorMemoryAllocation ? LBM_ERR_OOM   \
                                                             : LBM_ERR_CUDA, \
                        "%s: %s", #call, cudaGetErrorString(e_));            \
    } while (0)

// ---------------------------------------------------------------------------
// Thermodynamics on the host.  p0(rho) of Eqs. 16, 19, 22, 25 is evaluated
// on second-order forward-mode dual numbers, which carry p0, dp0/drho and
// d2p0/drho2 through the printed formula exactly (to rounding).
// ---------------------------------------------------------------------------
struct D2 {
    double v, d, dd;
};
D2 operator+(D2 a, D2 b) { return {a.v + b.v, a.d + b.d, a.dd + b.dd}; }
D2 operator-(D2 a, D2 b) { return {a.v - b.v, a.d - b.d, a.dd - b.dd}; }
D2 operator*(D2 a, D2 b)
{
    return {a.v * b.v, a.d * b.v + a.v * b.d,
            a.dd * b.v + 2 * a.d * b.d + a.v * b.dd};
}
D2 recip(D2 b)
{
    const double i = 1.0 / b.v;
    return {i, -b.d * i * i, 2 * b.d * b.d * i * i * i - b.dd * i * i};
}
D2 operator/(D2 a, D2 b) { return a * recip(b); }
D2 cst(double c) { return {c, 0, 0}; }

// p0 with temperature factor RT and attraction aa (a alpha).
D2 p0_dual(int kind, double aa, double b, double RT, D2 rho)
{
    const D2 one = cst(1), br = cst(b) * rho;
    switch (kind) {
    case EOS_VDW:
        return cst(RT) * rho / (one - br) - cst(aa) * rho * rho;
    case EOS_RKS:
        return cst(RT) * rho / (one - br) - cst(aa) * rho * rho / (one + br);
    case EOS_PR:
        return cst(RT) * rho / (one - br) -
               cst(aa) * rho * rho / (one + cst(2) * br - br * br);
    default: {  // CS
        const D2 h = cst(0.25) * br;
        const D2 q = one - h;
        return cst(RT) * rho * (one + h + h * h - h * h * h) / (q * q * q) -
               cst(aa) * rho * rho;
    }
    }
}

double pole(int kind, double b) { return (kind == EOS_CS ? 4.0 : 1.0) / b; }

// Critical point with alpha = 1.  p0 = T A(rho) - B(rho): A from
// p0(RT = R, aa = 0), B from -p0(RT = 0, aa = a).  Where p0' = p0'' = 0,
// T = B'/A' = B''/A'', so rho_c is the root of B' A'' - B'' A' (one sign
// change on (0, pole)); bisection to the last bit.
bool critical(int kind, double a, double b, double R, double *Tc, double *rc)
{
    auto g = [&](double r, double *T) {
        const D2 A = p0_dual(kind, 0.0, b, R, D2{r, 1, 0});
        const D2 B = p0_dual(kind, a, b, 0.0, D2{r, 1, 0});
        const double A1 = A.d, A2 = A.dd, B1 = -B.d, B2 = -B.dd;
        if (T) *T = B1 / A1;
        return B1 * A2 - B2 * A1;
    };
    double lo = 1e-9 * pole(kind, b), hi = (1 - 1e-9) * pole(kind, b);
    double glo = g(lo, nullptr), ghi = g(hi, nullptr);
    if (!(glo * ghi < 0)) return false;
    for (int it = 0; it < 2000; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        const double gm = g(mid, nullptr);
        if ((gm < 0) == (glo < 0)) { lo = mid; glo = gm; } else { hi = mid; }
    }
    *rc = 0.5 * (lo + hi);
    g(*rc, Tc);
    return std::isfinite(*Tc) && *Tc > 0;
}

// alpha(T) of PR (text under Eq. 22) and RKS (text under Eq. 19).
double alpha_of(int kind, double Tr, double omega)
{
    double m;
    if (kind == EOS_PR) m = 0.37464 + 1.54226 * omega - 0.26992 * omega * omega;
    else if (kind == EOS_RKS) m = 0.480 + 1.574 * omega - 0.176 * omega * omega;
    else return 1.0;
    const double s = 1.0 + m * (1.0 - std::sqrt(Tr));
    return s * s;
}

// Printed bulk chemical potential psi'(rho) (Eqs. 18, 21, 24, 27 without
// the gradient term), host FP64, for the coexistence solver.
double host_mu(int kind, double a, double aa, double b, double RT, double r)
{
    const double q = 1.0 - b * r;
    switch (kind) {
    case EOS_VDW:
        return RT * (std::log(r / q) + 1.0 / q) - 2.0 * a * r;
    case EOS_RKS:
        return RT * std::log(r / q) + RT / q - aa / b * std::log(1.0 + b * r) -
               aa * r / (1.0 + b * r);
    case EOS_PR: {
        const double s2 = std::sqrt(2.0);
        return RT * std::log(r / q) -
               aa / (2.0 * s2 * b) * std::log((s2 - 1.0 + b * r) / (s2 + 1.0 - b * r)) +
               RT / q - aa * r / (1.0 + 2.0 * b * r - b * b * r * r);
    }
    default: {  // CS
        const double h = 0.25 * b * r, qc = 1.0 - h;
        return RT * ((3.0 - h) / (qc * qc * qc) + std::log(r) + 1.0) - 2.0 * a * r;
    }
    }
}

// Root of a monotonic f on [lo, hi] (f(lo), f(hi) of opposite signs) by
// bisection to the last representable midpoint.
template <class F>
double bisect(F f, double lo, double hi)
{
    double flo = f(lo);
    for (int it = 0; it < 2000; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        const double fm = f(mid);
        if ((fm < 0) == (flo < 0)) { lo = mid; flo = fm; } else { hi = mid; }
    }
    return 0.5 * (lo + hi);
}

// Coexisting densities by the Maxwell construction (Sec. III): the pressure
// p_s at which the vapour and liquid branches of p0 have equal chemical
// potential, found by bisection in p_s between the spinodal pressures.
bool coexistence(int kind, double a, double b, double R, double Tr,
                 double omega, double *rv, double *rl, double *muc)
{
    double Tc, rc;
    if (!(Tr > 0 && Tr < 1) || !critical(kind, a, b, R, &Tc, &rc)) return false;
    const double RT = R * Tr * Tc, aa = a * alpha_of(kind, Tr, omega);
    const double top = pole(kind, b);
    auto p = [&](double r) { return p0_dual(kind, aa, b, RT, D2{r, 1, 0}).v; };
    auto dp = [&](double r) { return p0_dual(kind, aa, b, RT, D2{r, 1, 0}).d; };
    if (!(dp(rc) < 0)) return false;
    const double s1 = bisect(dp, 1e-12 * top, rc);   // dp0/drho = 0, vapour side
    const double s2 = bisect(dp, rc, (1 - 1e-12) * top);
    const double phi = p(s1), plo = std::max(p(s2), 0.0);
    auto roots = [&](double ps, double *v, double *l) {
        *v = bisect([&](double r) { return p(r) - ps; }, 1e-300, s1);
        *l = bisect([&](double r) { return p(r) - ps; }, s2, (1 - 1e-14) * top);
    };
    auto g = [&](double ps) {
        double v, l;
        roots(ps, &v, &l);
        return host_mu(kind, a, aa, b, RT, v) - host_mu(kind, a, aa, b, RT, l);
    };
    const double ps = bisect(g, plo + 1e-14 * std::fabs(phi), phi * (1 - 1e-12));
    roots(ps, rv, rl);
    *muc = 0.5 * (host_mu(kind, a, aa, b, RT, *rv) + host_mu(kind, a, aa, b, RT, *rl));
    return std::isfinite(*rv) && std::isfinite(*rl) && *rv < *rl;
}

lbm_status ensure_tmp(lbm_ctx *c, size_t bytes)
{
    if (c->tmp_bytes >= bytes) return LBM_OK;
    dev_free(c->d_tmp);
    c->d_tmp = nullptr;
    c->tmp_bytes = 0;
    CUDA_TRY(c, dev_alloc((void **)&c->d_tmp, bytes));
    c->tmp_bytes = bytes;
    return LBM_OK;
}

// Queue the zeroing of both generations of partial sums.
cudaError_t clear_rings(const Lattice &L, cudaStream_t s)
{
    const size_t rb = rho_bytes(L.precision);
    for (int k = 0; k < 2; ++k)
        for (int r = 0; r < R_COUNT; ++r) {
            cudaError_t e = cudaMemsetAsync(L.ring[k][r], 0, ring_elems(L, r) * rb, s);
            if (e != cudaSuccess) return e;
        }
    return cudaSuccess;
}

void free_all(lbm_ctx *c)
{
    if (c->graph) cudaGraphExecDestroy(c->graph);
    if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
    c->graph = nullptr;
    c->capture_stream = nullptr;
    Lattice &L = c->L;
    dev_free(L.pops);
    for (int k = 0; k < 2; ++k) {
        dev_free(L.rho[k]);
        for (int r = 0; r < R_COUNT; ++r) dev_free(L.ring[k][r]);
    }
    dev_free(c->d_red);
    dev_free(c->d_bad);
    dev_free(c->d_prev);
    dev_free(c->d_tmp);
    dev_free(c->d_err);
}

// Tensor maps for the current tile shape (the TMA path is skipped when they
// cannot be built, e.g. for FP16 storage).
void refresh_maps(lbm_ctx *c)
{
    char msg[256];
    c->maps.valid = 0;
    if (c->use_tma) build_tma_maps(c->L, &c->maps, msg, sizeof msg);
}

// Kernel error flags: a bounded wait inside a kernel gave up.
lbm_status check_kernel_flags(lbm_ctx *c)
{
    int flags = 0;
    CUDA_TRY(c, cudaMemcpy(&flags, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (flags) {
        CUDA_TRY(c, cudaMemset(c->d_err, 0, sizeof(int)));
        if (flags & ERR_BOUNDS)
            return fail(c, LBM_ERR_CUDA, "a kernel accessed memory outside its buffer "
                        "(bounds-checked build; flags %d); the access was skipped", flags);
        return fail(c, LBM_ERR_CUDA, "a step kernel's wait for its data timed out "
                    "(flags %d); the affected tiles were not updated", flags);
    }
    return LBM_OK;
}

struct StateHeader {
    char magic[8];  // "CPLBMST1"
    int nx, ny, walls, precision;
    long long t;
};

// Steps replayed per CUDA graph launch (from an even step: both in-place
// parities in turn).
constexpr int STEP_GRAPH_STEPS = 16;

cudaError_t launch_one_step(lbm_ctx *c, cudaStream_t s)
{
    const int p = (int)(c->t & 1);
    return c->force_model == 1 ? launch_step_pt(c->L, p, p, s, &c->maps)
                               : launch_step(c->L, p, p, s, &c->maps);
}

// The graph of STEP_GRAPH_STEPS steps from an even step, captured on a
// private stream (the caller's may be the legacy stream, which cannot
// capture) and launched on the caller's.  Its kernels carry the lattice
// descriptor and tensor maps by value: a change of tile shape, physics,
// force model or wait limit since the capture makes a new one.  Returns
// false (direct launches) when capture is not possible.
bool step_graph(lbm_ctx *c)
{
    if (c->graph_failed) return false;
    // the caller capturing on its stream: direct launches join its graph
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (c->stream && (cudaStreamIsCapturing(c->stream, &cs) != cudaSuccess ||
                      cs != cudaStreamCaptureStatusNone))
        return false;
    if (c->graph && std::memcmp(&c->graph_L, &c->L, sizeof(Lattice)) == 0 &&
        std::memcmp(&c->graph_maps, &c->maps, sizeof(TmaMaps)) == 0 &&
        c->graph_force == c->force_model)
        return true;
    if (c->graph) cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
    if (!c->capture_stream &&
        cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
        c->capture_stream = nullptr;
        c->graph_failed = true;
        return false;
    }
    const long long t0 = c->t;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(c->capture_stream, cudaStreamCaptureModeThreadLocal);
    const bool capturing = e == cudaSuccess;
    for (int k = 0; k < STEP_GRAPH_STEPS && e == cudaSuccess; ++k, ++c->t)
        e = launch_one_step(c, c->capture_stream);
    c->t = t0;
    const cudaError_t e2 = capturing ? cudaStreamEndCapture(c->capture_stream, &g) : cudaSuccess;
    if (e == cudaSuccess && e2 == cudaSuccess)
        e = cudaGraphInstantiate(&c->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        cudaGetLastError();  // the direct launches report their own errors
        c->graph = nullptr;
        c->graph_failed = true;
        return false;
    }
    // byte copies: the comparison above covers padding bytes too
    std::memcpy(&c->graph_L, &c->L, sizeof(Lattice));
    std::memcpy(&c->graph_maps, &c->maps, sizeof(TmaMaps));
    c->graph_force = c->force_model;
    return true;
}

}  // namespace

namespace cplbm {
// Host helpers shared with the allocation-free entry point (noalloc.cu).
bool host_critical(int kind, double a, double b, double R, double *Tc,
                   double *rhoc)
{
    return critical(kind, a, b, R, Tc, rhoc);
}
double host_alpha(int kind, double Tr, double omega)
{
    return alpha_of(kind, Tr, omega);
}
void set_global_error(const char *msg) { g_err = msg; }
}  // namespace cplbm

extern "C" {

lbm_status lbm_create(const lbm_config *cfg, lbm_ctx **out)
{
    if (out) *out = nullptr;
    if (!cfg || !out) return fail(nullptr, LBM_ERR_ARG, "null argument");
    if (cfg->nx < 5 || cfg->ny < 5)
        return fail(nullptr, LBM_ERR_ARG, "nx and ny must be >= 5 (got %d, %d)",
                    cfg->nx, cfg->ny);
    if (cfg->walls != 0 && cfg->walls != 1)
        return fail(nullptr, LBM_ERR_ARG, "walls must be 0 or 1");
    if (cfg->walls && cfg->ny < 7)
        return fail(nullptr, LBM_ERR_ARG, "walls need ny >= 7");
    if (!(cfg->tau > 0.5) || !std::isfinite(cfg->tau))
        return fail(nullptr, LBM_ERR_ARG, "tau must be > 0.5 (got %g)", cfg->tau);
    if (!(cfg->kappa >= 0) || !std::isfinite(cfg->kappa))
        return fail(nullptr, LBM_ERR_ARG, "kappa must be >= 0");
    if (cfg->precision < LBM_F64 || cfg->precision > LBM_F16_OFFSET)
        return fail(nullptr, LBM_ERR_ARG, "unknown precision %d", cfg->precision);
    if (!std::isfinite(cfg->rho_ref))
        return fail(nullptr, LBM_ERR_ARG, "rho_ref must be finite");
    if ((long long)cfg->nx * cfg->ny > (1LL << 31))
        return fail(nullptr, LBM_ERR_ARG, "lattice larger than 2^31 nodes");

    lbm_ctx *c = new (std::nothrow) lbm_ctx();
    if (!c) return fail(nullptr, LBM_ERR_OOM, "host allocation failed");
    c->device = cfg->device;
    c->stream = (cudaStream_t)cfg->stream;
    cudaError_t e = cudaSetDevice(cfg->device);
    if (e != cudaSuccess) {
        delete c;
        return fail(nullptr, LBM_ERR_CUDA, "cudaSetDevice(%d): %s", cfg->device,
                    cudaGetErrorString(e));
    }
    Lattice &L = c->L;
    L.nx = cfg->nx;
    L.ny = cfg->ny;
    L.walls = cfg->walls;
    L.nyf = cfg->walls ? cfg->ny - 2 : cfg->ny;
    L.pitch = (cfg->nx + 31) / 32 * 32;
    L.nyf_pad = (L.nyf + 31) / 32 * 32;
    L.plane = (long long)L.nyf * L.pitch;
    L.tau = cfg->tau;
    L.kappa = cfg->kappa;
    L.rho_ref = (cfg->precision == LBM_F32_OFFSET ||
                 cfg->precision == LBM_F16_OFFSET) ? cfg->rho_ref : 0.0;
    L.precision = cfg->precision;
    L.top_mode = 0;
    set_consts(L);
    step_default_shape(L.precision, &L.tx, &L.ty);

    const size_t pb = pop_bytes(L.precision), rb = rho_bytes(L.precision);
    lbm_status st = LBM_OK;
    auto alloc = [&](void **p, size_t bytes) {
        if (st != LBM_OK) return;
        cudaError_t ea = dev_alloc(p, bytes);
        if (ea != cudaSuccess) {
            *p = nullptr;
            st = fail(nullptr, LBM_ERR_OOM, "device allocation of %zu bytes: %s", bytes,
                      cudaGetErrorString(ea));
        }
    };
    alloc(&L.pops, 8 * (size_t)L.plane * pb);
#ifdef CPLBM_CHECK_BOUNDS
    set_bounds(L, 8 * L.plane * (long long)pb, L.plane * (long long)rb);
#endif
    for (int k = 0; k < 2; ++k) {
        alloc(&L.rho[k], (size_t)L.plane * rb);
        for (int r = 0; r < R_COUNT; ++r) alloc(&L.ring[k][r], ring_elems(L, r) * rb);
    }
    alloc((void **)&c->d_red, 4 * sizeof(double));
    alloc((void **)&c->d_bad, sizeof(int));
    alloc((void **)&c->d_prev, (size_t)L.nx * L.ny * sizeof(double));
    alloc((void **)&c->d_err, sizeof(int));
    if (st == LBM_OK && cudaMemset(c->d_err, 0, sizeof(int)) != cudaSuccess)
        st = fail(nullptr, LBM_ERR_CUDA, "cudaMemset failed");
    if (st != LBM_OK) {
        free_all(c);
        delete c;
        return st;
    }
    L.err = c->d_err;
    L.wait_cycles = WAIT_CYCLES_DEFAULT;
    const char *no_tma = getenv("CPLBM_NO_TMA");
    c->use_tma = !(no_tma && no_tma[0] == '1');
    refresh_maps(c);
    *out = c;
    return LBM_OK;
}

lbm_status lbm_eos_critical(int eos, double a, double b, double R, double *Tc,
                            double *rhoc)
{
    if (!Tc || !rhoc) return fail(nullptr, LBM_ERR_ARG, "null output");
    if (eos < LBM_EOS_VDW || eos > LBM_EOS_RKS)
        return fail(nullptr, LBM_ERR_ARG, "unknown EOS %d", eos);
    if (!(a > 0 && b > 0 && R > 0))
        return fail(nullptr, LBM_ERR_ARG, "a, b, R must be positive");
    if (!critical(eos, a, b, R, Tc, rhoc))
        return fail(nullptr, LBM_ERR_NUMERIC, "critical point not found");
    return LBM_OK;
}

lbm_status lbm_eos_coexistence(int eos, double a, double b, double R,
                               double T_over_Tc, double omega, double *rho_v,
                               double *rho_l, double *mu_coex)
{
    if (!rho_v || !rho_l) return fail(nullptr, LBM_ERR_ARG, "null output");
    if (eos < LBM_EOS_VDW || eos > LBM_EOS_RKS || !(a > 0 && b > 0 && R > 0))
        return fail(nullptr, LBM_ERR_ARG, "invalid EOS parameters");
    if (!(T_over_Tc > 0 && T_over_Tc < 1))
        return fail(nullptr, LBM_ERR_ARG, "coexistence needs 0 < T/T_c < 1");
    double mu = 0;
    if (!coexistence(eos, a, b, R, T_over_Tc, omega, rho_v, rho_l, &mu))
        return fail(nullptr, LBM_ERR_NUMERIC, "Maxwell construction failed");
    if (mu_coex) *mu_coex = mu;
    return LBM_OK;
}

lbm_status lbm_eos_pressure(int eos, double a, double b, double R,
                            double T_over_Tc, double omega, const double *rho,
                            double *p, size_t n)
{
    if ((!rho || !p) && n) return fail(nullptr, LBM_ERR_ARG, "null array");
    if (eos < LBM_EOS_VDW || eos > LBM_EOS_RKS || !(a > 0 && b > 0 && R > 0))
        return fail(nullptr, LBM_ERR_ARG, "invalid EOS parameters");
    if (!(T_over_Tc > 0) || !std::isfinite(T_over_Tc) || !std::isfinite(omega))
        return fail(nullptr, LBM_ERR_ARG, "T_over_Tc must be positive and finite");
    double Tc, rc;
    if (!critical(eos, a, b, R, &Tc, &rc))
        return fail(nullptr, LBM_ERR_NUMERIC, "critical point not found");
    const double RT = R * T_over_Tc * Tc, aa = a * alpha_of(eos, T_over_Tc, omega);
    const double top = pole(eos, b);
    for (size_t k = 0; k < n; ++k) {
        if (!(rho[k] > 0 && rho[k] < top))
            return fail(nullptr, LBM_ERR_ARG, "density %g outside (0, %g)", rho[k], top);
        p[k] = p0_dual(eos, aa, b, RT, D2{rho[k], 1, 0}).v;
    }
    return LBM_OK;
}

lbm_status lbm_tile_kinds(int nx, int ny, int walls, int tx, int ty, int seams,
                          int *kinds, size_t max)
{
    if (!kinds) return fail(nullptr, LBM_ERR_ARG, "null array");
    if (nx < 5 || ny < (walls ? 7 : 5))
        return fail(nullptr, LBM_ERR_ARG, "lattice %d x %d too small", nx, ny);
    int sx[16], sy[16];
    const int ns = step_shapes(sx, sy, 16);
    bool known = false;
    for (int k = 0; k < ns && k < 16; ++k) known = known || (sx[k] == tx && sy[k] == ty);
    if (!known) return fail(nullptr, LBM_ERR_ARG, "no step kernel for tile %d x %d", tx, ty);
    Lattice L{};
    L.nx = nx;
    L.ny = ny;
    L.walls = walls ? 1 : 0;
    L.nyf = walls ? ny - 2 : ny;
    const int ntx = (nx + tx - 1) / tx, nty = (L.nyf + ty - 1) / ty;
    if ((size_t)ntx * nty > max)
        return fail(nullptr, LBM_ERR_ARG, "kinds holds %zu entries, %d x %d needed", max, ntx,
                    nty);
    const int sb = seams ? seam_bits(L, tx, ty) : 0;
    for (int by = 0; by < nty; ++by)
        for (int bx = 0; bx < ntx; ++bx)
            kinds[(size_t)by * ntx + bx] = tile_kind(L, tx, ty, bx, by, sb);
    return LBM_OK;
}

lbm_status lbm_set_eos(lbm_ctx *c, int eos, double a, double b, double R,
                       double T_over_Tc, double omega)
{
    if (!c) return fail(nullptr, LBM_ERR_ARG, "null context");
    if (eos < LBM_EOS_VDW || eos > LBM_EOS_RKS)
        return fail(c, LBM_ERR_ARG, "unknown EOS %d", eos);
    if (!(a > 0 && b > 0 && R > 0))
        return fail(c, LBM_ERR_ARG, "a, b, R must be positive");
    if (!(T_over_Tc > 0) || !std::isfinite(T_over_Tc) || !std::isfinite(omega))
        return fail(c, LBM_ERR_ARG, "T_over_Tc must be positive and finite");
    double Tc, rc;
    if (!critical(eos, a, b, R, &Tc, &rc))
        return fail(c, LBM_ERR_NUMERIC, "critical point not found");
    c->Tc = Tc;
    c->rhoc = rc;
    c->T = T_over_Tc * Tc;
    c->alpha = alpha_of(eos, T_over_Tc, omega);
    EosParams &E = c->L.eos;
    E.kind = eos;
    E.a = a;
    E.b = b;
    E.RT = R * c->T;
    E.aalpha = a * c->alpha;
    set_consts(c->L);
    c->eos_set = true;
    return LBM_OK;
}

lbm_status lbm_eos_info(const lbm_ctx *c, double *T, double *alpha,
                        double *Tc, double *rhoc)
{
    if (!c) return fail(nullptr, LBM_ERR_ARG, "null context");
    if (!c->eos_set)
        return fail(const_cast<lbm_ctx *>(c), LBM_ERR_STATE, "EOS not set");
    if (T) *T = c->T;
    if (alpha) *alpha = c->alpha;
    if (Tc) *Tc = c->Tc;
    if (rhoc) *rhoc = c->rhoc;
    return LBM_OK;
}

lbm_status lbm_set_tile(lbm_ctx *c, int tx, int ty)
{
    CPLBM_TRACE("lbm_set_tile");
    if (!c) return fail(nullptr, LBM_ERR_ARG, "null context");
    if (!step_shape_supported(c->L.precision, tx, ty))
        return fail(c, LBM_ERR_ARG, "no step kernel for tile %d x %d", tx, ty);
    if (c->force_model == 1 && !pt_shape_supported(c->L.precision, tx, ty))
        return fail(c, LBM_ERR_ARG, "the pressure-tensor baseline has no "
                    "kernel for tile %d x %d", tx, ty);
    if (c->initialized && (tx != c->L.tx || ty != c->L.ty)) {
        // The tile grid defines how the current density is split between
        // rho and the partial sums: gather it whole before switching.
        CUDA_TRY(c, cudaSetDevice(c->device));
        Lattice &L = c->L;
        const int p = (int)(c->t & 1);
        CUDA_TRY(c, launch_gather_rho(L, p, L.rho[p ^ 1], c->stream));
        const size_t rb = rho_bytes(L.precision);
        CUDA_TRY(c, clear_rings(L, c->stream));
        CUDA_TRY(c, cudaMemcpyAsync(L.rho[p], L.rho[p ^ 1], (size_t)L.plane * rb,
                                    cudaMemcpyDeviceToDevice, c->stream));
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    }
    c->L.tx = tx;
    c->L.ty = ty;
    refresh_maps(c);
    return LBM_OK;
}

namespace {
// Copy the current state (populations and whole density) into snap, or back
// from it, leaving the partial sums zero.  snap holds pops then density.
lbm_status snapshot(lbm_ctx *c, char *snap, bool save)
{
    Lattice &L = c->L;
    const int p = (int)(c->t & 1);
    const size_t pb = 8 * (size_t)L.plane * pop_bytes(L.precision);
    const size_t rb = (size_t)L.plane * rho_bytes(L.precision);
    if (save) {
        CUDA_TRY(c, launch_gather_rho(L, p, snap + pb, c->stream));
        CUDA_TRY(c, cudaMemcpyAsync(snap, L.pops, pb, cudaMemcpyDeviceToDevice,
                                    c->stream));
    } else {
        CUDA_TRY(c, clear_rings(L, c->stream));
        CUDA_TRY(c, cudaMemcpyAsync(L.pops, snap, pb, cudaMemcpyDeviceToDevice,
                                    c->stream));
        CUDA_TRY(c, cudaMemcpyAsync(L.rho[p], snap + pb, rb,
                                    cudaMemcpyDeviceToDevice, c->stream));
    }
    return LBM_OK;
}
}  // namespace

lbm_status lbm_autotune(lbm_ctx *c, int nsteps, int *best_tx, int *best_ty)
{
    CPLBM_TRACE("lbm_autotune");
    if (!c) return fail(nullptr, LBM_ERR_ARG, "null context");
    if (!c->initialized) return fail(c, LBM_ERR_STATE, "lbm_init must come first");
    if (nsteps < 2) nsteps = 2;
    nsteps &= ~1;
    CUDA_TRY(c, cudaSetDevice(c->device));
    Lattice &L = c->L;
    const size_t bytes = 8 * (size_t)L.plane * pop_bytes(L.precision) +
                         (size_t)L.plane * rho_bytes(L.precision);
    char *snap = nullptr;
    CUDA_TRY(c, dev_alloc((void **)&snap, bytes));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int tx[16], ty[16];
    const int n = step_shapes(tx, ty, 16);
    const long long t0 = c->t;
    int best = -1;
    float best_ms = 0.f;
    lbm_status st = snapshot(c, snap, true);
    cudaError_t e = cudaSuccess;
    if (st == LBM_OK) e = cudaEventCreate(&e0);
    if (st == LBM_OK && e == cudaSuccess) e = cudaEventCreate(&e1);
    for (int k = 0; k < n && st == LBM_OK && e == cudaSuccess; ++k) {
        // the shapes of the force model in use, timed with its step
        if (!step_shape_supported(L.precision, tx[k], ty[k])) continue;
        if (c->force_model == 1 && !pt_shape_supported(L.precision, tx[k], ty[k])) continue;
        L.tx = tx[k];
        L.ty = ty[k];
        refresh_maps(c);
        st = snapshot(c, snap, false);
        c->t = t0;
        for (int w = 0; w < 2 && e == cudaSuccess; ++w, ++c->t)
            e = launch_one_step(c, c->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
        for (int s = 0; s < nsteps && e == cudaSuccess; ++s, ++c->t)
            e = launch_one_step(c, c->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && (best < 0 || ms < best_ms)) {
            best = k;
            best_ms = ms;
        }
    }
    if (st == LBM_OK && e == cudaSuccess && best >= 0) {
        L.tx = tx[best];
        L.ty = ty[best];
        refresh_maps(c);
        st = snapshot(c, snap, false);
        c->t = t0;
        if (st == LBM_OK) e = cudaStreamSynchronize(c->stream);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    dev_free(snap);
    if (st != LBM_OK) return st;
    if (e != cudaSuccess)
        return fail(c, LBM_ERR_CUDA, "autotune: %s", cudaGetErrorString(e));
    if (best_tx) *best_tx = L.tx;
    if (best_ty) *best_ty = L.ty;
    return LBM_OK;
}

lbm_status lbm_set_force_model(lbm_ctx *c, int model)
{
    if (!c) return fail(nullptr, LBM_ERR_ARG, "null context");
    if (model == 0) {
        c->force_model = 0;
        return LBM_OK;
    }
    if (model != 1) return fail(c, LBM_ERR_ARG, "unknown force model %d", model);
    if (c->L.walls)
        return fail(c, LBM_ERR_ARG, "the pressure-tensor force has no wall rule "
                    "(Sec. IV defines the chemical-potential one)");
    if (c->L.precision != LBM_F64 && c->L.precision != LBM_F32)
        return fail(c, LBM_ERR_ARG, "the pressure-tensor baseline runs in "
                    "LBM_F64 or LBM_F32");
    int tx, ty;
    pt_shape(c->L.precision, &tx, &ty);
    lbm_status st = lbm_set_tile(c, tx, ty);
    if (st != LBM_OK) return st;
    c->force_model = 1;
    return LBM_OK;
}

lbm_status lbm_get_tile(const lbm_ctx *c, int *tx, int *ty)
{
    if (!c || !tx || !ty) return fail(nullptr, LBM_ERR_ARG, "null argument");
    *tx = c->L.tx;
    *ty = c->L.ty;
    return LBM_OK;
}

lbm_status lbm_set_wall_mu(lbm_ctx *c, double mu_bottom, int top_mode,
                           double mu_top)
{
    if (!c) return fail(nullptr, LBM_ERR_ARG, "null context");
    if (top_mode != 0 && top_mode != 1)
        return fail(c, LBM_ERR_ARG, "top_mode must be 0 or 1");
    if (!std::isfinite(mu_bottom) || !std::isfinite(mu_top))
        return fail(c, LBM_ERR_ARG, "surface chemical potentials must be finite");
    c->L.mu_bottom = mu_bottom;
    c->L.top_mode = top_mode;
    c->L.mu_top = mu_top;
    set_consts(c->L);
    return LBM_OK;
}

lbm_status lbm_init(lbm_ctx *c, const double *rho, const double *ux,
                    const double *uy, int on_device)
{
    CPLBM_TRACE("lbm_init");
    if (!c) return fail(nullptr, LBM_ERR_ARG, "null context");
    if (!rho) return fail(c, LBM_ERR_ARG, "rho is required");
    if (!c->eos_set) return fail(c, LBM_ERR_STATE, "lbm_set_eos must come first");
    CUDA_TRY(c, cudaSetDevice(c->device));
    Lattice &L = c->L;
    const size_t field = (size_t)L.nx * L.ny * sizeof(double);
    const double *drho = rho, *dux = ux, *duy = uy;
    if (!on_device) {
        lbm_status s = ensure_tmp(c, 3 * field);
        if (s != LBM_OK) return s;
        double *t0 = c->d_tmp, *t1 = t0 + (size_t)L.nx * L.ny,
               *t2 = t1 + (size_t)L.nx * L.ny;
        CUDA_TRY(c, cudaMemcpyAsync(t0, rho, field, cudaMemcpyHostToDevice, c->stream));
        drho = t0;
        dux = duy = nullptr;
        if (ux) {
            CUDA_TRY(c, cudaMemcpyAsync(t1, ux, field, cudaMemcpyHostToDevice, c->stream));
            dux = t1;
        }
        if (uy) {
            CUDA_TRY(c, cudaMemcpyAsync(t2, uy, field, cudaMemcpyHostToDevice, c->stream));
            duy = t2;
        }
    }
    const size_t rb = rho_bytes(L.precision);
    for (int k = 0; k < 2; ++k)
        CUDA_TRY(c, cudaMemsetAsync(L.rho[k], 0, (size_t)L.plane * rb, c->stream));
    CUDA_TRY(c, clear_rings(L, c->stream));
    CUDA_TRY(c, cudaMemsetAsync(c->d_bad, 0, sizeof(int), c->stream));
    CUDA_TRY(c, launch_init(L, drho, dux, duy, c->d_bad, c->stream));
    // the reduction snapshot starts at the initial density
    CUDA_TRY(c, cudaMemsetAsync(c->d_prev, 0, field, c->stream));
    CUDA_TRY(c, launch_macro(L, 0, 0, c->d_prev, nullptr, nullptr, nullptr,
                             nullptr, nullptr, nullptr, c->stream));
    int bad = 0;
    CUDA_TRY(c, cudaMemcpyAsync(&bad, c->d_bad, sizeof(int), cudaMemcpyDeviceToHost,
                                c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    c->t = 0;
    if (bad) {
        c->initialized = false;
        return fail(c, LBM_ERR_ARG,
                    "%d fluid node(s) with density outside (0, %g) or non-finite "
                    "velocity", bad, pole(L.eos.kind, L.eos.b));
    }
    c->initialized = true;
    return LBM_OK;
}

lbm_status lbm_step(lbm_ctx *c, int nsteps)
{
    CPLBM_TRACE("lbm_step");
    if (!c) return fail(nullptr, LBM_ERR_ARG, "null context");
    if (nsteps < 0) return fail(c, LBM_ERR_ARG, "nsteps must be >= 0");
    if (!c->initialized) return fail(c, LBM_ERR_STATE, "lbm_init must come first");
    CUDA_TRY(c, cudaSetDevice(c->device));
    int left = nsteps;
    if (left > 0 && (c->t & 1)) {  // graphs start on an even step
        CUDA_TRY(c, launch_one_step(c, c->stream));
        ++c->t;
        --left;
    }
    while (left >= STEP_GRAPH_STEPS && step_graph(c)) {
        CUDA_TRY(c, cudaGraphLaunch(c->graph, c->stream));
        c->t += STEP_GRAPH_STEPS;
        left -= STEP_GRAPH_STEPS;
    }
    for (; left > 0; --left) {
        CUDA_TRY(c, launch_one_step(c, c->stream));
        ++c->t;
    }
    return LBM_OK;
}

lbm_status lbm_moments(lbm_ctx *c, double *rho, double *vx, double *vy,
                       double *mu, int on_device)
{
    CPLBM_TRACE("lbm_moments");
    if (!c) return fail(nullptr, LBM_ERR_ARG, "null context");
    if (!c->initialized) return fail(c, LBM_ERR_STATE, "lbm_init must come first");
    CUDA_TRY(c, cudaSetDevice(c->device));
    Lattice &L = c->L;
    const int p = (int)(c->t & 1);
    const size_t n = (size_t)L.nx * L.ny, field = n * sizeof(double);
    if (on_device) {
        CUDA_TRY(c, launch_macro(L, p, p, rho, vx, vy, mu, nullptr, nullptr,
                                 nullptr, c->stream));
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        return check_kernel_flags(c);
    }
    lbm_status s = ensure_tmp(c, 4 * field);
    if (s != LBM_OK) return s;
    double *d[4] = {c->d_tmp, c->d_tmp + n, c->d_tmp + 2 * n, c->d_tmp + 3 * n};
    double *h[4] = {rho, vx, vy, mu};
    CUDA_TRY(c, launch_macro(L, p, p, rho ? d[0] : nullptr, vx ? d[1] : nullptr,
                             vy ? d[2] : nullptr, mu ? d[3] : nullptr, nullptr,
                             nullptr, nullptr, c->stream));
    for (int k = 0; k < 4; ++k)
        if (h[k])
            CUDA_TRY(c, cudaMemcpyAsync(h[k], d[k], field, cudaMemcpyDeviceToHost,
                                        c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    {
        lbm_status fs = check_kernel_flags(c);
        if (fs != LBM_OK) return fs;
    }
    return LBM_OK;
}

lbm_status lbm_get_populations(lbm_ctx *c, double *f, int on_device)
{
    CPLBM_TRACE("lbm_get_populations");
    if (!c) return fail(nullptr, LBM_ERR_ARG, "null context");
    if (!f) return fail(c, LBM_ERR_ARG, "null output");
    if (!c->initialized) return fail(c, LBM_ERR_STATE, "lbm_init must come first");
    CUDA_TRY(c, cudaSetDevice(c->device));
    Lattice &L = c->L;
    const int p = (int)(c->t & 1);
    const size_t bytes = 9 * (size_t)L.nx * L.ny * sizeof(double);
    double *dst = f;
    if (!on_device) {
        lbm_status s = ensure_tmp(c, bytes);
        if (s != LBM_OK) return s;
        dst = c->d_tmp;
    }
    CUDA_TRY(c, cudaMemsetAsync(dst, 0, bytes, c->stream));
    CUDA_TRY(c, launch_populations(L, p, p, dst, c->stream));
    if (!on_device)
        CUDA_TRY(c, cudaMemcpyAsync(f, dst, bytes, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    {
        lbm_status fs = check_kernel_flags(c);
        if (fs != LBM_OK) return fs;
    }
    return LBM_OK;
}

lbm_status lbm_reduce(lbm_ctx *c, double out[4])
{
    CPLBM_TRACE("lbm_reduce");
    if (!c) return fail(nullptr, LBM_ERR_ARG, "null context");
    if (!out) return fail(c, LBM_ERR_ARG, "null output");
    if (!c->initialized) return fail(c, LBM_ERR_STATE, "lbm_init must come first");
    CUDA_TRY(c, cudaSetDevice(c->device));
    const int p = (int)(c->t & 1);
    CUDA_TRY(c, cudaMemsetAsync(c->d_red, 0, 4 * sizeof(double), c->stream));
    CUDA_TRY(c, cudaMemsetAsync(c->d_bad, 0, sizeof(int), c->stream));
    CUDA_TRY(c, launch_macro(c->L, p, p, nullptr, nullptr, nullptr, nullptr,
                             c->d_red, c->d_prev, c->d_bad, c->stream));
    double h[4];
    int bad = 0;
    CUDA_TRY(c, cudaMemcpyAsync(h, c->d_red, sizeof h, cudaMemcpyDeviceToHost,
                                c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(&bad, c->d_bad, sizeof(int), cudaMemcpyDeviceToHost,
                                c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    {
        lbm_status fs = check_kernel_flags(c);
        if (fs != LBM_OK) return fs;
    }
    for (int k = 0; k < 4; ++k) out[k] = h[k];
    if (bad)
        return fail(c, LBM_ERR_NUMERIC, "%d fluid node(s) with non-finite "
                    "density or momentum", bad);
    return LBM_OK;
}

size_t lbm_state_size(const lbm_ctx *c)
{
    if (!c) return 0;
    const Lattice &L = c->L;
    return sizeof(StateHeader) + 8 * (size_t)L.plane * pop_bytes(L.precision) +
           (size_t)L.plane * rho_bytes(L.precision);
}

lbm_status lbm_get_state(lbm_ctx *c, void *buf, size_t bytes)
{
    CPLBM_TRACE("lbm_get_state");
    if (!c) return fail(nullptr, LBM_ERR_ARG, "null context");
    if (!buf || bytes < lbm_state_size(c))
        return fail(c, LBM_ERR_ARG, "buffer smaller than lbm_state_size()");
    if (!c->initialized) return fail(c, LBM_ERR_STATE, "lbm_init must come first");
    CUDA_TRY(c, cudaSetDevice(c->device));
    Lattice &L = c->L;
    const int p = (int)(c->t & 1);
    StateHeader h{};
    memcpy(h.magic, "CPLBMST1", 8);
    h.nx = L.nx; h.ny = L.ny; h.walls = L.walls; h.precision = L.precision;
    h.t = c->t;
    char *o = (char *)buf;
    memcpy(o, &h, sizeof h);
    o += sizeof h;
    const size_t pbytes = 8 * (size_t)L.plane * pop_bytes(L.precision);
    const size_t rbytes = (size_t)L.plane * rho_bytes(L.precision);
    // the next-step density buffer is free between steps: gather into it
    CUDA_TRY(c, launch_gather_rho(L, p, L.rho[p ^ 1], c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(o, L.pops, pbytes, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(o + pbytes, L.rho[p ^ 1], rbytes,
                                cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

lbm_status lbm_set_state(lbm_ctx *c, const void *buf, size_t bytes)
{
    CPLBM_TRACE("lbm_set_state");
    if (!c) return fail(nullptr, LBM_ERR_ARG, "null context");
    if (!buf || bytes < lbm_state_size(c))
        return fail(c, LBM_ERR_ARG, "buffer smaller than lbm_state_size()");
    if (!c->eos_set) return fail(c, LBM_ERR_STATE, "lbm_set_eos must come first");
    StateHeader h;
    memcpy(&h, buf, sizeof h);
    Lattice &L = c->L;
    if (memcmp(h.magic, "CPLBMST1", 8) != 0 || h.nx != L.nx || h.ny != L.ny ||
        h.walls != L.walls || h.precision != L.precision || h.t < 0)
        return fail(c, LBM_ERR_ARG, "state does not match this context");
    CUDA_TRY(c, cudaSetDevice(c->device));
    const char *in = (const char *)buf + sizeof h;
    const size_t pbytes = 8 * (size_t)L.plane * pop_bytes(L.precision);
    const size_t rbytes = (size_t)L.plane * rho_bytes(L.precision);
    const int p = (int)(h.t & 1);
    CUDA_TRY(c, clear_rings(L, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(L.pops, in, pbytes, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(L.rho[p], in + pbytes, rbytes,
                                cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    c->t = h.t;
    c->initialized = true;
    return LBM_OK;
}

long long lbm_step_count(const lbm_ctx *c) { return c ? c->t : -1; }

void lbm_destroy(lbm_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    free_all(c);
    delete c;
}

lbm_status lbm_test_set_wait_cycles(lbm_ctx *c, long long cycles)
{
    if (!c) return fail(nullptr, LBM_ERR_ARG, "null context");
    c->L.wait_cycles = cycles < 0 ? WAIT_CYCLES_DEFAULT : cycles;
    return LBM_OK;
}

void lbm_test_fail_device_alloc(int after) { g_fail_countdown = after < 0 ? -1 : after; }

long long lbm_test_device_allocs(void) { return g_live_allocs.load(); }

lbm_status lbm_test_shrink_bounds(lbm_ctx *c, long long rho_bytes)
{
    if (!c) return fail(nullptr, LBM_ERR_ARG, "null context");
#ifdef CPLBM_CHECK_BOUNDS
    if (rho_bytes < 0 || rho_bytes > c->L.b_rho)
        return fail(c, LBM_ERR_ARG, "extent must be 0 .. %lld bytes", c->L.b_rho);
    c->L.b_rho = rho_bytes;
    return LBM_OK;
#else
    (void)rho_bytes;
    return fail(c, LBM_ERR_STATE, "bounds checks exist in the checked build only");
#endif
}

lbm_status lbm_test_fp64_math(const double *x, int n, double *log_out, double *rcp_out)
{
    if (!x || !log_out || !rcp_out || n < 0)
        return fail(nullptr, LBM_ERR_ARG, "null buffer or negative count");
    if (n == 0) return LBM_OK;
    const size_t bytes = (size_t)n * sizeof(double);
    double *d = nullptr;
    cudaError_t e = dev_alloc((void **)&d, 3 * bytes);
    if (e != cudaSuccess)
        return fail(nullptr, e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA,
                    "device allocation: %s", cudaGetErrorString(e));
    e = cudaMemcpy(d, x, bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_fp64_math(d, n, d + n, d + 2 * (size_t)n, 0);
    if (e == cudaSuccess) e = cudaMemcpy(log_out, d + n, bytes, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(rcp_out, d + 2 * (size_t)n, bytes, cudaMemcpyDeviceToHost);
    dev_free(d);
    if (e != cudaSuccess)
        return fail(nullptr, LBM_ERR_CUDA, "fp64 math: %s", cudaGetErrorString(e));
    return LBM_OK;
}

const char *lbm_last_error(const lbm_ctx *c)
{
    return c ? c->err.c_str() : g_err.c_str();
}

}  // extern "C"

namespace cplbm {
size_t ctx_state_bytes(const lbm_ctx *c)
{
    const Lattice &L = c->L;
    return 8 * (size_t)L.plane * pop_bytes(L.precision) +
           (size_t)L.plane * rho_bytes(L.precision);
}
lbm_status ctx_snapshot(lbm_ctx *c, char *snap, bool save)
{
    return snapshot(c, snap, save);
}
void ctx_refresh_maps(lbm_ctx *c) { refresh_maps(c); }
}  // namespace cplbm
