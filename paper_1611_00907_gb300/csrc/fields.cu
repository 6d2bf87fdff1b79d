// Field kernels around the fused step: equilibrium initialisation (Eq. 14),
// macroscopic fields and FP64 reductions, natural-order populations, and
// the density gather used by checkpoints.
#include <cuda_fp16.h>

#include "device_common.cuh"

namespace cplbm {

// ---------------------------------------------------------------------------
// Initial state f_i = f_i^eq(rho, u) (Eq. 14) at every fluid node.
// ---------------------------------------------------------------------------
template <class S>
__global__ void init_kernel(const Lattice L, const double *rho_in,
                            const double *ux_in, const double *uy_in, int *bad)
{
    using pop_t = typename S::pop_t;
    using rho_t = typename S::rho_t;
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= (long long)L.nx * L.nyf) return;
    const int x = (int)(n % L.nx), r = (int)(n / L.nx);
    const long long g = (long long)(r + L.walls) * L.nx + x;  // lattice index
    const double rho = rho_in[g];
    const double ux = ux_in ? ux_in[g] : 0.0, uy = uy_in ? uy_in[g] : 0.0;
    const double pole = (L.eos.kind == EOS_CS ? 4.0 : 1.0) / L.eos.b;
    if (!(rho > 0.0 && rho < pole && isfinite(ux) && isfinite(uy)))
        atomicAdd(bad, 1);
    const double ref = S::offset ? L.rho_ref : 0.0;
    const double usq = 1.5 * (ux * ux + uy * uy);
    pop_t *A = (pop_t *)L.pops;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const double eu = ex(i) * ux + ey(i) * uy;
        const double feq =
            wgt<double>(i) * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - usq);
        pop_t *p = A + pidx(L, i, r, x);
        if (CPLBM_IN_POPS(L, p, 1)) st_real(p, (typename S::real)(feq - wgt<double>(i) * ref));
    }
    rho_t *q = (rho_t *)L.rho[0] + fidx(L, r, x);
    if (CPLBM_IN_RHO(L, 0, q, 1)) *q = (rho_t)(rho - ref);
}

// ---------------------------------------------------------------------------
// Macroscopic fields (rho, v = u + F / (2 rho), mu) on the lattice rows of
// the output, plus optional FP64 reductions.  Tiled like the step so that
// mu and F come from the same stencil code.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void atomic_max_nonneg(double *addr, double v)
{
    // non-negative doubles order like their bit patterns
    atomicMax((unsigned long long *)addr, (unsigned long long)__double_as_longlong(v));
}

template <class S, int TX, int TY>
__global__ void macro_kernel(const Lattice L, int parity, int cur,
                             double *o_rho, double *o_vx, double *o_vy,
                             double *o_mu, double *red, double *prev, int *bad)
{
    using real = typename S::real;
    using pop_t = typename S::pop_t;
    constexpr int WR = TX + 4, WM = TX + 2;
    extern __shared__ unsigned char smem_raw[];
    real *s_rho = reinterpret_cast<real *>(smem_raw);
    real *s_mu = s_rho + (TY + 4) * WR;
    __shared__ double s_red[4][32];
    __shared__ int s_bad;

    const int X0 = blockIdx.x * TX, Y0 = blockIdx.y * TY;
    const int wx = min(TX, L.nx - X0), wy = min(TY, L.nyf - Y0);
    if (threadIdx.x == 0) s_bad = 0;
    load_rho_tile<S, TX, TY>(L, cur, X0, Y0, s_rho);
    __syncthreads();
    mu_tile<S, TX, TY>(L, X0, Y0, s_rho, s_mu);
    __syncthreads();

    const real rho_ref = S::offset ? consts<real>(L).rho_ref : real(0);
    const pop_t *A = (const pop_t *)L.pops;
    double acc_m = 0.0, acc_x = 0.0, acc_y = 0.0, acc_d = 0.0;
    // s_rho holds the stored form; rho_ref makes it absolute
    int nbad = 0;
    for (int n = threadIdx.x; n < TX * TY; n += blockDim.x) {
        const int lx = n % TX, ly = n / TX;
        if (lx >= wx || ly >= wy) continue;
        const int x = X0 + lx, r = Y0 + ly;
        const int cr = (ly + 2) * WR + lx + 2, cm = (ly + 1) * WM + lx + 1;
        real f[9];
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            const pop_t *p = A + aa_read_index(L, parity, i, r, x);
            f[i] = CPLBM_IN_POPS(L, p, 1) ? ld_real(p) : real(0);
        }
        const real rho = s_rho[cr] + rho_ref;
        real gmx, gmy, grx, gry;
        grad9<real, WM>(s_mu, cm, gmx, gmy);
        grad9<real, WR>(s_rho, cr, grx, gry);
        const real Fx = -rho * gmx + grx / real(3);
        const real Fy = -rho * gmy + gry / real(3);
        const real jx = f[1] - f[3] + f[5] - f[6] - f[7] + f[8];
        const real jy = f[2] - f[4] + f[5] + f[6] - f[7] - f[8];
        const double px = (double)jx + 0.5 * (double)Fx;  // rho v
        const double py = (double)jy + 0.5 * (double)Fy;
        const long long g = (long long)(r + L.walls) * L.nx + x;
        if (o_rho) o_rho[g] = (double)rho;
        if (o_vx) o_vx[g] = px / (double)rho;
        if (o_vy) o_vy[g] = py / (double)rho;
        if (o_mu) o_mu[g] = (double)s_mu[cm];
        if (red) {
            acc_m += (double)rho;
            acc_x += px;
            acc_y += py;
            if (!(isfinite((double)rho) && isfinite(px) && isfinite(py)))
                ++nbad;
            if (prev) {
                const double d = fabs((double)rho - prev[g]);
                acc_d = fmax(acc_d, isfinite(d) ? d : 0.0);
                prev[g] = (double)rho;
            }
        }
    }
    // Solid rows: rho by Eq. 28 and the wall mu from the shared tiles.
    if (L.walls && (o_rho || o_mu || o_vx || o_vy)) {
        for (int lx = threadIdx.x; lx < wx; lx += blockDim.x) {
            const int x = X0 + lx;
            if (Y0 == 0) {
                const long long g = x;
                if (o_rho) o_rho[g] = (double)(s_rho[1 * WR + lx + 2] + rho_ref);
                if (o_mu) o_mu[g] = (double)s_mu[0 * WM + lx + 1];
                if (o_vx) o_vx[g] = 0.0;
                if (o_vy) o_vy[g] = 0.0;
            }
            if (Y0 + wy == L.nyf) {
                const long long g = (long long)(L.ny - 1) * L.nx + x;
                if (o_rho) o_rho[g] = (double)(s_rho[(wy + 2) * WR + lx + 2] + rho_ref);
                if (o_mu) o_mu[g] = (double)s_mu[(wy + 1) * WM + lx + 1];
                if (o_vx) o_vx[g] = 0.0;
                if (o_vy) o_vy[g] = 0.0;
            }
        }
    }
    if (red) {
        // warp then block reduction, fixed order within the block
        for (int o = 16; o > 0; o >>= 1) {
            acc_m += __shfl_down_sync(0xffffffffu, acc_m, o);
            acc_x += __shfl_down_sync(0xffffffffu, acc_x, o);
            acc_y += __shfl_down_sync(0xffffffffu, acc_y, o);
            acc_d = fmax(acc_d, __shfl_down_sync(0xffffffffu, acc_d, o));
        }
        const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
        if (nbad) atomicAdd(&s_bad, nbad);
        if (lane == 0) {
            s_red[0][warp] = acc_m; s_red[1][warp] = acc_x;
            s_red[2][warp] = acc_y; s_red[3][warp] = acc_d;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double m = 0, sx = 0, sy = 0, d = 0;
            for (int w = 0; w < (int)(blockDim.x / 32); ++w) {
                m += s_red[0][w]; sx += s_red[1][w]; sy += s_red[2][w];
                d = fmax(d, s_red[3][w]);
            }
            atomicAdd(&red[0], m);
            atomicAdd(&red[1], sx);
            atomicAdd(&red[2], sy);
            atomic_max_nonneg(&red[3], d);
            if (s_bad) atomicAdd(bad, s_bad);
        }
    }
}

// ---------------------------------------------------------------------------
// Natural-order FP64 populations [9][ny][nx] (solid rows untouched).
// ---------------------------------------------------------------------------
template <class S>
__global__ void populations_kernel(const Lattice L, int parity, int cur,
                                   double *f)
{
    using pop_t = typename S::pop_t;
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= (long long)L.nx * L.nyf) return;
    const int x = (int)(n % L.nx), r = (int)(n / L.nx);
    const long long N = (long long)L.nx * L.ny;
    const long long g = (long long)(r + L.walls) * L.nx + x;
    const double ref = S::offset ? L.rho_ref : 0.0;
    const pop_t *A = (const pop_t *)L.pops;
    double sum = 0.0;
    for (int i = 1; i < 9; ++i) {
        const pop_t *p = A + aa_read_index(L, parity, i, r, x);
        const double v = (CPLBM_IN_POPS(L, p, 1) ? (double)ld_real(p) : 0.0) +
                         wgt<double>(i) * ref;
        f[i * N + g] = v;
        sum += v;
    }
    f[g] = (double)load_rho<S>(L, cur, r, x) - sum;
}

// Stored-form density sum of every fluid node into dst (see load_rho).
template <class S>
__global__ void gather_rho_kernel(const Lattice L, int cur, void *dst)
{
    using rho_t = typename S::rho_t;
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= (long long)L.nx * L.nyf) return;
    const int x = (int)(n % L.nx), r = (int)(n / L.nx);
    ((rho_t *)dst)[fidx(L, r, x)] = (rho_t)load_rho_stored<S>(L, cur, r, x);
}

// ---------------------------------------------------------------------------
// Launchers.
// ---------------------------------------------------------------------------
static inline unsigned blocks_for(long long n, int t)
{
    return (unsigned)((n + t - 1) / t);
}

template <class S>
static cudaError_t launch_init_t(const Lattice &L, const double *rho,
                                 const double *ux, const double *uy, int *bad,
                                 cudaStream_t s)
{
    const long long n = (long long)L.nx * L.nyf;
    init_kernel<S><<<blocks_for(n, 256), 256, 0, s>>>(L, rho, ux, uy, bad);
    return cudaGetLastError();
}

template <class S>
static cudaError_t launch_macro_t(const Lattice &L, int parity, int cur,
                                  double *rho, double *vx, double *vy,
                                  double *mu, double *red, double *prev,
                                  int *bad, cudaStream_t s)
{
    using real = typename S::real;
    constexpr int TX = FIELD_TILE_X, TY = FIELD_TILE_Y;
    const size_t smem =
        sizeof(real) * ((TY + 4) * (TX + 4) + (TY + 2) * (TX + 2));
    dim3 grid((L.nx + TX - 1) / TX, (L.nyf + TY - 1) / TY);
    macro_kernel<S, TX, TY><<<grid, 256, smem, s>>>(L, parity, cur, rho, vx,
                                                     vy, mu, red, prev, bad);
    return cudaGetLastError();
}

template <class S>
static cudaError_t launch_pop_t(const Lattice &L, int parity, int cur,
                                double *f, cudaStream_t s)
{
    const long long n = (long long)L.nx * L.nyf;
    populations_kernel<S><<<blocks_for(n, 256), 256, 0, s>>>(L, parity, cur, f);
    return cudaGetLastError();
}

template <class S>
static cudaError_t launch_gather_t(const Lattice &L, int cur, void *dst,
                                   cudaStream_t s)
{
    const long long n = (long long)L.nx * L.nyf;
    gather_rho_kernel<S><<<blocks_for(n, 256), 256, 0, s>>>(L, cur, dst);
    return cudaGetLastError();
}

#define CPLBM_DISPATCH(prec, call)                                   \
    switch (prec) {                                                  \
    case P_F64: { using S = SF64; return call; }                     \
    case P_F32: { using S = SF32; return call; }                     \
    case P_F32_OFF: { using S = SF32Off; return call; }              \
    case P_F16_OFF: { using S = SF16Off; return call; }              \
    }                                                                \
    return cudaErrorInvalidValue;

cudaError_t launch_init(const Lattice &L, const double *rho, const double *ux,
                        const double *uy, int *bad, cudaStream_t s)
{
    CPLBM_DISPATCH(L.precision, launch_init_t<S>(L, rho, ux, uy, bad, s))
}

cudaError_t launch_macro(const Lattice &L, int parity, int cur, double *rho,
                         double *vx, double *vy, double *mu, double *red,
                         double *prev, int *bad, cudaStream_t s)
{
    CPLBM_DISPATCH(L.precision, launch_macro_t<S>(L, parity, cur, rho, vx, vy,
                                                  mu, red, prev, bad, s))
}

cudaError_t launch_populations(const Lattice &L, int parity, int cur,
                               double *f, cudaStream_t s)
{
    CPLBM_DISPATCH(L.precision, launch_pop_t<S>(L, parity, cur, f, s))
}

cudaError_t launch_gather_rho(const Lattice &L, int cur, void *dst,
                              cudaStream_t s)
{
    CPLBM_DISPATCH(L.precision, launch_gather_t<S>(L, cur, dst, s))
}

// The FP64 logarithm and reciprocal of the step kernels on n values
// (lbm_test_fp64_math).
__global__ void fp64_math_kernel(const double *__restrict__ x, int n,
                                 double *__restrict__ lg, double *__restrict__ rc)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        lg[i] = log_tab(x[i]);
        rc[i] = rcp_nr(x[i]);
    }
}

cudaError_t launch_fp64_math(const double *x, int n, double *lg, double *rc,
                             cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    fp64_math_kernel<<<(n + 255) / 256, 256, 0, s>>>(x, n, lg, rc);
    return cudaGetLastError();
}

}  // namespace cplbm
