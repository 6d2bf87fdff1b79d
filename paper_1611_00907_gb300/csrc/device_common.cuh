// Device building blocks of the chemical-potential LBM step (arXiv
// 1611.00907): D2Q9 lattice, storage types, the EOS chemical potentials,
// the AA-pattern addressing and the tile loaders shared by the fused step
// kernel and the field kernels.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "cplbm_internal.h"
#include "log_table.h"

namespace cplbm {

// ---------------------------------------------------------------------------
// D2Q9 lattice (Eq. 13-14).  e_0 = (0,0); e_1..4 = (1,0),(0,1),(-1,0),(0,-1);
// e_5..8 = (1,1),(-1,1),(-1,-1),(1,-1).
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int ex(int i)
{
    return (i == 1 || i == 5 || i == 8) ? 1 : (i == 3 || i == 6 || i == 7) ? -1 : 0;
}
__host__ __device__ constexpr int ey(int i)
{
    return (i == 2 || i == 5 || i == 6) ? 1 : (i == 4 || i == 7 || i == 8) ? -1 : 0;
}
__host__ __device__ constexpr int opp(int i)
{
    return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 3) % 4) + 5);
}
static_assert(opp(1) == 3 && opp(2) == 4 && opp(3) == 1 && opp(4) == 2, "");
static_assert(opp(5) == 7 && opp(6) == 8 && opp(7) == 5 && opp(8) == 6, "");

template <class T>
__host__ __device__ constexpr T wgt(int i)
{
    return i == 0 ? T(4) / T(9) : (i <= 4 ? T(1) / T(9) : T(1) / T(36));
}

// ---------------------------------------------------------------------------
// Storage variants: population storage type, density storage type, the
// arithmetic type, and whether values are stored as offsets from the
// reference state (f_i - w_i rho_ref, rho - rho_ref).
// ---------------------------------------------------------------------------
struct SF64 {
    using pop_t = double; using rho_t = double; using real = double;
    static constexpr bool offset = false;
};
struct SF32 {
    using pop_t = float; using rho_t = float; using real = float;
    static constexpr bool offset = false;
};
struct SF32Off {
    using pop_t = float; using rho_t = float; using real = float;
    static constexpr bool offset = true;
};
struct SF16Off {
    using pop_t = __half; using rho_t = float; using real = float;
    static constexpr bool offset = true;
};

template <class T> __device__ __forceinline__ float to_f(T v) { return (float)v; }
__device__ __forceinline__ double ld_real(const double *p) { return *p; }
__device__ __forceinline__ float ld_real(const float *p) { return *p; }
__device__ __forceinline__ float ld_real(const __half *p) { return __half2float(*p); }
__device__ __forceinline__ void st_real(double *p, double v) { *p = v; }
__device__ __forceinline__ void st_real(float *p, float v) { *p = v; }
__device__ __forceinline__ void st_real(__half *p, float v) { *p = __float2half_rn(v); }

// ---------------------------------------------------------------------------
// Bounds-checked build (CPLBM_CHECK_BOUNDS; a debug build that stands in for
// a memory checker): the global accesses of the step and field kernels are
// checked against the buffer they belong to first; an access outside it
// raises ERR_BOUNDS in L.err and is skipped (a load reads zero, a copy
// leaves its destination as it was).  TMA loads need no check: the tensor
// map bounds them.  In the normal build every check is the constant true,
// its arguments are not evaluated, and the accesses compile as before.
// n: elements accessed from p on.
// ---------------------------------------------------------------------------
#ifdef CPLBM_CHECK_BOUNDS
__device__ __forceinline__ bool in_buffer(const Lattice &L, const void *base, long long bytes,
                                          const void *p, long long size)
{
    const long long off = (const char *)p - (const char *)base;
    if (off >= 0 && off + size <= bytes) return true;
    if (L.err) atomicOr(L.err, ERR_BOUNDS);
    return false;
}
#define CPLBM_IN_POPS(L, p, n) \
    ::cplbm::in_buffer(L, (L).pops, (L).b_pops, p, (long long)(n) * sizeof(*(p)))
#define CPLBM_IN_RHO(L, k, p, n) \
    ::cplbm::in_buffer(L, (L).rho[k], (L).b_rho, p, (long long)(n) * sizeof(*(p)))
#define CPLBM_IN_RING(L, k, c, p, n) \
    ::cplbm::in_buffer(L, (L).ring[k][c], (L).b_ring[c], p, (long long)(n) * sizeof(*(p)))
#else
#define CPLBM_IN_POPS(L, p, n) true
#define CPLBM_IN_RHO(L, k, p, n) true
#define CPLBM_IN_RING(L, k, c, p, n) true
#endif

// ---------------------------------------------------------------------------
// Bulk chemical potential psi'(rho): Eq. 18 (vdW), Eq. 21 (RK/RKS), Eq. 24
// (PR), Eq. 27 (CS) without the -kappa lap(rho) term.
// ---------------------------------------------------------------------------
// FP64 reciprocal: the hardware's approximate reciprocal (PTX
// rcp.approx.ftz.f64) refined by two Newton-Raphson steps r <- r + r (1 -
// x r), each of which doubles the number of correct bits.  Within one ulp of
// 1/x for normal x with a normal reciprocal (measured: the correctly
// rounded value on 800 000 log-uniform samples), not guaranteed correctly
// rounded as IEEE division is, at a fraction of its FP64-pipe instructions
// (the GB300 FP64 pipe bounds the FP64 step).  Zero, infinite and NaN x give
// NaN.
__device__ __forceinline__ double rcp_nr(double x)
{
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    r = fma(r, fma(-x, r, 1.0), r);
    return fma(r, fma(-x, r, 1.0), r);
}

// FP64 natural logarithm after Tang's table-driven method (P. T. P. Tang,
// ACM TOMS 16(4), 1990).  x = 2^m y with y in [1, 2); F = 1 + j/128 the
// breakpoint next to y, f = y - F (exact, |f| <= 2^-8), r = f/F from the
// tabulated 1/F; ln x = m ln 2 + ln F + ln(1 + r), the last by its Taylor
// series through r^7 (the rest is below 2^-59 of r).  ln 2 and ln F are
// tabulated as hi + lo with hi a multiple of 2^-32, so m ln2_hi + lnF_hi is
// exact: just below 1 the two cancel almost entirely, and only the small
// terms carry rounding errors.  For x in [1 - 2^-9, 1) (m = -1, j = 128) the
// series takes r = x - 1 directly.  Within about two ulp for positive
// normal x; zero, negative, subnormal, infinite and NaN x go to log().
__device__ __forceinline__ double log_tab(double x)
{
    const int hi = __double2hiint(x);
    if ((unsigned)(hi - 0x00100000) >= 0x7FE00000u) return log(x);
    int m = (hi >> 20) - 1023;
    const int mant = hi & 0x000FFFFF;        // top 20 bits of the significand
    int j = (mant + (1 << 12)) >> 13;        // nearest multiple of 1/128: 0 .. 128
    double y = __hiloint2double(mant | 0x3FF00000, __double2loint(x));
    if (m == -1 && j == LOG_TABLE_N) {       // x in [1 - 2^-9, 1)
        y = x;
        m = 0;
        j = 0;
    }
    const double F = __hiloint2double(0x3FF00000 + (j << 13), 0);
    const double2 t = __ldg(&kLogTable[j]);  // {1/F, hi of ln F}
    const double r = (y - F) * t.x;
    double q = fma(r, 1.0 / 7.0, -1.0 / 6.0);
    q = fma(q, r, 1.0 / 5.0);
    q = fma(q, r, -1.0 / 4.0);
    q = fma(q, r, 1.0 / 3.0);
    q = fma(q, r, -0.5);
    const double p = fma(r * r, q, r);       // ln(1 + r)
    const double dm = (double)m;
    return fma(dm, LN2_HI, t.y) + (fma(dm, LN2_LO, __ldg(&kLogTableLo[j])) + p);
}

// Division and logarithm of the arithmetic type: the FP32 kernels use the
// fast hardware forms (__fdividef, __logf), whose few-ulp errors sit far
// below the FP32 storage error; FP64 the reciprocal and logarithm above,
// within one or two ulp of IEEE division and log().
__device__ __forceinline__ float fdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double fdiv(double a, double b) { return a * rcp_nr(b); }
__device__ __forceinline__ float flog(float x) { return __logf(x); }
__device__ __forceinline__ double flog(double x) { return log_tab(x); }

template <class T>
__device__ __forceinline__ T mu_bulk(const EosT<T> &e, T rho)
{
    switch (e.kind) {
    case EOS_VDW: {
        const T iq = fdiv(T(1), T(1) - e.b * rho);
        return e.RT * (flog(rho * iq) + iq) - T(2) * e.a * rho;
    }
    case EOS_CS: {
        const T h = e.quarter_b * rho;
        const T iq = fdiv(T(1), T(1) - h);
        return e.RT * ((T(3) - h) * (iq * iq * iq) + flog(rho) + T(1)) -
               T(2) * e.a * rho;
    }
    case EOS_PR: {
        const T br = e.b * rho;
        const T iq = fdiv(T(1), T(1) - br);
        return e.RT * flog(rho * iq) -
               e.pr_c * flog(fdiv(e.pr_s2m1 + br, e.pr_s2p1 - br)) +
               e.RT * iq - fdiv(e.aalpha * rho, T(1) + T(2) * br - br * br);
    }
    default: {  // EOS_RKS
        const T br = e.b * rho;
        const T iq = fdiv(T(1), T(1) - br);
        return e.RT * (flog(rho * iq) + iq) - e.rks_c * flog(T(1) + br) -
               fdiv(e.aalpha * rho, T(1) + br);
    }
    }
}

// Equation of state p0(rho): Eq. 16 (vdW), Eq. 19 (RK/RKS), Eq. 22 (PR),
// Eq. 25 (CS).  Used only by the pressure-tensor force of Eq. 5.
template <class T>
__device__ __forceinline__ T p0_bulk(const EosT<T> &e, T rho)
{
    const T br = e.b * rho;
    switch (e.kind) {
    case EOS_VDW:
        return fdiv(rho * e.RT, T(1) - br) - e.a * rho * rho;
    case EOS_CS: {
        const T h = e.quarter_b * rho, q = T(1) - h;
        return fdiv(rho * e.RT * (T(1) + h + h * h - h * h * h), q * q * q) -
               e.a * rho * rho;
    }
    case EOS_PR:
        return fdiv(rho * e.RT, T(1) - br) -
               fdiv(e.aalpha * rho * rho, T(1) + T(2) * br - br * br);
    default:  // EOS_RKS
        return fdiv(rho * e.RT, T(1) - br) - fdiv(e.aalpha * rho * rho, T(1) + br);
    }
}

// ---------------------------------------------------------------------------
// Asynchronous global -> shared copies of single elements (sm_80+ cp.async).
// A thread's copies become visible to that thread after cp_async_wait_all.
// ---------------------------------------------------------------------------
template <int BYTES>
__device__ __forceinline__ void cp_async(void *smem, const void *gmem)
{
    static_assert(BYTES == 4 || BYTES == 8 || BYTES == 16, "cp.async size");
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s),
                 "l"(gmem), "n"(BYTES)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}
// Wait until at most N of the thread's most recent copy groups are pending.
template <int N>
__device__ __forceinline__ void cp_async_wait_group()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ---------------------------------------------------------------------------
// TMA (cp.async.bulk.tensor) loads completing on a shared-memory mbarrier.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_addr(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)),
                 "r"(count)
                 : "memory");
    // make the initialised barrier visible to the asynchronous proxy
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(
                     smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}
// Wait for phase `parity` of the barrier: poll while fewer than max_cycles
// SM clocks have passed; false when the limit was reached (max_cycles <= 0:
// at once, without polling).
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity,
                                          long long max_cycles)
{
    const unsigned a = smem_addr(bar);
    const long long t0 = clock64();
    while (clock64() - t0 < max_cycles) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n"
            " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map,
                                            int x, int y, unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];\n" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y),
        "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map,
                                            int x, int y, int z,
                                            unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z),
        "r"(smem_addr(bar))
        : "memory");
}

// ---------------------------------------------------------------------------
// Addressing.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int wrapi(int v, int n)
{
    return v < 0 ? v + n : (v >= n ? v - n : v);
}

// Index of population i (1..8) of fluid node (x, r) in the pops array.
__device__ __forceinline__ long long pidx(const Lattice &L, int i, int r, int x)
{
    return (long long)(i - 1) * L.plane + (long long)r * L.pitch + x;
}
__device__ __forceinline__ long long fidx(const Lattice &L, int r, int x)
{
    return (long long)r * L.pitch + x;
}
// Index of the partial sum of class c for the receiving node (r, x), whose
// tile is (bx, by): classes L and R keep one column per tile column, B and
// T one row per tile row, the corners one entry per tile.
__device__ __forceinline__ long long ring_index(const Lattice &L, int c, int bx,
                                                int by, int r, int x)
{
    if (c == R_L || c == R_R) return (long long)bx * L.nyf_pad + r;
    if (c == R_B || c == R_T) return (long long)by * L.pitch + x;
    return (long long)by * ((L.nx + 31) >> 5) + bx;
}

// Row r + dy of a fluid node; with walls, -1 / nyf mean the solid rows.
__device__ __forceinline__ bool row_is_solid(const Lattice &L, int r)
{
    return L.walls && (r < 0 || r >= L.nyf);
}
__device__ __forceinline__ int row_wrap(const Lattice &L, int r)
{
    return L.walls ? r : wrapi(r, L.nyf);
}

// AA pattern (in place).  Even step: node x reads f_i from its own slot i
// and writes f*_i into its own slot opp(i).  Odd step: node x reads f_i from
// slot opp(i) of x - e_i and writes f*_i into slot i of x + e_i.  Every slot
// a node reads is one it writes, so no two nodes touch the same slot in a
// step.  Halfway bounce-back (Sec. IV): on an odd step, a population whose
// source x - e_i is solid is read from slot i of x itself, where the even
// step left f*_opp(i); a population whose target x + e_i is solid is written
// to slot opp(i) of x, where the next even step reads it.
__device__ __forceinline__ long long aa_read_index(const Lattice &L, int parity,
                                                   int i, int r, int x)
{
    if (parity == 0) return pidx(L, i, r, x);
    const int rs = r - ey(i);
    if (row_is_solid(L, rs)) return pidx(L, i, r, x);
    return pidx(L, opp(i), row_wrap(L, rs), wrapi(x - ex(i), L.nx));
}
__device__ __forceinline__ long long aa_write_index(const Lattice &L,
                                                    int parity, int i, int r,
                                                    int x)
{
    if (parity == 0) return pidx(L, opp(i), r, x);
    const int rt = r + ey(i);
    if (row_is_solid(L, rt)) return pidx(L, opp(i), r, x);
    return pidx(L, i, row_wrap(L, rt), wrapi(x + ex(i), L.nx));
}

// ---------------------------------------------------------------------------
// Density of the current step at fluid node (x, r) in stored form (offset
// precisions: rho - rho_ref): the tile-local sum in rho[cur] plus the
// partial sums written by neighbouring tiles for nodes on the edge of their
// tile (see step.cu), always added in this order.
// ---------------------------------------------------------------------------
template <class S>
__device__ __forceinline__ typename S::real load_rho_stored(const Lattice &L,
                                                            int cur, int r,
                                                            int x)
{
    using rt = typename S::rho_t;
    using real = typename S::real;
    const rt *R = (const rt *)L.rho[cur];
    const rt *rp = R + fidx(L, r, x);
    real v = CPLBM_IN_RHO(L, cur, rp, 1) ? (real)*rp : real(0);
    const int bx = x / L.tx, by = r / L.ty;
    const int lx = x - bx * L.tx, ly = r - by * L.ty;
    const int wx = min(L.tx, L.nx - bx * L.tx);
    const int wy = min(L.ty, L.nyf - by * L.ty);
    const bool left = lx == 0, right = lx == wx - 1;
    const bool below = ly == 0 && !(L.walls && r == 0);
    const bool above = ly == wy - 1 && !(L.walls && r == L.nyf - 1);
    if (left | right | below | above) {
        rt *const *ring = (rt *const *)L.ring[cur];
        auto at = [&](int c) {
            const rt *q = ring[c] + ring_index(L, c, bx, by, r, x);
            return CPLBM_IN_RING(L, cur, c, q, 1) ? *q : rt(0);
        };
        if (left) v += (real)at(R_L);
        if (right) v += (real)at(R_R);
        if (below) {
            v += (real)at(R_B);
            if (left) v += (real)at(R_BL);
            if (right) v += (real)at(R_BR);
        }
        if (above) {
            v += (real)at(R_T);
            if (left) v += (real)at(R_TL);
            if (right) v += (real)at(R_TR);
        }
    }
    return v;
}

// Absolute density.
template <class S>
__device__ __forceinline__ typename S::real load_rho(const Lattice &L, int cur,
                                                     int r, int x)
{
    using real = typename S::real;
    const real v = load_rho_stored<S>(L, cur, r, x);
    return S::offset ? v + consts<real>(L).rho_ref : v;
}

// Fill s_rho[(TY + 4) x (TX + 4)] with the stored-form density of the tile
// at (X0, Y0) and a halo of two nodes; solid rows get the Eq. 28 average of
// the adjacent fluid row (the top row mirrors it from row nyf - 1).
template <class S, int TX, int TY>
__device__ void load_rho_tile(const Lattice &L, int cur, int X0, int Y0,
                              typename S::real *s_rho)
{
    using real = typename S::real;
    constexpr int W = TX + 4, H = TY + 4;
    const int wx = min(TX, L.nx - X0), wy = min(TY, L.nyf - Y0);
    for (int k = threadIdx.x; k < W * H; k += blockDim.x) {
        const int lx = k % W, ly = k / W;
        if (lx > wx + 3 || ly > wy + 3) {  // beyond a ragged tile's halo
            s_rho[k] = real(0);
            continue;
        }
        // X0 - 2 <= x < X0 + wx + 2 <= nx + 2: one wrap suffices (nx >= 5)
        const int x = wrapi(X0 + lx - 2, L.nx);
        const int r = Y0 + ly - 2;
        real v;
        if (!L.walls) {
            v = load_rho_stored<S>(L, cur, wrapi(r, L.nyf), x);
        } else if (r >= 0 && r < L.nyf) {
            v = load_rho_stored<S>(L, cur, r, x);
        } else if (r == -1 || r == L.nyf) {
            // Eq. 28: rho(x, wall) = 2/3 rho(x, 1) + 1/6 rho(x-1, 1) + 1/6 rho(x+1, 1)
            // (the weights sum to one, so the stored form averages the same)
            const int rf = r < 0 ? 0 : L.nyf - 1;
            v = real(2.0 / 3.0) * load_rho_stored<S>(L, cur, rf, x) +
                real(1.0 / 6.0) * load_rho_stored<S>(L, cur, rf, wrapi(x - 1, L.nx)) +
                real(1.0 / 6.0) * load_rho_stored<S>(L, cur, rf, wrapi(x + 1, L.nx));
        } else {
            v = real(0);  // beyond a wall: never read
        }
        s_rho[k] = v;
    }
}

// Isotropic D2Q9 Laplacian and gradient on a shared-memory tile of row
// width W at linear index c.
template <class T, int W>
__device__ __forceinline__ T lap9(const T *s, int c)
{
    const T axial = s[c + 1] + s[c - 1] + s[c + W] + s[c - W];
    const T diag = (s[c + W + 1] + s[c + W - 1]) + (s[c - W + 1] + s[c - W - 1]);
    return (T(4) * axial + diag - T(20) * s[c]) * T(1.0 / 6.0);
}
template <class T, int W>
__device__ __forceinline__ void grad9(const T *s, int c, T &gx, T &gy)
{
    // 3 sum_i w_i phi(x + e_i) e_i = [4 (E - W) + (NE - NW + SE - SW)] / 12
    const T ne = s[c + W + 1], nw = s[c + W - 1];
    const T se = s[c - W + 1], sw = s[c - W - 1];
    gx = (T(4) * (s[c + 1] - s[c - 1]) + (ne - nw) + (se - sw)) * T(1.0 / 12.0);
    gy = (T(4) * (s[c + W] - s[c - W]) + (ne + nw) - (se + sw)) * T(1.0 / 12.0);
}

// Fill s_mu[(TY + 2) x (TX + 2)] with mu on the tile and a one-node halo
// (Eq. 8) from the stored-form densities in s_rho; solid rows carry the
// surface values (Sec. IV, V).
template <class S, int TX, int TY>
__device__ void mu_tile(const Lattice &L, int X0, int Y0,
                        const typename S::real *s_rho, typename S::real *s_mu)
{
    using real = typename S::real;
    constexpr int W = TX + 2, H = TY + 2, WR = TX + 4;
    const Consts<real> &K = consts<real>(L);
    const EosT<real> &eos = K.eos;
    const real kappa = K.kappa;
    const real ref = S::offset ? K.rho_ref : real(0);
    const int wx = min(TX, L.nx - X0), wy = min(TY, L.nyf - Y0);
    for (int k = threadIdx.x; k < W * H; k += blockDim.x) {
        const int lx = k % W, ly = k / W;
        if (lx > wx + 1 || ly > wy + 1) {  // beyond a ragged tile's halo
            s_mu[k] = real(0);
            continue;
        }
        const int r = Y0 + ly - 1;
        const int c = (ly + 1) * WR + lx + 1;  // same node in s_rho
        real m;
        if (L.walls && r == -1) {
            m = K.mu_bottom;
        } else if (L.walls && r == L.nyf) {
            if (L.top_mode == 0) {
                const int cb = c - WR;  // fluid neighbour below (row nyf-1)
                m = mu_bulk(eos, s_rho[cb] + ref) - kappa * lap9<real, WR>(s_rho, cb);
            } else {
                m = K.mu_top;
            }
        } else if (L.walls && (r < -1 || r > L.nyf)) {
            m = real(0);
        } else {
            m = mu_bulk(eos, s_rho[c] + ref) - kappa * lap9<real, WR>(s_rho, c);
        }
        s_mu[k] = m;
    }
}

}  // namespace cplbm
