// Fused time step of the chemical-potential lattice Boltzmann method (arXiv
// 1611.00907): one kernel launch per step does density, Eq. 28 wall density,
// chemical potential (Eq. 8), nonideal force (Eq. 12), BGK collision with
// the velocity-shift forcing (Eq. 13-14, Sec. II) and streaming with halfway
// bounce-back (Sec. IV), in place (AA pattern).
//
// State.  The eight moving populations live in one array, updated in place
// in the AA order (device_common.cuh).  The rest population f_0 is not
// stored: the density field replaces it (f_0 = rho - sum_{i>0} f_i), so
// each node moves 8 populations plus one density in and out per step, the
// same 9 + 9 values as a plain in-place D2Q9 step.
//
// Density hand-over.  Every CTA owns a TX x TY tile.  After the collision it
// has all post-collision populations of its tile in shared memory and sums,
// for every node of the tile and of the one-node ring around it, the
// populations that stream there from inside the tile (bounce-back returns
// included).  A tile node's sum goes to rho[next]; the ring sums go to the
// partial-sum buffers ring[next][class], class = direction from the ring
// node's own tile to this one.  Each entry has exactly one writer, so the
// hand-over needs no atomics and no clearing, and the next step adds the
// parts in a fixed order (load_rho_stored): results do not depend on
// scheduling.
//
// Memory pipeline.  Every global load a CTA needs is issued at its start as
// an asynchronous copy into shared memory (cp.async): the density halo and
// the partial sums first, then the eight populations of each node, which
// land in the planes of the post-collision buffer the node later overwrites.
// The chemical potential is computed while the populations are in flight.
//
// Two code paths share this structure.  Tiles whose halo and ring touch no
// domain edge and whose neighbours' edges sit where full tiles' would
// (tile_kind; nearly all of a large lattice) take the interior path:
// constant address offsets, no periodic wrap, no wall tests, asynchronous
// density loads.  All other tiles take the general path.  Both add the same
// terms in the same order, so a node's values do not depend on which path
// a tile took.  The TMA paths further below take the interior tiles and,
// in a variant, the tiles whose halo wraps around a periodic edge; they
// sum the density hand-over in registers, in another order.
#pragma once
#include "device_common.cuh"

namespace cplbm {

// Shared-memory carve-up of one CTA.
template <class real, int TX, int TY>
struct StepSmem {
    static constexpr int WR = TX + 4, HR = TY + 4;   // rho + 2-node halo
    static constexpr int WM = TX + 2, HM = TY + 2;   // mu + 1-node halo
    static constexpr int NPOST = 8 * TX * TY;        // f*_1..8 of the tile
    static constexpr int NRING = 4 * HR + 4 * WR + 16;  // staged partial sums
    static constexpr size_t bytes =
        sizeof(real) * (WR * HR + WM * HM + NPOST + NRING);
};

// In an interior tile's density halo the tile grid's edges sit at fixed
// columns (1, 2, TX + 1, TX + 2) and rows (1, 2, TY + 1, TY + 2).  Columns 2
// and TX + 2 are left edges of their tile (class L), 1 and TX + 1 right
// edges (R); rows 2 and TY + 2 are bottom edges (B), 1 and TY + 1 top edges.
template <int T>
__device__ __forceinline__ int edge_col(int ci)
{
    return ci == 0 ? 1 : ci == 1 ? 2 : ci == 2 ? T + 1 : T + 2;
}
// The same for an edge tile of width (height) w: a ragged last tile has
// its far edge at column (row) w + 1 and the next tile's near edge at w + 2.
__device__ __forceinline__ int edge_col(int ci, int w)
{
    return ci == 0 ? 1 : ci == 1 ? 2 : ci == 2 ? w + 1 : w + 2;
}
__device__ __forceinline__ int col_index(int l, int w)
{
    return l == 1 ? 0 : l == 2 ? 1 : l == w + 1 ? 2 : l == w + 2 ? 3 : -1;
}
__device__ __forceinline__ bool col_is_left(int ci) { return ci & 1; }
__device__ __forceinline__ bool row_is_below(int ri) { return ri & 1; }
template <int T>
__device__ __forceinline__ int col_index(int l)
{
    return l == 1 ? 0 : l == 2 ? 1 : l == T + 1 ? 2 : l == T + 2 ? 3 : -1;
}
// Tile of halo edge index ci (as edge_col) relative to this tile.
__device__ __forceinline__ int edge_tile(int ci) { return ci == 0 ? -1 : ci == 3 ? 1 : 0; }

// Issue the asynchronous loads of an interior tile's stored density and of
// the partial sums its halo needs.
template <class S, int TX, int TY, int NT>
__device__ __forceinline__ void issue_rho_interior(const Lattice &L, int cur,
                                                   int X0, int Y0,
                                                   typename S::real *s_rho,
                                                   typename S::real *s_ring)
{
    using real = typename S::real;
    using rt = typename S::rho_t;
    static_assert(sizeof(rt) == sizeof(real), "density staged as stored");
    using SM = StepSmem<real, TX, TY>;
    constexpr int WR = SM::WR, HR = SM::HR;
    const rt *R = (const rt *)L.rho[cur];
    rt *const *ring = (rt *const *)L.ring[cur];
    for (int k = threadIdx.x; k < WR * HR; k += NT) {
        const int lx = k % WR, ly = k / WR;
        const long long fi = (long long)(Y0 + ly - 2) * L.pitch + X0 + lx - 2;
        if (CPLBM_IN_RHO(L, cur, R + fi, 1)) cp_async<sizeof(rt)>(&s_rho[k], R + fi);
    }
    for (int p = threadIdx.x; p < SM::NRING; p += NT) {
        int c, lx, ly, dbx = 0, dby = 0;  // receiving tile - this tile
        if (p < 4 * HR) {  // edge columns: class L or R, column-major storage
            const int ci = p / HR;
            dbx = edge_tile(ci);
            ly = p % HR;
            lx = edge_col<TX>(ci);
            c = col_is_left(ci) ? R_L : R_R;
        } else if (p < 4 * HR + 4 * WR) {  // edge rows: class B or T
            const int q = p - 4 * HR, ri = q / WR;
            dby = edge_tile(ri);
            lx = q % WR;
            ly = edge_col<TY>(ri);
            c = row_is_below(ri) ? R_B : R_T;
        } else {  // the 16 crossings: corner classes
            const int q = p - 4 * HR - 4 * WR, ci = q / 4, ri = q % 4;
            dbx = edge_tile(ci);
            dby = edge_tile(ri);
            lx = edge_col<TX>(ci);
            ly = edge_col<TY>(ri);
            c = row_is_below(ri) ? (col_is_left(ci) ? R_BL : R_BR)
                                 : (col_is_left(ci) ? R_TL : R_TR);
        }
        const int x = X0 + lx - 2, r = Y0 + ly - 2;
        const long long idx = ring_index(L, c, X0 / TX + dbx, Y0 / TY + dby, r, x);
        if (CPLBM_IN_RING(L, cur, c, ring[c] + idx, 1))
            cp_async<sizeof(rt)>(&s_ring[p], ring[c] + idx);
    }
}

// Add the staged partial sums to the halo's edge nodes, in the order of
// load_rho_stored.
template <class S, int TX, int TY, int NT>
__device__ __forceinline__ void combine_rho_interior(typename S::real *s_rho,
                                                     const typename S::real *s_ring)
{
    using real = typename S::real;
    using SM = StepSmem<real, TX, TY>;
    constexpr int WR = SM::WR, HR = SM::HR;
    for (int q = threadIdx.x; q < 4 * HR + 4 * WR; q += NT) {
        int lx, ly;
        if (q < 4 * HR) {
            lx = edge_col<TX>(q / HR);
            ly = q % HR;
        } else {
            const int t = q - 4 * HR;
            lx = t % WR;
            ly = edge_col<TY>(t / WR);
            if (col_index<TX>(lx) >= 0) continue;  // done by its column entry
        }
        const int ci = col_index<TX>(lx), ri = col_index<TY>(ly);
        const bool lr = ci >= 0, ba = ri >= 0;
        real v = s_rho[ly * WR + lx];
        if (lr) v += s_ring[ci * HR + ly];
        if (ba) {
            v += s_ring[4 * HR + ri * WR + lx];
            if (lr) v += s_ring[4 * HR + 4 * WR + ci * 4 + ri];
        }
        s_rho[ly * WR + lx] = v;
    }
}

template <class S, int TX, int TY, int NT>
__device__ __forceinline__ void mu_interior(const Lattice &L,
                                            const typename S::real *s_rho,
                                            typename S::real *s_mu)
{
    using real = typename S::real;
    constexpr int W = TX + 2, H = TY + 2, WR = TX + 4;
    const Consts<real> &K = consts<real>(L);
    const EosT<real> &eos = K.eos;
    const real kappa = K.kappa;
    const real ref = S::offset ? K.rho_ref : real(0);
    for (int k = threadIdx.x; k < W * H; k += NT) {
        const int lx = k % W, ly = k / W;
        const int c = (ly + 1) * WR + lx + 1;
        s_mu[k] = mu_bulk(eos, s_rho[c] + ref) - kappa * lap9<real, WR>(s_rho, c);
    }
}

// BGK collision of one node with the velocity-shift forcing.  f[1..8] are
// the node's stored populations (f_0 = drho - sum f_i is implicit), drho
// its stored density (rho - rho_ref) and rho the absolute one; fp[0..8]
// receive the post-collision values in stored form.
template <class real>
__device__ __forceinline__ void collide(const real *f, real drho, real rho,
                                        real Fx, real Fy, real tau, real omega,
                                        real *fp)
{
    // u = sum f_i e_i / rho; u_eq = u + tau F / rho (Sec. II)
    const real jx = (f[1] - f[3]) + (f[5] - f[7]) + (f[8] - f[6]);
    const real jy = (f[2] - f[4]) + (f[5] - f[7]) + (f[6] - f[8]);
    const real inv_rho = fdiv(real(1), rho);
    const real ux = (jx + tau * Fx) * inv_rho;
    const real uy = (jy + tau * Fy) * inv_rho;
    const real usq = real(1.5) * (ux * ux + uy * uy);
    // Eq. 14 in stored form: f_eq - w_i rho_ref = w_i (drho + rho P_i(u)),
    // P_i = 3 e.u + 4.5 (e.u)^2 - 1.5 u^2; opposite directions share the
    // even part of P.
    const real w1 = real(1.0 / 9.0), w5 = real(1.0 / 36.0);
    {
        const real ex2 = real(4.5) * ux * ux - usq, ey2 = real(4.5) * uy * uy - usq;
        const real ax = w1 * (drho + rho * ex2), bx = w1 * rho * real(3) * ux;
        const real ay = w1 * (drho + rho * ey2), by = w1 * rho * real(3) * uy;
        fp[1] = f[1] + omega * ((ax + bx) - f[1]);
        fp[3] = f[3] + omega * ((ax - bx) - f[3]);
        fp[2] = f[2] + omega * ((ay + by) - f[2]);
        fp[4] = f[4] + omega * ((ay - by) - f[4]);
    }
    {
        const real sp = ux + uy, sm = ux - uy;
        const real ep = real(4.5) * sp * sp - usq, em = real(4.5) * sm * sm - usq;
        const real a5 = w5 * (drho + rho * ep), b5 = w5 * rho * real(3) * sp;
        const real a8 = w5 * (drho + rho * em), b8 = w5 * rho * real(3) * sm;
        fp[5] = f[5] + omega * ((a5 + b5) - f[5]);
        fp[7] = f[7] + omega * ((a5 - b5) - f[7]);
        fp[8] = f[8] + omega * ((a8 + b8) - f[8]);
        fp[6] = f[6] + omega * ((a8 - b8) - f[6]);
    }
    // The rest population takes what the moving ones leave of the density:
    // in exact arithmetic this equals f_0 + omega (f_0^eq - f_0) with
    // f_0 = drho - sum_{i>0} f_i, and it keeps the collision's mass exact
    // instead of biased by the rounding of f_eq.
    fp[0] = drho - (((fp[1] + fp[2]) + (fp[3] + fp[4])) +
                    ((fp[5] + fp[6]) + (fp[7] + fp[8])));
}

// Index of f*_i (i = 1..8) of tile node (lx, ly) in s_post.
template <int TX, int TY>
__device__ __forceinline__ int post_idx(int i, int ly, int lx)
{
    return ((i - 1) * TY + ly) * TX + lx;
}

// Partial density at position (ox, oy) of the tile or its ring from the
// tile's post-collision populations, with the general checks.  self0 is
// f*_0 of the node when the position is inside the tile.
template <class real, int TX, int TY>
__device__ __forceinline__ real handover_sum(const Lattice &L, const real *s_post,
                                             int ox, int oy, int wx, int wy,
                                             int r, bool inside, real self0)
{
    real s = inside ? self0 : real(0);
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const int sx = ox - ex(i), sy = oy - ey(i);
        if (inside && L.walls && row_is_solid(L, r - ey(i))) {
            // bounce-back: f*_opp(i) of this node comes back as f_i
            s += s_post[post_idx<TX, TY>(opp(i), oy, ox)];
        } else if (sx >= 0 && sx < wx && sy >= 0 && sy < wy) {
            s += s_post[post_idx<TX, TY>(i, sy, sx)];
        }
    }
    return s;
}

__device__ __forceinline__ int ring_class(int ox, int oy, int wx, int wy)
{
    if (ox < 0) return oy < 0 ? R_TR : (oy >= wy ? R_BR : R_R);
    if (ox >= wx) return oy < 0 ? R_TL : (oy >= wy ? R_BL : R_L);
    return oy < 0 ? R_T : R_B;
}

// Ring position p (0 .. 2 (wx + wy) + 3) of a wx x wy tile, walking the
// bottom row, the top row, then the left and right columns.
__device__ __forceinline__ void ring_position(int p, int wx, int wy, int &ox,
                                              int &oy)
{
    if (p < wx + 2) { ox = p - 1; oy = -1; return; }
    p -= wx + 2;
    if (p < wx + 2) { ox = p - 1; oy = wy; return; }
    p -= wx + 2;
    if (p < wy) { ox = -1; oy = p; return; }
    ox = wx; oy = p - wy;
}

// Pressure-tensor fields of Eq. 9 on the tile and a one-node halo, in
// three planes of s_p (xx, xy, yy), from the stored-form densities.  Only
// the baseline force model uses them (periodic lattices).
template <class S, int TX, int TY>
__device__ void pt_tile(const Lattice &L, int X0, int Y0,
                        const typename S::real *s_rho, typename S::real *s_p)
{
    using real = typename S::real;
    constexpr int W = TX + 2, H = TY + 2, WR = TX + 4, N = W * H;
    const Consts<real> &K = consts<real>(L);
    const EosT<real> &eos = K.eos;
    const real kappa = K.kappa;
    const real ref = S::offset ? K.rho_ref : real(0);
    const int wx = min(TX, L.nx - X0), wy = min(TY, L.nyf - Y0);
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const int lx = k % W, ly = k / W;
        if (lx > wx + 1 || ly > wy + 1) {
            s_p[k] = s_p[N + k] = s_p[2 * N + k] = real(0);
            continue;
        }
        const int c = (ly + 1) * WR + lx + 1;
        const real rho = s_rho[c] + ref;
        real gx, gy;
        grad9<real, WR>(s_rho, c, gx, gy);
        const real lap = lap9<real, WR>(s_rho, c);
        const real iso = p0_bulk(eos, rho) - kappa * rho * lap -
                         real(0.5) * kappa * (gx * gx + gy * gy);
        s_p[k] = iso + kappa * gx * gx;
        s_p[N + k] = kappa * gx * gy;
        s_p[2 * N + k] = iso + kappa * gy * gy;
    }
}

template <class S, int TX, int TY, int NT, int PARITY, bool INTERIOR,
          bool PT = false>
__device__ __forceinline__ void step_tile(const Lattice &L, int cur, int X0,
                                          int Y0, unsigned char *smem_raw)
{
    using real = typename S::real;
    using pop_t = typename S::pop_t;
    using rho_t = typename S::rho_t;
    using SM = StepSmem<real, TX, TY>;
    constexpr int WR = SM::WR, WM = SM::WM;
    constexpr int PER = TX * TY / NT;
    constexpr int DY = NT / TX;  // rows between a thread's nodes
    static_assert((TX * TY) % NT == 0 && NT % TX == 0, "thread mapping");
    real *s_rho = reinterpret_cast<real *>(smem_raw);
    real *s_mu = s_rho + SM::WR * SM::HR;  // mu, or three P planes (PT)
    real *s_post = s_mu + (PT ? 3 : 1) * SM::WM * SM::HM;  // [8][TY][TX]
    real *s_ring = s_post + SM::NPOST;

    const int wx = INTERIOR ? TX : min(TX, L.nx - X0);
    const int wy = INTERIOR ? TY : min(TY, L.nyf - Y0);
    const int nxt = cur ^ 1;
    pop_t *A = (pop_t *)L.pops;
    const int lx = threadIdx.x % TX, ly0 = threadIdx.x / TX;
    // Storage and arithmetic of the same width: populations are staged
    // asynchronously (FP16 storage is loaded directly instead).
    constexpr bool ASYNC = sizeof(pop_t) == sizeof(real);

    // per-direction offsets of the in-place pattern (interior tiles)
    long long roff[9], woff[9];
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        if (PARITY == 0) {
            roff[i] = (long long)(i - 1) * L.plane;
            woff[i] = (long long)(opp(i) - 1) * L.plane;
        } else {
            roff[i] = (long long)(opp(i) - 1) * L.plane -
                      (long long)ey(i) * L.pitch - ex(i);
            woff[i] = (long long)(i - 1) * L.plane +
                      (long long)ey(i) * L.pitch + ex(i);
        }
    }

    // 1. Issue the loads: density (interior tiles), then the populations.
    if (INTERIOR) {
        issue_rho_interior<S, TX, TY, NT>(L, cur, X0, Y0, s_rho, s_ring);
        cp_async_commit();
    }
    if constexpr (ASYNC) {
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int ly = ly0 + k * DY;
            if (!INTERIOR && (lx >= wx || ly >= wy)) continue;
            const int x = X0 + lx, r = Y0 + ly;
            const long long base = (long long)r * L.pitch + x;
#pragma unroll
            for (int i = 1; i < 9; ++i) {
                const pop_t *src = INTERIOR
                    ? A + base + roff[i]
                    : A + aa_read_index(L, PARITY, i, r, x);
                if (CPLBM_IN_POPS(L, src, 1))
                    cp_async<sizeof(pop_t)>(&s_post[post_idx<TX, TY>(i, ly, lx)], src);
            }
        }
        cp_async_commit();
    }

    // 2. Density with halo, then mu on the tile and a one-node halo.
    if (INTERIOR) {
        if constexpr (ASYNC) cp_async_wait_group<1>();  // density group only
        else cp_async_wait_all();
        __syncthreads();
        combine_rho_interior<S, TX, TY, NT>(s_rho, s_ring);
        __syncthreads();
        if constexpr (PT) pt_tile<S, TX, TY>(L, X0, Y0, s_rho, s_mu);
        else mu_interior<S, TX, TY, NT>(L, s_rho, s_mu);
    } else {
        load_rho_tile<S, TX, TY>(L, cur, X0, Y0, s_rho);
        __syncthreads();
        if constexpr (PT) pt_tile<S, TX, TY>(L, X0, Y0, s_rho, s_mu);
        else mu_tile<S, TX, TY>(L, X0, Y0, s_rho, s_mu);
    }
    __syncthreads();

    // 3. Force, collision, in-place streaming.
    const real tau = consts<real>(L).tau;
    const real omega = consts<real>(L).omega;
    const real rho_ref = S::offset ? consts<real>(L).rho_ref : real(0);
    if constexpr (ASYNC) cp_async_wait_all();
    real self0[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        self0[k] = real(0);
        const int ly = ly0 + k * DY;
        if (!INTERIOR && (lx >= wx || ly >= wy)) continue;
        const int x = X0 + lx, r = Y0 + ly;
        const long long base = (long long)r * L.pitch + x;
        real f[9];
        if constexpr (ASYNC) {
#pragma unroll
            for (int i = 1; i < 9; ++i) f[i] = s_post[post_idx<TX, TY>(i, ly, lx)];
        } else {
#pragma unroll
            for (int i = 1; i < 9; ++i) {
                const pop_t *src = INTERIOR ? A + base + roff[i]
                                            : A + aa_read_index(L, PARITY, i, r, x);
                f[i] = CPLBM_IN_POPS(L, src, 1) ? ld_real(src) : real(0);
            }
        }
        const int cr = (ly + 2) * WR + lx + 2, cm = (ly + 1) * WM + lx + 1;
        const real drho = s_rho[cr];
        const real rho = drho + rho_ref;
        real Fx, Fy, grx, gry;
        grad9<real, WR>(s_rho, cr, grx, gry);
        if constexpr (PT) {
            // Eq. 5: F = -div(P) + grad(cs^2 rho)
            constexpr int N = SM::WM * SM::HM;
            real pxx_x, pxx_y, pxy_x, pxy_y, pyy_x, pyy_y;
            grad9<real, WM>(s_mu, cm, pxx_x, pxx_y);
            grad9<real, WM>(s_mu + N, cm, pxy_x, pxy_y);
            grad9<real, WM>(s_mu + 2 * N, cm, pyy_x, pyy_y);
            Fx = grx * real(1.0 / 3.0) - (pxx_x + pxy_y);
            Fy = gry * real(1.0 / 3.0) - (pxy_x + pyy_y);
        } else {
            // Eq. 12: F = -rho grad(mu) + grad(cs^2 rho)
            real gmx, gmy;
            grad9<real, WM>(s_mu, cm, gmx, gmy);
            Fx = grx * real(1.0 / 3.0) - rho * gmx;
            Fy = gry * real(1.0 / 3.0) - rho * gmy;
        }
        real fp[9];
        collide<real>(f, drho, rho, Fx, Fy, tau, omega, fp);
        self0[k] = fp[0];
#pragma unroll
        for (int i = 1; i < 9; ++i) s_post[post_idx<TX, TY>(i, ly, lx)] = fp[i];
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            pop_t *dst = INTERIOR ? A + base + woff[i]
                                  : A + aa_write_index(L, PARITY, i, r, x);
            if (CPLBM_IN_POPS(L, dst, 1)) st_real(dst, fp[i]);
        }
    }
    __syncthreads();

    // 4. Density hand-over, tile nodes: the thread's own nodes.
    rho_t *Rn = (rho_t *)L.rho[nxt];
    rho_t *const *ring = (rho_t *const *)L.ring[nxt];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int ly = ly0 + k * DY;
        if (!INTERIOR && (lx >= wx || ly >= wy)) continue;
        const int r = Y0 + ly;
        real s;
        const bool deep = lx >= 1 && lx <= wx - 2 && ly >= 1 && ly <= wy - 2 &&
                          (INTERIOR || !L.walls || (r >= 1 && r <= L.nyf - 2));
        if (deep) {  // all nine sources inside the tile
            s = self0[k];
#pragma unroll
            for (int i = 1; i < 9; ++i)
                s += s_post[post_idx<TX, TY>(i, ly - ey(i), lx - ex(i))];
        } else {
            s = handover_sum<real, TX, TY>(L, s_post, lx, ly, wx, wy, r, true,
                                           self0[k]);
        }
        rho_t *q = Rn + (long long)r * L.pitch + X0 + lx;
        if (CPLBM_IN_RHO(L, nxt, q, 1)) *q = (rho_t)s;
    }
    // Ring around the tile: partial sums for the neighbouring tiles.
    const int nring = 2 * (wx + wy) + 4;
    for (int p = threadIdx.x; p < nring; p += NT) {
        int ox, oy;
        ring_position(p, wx, wy, ox, oy);
        const int r = Y0 + oy;
        if (!INTERIOR && L.walls && (r < 0 || r >= L.nyf)) continue;
        const real s = handover_sum<real, TX, TY>(L, s_post, ox, oy, wx, wy, r,
                                                  false, real(0));
        const int x = INTERIOR ? X0 + ox : wrapi(X0 + ox, L.nx);
        const int rw = INTERIOR ? r : row_wrap(L, r);
        const int c = ring_class(ox, oy, wx, wy);
        rho_t *q = ring[c] + ring_index(L, c, x / TX, rw / TY, rw, x);
        if (CPLBM_IN_RING(L, nxt, c, q, 1)) *q = (rho_t)s;
    }
}

// ---------------------------------------------------------------------------
// Interior tiles with TMA.  One thread issues nine tensor copies per tile:
// the density halo (a (TX + 8) x (TY + 4) box from x = X0 - 4, the nearest
// 16-byte-aligned column; staged rows of pitch RP = TX + 8, the tile's
// column 0 at offset 4) and, per direction, the (TX + 4) x TY box of the
// plane and rows that direction is read from in this step's AA order
// (pin_x0 / pin_col below).  They complete on one mbarrier; the partial sums
// of the halo's edge nodes come by per-element cp.async into a buffer that
// the warps' exchange slots reuse once the sums are added.
//
// Lanes map to x (TX = 32) and each warp owns PER consecutive rows, walked
// bottom to top.  Stencil windows roll with the rows, and the density
// hand-over is done in registers: a node's next density is
//   same(k) + up(k - 1) + down(k + 1),
// same = f*_0 + f*_1 from the left lane + f*_3 from the right lane,
// up   = f*_2 + f*_5 from the left + f*_6 from the right (to the row above),
// down = f*_4 + f*_8 from the left + f*_7 from the right (to the row below),
// with lane neighbours by warp shuffles.  Only each warp's first "down" and
// last "up" cross to the neighbouring warp, through shared memory.  Lane 0
// and lane 31 carry the same sums for the tile's left and right ring
// columns; the first and last warps write the bottom and top ring rows.
// ---------------------------------------------------------------------------
// Population staging of the TMA paths: per direction a (TX + PX) x TY box,
// PX = 16 bytes in elements (the step of a TMA x coordinate), from
// x = X0 + pin_x0(i): X0 - PX for the directions an odd step reads from
// x - 1, X0 otherwise.  Tile column lx of direction i then sits at staged
// column lx + pin_col(i).
template <int PARITY, int PX>
__device__ __forceinline__ constexpr int pin_x0(int i)
{
    return (PARITY == 1 && ex(i) == 1) ? -PX : 0;
}
template <int PARITY, int PX>
__device__ __forceinline__ constexpr int pin_col(int i)
{
    return PARITY == 0 ? 0 : (ex(i) == 1 ? PX - 1 : (ex(i) == -1 ? 1 : 0));
}

// All threads: wait (bounded) for phase `phase` of barrier k of the tile's
// copies (0: the density halo and partial sums, 1: the populations), then a
// block barrier.  false when any thread gave up: the flag is raised, every
// copy of the tile is given another bounded wait so none is left writing
// into this block's shared memory, and the caller leaves the tile untouched.
// `limit` bounds the first wait (Lattice::wait_cycles); the drain waits keep
// the long default so that no copy lands after the block has moved on.
__device__ __forceinline__ bool tma_landed(unsigned long long *bar, int k,
                                           unsigned phase, int *err, long long limit)
{
    const bool ok = mbar_wait(&bar[k], phase, limit);
    if (!__syncthreads_or(!ok)) return true;
    if (threadIdx.x == 0 && err) atomicOr(err, ERR_WAIT_TIMEOUT);
    mbar_wait(&bar[0], phase, WAIT_CYCLES_DEFAULT);
    mbar_wait(&bar[1], phase, WAIT_CYCLES_DEFAULT);
    __syncthreads();
    return false;
}

// Partial sums of an interior tile's halo edges, staged for the TMA paths.
// In the compact ring layout each of the four halo edge columns is one
// contiguous run of a class's column (rows Y0 - 4 .. Y0 + TY + 3) and each
// of the four edge rows one run of a class's row (columns X0 - 4 ..
// X0 + TX + 3), both 16-byte aligned, so thread 0 copies them whole with
// cp.async.bulk on the density's mbarrier; the 16 corner entries come by
// per-element cp.async.  Staged: [4][CL] columns (halo row ly at ly + 2),
// [4][RL] rows (halo column lx at lx + 2), [16] corners (ci * 4 + ri).
template <class rt, int TX, int TY>
struct RingStage {
    static constexpr int CL = TY + 8, RL = TX + 8;
    static constexpr int NCOL = 4 * CL, NROW = 4 * RL, N = NCOL + NROW + 16;
    static constexpr unsigned bulk_bytes = sizeof(rt) * (NCOL + NROW);
    static_assert((CL * sizeof(rt)) % 16 == 0 && (RL * sizeof(rt)) % 16 == 0,
                  "bulk copies are whole 16-byte units");
};

// Stores of the density hand-over into generation `gen` (element type T,
// value type V: one element or a packed pair), checked in the
// bounds-checked build.
template <class T, class V>
__device__ __forceinline__ void put_rho(const Lattice &L, int gen, T *R, long long idx, V v)
{
    T *q = R + idx;
    if (CPLBM_IN_RHO(L, gen, q, sizeof(V) / sizeof(T))) *reinterpret_cast<V *>(q) = v;
}
template <class T, class V>
__device__ __forceinline__ void put_ring(const Lattice &L, int gen, T *const *ring, int c,
                                         long long idx, V v)
{
    T *q = ring[c] + idx;
    if (CPLBM_IN_RING(L, gen, c, q, sizeof(V) / sizeof(T))) *reinterpret_cast<V *>(q) = v;
}

__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes,
                                          unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1], %2, [%3];\n" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<unsigned long long>(src)), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Thread 0 issues the eight bulk copies (the caller has added
// RingStage::bulk_bytes to bar's expected transactions); threads 0..15 the
// corner entries, committed as one cp.async group.
template <class rt, int TX, int TY>
__device__ __forceinline__ void stage_ring(const Lattice &L, int cur, int X0, int Y0,
                                           rt *s_ring, unsigned long long *bar)
{
    using RS = RingStage<rt, TX, TY>;
    rt *const *ring = (rt *const *)L.ring[cur];
    const int bx = X0 / TX, by = Y0 / TY;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int ci = 0; ci < 4; ++ci) {
            const int c = col_is_left(ci) ? R_L : R_R;
            const rt *src = ring[c] + ring_index(L, c, bx + edge_tile(ci), by, Y0 - 4, X0);
            // a skipped copy leaves its bytes owed to bar: the bounded wait
            // then gives up and reports it too
            if (CPLBM_IN_RING(L, cur, c, src, RS::CL))
                bulk_load(s_ring + ci * RS::CL, src, RS::CL * sizeof(rt), bar);
        }
#pragma unroll
        for (int ri = 0; ri < 4; ++ri) {
            const int c = row_is_below(ri) ? R_B : R_T;
            const rt *src = ring[c] + ring_index(L, c, bx, by + edge_tile(ri), Y0, X0 - 4);
            if (CPLBM_IN_RING(L, cur, c, src, RS::RL))
                bulk_load(s_ring + RS::NCOL + ri * RS::RL, src, RS::RL * sizeof(rt), bar);
        }
    }
    if (threadIdx.x < 16) {
        const int ci = threadIdx.x / 4, ri = threadIdx.x % 4;
        const int c = row_is_below(ri) ? (col_is_left(ci) ? R_BL : R_BR)
                                       : (col_is_left(ci) ? R_TL : R_TR);
        const rt *src = ring[c] + ring_index(L, c, bx + edge_tile(ci), by + edge_tile(ri), 0, 0);
        if (CPLBM_IN_RING(L, cur, c, src, 1))
            cp_async<sizeof(rt)>(s_ring + RS::NCOL + RS::NROW + threadIdx.x, src);
    }
    cp_async_commit();
}

// Tile of the neighbour d (-1, 0, 1) of the tile starting at coordinate c0
// (size T) along a lattice direction of n nodes: the tile of node c0 - 1,
// c0 or c0 + T, wrapped around the periodic edge on seam tiles.  Taken from
// the node, so a ragged last tile counts as the tile it is.
__device__ __forceinline__ int neighbour_tile(int c0, int d, int T, int n, bool seam)
{
    const int c = d < 0 ? c0 - 1 : (d > 0 ? c0 + T : c0);
    return (seam ? wrapi(c, n) : c) / T;
}

// Edge tiles (tile_kind TILE_SEAM): the halo wraps around a periodic edge
// or meets a wall, so the partial sums are staged element by element, in
// the layout of stage_ring (column entry j <-> row Y0 - 4 + j, row entry j
// <-> column X0 - 4 + j), by cp.async in one group.  Across a periodic edge
// the coordinates wrap: at least three full tiles span each wrapped
// direction and its last tile is full or at least 4 nodes wide (seam_bits),
// so the neighbour tiles are distinct, their near edges sit where a full
// tile's would, and one wrap step brings every coordinate into the lattice.
// With walls, entries of rows outside the fluid and of tile rows beyond a
// wall (below a bottom wall tile: edge rows 0 and 1; above a top wall
// tile: 2 and 3) have no writer and are staged as zeros.  WALLS: the
// variant that handles walled lattices (false: periodic ones only).
template <class rt, int TX, int TY, int NT, bool WALLS>
__device__ __forceinline__ void stage_ring_wrapped(const Lattice &L, int cur, int X0,
                                                   int Y0, rt *s_ring)
{
    using RS = RingStage<rt, TX, TY>;
    rt *const *ring = (rt *const *)L.ring[cur];
    const bool walls = WALLS && L.walls != 0;
    const bool wb = walls && Y0 == 0, wt = walls && Y0 + TY >= L.nyf;
    for (int p = threadIdx.x; p < RS::N; p += NT) {
        long long idx = 0;
        int c = 0;
        bool valid = true;
        if (p < RS::NCOL) {
            const int ci = p / RS::CL, j = p - ci * RS::CL;
            const int r = Y0 - 4 + j;
            c = col_is_left(ci) ? R_L : R_R;
            valid = !walls || (r >= 0 && r < L.nyf);
            idx = ring_index(L, c, neighbour_tile(X0, edge_tile(ci), TX, L.nx, true), 0,
                             walls ? r : wrapi(r, L.nyf), 0);
        } else if (p < RS::NCOL + RS::NROW) {
            const int q = p - RS::NCOL, ri = q / RS::RL, j = q - ri * RS::RL;
            c = row_is_below(ri) ? R_B : R_T;
            valid = !(wb && ri <= 1) && !(wt && ri >= 2);
            idx = ring_index(L, c, 0,
                             neighbour_tile(Y0, edge_tile(ri), TY, L.nyf, !walls), 0,
                             wrapi(X0 - 4 + j, L.nx));
        } else {
            const int q = p - RS::NCOL - RS::NROW, ci = q / 4, ri = q % 4;
            c = row_is_below(ri) ? (col_is_left(ci) ? R_BL : R_BR)
                                 : (col_is_left(ci) ? R_TL : R_TR);
            valid = !(wb && ri <= 1) && !(wt && ri >= 2);
            idx = ring_index(L, c, neighbour_tile(X0, edge_tile(ci), TX, L.nx, true),
                             neighbour_tile(Y0, edge_tile(ri), TY, L.nyf, !walls), 0, 0);
        }
        if (valid && CPLBM_IN_RING(L, cur, c, ring[c] + idx, 1))
            cp_async<sizeof(rt)>(s_ring + p, ring[c] + idx);
        else s_ring[p] = rt(0);
    }
    cp_async_commit();
}

// Edge tiles: where the TMA boxes leave the lattice they fill zeros.  The
// entries the step reads there are fetched from the lattice while the boxes
// are in flight, into staging slots (seam_fix_load), and copied over the
// zeros once the boxes have landed (seam_rho_apply, seam_pop_apply).
//   density halo (rows of pitch RP from x = X0 - 4, y = Y0 - 2): the two
//   halo columns or rows across a periodic edge, the right and top ones
//   after the tile's own width hx and height hy (SeamEdges), columns X0 - 2
//   .. X0 + TX + 1 (with walls, only rows of the fluid); on a wall tile at a periodic
//   x edge also the wall-adjacent row's density one column further out,
//   which the Eq. 28 average of the outermost halo column needs;
//   populations, odd steps (pin_x0 / pin_col layout): the three directions
//   whose source x - e_i lies across a periodic edge, at the edge column or
//   row, and on a wall tile the three directions whose source lies in the
//   solid row, at the wall-adjacent row (halfway bounce-back: read from the
//   node's own slot i); all taken with aa_read_index.
// Slot t of each list is fixed by the enumeration below, so loading and
// applying agree without storing positions.
struct SeamEdges {
    bool xl, xr, yb, yt;  // the tile's halo wraps the left / right / bottom / top edge
    bool wb, wt;          // the tile meets the bottom / top wall
    int hx, hy;           // columns and fluid rows of the tile (below TX, TY only
                          // on the ragged last tile of a direction)
    int vlo, vhi;         // staged density rows holding fluid nodes: [vlo, vhi)
};
template <bool WALLS>
__device__ __forceinline__ SeamEdges seam_edges(const Lattice &L, int X0, int Y0, int TX,
                                                int TY)
{
    const bool w = WALLS && L.walls != 0;
    const bool wb = w && Y0 == 0, wt = w && Y0 + TY >= L.nyf;
    const int hx = min(TX, L.nx - X0), hy = min(TY, L.nyf - Y0);
    return {X0 == 0, X0 + TX >= L.nx, !w && Y0 == 0, !w && Y0 + TY >= L.nyf,
            wb,     wt,              hx, hy,  wb ? 2 : 0,  wt ? hy + 2 : TY + 4};
}
template <int TX, int TY>
struct SeamLists {
    static constexpr int RHO_C = 2 * (TY + 4), RHO_R = RHO_C + 2 * (TX + 4);
    static constexpr int RHO = RHO_R + 4;
    static constexpr int POP_C = 3 * TY, POP = POP_C + 3 * TX;
};
// Density slot t: staged (ly, c); false when the slot is not used.
template <int TX, int TY>
__device__ __forceinline__ bool seam_rho_slot(const SeamEdges &e, int t, int &ly, int &c)
{
    using SL = SeamLists<TX, TY>;
    if (t < SL::RHO_C) {
        if (!e.xl && !e.xr) return false;
        ly = t >> 1;
        c = (e.xl ? 2 : e.hx + 4) + (t & 1);
        return ly >= e.vlo && ly < e.vhi;
    }
    if (t < SL::RHO_R) {
        if (!e.yb && !e.yt) return false;
        const int q = t - SL::RHO_C, sel = q / (TX + 4);
        ly = (e.yb ? 0 : e.hy + 2) + sel;
        c = 2 + q - sel * (TX + 4);
        return true;
    }
    // wall rows at a periodic x edge: t = base + 2 * top + right
    const int k = t - SL::RHO_R, top = k >> 1, right = k & 1;
    if (!(top ? e.wt : e.wb) || !(right ? e.xr : e.xl)) return false;
    ly = top ? e.hy + 1 : 2;
    c = right ? e.hx + 6 : 1;
    return true;
}
// Population slot t: direction i at tile node (lx, ly).
template <int TX, int TY>
__device__ __forceinline__ bool seam_pop_slot(const SeamEdges &e, int t, int &i, int &lx,
                                              int &ly)
{
    using SL = SeamLists<TX, TY>;
    if (t < SL::POP_C) {
        if (!e.xl && !e.xr) return false;
        const int d = t / TY;
        ly = t - d * TY;
        lx = e.xl ? 0 : e.hx - 1;
        // left edge: e_x = +1 reads x - 1 = -1; right edge: e_x = -1 reads x + 1 = nx
        i = e.xl ? (d == 0 ? 1 : d == 1 ? 5 : 8) : (d == 0 ? 3 : d == 1 ? 6 : 7);
        return ly < e.hy;
    }
    const bool bottom = e.yb || e.wb;
    if (!bottom && !e.yt && !e.wt) return false;
    const int q = t - SL::POP_C, d = q / TX;
    lx = q - d * TX;
    ly = bottom ? 0 : e.hy - 1;
    i = bottom ? (d == 0 ? 2 : d == 1 ? 5 : 6) : (d == 0 ? 4 : d == 1 ? 7 : 8);
    return lx < e.hx;
}
template <class S, int TX, int TY, int NT, int PARITY, bool WALLS>
__device__ __forceinline__ void seam_fix_load(const Lattice &L, int cur, int X0, int Y0,
                                              typename S::real *fix_rho,
                                              typename S::pop_t *fix_pop)
{
    using rt = typename S::rho_t;
    using pop_t = typename S::pop_t;
    using SL = SeamLists<TX, TY>;
    const SeamEdges e = seam_edges<WALLS>(L, X0, Y0, TX, TY);
    const rt *R = (const rt *)L.rho[cur];
    for (int t = threadIdx.x; t < SL::RHO; t += NT) {
        int ly, c;
        if (!seam_rho_slot<TX, TY>(e, t, ly, c)) continue;
        // fluid rows only: with walls the row needs no wrap
        const int x = wrapi(X0 - 4 + c, L.nx), r = wrapi(Y0 - 2 + ly, L.nyf);
        const rt *q = R + (long long)r * L.pitch + x;
        fix_rho[t] = CPLBM_IN_RHO(L, cur, q, 1) ? (typename S::real)*q : typename S::real(0);
    }
    if (PARITY == 1) {
        const pop_t *A = (const pop_t *)L.pops;
        for (int t = threadIdx.x; t < SL::POP; t += NT) {
            int i, lx, ly;
            if (!seam_pop_slot<TX, TY>(e, t, i, lx, ly)) continue;
            const pop_t *q = WALLS ? A + aa_read_index(L, 1, i, Y0 + ly, X0 + lx)
                                   : A + pidx(L, opp(i), wrapi(Y0 + ly - ey(i), L.nyf),
                                              wrapi(X0 + lx - ex(i), L.nx));
            fix_pop[t] = CPLBM_IN_POPS(L, q, 1) ? *q : pop_t(0);
        }
    }
}
template <class real, int TX, int TY, int NT, int RP, bool WALLS>
__device__ __forceinline__ void seam_rho_apply(const Lattice &L, int X0, int Y0,
                                               const real *fix_rho, real *s_rho)
{
    const SeamEdges e = seam_edges<WALLS>(L, X0, Y0, TX, TY);
    for (int t = threadIdx.x; t < SeamLists<TX, TY>::RHO; t += NT) {
        int ly, c;
        if (seam_rho_slot<TX, TY>(e, t, ly, c)) s_rho[ly * RP + c] = fix_rho[t];
    }
}
template <class pop_t, int TX, int TY, int NT, int PLANE, int PP, int PX, bool WALLS>
__device__ __forceinline__ void seam_pop_apply(const Lattice &L, int X0, int Y0,
                                               const pop_t *fix_pop, pop_t *s_pin)
{
    const SeamEdges e = seam_edges<WALLS>(L, X0, Y0, TX, TY);
    for (int t = threadIdx.x; t < SeamLists<TX, TY>::POP; t += NT) {
        int i, lx, ly;
        if (seam_pop_slot<TX, TY>(e, t, i, lx, ly))
            s_pin[(i - 1) * PLANE + ly * PP + lx + pin_col<1, PX>(i)] = fix_pop[t];
    }
}

// Edge tiles at a wall: the solid row's density by Eq. 28 from the
// wall-adjacent fluid row (both after the partial sums were added), at
// staged columns 2 .. TX + 5 (x = X0 - 2 .. X0 + TX + 1), in the order of
// load_rho_tile; the top solid row mirrors it (staged row hy + 2 from hy +
// 1).  Ends with a block barrier when the tile meets a wall (CTA-uniform).
template <class real, int TX, int NT, int RP>
__device__ __forceinline__ void wall_rho_rows(const SeamEdges &e, real *s_rho)
{
    if (!e.wb && !e.wt) return;
    constexpr int W = TX + 4;
    for (int t = threadIdx.x; t < 2 * W; t += NT) {
        const int top = t >= W;
        if (!(top ? e.wt : e.wb)) continue;
        const int c = 2 + t - top * W;
        const real *src = s_rho + (top ? e.hy + 1 : 2) * RP + c;
        s_rho[(top ? e.hy + 2 : 1) * RP + c] =
            real(2.0 / 3.0) * src[0] + real(1.0 / 6.0) * src[-1] + real(1.0 / 6.0) * src[1];
    }
    __syncthreads();
}

// mu of halo row b (r = Y0 - 1 + b) of an edge tile when that row is not a
// fluid row: mu_s on the bottom solid row (Sec. IV); on the top solid row
// the value of its fluid neighbour below (Sec. V, top_mode 0: computed here
// from the staged density, as mu_tile does) or mu_top; zero beyond a ragged
// top wall tile (never read).  false for fluid rows.  c: staged density
// index of the halo node.
template <class S, int RP>
__device__ __forceinline__ bool wall_mu(const Lattice &L, const SeamEdges &e, int b, int c,
                                        const typename S::real *s_rho, typename S::real &m)
{
    using real = typename S::real;
    const Consts<real> &K = consts<real>(L);
    if (e.wb && b == 0) {
        m = K.mu_bottom;
        return true;
    }
    if (e.wt && b >= e.hy + 1) {
        if (b > e.hy + 1) {
            m = real(0);
        } else if (L.top_mode == 0) {
            const int cb = c - RP;  // fluid neighbour below (row nyf - 1)
            const real ref = S::offset ? K.rho_ref : real(0);
            m = mu_bulk(K.eos, s_rho[cb] + ref) - K.kappa * lap9<real, RP>(s_rho, cb);
        } else {
            m = K.mu_top;
        }
        return true;
    }
    return false;
}

// Add the staged partial sums to the halo's tile-edge nodes of s_rho (rows
// of pitch RP, halo node (lx, ly) at column lx + 2), in the order of
// load_rho_stored.  Items 0 .. 4 HR - 1 take the four edge columns whole,
// crossings with the edge rows included; the rest take the edge rows
// without those crossings (halo columns 0, 3 .. hx, hx + 3).  hx, hy: the
// tile's width and height (TX, TY but on a ragged last tile, whose halo
// ends at column hx + 3 and row hy + 3; what lies beyond is not read).
template <class real, int TX, int TY, int NT, int RP>
__device__ __forceinline__ void combine_ring(real *s_rho, const real *s_ring, int hx,
                                             int hy)
{
    using RS = RingStage<real, TX, TY>;
    constexpr int HR = TY + 4, NC = 4 * HR, NI = NC + 4 * TX;
    for (int q = threadIdx.x; q < NI; q += NT) {
        if (q < NC) {
            const int ci = q / HR, ly = q - ci * HR, lx = edge_col(ci, hx);
            const int ri = col_index(ly, hy);
            real v = s_rho[ly * RP + lx + 2] + s_ring[ci * RS::CL + ly + 2];
            if (ri >= 0)
                v = (v + s_ring[RS::NCOL + ri * RS::RL + lx + 2]) +
                    s_ring[RS::NCOL + RS::NROW + ci * 4 + ri];
            s_rho[ly * RP + lx + 2] = v;
        } else {
            const int t = q - NC, ri = t / TX, k = t - ri * TX;
            if (k >= hx) continue;
            const int lx = k == 0 ? 0 : (k == hx - 1 ? hx + 3 : k + 2);
            const int ly = edge_col(ri, hy);
            s_rho[ly * RP + lx + 2] += s_ring[RS::NCOL + ri * RS::RL + lx + 2];
        }
    }
}

// Shared memory of a TMA tile: the staged populations in their storage
// type, then density, partial sums / exchange slots and mu in the
// arithmetic type.
// The two tensor maps one tile's TMA loads read: the populations and the
// density buffer of this step.  Addresses in kernel-parameter space (the
// maps are __grid_constant__ arguments of the launching kernel).
struct TileMaps {
    const CUtensorMap *pops;
    const CUtensorMap *rho;
};

template <class S, int TX, int TY, int NP = 1>
struct TmaSmem {
    using real = typename S::real;
    using pop_t = typename S::pop_t;
    static constexpr int PX = 16 / sizeof(pop_t);
    static constexpr int RP = TX + 8;   // density rows (from X0 - 4)
    static constexpr int PP = TX + PX;  // population rows
    static constexpr int PLANE = TY * PP;
    static constexpr size_t PIN_BYTES = sizeof(pop_t) * 8 * PLANE;
    static constexpr int NRHO = (TY + 4) * RP;
    static constexpr int MP = TX + 2, MH = TY + 2;
    static constexpr int NRING = RingStage<real, TX, TY>::N;
    static constexpr int NMU = NP * MP * MH;  // mu, or (NP = 3) the tensor of Eq. 9
    static constexpr int NXCH = 2 * (STEP_THREADS / 32) * (TX + 2);
    // ring (and on seam tiles the staged population fix-ups after it), then
    // the exchange slots
    static constexpr int NFIXP = (SeamLists<TX, TY>::POP * sizeof(pop_t) + sizeof(real) - 1) /
                                 sizeof(real);
    static constexpr int NSHARE = NRING + NFIXP > NXCH ? NRING + NFIXP : NXCH;
    static_assert(MP * MH >= SeamLists<TX, TY>::RHO, "density fix-ups staged in s_mu");
    static constexpr size_t bar_offset =
        (PIN_BYTES + sizeof(real) * (NRHO + NSHARE + NMU) + 15) / 16 * 16;
    static constexpr size_t bytes = bar_offset + 16;
    static constexpr unsigned tx_rho = sizeof(real) * NRHO;
    static constexpr unsigned tx_pops = PIN_BYTES;
    static_assert((PLANE * sizeof(pop_t)) % 128 == 0, "TMA destinations");
};

// Gradient of the isotropic stencil from a 3 x 3 window w[row][col] (row 0
// below, col 0 left), same arithmetic as grad9.
template <class T>
__device__ __forceinline__ void grad_w(const T (&w)[3][3], T &gx, T &gy)
{
    const T ne = w[2][2], nw = w[2][0], se = w[0][2], sw = w[0][0];
    gx = (T(4) * (w[1][2] - w[1][0]) + (ne - nw) + (se - sw)) * T(1.0 / 12.0);
    gy = (T(4) * (w[2][1] - w[0][1]) + (ne + nw) - (se + sw)) * T(1.0 / 12.0);
}
// Laplacian of the isotropic stencil from a 3 x 3 window, as lap9.
template <class T>
__device__ __forceinline__ T lap_w(const T (&w)[3][3])
{
    const T axial = w[1][2] + w[1][0] + w[2][1] + w[0][1];
    const T diag = (w[2][2] + w[2][0]) + (w[0][2] + w[0][0]);
    return (T(4) * axial + diag - T(20) * w[1][1]) * T(1.0 / 6.0);
}

// PT: the baseline force of Eq. 5 (the pressure tensor of Eq. 9 in three
// planes where the chemical potential would be; periodic lattices only).
template <class S, int TX, int TY, int NT, int PARITY, int EDGE, bool PT = false>
__device__ __forceinline__ bool step_tile_tma(const Lattice &L, int cur, int X0,
                                              int Y0, unsigned char *smem_raw,
                                              TileMaps maps,
                                              unsigned long long *bar, unsigned phase)
{
    using real = typename S::real;
    using pop_t = typename S::pop_t;
    using rho_t = typename S::rho_t;
    using TS = TmaSmem<S, TX, TY, PT ? 3 : 1>;
    static_assert(TX == 32, "lanes map to x");
    static_assert(!PT || EDGE != 2, "the pressure-tensor force has no wall rule");
    constexpr int NW = NT / 32, PER = TY / NW;
    static_assert(PER * NW == TY && PER >= 2, "warps own whole row blocks");
    constexpr int RP = TS::RP, PP = TS::PP, PLANE = TS::PLANE, MP = TS::MP, MH = TS::MH;
    constexpr int XW = TX + 2;               // exchange slots per warp
    pop_t *s_pin = reinterpret_cast<pop_t *>(smem_raw);            // [8][TY][PP]
    real *s_rho = reinterpret_cast<real *>(smem_raw + TS::PIN_BYTES);  // [TY + 4][RP]
    real *s_ring = s_rho + TS::NRHO;
    real *s_mu = s_ring + TS::NSHARE;                    // [MH][MP]
    real *s_up = s_ring;                                 // [NW][XW], after step 2
    real *s_down = s_up + NW * XW;                       // [NW][XW]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nxt = cur ^ 1;
    // EDGE: 0 interior tile; an edge tile (tile_kind TILE_SEAM), whose halo
    // wraps around a periodic edge, of a periodic lattice (1) or of any
    // lattice, walls included (2)
    constexpr bool seam = EDGE != 0, walls_ok = EDGE == 2;

    // 1. Loads (bar: the caller's two initialised mbarriers, this tile
    //    completing phase `phase` of each).  Density halo and populations by
    //    TMA and the partial sums by bulk copies (thread 0), the corner sums
    //    by cp.async; on seam tiles all partial sums by cp.async, wrapped.
    if (threadIdx.x == 0) {
        mbar_expect_tx(&bar[0],
                       TS::tx_rho + (seam ? 0u : RingStage<real, TX, TY>::bulk_bytes));
        tma_load_2d(s_rho, maps.rho, X0 - 4, Y0 - 2, &bar[0]);
        mbar_expect_tx(&bar[1], TS::tx_pops);
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            const int plane = PARITY == 0 ? i - 1 : opp(i) - 1;
            const int y0 = PARITY == 0 ? Y0 : Y0 - ey(i);
            tma_load_3d(s_pin + (i - 1) * PLANE, maps.pops,
                        X0 + pin_x0<PARITY, TS::PX>(i), y0, plane, &bar[1]);
        }
    }
    pop_t *fix_pop = reinterpret_cast<pop_t *>(s_ring + TS::NRING);
    if (seam) {
        stage_ring_wrapped<real, TX, TY, NT, walls_ok>(L, cur, X0, Y0, s_ring);
        seam_fix_load<S, TX, TY, NT, PARITY, walls_ok>(L, cur, X0, Y0, s_mu, fix_pop);
    } else {
        stage_ring<real, TX, TY>(L, cur, X0, Y0, s_ring, &bar[0]);
    }
    cp_async_wait_all();
    if (!tma_landed(bar, 0, phase, L.err, L.wait_cycles)) return false;
    if (seam) {
        seam_rho_apply<real, TX, TY, NT, RP, walls_ok>(L, X0, Y0, s_mu, s_rho);
        __syncthreads();
    }

    // 2. Partial sums into the halo's tile-edge nodes (order of
    //    load_rho_stored).  Halo (lx, ly) of the (TX + 4)-wide convention is
    //    staged row ly, column lx + 2.  Edge tiles may be the ragged last
    //    tile of a periodic direction: hx columns, hy rows (its right and
    //    top edges, the wrap and the partial sums across them sit there);
    //    lanes at hx and beyond and rows at hy and beyond compute but store
    //    nothing.
    const SeamEdges edge = seam_edges<walls_ok>(L, X0, Y0, TX, TY);
    const int hx = seam ? edge.hx : TX, hy = seam ? edge.hy : TY;
    combine_ring<real, TX, TY, NT, RP>(s_rho, s_ring, hx, hy);
    __syncthreads();
    // edge tiles at a wall: the solid row's density (Eq. 28)
    if (walls_ok) wall_rho_rows<real, TX, NT, RP>(edge, s_rho);

    // 3. mu at (a, b), a in [0, TX + 2) <-> x = X0 - 1 + a, b in [0, TY + 2)
    //    <-> r = Y0 - 1 + b; its density sits at staged (b + 1, a + 3).
    //    Columns 1..TX: lane a - 1, each warp a run of consecutive rows with
    //    a rolling 3 x 3 window; columns 0 and TX + 1 separately.  Solid
    //    rows of wall tiles take the surface values (wall_mu).  The
    //    pressure-tensor baseline (PT) fills the three planes of Eq. 9
    //    instead, in the arithmetic of pt_tile.
    if constexpr (PT) {
        const Consts<real> &K = consts<real>(L);
        const real kappa = K.kappa;
        const real ref = S::offset ? K.rho_ref : real(0);
        constexpr int N = MP * MH;
        for (int k = threadIdx.x; k < N; k += NT) {
            const int a = k % MP, b = k / MP;
            const int c = (b + 1) * RP + a + 3;
            const real rho = s_rho[c] + ref;
            real gx, gy;
            grad9<real, RP>(s_rho, c, gx, gy);
            const real lap = lap9<real, RP>(s_rho, c);
            const real iso = p0_bulk(K.eos, rho) - kappa * rho * lap -
                             real(0.5) * kappa * (gx * gx + gy * gy);
            s_mu[k] = iso + kappa * gx * gx;
            s_mu[N + k] = kappa * gx * gy;
            s_mu[2 * N + k] = iso + kappa * gy * gy;
        }
    } else {
        const Consts<real> &K = consts<real>(L);
        const EosT<real> &eos = K.eos;
        const real kappa = K.kappa;
        const real ref = S::offset ? K.rho_ref : real(0);
        const int b0 = (warp * MH) / NW, b1 = ((warp + 1) * MH) / NW;
        const int a = lane + 1;
        real w[3][3];
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int d = 0; d < 3; ++d) w[j][d] = s_rho[(b0 + j) * RP + a + 2 + d];
        for (int b = b0; b < b1; ++b) {
#pragma unroll
            for (int d = 0; d < 3; ++d) w[2][d] = s_rho[(b + 2) * RP + a + 2 + d];
            real m;
            if (!(walls_ok && wall_mu<S, RP>(L, edge, b, (b + 1) * RP + a + 3, s_rho, m)))
                m = mu_bulk(eos, w[1][1] + ref) - kappa * lap_w(w);
            s_mu[b * MP + a] = m;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                w[0][d] = w[1][d];
                w[1][d] = w[2][d];
            }
        }
        for (int t = threadIdx.x; t < 2 * MH; t += NT) {
            const int ae = (t & 1) ? TX + 1 : 0, b = t >> 1;
            const int c = (b + 1) * RP + ae + 3;
            real m;
            if (!(walls_ok && wall_mu<S, RP>(L, edge, b, c, s_rho, m)))
                m = mu_bulk(eos, s_rho[c] + ref) - kappa * lap9<real, RP>(s_rho, c);
            s_mu[b * MP + ae] = m;
        }
    }
    // the populations were in flight during steps 2 and 3; the barrier also
    // publishes s_mu
    if (!tma_landed(bar, 1, phase, L.err, L.wait_cycles)) return false;
    if (PARITY == 1 && seam) {
        seam_pop_apply<pop_t, TX, TY, NT, PLANE, PP, TS::PX, walls_ok>(L, X0, Y0, fix_pop, s_pin);
        __syncthreads();
    }

    // 4. Force, collision, in-place streaming and the register hand-over for
    //    the thread's PER nodes at rows ly0 .. ly0 + PER - 1, column lx.
    const int lx = lane, ly0 = warp * PER;
    const real tau = consts<real>(L).tau;
    const real omega = consts<real>(L).omega;
    const real rho_ref = S::offset ? consts<real>(L).rho_ref : real(0);
    pop_t *A = (pop_t *)L.pops;
    rho_t *Rn = (rho_t *)L.rho[nxt];
    rho_t *const *ring = (rho_t *const *)L.ring[nxt];
    // 32-bit write offsets (the TMA maps exist only when 8 planes fit); on
    // odd steps of seam tiles an x target across a periodic edge is brought
    // back by nx (lanes 0 and hx - 1), a row target by the lattice height
    // (rows 0 and hy - 1, wrap_y below)
    const int lr = hx - 1;  // lane of the tile's last column
    const int cxl = (PARITY == 1 && seam && X0 == 0 && lane == 0) ? L.nx : 0;
    const int cxr = (PARITY == 1 && seam && X0 + TX >= L.nx && lane == lr) ? -L.nx : 0;
    int woff[9];
#pragma unroll
    for (int i = 1; i < 9; ++i)
        woff[i] = PARITY == 0 ? (opp(i) - 1) * (int)L.plane
                              : (i - 1) * (int)L.plane + ey(i) * L.pitch + ex(i) +
                                    (ex(i) < 0 ? cxl : ex(i) > 0 ? cxr : 0);
    // rows 0 .. hy - 1 and columns 0 .. hx - 1 are the tile's (below TY, TX
    // on a ragged last tile, and on a ragged top wall tile rows hy and up are
    // not fluid); the others are not updated and contribute nothing
    const bool has_l = lane > 0, has_r = lane < lr;
    const bool lane_ok = lane < hx;
    real wr[3][3], wm[3][3];
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            wr[j][d] = s_rho[(ly0 + 1 + j) * RP + lx + 3 + d];
            wm[j][d] = s_mu[(ly0 + j) * MP + lx + d];
        }
    // Rolling hand-over.  pend: row k - 1 without its "down" part;
    // first: row 0 of the warp without the warp below's "up"; *_c: the same
    // for the ring column a lane 0 / lane hx - 1 feeds; up_top: the "up" of
    // the tile's last row hy - 1, for the ring row above the tile.
    real pend = real(0), up_prev = real(0), first = real(0);
    real pend_c = real(0), up_prev_c = real(0), first_c = real(0);
    real up_top = real(0), up_top_c = real(0);
    const int slot_c = TX + (lane == lr);         // exchange slot of a column
    const int xc = lane == 0 ? X0 - 1 : X0 + hx;  // ring column of the lane
    const int cls_c = lane == 0 ? R_R : R_L;
    // this tile, and the tile of the ring column a lane feeds (classes L and
    // R share one index layout)
    const int bx = X0 / TX, by = Y0 / TY;
    const int bxc = neighbour_tile(X0, lane == 0 ? -1 : 1, TX, L.nx, seam);
    const bool col_lane = lane == 0 || lane == lr;
    pop_t *Arow = A + (long long)(Y0 + ly0) * L.pitch + X0 + lx;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int ly = ly0 + k;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            wr[2][d] = s_rho[(ly + 3) * RP + lx + 3 + d];
            wm[2][d] = s_mu[(ly + 2) * MP + lx + d];
        }
        real same = real(0), up = real(0), down = real(0);
        real same_c = real(0), up_c = real(0), down_c = real(0);
        if (!seam || ly < hy) {  // warp-uniform
            real f[9];
#pragma unroll
            for (int i = 1; i < 9; ++i)
                f[i] = ld_real(s_pin + (i - 1) * PLANE + ly * PP + lx + pin_col<PARITY, TS::PX>(i));
            const real drho = wr[1][1];
            const real rho = drho + rho_ref;
            real gmx, gmy, grx, gry;
            grad_w(wr, grx, gry);
            real Fx, Fy;
            if constexpr (PT) {
                // Eq. 5: F = -div(P) + grad(cs^2 rho), as step_tile
                constexpr int N = MP * MH;
                const int cm = (ly + 1) * MP + lx + 1;
                real pxx_x, pxx_y, pxy_x, pxy_y, pyy_x, pyy_y;
                grad9<real, MP>(s_mu, cm, pxx_x, pxx_y);
                grad9<real, MP>(s_mu + N, cm, pxy_x, pxy_y);
                grad9<real, MP>(s_mu + 2 * N, cm, pyy_x, pyy_y);
                Fx = grx * real(1.0 / 3.0) - (pxx_x + pxy_y);
                Fy = gry * real(1.0 / 3.0) - (pxy_x + pyy_y);
            } else {
                grad_w(wm, gmx, gmy);
                Fx = grx * real(1.0 / 3.0) - rho * gmx;
                Fy = gry * real(1.0 / 3.0) - rho * gmy;
            }
            real fp[9];
            collide<real>(f, drho, rho, Fx, Fy, tau, omega, fp);
            // wall rows (halfway bounce-back, Sec. IV): what leaves into the
            // solid row comes back to the node
            const bool wall_b = walls_ok && edge.wb && ly == 0;
            const bool wall_t = walls_ok && edge.wt && ly == hy - 1;
            {
                const int wrap_y = L.nyf * L.pitch;
                const int cyb = (PARITY == 1 && seam && edge.yb && ly == 0) ? wrap_y : 0;
                const int cyt = (PARITY == 1 && seam && edge.yt && ly == hy - 1) ? -wrap_y : 0;
#pragma unroll
                for (int i = 1; i < 9; ++i) {
                    // odd steps: a population heading into a solid row goes
                    // to the node's own slot opp(i)
                    const bool into_wall = PARITY == 1 && ((ey(i) < 0 && wall_b) ||
                                                           (ey(i) > 0 && wall_t));
                    const int o = into_wall ? (opp(i) - 1) * (int)L.plane
                                            : woff[i] + (ey(i) < 0 ? cyb : ey(i) > 0 ? cyt : 0);
                    if ((!seam || lane_ok) && CPLBM_IN_POPS(L, Arow + o, 1))
                        st_real(Arow + o, fp[i]);
                }
            }

            // lane-neighbour parts of the hand-over
            const real f1l = __shfl_up_sync(0xffffffffu, fp[1], 1);
            const real f5l = __shfl_up_sync(0xffffffffu, fp[5], 1);
            const real f8l = __shfl_up_sync(0xffffffffu, fp[8], 1);
            const real f3r = __shfl_down_sync(0xffffffffu, fp[3], 1);
            const real f6r = __shfl_down_sync(0xffffffffu, fp[6], 1);
            const real f7r = __shfl_down_sync(0xffffffffu, fp[7], 1);
            same = fp[0] + (has_l ? f1l : real(0)) + (has_r ? f3r : real(0));
            up = fp[2] + (has_l ? f5l : real(0)) + (has_r ? f6r : real(0));
            down = fp[4] + (has_l ? f8l : real(0)) + (has_r ? f7r : real(0));
            if (wall_b) same += (fp[4] + fp[7]) + fp[8];
            if (wall_t) same += (fp[2] + fp[5]) + fp[6];
            // ring columns: lane 0 feeds x = X0 - 1 (f*_3; f*_6 up; f*_7
            // down), lane hx - 1 feeds x = X0 + hx (f*_1; f*_5 up; f*_8 down)
            same_c = lane == 0 ? fp[3] : fp[1];
            up_c = lane == 0 ? fp[6] : fp[5];
            down_c = lane == 0 ? fp[7] : fp[8];
        }
        if (seam && ly == hy - 1) {
            up_top = up;
            up_top_c = up_c;
        }
        Arow += L.pitch;
        // rows of the lattice this warp may write (the tile's rows
        // 0 .. hy - 1) and its lanes that hold a node of the tile
        const bool row_ok = !seam || ly - 1 < hy;
        const bool put_ok = !seam || lane_ok;
        if (k == 0) {
            // this row's "down" belongs to the warp below (or the ring row
            // under the tile)
            s_down[warp * XW + lane] = down;
            if (col_lane) s_down[warp * XW + slot_c] = down_c;
            pend = same;
            pend_c = same_c;
        } else {
            const real done = pend + down;        // row ly - 1
            const real done_c = pend_c + down_c;
            if (k == 1) {
                first = done;
                first_c = done_c;
            } else if (row_ok) {
                if (put_ok) put_rho(L, nxt, Rn, (long long)(Y0 + ly - 1) * L.pitch + X0 + lx, (rho_t)done);
                if (col_lane) put_ring(L, nxt, ring, cls_c, ring_index(L, R_L, bxc, by, Y0 + ly - 1, xc), (rho_t)done_c);
            }
            pend = same + up_prev;
            pend_c = same_c + up_prev_c;
        }
        up_prev = up;
        up_prev_c = up_c;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            wr[0][d] = wr[1][d]; wr[1][d] = wr[2][d];
            wm[0][d] = wm[1][d]; wm[1][d] = wm[2][d];
        }
    }
    // up_prev: the warp's last-row "up", for the warp above (or the ring
    // row over the tile).
    s_up[warp * XW + lane] = up_prev;
    if (col_lane) s_up[warp * XW + slot_c] = up_prev_c;
    __syncthreads();
    {
        // last row: add the warp above's first-row "down"
        real top = pend, top_c = pend_c;
        if (warp + 1 < NW) {
            top += s_down[(warp + 1) * XW + lane];
            top_c += s_down[(warp + 1) * XW + slot_c];
        }
        if (!seam || ly0 + PER - 1 < hy) {
            if (!seam || lane_ok)
                put_rho(L, nxt, Rn, (long long)(Y0 + ly0 + PER - 1) * L.pitch + X0 + lx, (rho_t)top);
            if (col_lane) put_ring(L, nxt, ring, cls_c, ring_index(L, R_L, bxc, by, Y0 + ly0 + PER - 1, xc), (rho_t)top_c);
        }
        // first row: add the warp below's last-row "up"
        if (warp > 0) {
            first += s_up[(warp - 1) * XW + lane];
            first_c += s_up[(warp - 1) * XW + slot_c];
        }
        if (!seam || ly0 < hy) {
            if (!seam || lane_ok)
                put_rho(L, nxt, Rn, (long long)(Y0 + ly0) * L.pitch + X0 + lx, (rho_t)first);
            if (col_lane) put_ring(L, nxt, ring, cls_c, ring_index(L, R_L, bxc, by, Y0 + ly0, xc), (rho_t)first_c);
        }
    }
    // ring rows below and above the tile, with their corners (none across a
    // wall); the row above takes the "up" of the tile's last row hy - 1 (the
    // last row of the last warp but on a ragged last tile)
    const int bxl = neighbour_tile(X0, -1, TX, L.nx, seam);
    const int bxr = neighbour_tile(X0, 1, TX, L.nx, seam);
    if (warp == 0 && !(walls_ok && edge.wb)) {
        const int byb = neighbour_tile(Y0, -1, TY, L.nyf, seam);
        if (!seam || lane_ok)
            put_ring(L, nxt, ring, R_T, ring_index(L, R_T, bx, byb, Y0 - 1, X0 + lx), (rho_t)s_down[lane]);
        if (lane == 0) put_ring(L, nxt, ring, R_TR, ring_index(L, R_TR, bxl, byb, Y0 - 1, X0 - 1), (rho_t)s_down[TX]);
        if (lane == lr) put_ring(L, nxt, ring, R_TL, ring_index(L, R_TL, bxr, byb, Y0 - 1, X0 + hx), (rho_t)s_down[TX + 1]);
    }
    const real upt = seam ? up_top : up_prev, upt_c = seam ? up_top_c : up_prev_c;
    if (warp == (hy - 1) / PER && !(walls_ok && edge.wt)) {
        const int byt = neighbour_tile(Y0, 1, TY, L.nyf, seam);
        if (!seam || lane_ok)
            put_ring(L, nxt, ring, R_B, ring_index(L, R_B, bx, byt, Y0 + hy, X0 + lx), (rho_t)upt);
        if (lane == 0) put_ring(L, nxt, ring, R_BR, ring_index(L, R_BR, bxl, byt, Y0 + hy, X0 - 1), (rho_t)upt_c);
        if (lane == lr) put_ring(L, nxt, ring, R_BL, ring_index(L, R_BL, bxr, byt, Y0 + hy, X0 + hx), (rho_t)upt_c);
    }
    return true;
}

// ---------------------------------------------------------------------------
// FP32 interior tiles with TMA, two nodes per lane.  Tiles are TX = 64 wide:
// lane l owns columns 2l and 2l + 1 of each of its warp's PER rows, and the
// pair's arithmetic runs on packed FP32 pairs (the two-wide FFMA / FADD /
// FMUL of sm_100 and later), so one instruction serves both nodes.  Loads,
// partial sums and the density hand-over are those of step_tile_tma; even
// steps also move the pair's populations as aligned 64-bit words (odd steps
// read and write the x-shifted directions one node at a time).
//
// Stencils on a pair.  For a field v and one row of the pair's window, with
// (v0, v1) the pair and wl = v(x0 - 1), wr = v(x1 + 1):
//   C = (v0, v1),  H = W + E = (v1 + wl, wr + v0),  D = E - W = (v1 - wl, wr - v0),
// and with rows u (above), m and d (below):
//   grad_x = (4 D_m + D_u + D_d) / 12,   grad_y = (4 (C_u - C_d) + H_u - H_d) / 12,
//   lap    = (4 (H_m + C_u + C_d) + (H_u + H_d) - 20 C_m) / 6,
// which are grad_w / lap_w term by term.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 p2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b as b * (-1) + a: the exact difference rounded once, as a subtraction
__device__ __forceinline__ float2 psub(float2 a, float2 b)
{
    return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}
__device__ __forceinline__ float2 prcp(float2 v)
{
    return make_float2(__fdividef(1.0f, v.x), __fdividef(1.0f, v.y));
}
__device__ __forceinline__ float2 pdiv(float2 a, float2 b)
{
    return make_float2(__fdividef(a.x, b.x), __fdividef(a.y, b.y));
}
__device__ __forceinline__ float2 plog(float2 v)
{
    return make_float2(__logf(v.x), __logf(v.y));
}

// One window row of a field around the pair at s + i (8-byte aligned).
struct Row2 {
    float2 c, h, d;
};
__device__ __forceinline__ Row2 row2(const float *s, int i)
{
    const float2 c = *reinterpret_cast<const float2 *>(s + i);
    const float wl = s[i - 1], wr = s[i + 2];
    return {c, make_float2(c.y + wl, wr + c.x), make_float2(c.y - wl, wr - c.x)};
}
__device__ __forceinline__ float2 lap2(const Row2 &u, const Row2 &m, const Row2 &d)
{
    const float2 axial = padd(padd(m.h, u.c), d.c);
    const float2 diag = padd(u.h, d.h);
    return pmul(pfma(p2(-20.0f), m.c, pfma(p2(4.0f), axial, diag)), p2(1.0f / 6.0f));
}
__device__ __forceinline__ void grad2(const Row2 &u, const Row2 &m, const Row2 &d,
                                      float2 &gx, float2 &gy)
{
    const float2 c = p2(1.0f / 12.0f), four = p2(4.0f);
    gx = pmul(padd(pfma(four, m.d, u.d), d.d), c);
    gy = pmul(psub(pfma(four, psub(u.c, d.c), u.h), d.h), c);
}

// mu_bulk on a pair of densities.
__device__ __forceinline__ float2 mu_bulk2(const EosT<float> &e, float2 rho)
{
    const float2 one = p2(1.0f), m2a = p2(-2.0f * e.a);
    switch (e.kind) {
    case EOS_VDW: {
        const float2 iq = prcp(psub(one, pmul(p2(e.b), rho)));
        return pfma(m2a, rho, pmul(p2(e.RT), padd(plog(pmul(rho, iq)), iq)));
    }
    case EOS_CS: {
        const float2 h = pmul(p2(e.quarter_b), rho);
        const float2 iq = prcp(psub(one, h));
        const float2 iq3 = pmul(pmul(iq, iq), iq);
        const float2 s = padd(padd(pmul(psub(p2(3.0f), h), iq3), plog(rho)), one);
        return pfma(m2a, rho, pmul(p2(e.RT), s));
    }
    case EOS_PR: {
        const float2 br = pmul(p2(e.b), rho);
        const float2 iq = prcp(psub(one, br));
        const float2 t1 = pmul(p2(e.RT), plog(pmul(rho, iq)));
        const float2 t2 = pmul(
            p2(e.pr_c), plog(pdiv(padd(p2(e.pr_s2m1), br), psub(p2(e.pr_s2p1), br))));
        const float2 den = psub(pfma(p2(2.0f), br, one), pmul(br, br));
        return psub(pfma(p2(e.RT), iq, psub(t1, t2)), pdiv(pmul(p2(e.aalpha), rho), den));
    }
    default: {  // EOS_RKS
        const float2 br = pmul(p2(e.b), rho);
        const float2 iq = prcp(psub(one, br));
        const float2 t1 = pmul(p2(e.RT), padd(plog(pmul(rho, iq)), iq));
        const float2 t2 = pmul(p2(e.rks_c), plog(padd(one, br)));
        return psub(psub(t1, t2), pdiv(pmul(p2(e.aalpha), rho), padd(one, br)));
    }
    }
}

// p0_bulk on a pair of densities (the pressure-tensor baseline).
__device__ __forceinline__ float2 p0_bulk2(const EosT<float> &e, float2 rho)
{
    const float2 one = p2(1.0f), ma = p2(-e.a);
    const float2 br = pmul(p2(e.b), rho), rrt = pmul(rho, p2(e.RT));
    switch (e.kind) {
    case EOS_VDW:
        return pfma(pmul(ma, rho), rho, pdiv(rrt, psub(one, br)));
    case EOS_CS: {
        const float2 h = pmul(p2(e.quarter_b), rho), q = psub(one, h), h2 = pmul(h, h);
        const float2 num = pmul(rrt, psub(padd(padd(one, h), h2), pmul(h2, h)));
        return pfma(pmul(ma, rho), rho, pdiv(num, pmul(pmul(q, q), q)));
    }
    case EOS_PR: {
        const float2 den = psub(pfma(p2(2.0f), br, one), pmul(br, br));
        return psub(pdiv(rrt, psub(one, br)), pdiv(pmul(pmul(p2(e.aalpha), rho), rho), den));
    }
    default:  // EOS_RKS
        return psub(pdiv(rrt, psub(one, br)),
                    pdiv(pmul(pmul(p2(e.aalpha), rho), rho), padd(one, br)));
    }
}

// collide() on a pair of nodes.
__device__ __forceinline__ void collide2(const float2 *f, float2 drho, float2 rho,
                                         float2 Fx, float2 Fy, float2 tau,
                                         float2 omega, float2 *fp)
{
    const float2 d57 = psub(f[5], f[7]);
    const float2 jx = padd(padd(psub(f[1], f[3]), d57), psub(f[8], f[6]));
    const float2 jy = padd(padd(psub(f[2], f[4]), d57), psub(f[6], f[8]));
    const float2 inv_rho = prcp(rho);
    const float2 ux = pmul(pfma(tau, Fx, jx), inv_rho);
    const float2 uy = pmul(pfma(tau, Fy, jy), inv_rho);
    const float2 nusq = pmul(p2(-1.5f), pfma(ux, ux, pmul(uy, uy)));  // -1.5 u^2
    const float2 c45 = p2(4.5f), c3 = p2(3.0f);
    {
        const float2 w1 = p2(1.0f / 9.0f);
        const float2 ex2 = pfma(pmul(c45, ux), ux, nusq);
        const float2 ey2 = pfma(pmul(c45, uy), uy, nusq);
        const float2 ax = pmul(w1, pfma(rho, ex2, drho));
        const float2 ay = pmul(w1, pfma(rho, ey2, drho));
        const float2 r3 = pmul(pmul(w1, rho), c3);
        const float2 bx = pmul(r3, ux), by = pmul(r3, uy);
        fp[1] = pfma(omega, psub(padd(ax, bx), f[1]), f[1]);
        fp[3] = pfma(omega, psub(psub(ax, bx), f[3]), f[3]);
        fp[2] = pfma(omega, psub(padd(ay, by), f[2]), f[2]);
        fp[4] = pfma(omega, psub(psub(ay, by), f[4]), f[4]);
    }
    {
        const float2 w5 = p2(1.0f / 36.0f);
        const float2 sp = padd(ux, uy), sm = psub(ux, uy);
        const float2 ep = pfma(pmul(c45, sp), sp, nusq);
        const float2 em = pfma(pmul(c45, sm), sm, nusq);
        const float2 a5 = pmul(w5, pfma(rho, ep, drho));
        const float2 a8 = pmul(w5, pfma(rho, em, drho));
        const float2 r3 = pmul(pmul(w5, rho), c3);
        const float2 b5 = pmul(r3, sp), b8 = pmul(r3, sm);
        fp[5] = pfma(omega, psub(padd(a5, b5), f[5]), f[5]);
        fp[7] = pfma(omega, psub(psub(a5, b5), f[7]), f[7]);
        fp[8] = pfma(omega, psub(padd(a8, b8), f[8]), f[8]);
        fp[6] = pfma(omega, psub(psub(a8, b8), f[6]), f[6]);
    }
    fp[0] = psub(drho, padd(padd(padd(fp[1], fp[2]), padd(fp[3], fp[4])),
                            padd(padd(fp[5], fp[6]), padd(fp[7], fp[8]))));
}

// Two adjacent stored populations (8- or 4-byte aligned) as a float pair.
__device__ __forceinline__ float2 ld_pair(const float *p)
{
    return *reinterpret_cast<const float2 *>(p);
}
__device__ __forceinline__ float2 ld_pair(const __half *p)
{
    return __half22float2(*reinterpret_cast<const __half2 *>(p));
}
__device__ __forceinline__ void st_pair(float *p, float2 v)
{
    *reinterpret_cast<float2 *>(p) = v;
}
__device__ __forceinline__ void st_pair(__half *p, float2 v)
{
    *reinterpret_cast<__half2 *>(p) = __floats2half2_rn(v.x, v.y);
}

template <class pop_t, int TX, int TY, int NT, int NP = 1>
struct TmaPairSmem {
    static constexpr int NW = NT / 32;
    static constexpr int PX = 16 / sizeof(pop_t);
    static constexpr int RP = TX + 8;              // density rows from x = X0 - 4
    static constexpr int PP = TX + PX;             // population rows (pin_x0)
    static constexpr int PLANE = TY * PP;
    static constexpr size_t PIN_BYTES = sizeof(pop_t) * 8 * PLANE;
    static constexpr int NRHO = (TY + 4) * RP;
    static constexpr int MP = TX + 4, MH = TY + 2;  // mu of halo column a at a + 1
    static constexpr int NRING = RingStage<float, TX, TY>::N;
    static constexpr int NMU = NP * MP * MH;        // mu, or (NP = 3) the tensor of Eq. 9
    static constexpr int XW = TX + 2;              // exchange slots per warp
    static constexpr int NXCH = 2 * NW * XW;
    // as TmaSmem
    static constexpr int NFIXP = (SeamLists<TX, TY>::POP * sizeof(pop_t) + 3) / 4;
    static constexpr int NSHARE = NRING + NFIXP > NXCH ? NRING + NFIXP : NXCH;
    static_assert(NMU >= SeamLists<TX, TY>::RHO, "density fix-ups staged in s_mu");
    static constexpr size_t bar_offset =
        (PIN_BYTES + sizeof(float) * (NRHO + NSHARE + NMU) + 15) / 16 * 16;
    static constexpr size_t bytes = bar_offset + 16;
    static constexpr unsigned tx_rho = sizeof(float) * NRHO;
    static constexpr unsigned tx_pops = PIN_BYTES;
    static_assert((PLANE * sizeof(pop_t)) % 128 == 0, "TMA destinations");
    static_assert(NRHO % 2 == 0 && NSHARE % 2 == 0 && NMU % 2 == 0 && XW % 2 == 0 &&
                      PP % 2 == 0,
                  "pair-aligned sub-arrays");
};

// PT: the baseline force of Eq. 5, as for step_tile_tma.
template <class S, int TX, int TY, int NT, int PARITY, int EDGE, bool PT = false>
__device__ __forceinline__ bool step_tile_tma_pair(const Lattice &L, int cur, int X0,
                                                   int Y0, unsigned char *smem_raw,
                                                   TileMaps maps,
                                                   unsigned long long *bar,
                                                   unsigned phase)
{
    using rho_t = typename S::rho_t;
    using pop_t = typename S::pop_t;
    using TS = TmaPairSmem<pop_t, TX, TY, NT, PT ? 3 : 1>;
    static_assert(TX == 64, "lanes map to x pairs");
    static_assert(sizeof(rho_t) == 4 && sizeof(typename S::real) == 4, "FP32 arithmetic");
    static_assert(!PT || EDGE != 2, "the pressure-tensor force has no wall rule");
    constexpr int NW = TS::NW, PER = TY / NW;
    static_assert(PER * NW == TY && PER >= 2, "warps own whole row blocks");
    constexpr int RP = TS::RP, PP = TS::PP, PLANE = TS::PLANE, MP = TS::MP, MH = TS::MH;
    constexpr int XW = TS::XW;
    pop_t *s_pin = reinterpret_cast<pop_t *>(smem_raw);             // [8][TY][PP]
    float *s_rho = reinterpret_cast<float *>(smem_raw + TS::PIN_BYTES);  // [TY + 4][RP]
    float *s_ring = s_rho + TS::NRHO;
    float *s_mu = s_ring + TS::NSHARE;                    // [MH][MP]
    float *s_up = s_ring;                                 // [NW][XW], after step 2
    float *s_down = s_up + NW * XW;                       // [NW][XW]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nxt = cur ^ 1;
    // EDGE: 0 interior tile; an edge tile (tile_kind TILE_SEAM), whose halo
    // wraps around a periodic edge, of a periodic lattice (1) or of any
    // lattice, walls included (2)
    constexpr bool seam = EDGE != 0, walls_ok = EDGE == 2;

    // 1. Loads (bar, phase, seam tiles: as step_tile_tma).
    if (threadIdx.x == 0) {
        mbar_expect_tx(&bar[0],
                       TS::tx_rho + (seam ? 0u : RingStage<float, TX, TY>::bulk_bytes));
        tma_load_2d(s_rho, maps.rho, X0 - 4, Y0 - 2, &bar[0]);
        mbar_expect_tx(&bar[1], TS::tx_pops);
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            const int plane = PARITY == 0 ? i - 1 : opp(i) - 1;
            const int y0 = PARITY == 0 ? Y0 : Y0 - ey(i);
            tma_load_3d(s_pin + (i - 1) * PLANE, maps.pops,
                        X0 + pin_x0<PARITY, TS::PX>(i), y0, plane, &bar[1]);
        }
    }
    pop_t *fix_pop = reinterpret_cast<pop_t *>(s_ring + TS::NRING);
    if (seam) {
        stage_ring_wrapped<float, TX, TY, NT, walls_ok>(L, cur, X0, Y0, s_ring);
        seam_fix_load<S, TX, TY, NT, PARITY, walls_ok>(L, cur, X0, Y0, s_mu, fix_pop);
    } else {
        stage_ring<float, TX, TY>(L, cur, X0, Y0, s_ring, &bar[0]);
    }
    cp_async_wait_all();
    if (!tma_landed(bar, 0, phase, L.err, L.wait_cycles)) return false;
    if (seam) {
        seam_rho_apply<float, TX, TY, NT, RP, walls_ok>(L, X0, Y0, s_mu, s_rho);
        __syncthreads();
    }

    // 2. Partial sums into the halo's tile-edge nodes (order of
    //    load_rho_stored); halo (lx, ly) is staged at row ly, column lx + 2.
    combine_ring<float, TX, TY, NT, RP>(s_rho, s_ring, TX, TY);
    __syncthreads();
    // edge tiles at a wall: the solid row's density (Eq. 28)
    const SeamEdges edge = seam_edges<walls_ok>(L, X0, Y0, TX, TY);
    if (walls_ok) wall_rho_rows<float, TX, NT, RP>(edge, s_rho);

    // 3. mu at halo column a (x = X0 - 1 + a) and row b (r = Y0 - 1 + b),
    //    stored at s_mu[b][a + 1]; its density is staged at (b + 1, a + 3).
    //    Lane l takes the pair a = 2l + 1, 2l + 2 down its warp's rows with a
    //    rolling window; columns 0 and TX + 1 one node at a time.
    const Consts<float> &K = consts<float>(L);
    const float ref = S::offset ? K.rho_ref : 0.0f;
    const float2 ref2 = p2(ref);
    constexpr int NP1 = MP * MH;  // one plane of s_mu
    if constexpr (PT) {
        // the tensor of Eq. 9 in three planes (xx, xy, yy), in the
        // arithmetic of pt_tile, with the window walk of the mu branch
        const EosT<float> &eos = K.eos;
        const float kappa = K.kappa;
        const float2 kap = p2(kappa), mkap = p2(-kappa), mhkap = p2(-0.5f * kappa);
        const int b0 = (warp * MH) / NW, b1 = ((warp + 1) * MH) / NW;
        const int c0 = 2 * lane + 4;
        Row2 d = row2(s_rho, b0 * RP + c0), m = row2(s_rho, (b0 + 1) * RP + c0);
        for (int b = b0; b < b1; ++b) {
            const Row2 u = row2(s_rho, (b + 2) * RP + c0);
            const float2 rho = S::offset ? padd(m.c, ref2) : m.c;
            float2 gx, gy;
            grad2(u, m, d, gx, gy);
            const float2 lap = lap2(u, m, d);
            const float2 iso = pfma(mhkap, pfma(gx, gx, pmul(gy, gy)),
                                    pfma(pmul(mkap, rho), lap, p0_bulk2(eos, rho)));
            float *o = s_mu + b * MP + 2 * lane + 2;
            *reinterpret_cast<float2 *>(o) = pfma(pmul(kap, gx), gx, iso);
            *reinterpret_cast<float2 *>(o + NP1) = pmul(pmul(kap, gx), gy);
            *reinterpret_cast<float2 *>(o + 2 * NP1) = pfma(pmul(kap, gy), gy, iso);
            d = m;
            m = u;
        }
        for (int t = threadIdx.x; t < 2 * MH; t += NT) {
            const int ae = (t & 1) ? TX + 1 : 0, b = t >> 1;
            const int c = (b + 1) * RP + ae + 3;
            const float rho = s_rho[c] + ref;
            float gx, gy;
            grad9<float, RP>(s_rho, c, gx, gy);
            const float lap = lap9<float, RP>(s_rho, c);
            const float iso = p0_bulk(eos, rho) - kappa * rho * lap -
                              0.5f * kappa * (gx * gx + gy * gy);
            float *o = s_mu + b * MP + ae + 1;
            o[0] = iso + kappa * gx * gx;
            o[NP1] = kappa * gx * gy;
            o[2 * NP1] = iso + kappa * gy * gy;
        }
    } else {
        const EosT<float> &eos = K.eos;
        const float2 mkappa = p2(-K.kappa);
        const int b0 = (warp * MH) / NW, b1 = ((warp + 1) * MH) / NW;
        const int c0 = 2 * lane + 4;
        Row2 d = row2(s_rho, b0 * RP + c0), m = row2(s_rho, (b0 + 1) * RP + c0);
        for (int b = b0; b < b1; ++b) {
            const Row2 u = row2(s_rho, (b + 2) * RP + c0);
            float2 mp;
            if (walls_ok && ((edge.wb && b == 0) || (edge.wt && b >= edge.hy + 1))) {
                // solid rows of wall tiles: surface values (wall_mu)
                wall_mu<S, RP>(L, edge, b, (b + 1) * RP + c0, s_rho, mp.x);
                wall_mu<S, RP>(L, edge, b, (b + 1) * RP + c0 + 1, s_rho, mp.y);
            } else {
                const float2 rho = S::offset ? padd(m.c, ref2) : m.c;
                mp = pfma(mkappa, lap2(u, m, d), mu_bulk2(eos, rho));
            }
            *reinterpret_cast<float2 *>(s_mu + b * MP + 2 * lane + 2) = mp;
            d = m;
            m = u;
        }
        for (int t = threadIdx.x; t < 2 * MH; t += NT) {
            const int ae = (t & 1) ? TX + 1 : 0, b = t >> 1;
            const int c = (b + 1) * RP + ae + 3;
            float mv;
            if (!(walls_ok && wall_mu<S, RP>(L, edge, b, c, s_rho, mv)))
                mv = mu_bulk(eos, s_rho[c] + ref) - K.kappa * lap9<float, RP>(s_rho, c);
            s_mu[b * MP + ae + 1] = mv;
        }
    }
    // the populations were in flight during steps 2 and 3; the barrier also
    // publishes s_mu
    if (!tma_landed(bar, 1, phase, L.err, L.wait_cycles)) return false;
    if (PARITY == 1 && seam) {
        seam_pop_apply<pop_t, TX, TY, NT, PLANE, PP, TS::PX, walls_ok>(L, X0, Y0, fix_pop, s_pin);
        __syncthreads();
    }

    // 4. Force, collision, in-place streaming and the register hand-over for
    //    the pair at columns x0, x0 + 1 of rows ly0 .. ly0 + PER - 1.
    const int x0 = 2 * lane, ly0 = warp * PER;
    const float2 tau = p2(K.tau), omega = p2(K.omega), third = p2(1.0f / 3.0f);
    pop_t *A = (pop_t *)L.pops;
    rho_t *Rn = (rho_t *)L.rho[nxt];
    rho_t *const *ring = (rho_t *const *)L.ring[nxt];
    int woff[9];  // 32-bit: the TMA maps exist only when 8 planes fit
#pragma unroll
    for (int i = 1; i < 9; ++i)
        woff[i] = PARITY == 0 ? (opp(i) - 1) * (int)L.plane
                              : (i - 1) * (int)L.plane + ey(i) * L.pitch + ex(i);
    // wall tiles: rows 0 .. hy - 1 hold fluid (as step_tile_tma)
    const int hy = walls_ok ? edge.hy : TY;
    const bool has_l = lane > 0, has_r = lane < 31;
    // windows: density of tile row ly at staged row ly + 2, column x0 + 4;
    // mu of tile row ly at s_mu row ly + 1, column x0 + 2
    Row2 rd = row2(s_rho, (ly0 + 1) * RP + x0 + 4), rm = row2(s_rho, (ly0 + 2) * RP + x0 + 4);
    Row2 md = row2(s_mu, ly0 * MP + x0 + 2), mm = row2(s_mu, (ly0 + 1) * MP + x0 + 2);
    // PT: md / mm hold P_xx; the windows of P_xy and P_yy
    Row2 xyd{}, xym{}, yyd{}, yym{};
    if constexpr (PT) {
        xyd = row2(s_mu + NP1, ly0 * MP + x0 + 2);
        xym = row2(s_mu + NP1, (ly0 + 1) * MP + x0 + 2);
        yyd = row2(s_mu + 2 * NP1, ly0 * MP + x0 + 2);
        yym = row2(s_mu + 2 * NP1, (ly0 + 1) * MP + x0 + 2);
    }
    float2 pend = p2(0.0f), up_prev = p2(0.0f), first = p2(0.0f);
    float pend_c = 0.0f, up_prev_c = 0.0f, first_c = 0.0f;
    const int slot_c = TX + (lane == 31);        // exchange slot of a column
    const int xc = lane == 0 ? X0 - 1 : X0 + TX;  // ring column of the lane
    const int cls_c = lane == 0 ? R_R : R_L;
    // this tile, and the tile of the ring column a lane feeds (classes L and
    // R share one index layout)
    const int bx = X0 / TX, by = Y0 / TY;
    const int bxl = neighbour_tile(X0, -1, TX, L.nx, seam), bxr = neighbour_tile(X0, 1, TX, L.nx, seam);
    const int byb = neighbour_tile(Y0, -1, TY, L.nyf, seam), byt = neighbour_tile(Y0, 1, TY, L.nyf, seam);
    const int bxc = lane == 0 ? bxl : bxr;
    const bool col_lane = lane == 0 || lane == 31;
    pop_t *Arow = A + (long long)(Y0 + ly0) * L.pitch + X0 + x0;
    // corrections of odd-step write offsets across the periodic edges
    const int wrap_y = L.nyf * L.pitch;
    const int cxl = (PARITY == 1 && seam && X0 == 0 && lane == 0) ? L.nx : 0;
    const int cxr = (PARITY == 1 && seam && X0 + TX >= L.nx && lane == 31) ? -L.nx : 0;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int ly = ly0 + k;
        const Row2 ru = row2(s_rho, (ly + 3) * RP + x0 + 4);
        const Row2 mu = row2(s_mu, (ly + 2) * MP + x0 + 2);
        Row2 xyu{}, yyu{};
        if constexpr (PT) {
            xyu = row2(s_mu + NP1, (ly + 2) * MP + x0 + 2);
            yyu = row2(s_mu + 2 * NP1, (ly + 2) * MP + x0 + 2);
        }
        float2 same = p2(0.0f), up = p2(0.0f), down = p2(0.0f);
        float same_c = 0.0f, up_c = 0.0f, down_c = 0.0f;
        if (!walls_ok || ly < hy) {  // warp-uniform
            float2 f[9];
#pragma unroll
            for (int i = 1; i < 9; ++i) {
                const pop_t *src =
                    s_pin + (i - 1) * PLANE + ly * PP + x0 + pin_col<PARITY, TS::PX>(i);
                if (PARITY == 0 || ex(i) == 0)
                    f[i] = ld_pair(src);
                else
                    f[i] = make_float2(ld_real(src), ld_real(src + 1));
            }
            const float2 drho = rm.c;
            const float2 rho = S::offset ? padd(drho, ref2) : drho;
            float2 grx, gry, gmx, gmy, Fx, Fy;
            grad2(ru, rm, rd, grx, gry);
            grad2(mu, mm, md, gmx, gmy);
            if constexpr (PT) {
                // Eq. 5: F = -div(P) + grad(cs^2 rho)
                float2 xy_x, xy_y, yy_x, yy_y;
                grad2(xyu, xym, xyd, xy_x, xy_y);
                grad2(yyu, yym, yyd, yy_x, yy_y);
                Fx = psub(pmul(grx, third), padd(gmx, xy_y));
                Fy = psub(pmul(gry, third), padd(xy_x, yy_y));
            } else {
                Fx = psub(pmul(grx, third), pmul(rho, gmx));
                Fy = psub(pmul(gry, third), pmul(rho, gmy));
            }
            float2 fp[9];
            collide2(f, drho, rho, Fx, Fy, tau, omega, fp);
            // wall rows (halfway bounce-back, Sec. IV)
            const bool wall_b = walls_ok && edge.wb && ly == 0;
            const bool wall_t = walls_ok && edge.wt && ly == hy - 1;
            {
                // odd steps on seam tiles: a target across a periodic edge is
                // brought back by one lattice length (the x-shifted directions
                // are stored one node at a time); a population heading into a
                // solid row goes to the node's own slot opp(i)
                const int cyb = (PARITY == 1 && seam && edge.yb && ly == 0) ? wrap_y : 0;
                const int cyt = (PARITY == 1 && seam && edge.yt && ly == TY - 1) ? -wrap_y : 0;
#pragma unroll
                for (int i = 1; i < 9; ++i) {
                    const bool into_wall = PARITY == 1 && ((ey(i) < 0 && wall_b) ||
                                                           (ey(i) > 0 && wall_t));
                    pop_t *dst = into_wall ? Arow + (opp(i) - 1) * (int)L.plane
                                           : Arow + woff[i] + (ey(i) < 0 ? cyb : ey(i) > 0 ? cyt : 0);
                    if (PARITY == 0 || ex(i) == 0 || into_wall) {
                        if (CPLBM_IN_POPS(L, dst, 2)) st_pair(dst, fp[i]);
                    } else {
                        pop_t *d0 = dst + (ex(i) < 0 ? cxl : 0), *d1 = dst + 1 + (ex(i) > 0 ? cxr : 0);
                        if (CPLBM_IN_POPS(L, d0, 1)) st_real(d0, fp[i].x);
                        if (CPLBM_IN_POPS(L, d1, 1)) st_real(d1, fp[i].y);
                    }
                }
            }

            // lane-neighbour parts of the hand-over
            const float f1l = __shfl_up_sync(0xffffffffu, fp[1].y, 1);
            const float f5l = __shfl_up_sync(0xffffffffu, fp[5].y, 1);
            const float f8l = __shfl_up_sync(0xffffffffu, fp[8].y, 1);
            const float f3r = __shfl_down_sync(0xffffffffu, fp[3].x, 1);
            const float f6r = __shfl_down_sync(0xffffffffu, fp[6].x, 1);
            const float f7r = __shfl_down_sync(0xffffffffu, fp[7].x, 1);
            same = make_float2((fp[0].x + (has_l ? f1l : 0.0f)) + fp[3].y,
                               (fp[0].y + fp[1].x) + (has_r ? f3r : 0.0f));
            up = make_float2((fp[2].x + (has_l ? f5l : 0.0f)) + fp[6].y,
                             (fp[2].y + fp[5].x) + (has_r ? f6r : 0.0f));
            down = make_float2((fp[4].x + (has_l ? f8l : 0.0f)) + fp[7].y,
                               (fp[4].y + fp[8].x) + (has_r ? f7r : 0.0f));
            // what leaves into a solid row comes back to the node
            if (wall_b) same = padd(same, padd(padd(fp[4], fp[7]), fp[8]));
            if (wall_t) same = padd(same, padd(padd(fp[2], fp[5]), fp[6]));
            // ring columns: lane 0 feeds x = X0 - 1 (f*_3; f*_6 up; f*_7 down)
            // from its first node, lane 31 feeds x = X0 + TX (f*_1; f*_5 up;
            // f*_8 down) from its second
            same_c = lane == 0 ? fp[3].x : fp[1].y;
            up_c = lane == 0 ? fp[6].x : fp[5].y;
            down_c = lane == 0 ? fp[7].x : fp[8].y;
        }
        Arow += L.pitch;
        const bool row_ok = !walls_ok || ly - 1 < hy;
        if (k == 0) {
            *reinterpret_cast<float2 *>(s_down + warp * XW + x0) = down;
            if (col_lane) s_down[warp * XW + slot_c] = down_c;
            pend = same;
            pend_c = same_c;
        } else {
            const float2 done = padd(pend, down);  // row ly - 1
            const float done_c = pend_c + down_c;
            if (k == 1) {
                first = done;
                first_c = done_c;
            } else if (row_ok) {
                put_rho(L, nxt, Rn, (long long)(Y0 + ly - 1) * L.pitch + X0 + x0, done);
                if (col_lane) put_ring(L, nxt, ring, cls_c, ring_index(L, R_L, bxc, by, Y0 + ly - 1, xc), done_c);
            }
            pend = padd(same, up_prev);
            pend_c = same_c + up_prev_c;
        }
        up_prev = up;
        up_prev_c = up_c;
        rd = rm;
        rm = ru;
        md = mm;
        mm = mu;
        if constexpr (PT) {
            xyd = xym;
            xym = xyu;
            yyd = yym;
            yym = yyu;
        }
    }
    *reinterpret_cast<float2 *>(s_up + warp * XW + x0) = up_prev;
    if (col_lane) s_up[warp * XW + slot_c] = up_prev_c;
    __syncthreads();
    {
        float2 top = pend;
        float top_c = pend_c;
        if (warp + 1 < NW) {
            top = padd(top, *reinterpret_cast<const float2 *>(s_down + (warp + 1) * XW + x0));
            top_c += s_down[(warp + 1) * XW + slot_c];
        }
        if (!walls_ok || ly0 + PER - 1 < hy) {
            put_rho(L, nxt, Rn, (long long)(Y0 + ly0 + PER - 1) * L.pitch + X0 + x0, top);
            if (col_lane) put_ring(L, nxt, ring, cls_c, ring_index(L, R_L, bxc, by, Y0 + ly0 + PER - 1, xc), top_c);
        }
        if (warp > 0) {
            first = padd(first, *reinterpret_cast<const float2 *>(s_up + (warp - 1) * XW + x0));
            first_c += s_up[(warp - 1) * XW + slot_c];
        }
        if (!walls_ok || ly0 < hy) {
            put_rho(L, nxt, Rn, (long long)(Y0 + ly0) * L.pitch + X0 + x0, first);
            if (col_lane) put_ring(L, nxt, ring, cls_c, ring_index(L, R_L, bxc, by, Y0 + ly0, xc), first_c);
        }
    }
    // ring rows below and above the tile, with their corners (none across a
    // wall)
    if (warp == 0 && !(walls_ok && edge.wb)) {
        put_ring(L, nxt, ring, R_T, ring_index(L, R_T, bx, byb, Y0 - 1, X0 + x0), *reinterpret_cast<const float2 *>(s_down + x0));
        if (lane == 0) put_ring(L, nxt, ring, R_TR, ring_index(L, R_TR, bxl, byb, Y0 - 1, X0 - 1), s_down[TX]);
        if (lane == 31) put_ring(L, nxt, ring, R_TL, ring_index(L, R_TL, bxr, byb, Y0 - 1, X0 + TX), s_down[TX + 1]);
    }
    if (warp == NW - 1 && !(walls_ok && edge.wt)) {
        put_ring(L, nxt, ring, R_B, ring_index(L, R_B, bx, byt, Y0 + TY, X0 + x0), up_prev);
        if (lane == 0) put_ring(L, nxt, ring, R_BR, ring_index(L, R_BR, bxl, byt, Y0 + TY, X0 - 1), up_prev_c);
        if (lane == 31) put_ring(L, nxt, ring, R_BL, ring_index(L, R_BL, bxr, byt, Y0 + TY, X0 + TX), up_prev_c);
    }
    return true;
}

// Whether a (precision, tile) pair has the two-nodes-per-lane TMA path (FP32
// arithmetic, FP32 or FP16 storage), and the CTA size of a shape: four rows
// per warp on that path.
template <class S>
struct IsPairStorage {
    static constexpr bool value = sizeof(typename S::real) == 4 &&
                                  sizeof(typename S::rho_t) == 4;
};
template <class S, int TX, int TY>
constexpr int step_threads()
{
    return (TX == 64 && IsPairStorage<S>::value) ? 8 * TY : STEP_THREADS;
}
template <class S, int TX, int TY, int NT>
struct HasTmaPair {
    static constexpr bool value = TX == 64 && IsPairStorage<S>::value &&
                                  TY % (NT / 32) == 0 && TY / (NT / 32) >= 2;
};

// Whether a (precision, tile) pair has the TMA interior path.
template <class S, int TX, int TY, int NT>
struct HasTma {
    static constexpr bool value = TX == 32 && (TY % (NT / 32)) == 0;
};

// Resident CTAs a pair-path kernel asks for (__launch_bounds__): 640 / NT,
// five of 128 threads at 96 registers; six for FP16 storage at 64 x 16
// (80 registers), whose TMA path needs 31 KB of shared memory, so six fit
// when a launch has no general tile (launch_shape).
template <class S, int TX, int TY, int NT>
constexpr int pair_min_ctas()
{
    return sizeof(typename S::pop_t) == 2 && NT == 128 ? 6 : 640 / NT;
}

// WALLS: the kernel of walled lattices, whose edge tiles include the wall
// rows; periodic lattices take the variant without the wall code, so that it
// does not weigh on the code the interior tiles run.
template <class S, int TX, int TY, int NT, int PARITY, bool WALLS>
__global__ void __launch_bounds__(NT, HasTmaPair<S, TX, TY, NT>::value
                                          ? pair_min_ctas<S, TX, TY, NT>() : 0)
    step_kernel(const Lattice L, int cur, int seams, const __grid_constant__ TmaMaps maps)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // Odd steps walk the tile grid backwards: the tiles a step writes last,
    // still in L2, are the first the next step reads.
    const int bx = PARITY ? gridDim.x - 1 - blockIdx.x : blockIdx.x;
    const int by = PARITY ? gridDim.y - 1 - blockIdx.y : blockIdx.y;
    const int X0 = bx * TX, Y0 = by * TY;
    // seams: seam_bits of the lattice, for the kernels whose TMA path takes
    // seam tiles (0 for the others)
    const int kind = tile_kind(L, TX, TY, bx, by, seams);
    const bool interior = kind == TILE_INTERIOR;
    if constexpr (HasTma<S, TX, TY, NT>::value || HasTmaPair<S, TX, TY, NT>::value) {
        if (kind != TILE_GENERAL && maps.valid) {
            __shared__ __align__(8) unsigned long long bar[2];
            if (threadIdx.x == 0) {
                mbar_init(&bar[0], 1);
                mbar_init(&bar[1], 1);
            }
            __syncthreads();
            const TileMaps tm{&maps.pops, &maps.rho[cur]};
            if constexpr (HasTma<S, TX, TY, NT>::value) {
                if (interior)
                    step_tile_tma<S, TX, TY, NT, PARITY, 0>(L, cur, X0, Y0, smem_raw,
                                                            tm, bar, 0);
                else
                    step_tile_tma<S, TX, TY, NT, PARITY, WALLS ? 2 : 1>(L, cur, X0, Y0,
                                                                        smem_raw, tm, bar, 0);
            } else {
                if (interior)
                    step_tile_tma_pair<S, TX, TY, NT, PARITY, 0>(L, cur, X0, Y0,
                                                                 smem_raw, tm, bar, 0);
                else
                    step_tile_tma_pair<S, TX, TY, NT, PARITY, WALLS ? 2 : 1>(
                        L, cur, X0, Y0, smem_raw, tm, bar, 0);
            }
            return;
        }
    }
    if (interior)
        step_tile<S, TX, TY, NT, PARITY, true>(L, cur, X0, Y0, smem_raw);
    else
        step_tile<S, TX, TY, NT, PARITY, false>(L, cur, X0, Y0, smem_raw);
}

template <class S, int TX, int TY>
static cudaError_t launch_shape(const Lattice &L, int parity, int cur,
                                cudaStream_t s, const TmaMaps *maps)
{
    using real = typename S::real;
    constexpr int NT = step_threads<S, TX, TY>();
    const size_t smem_v4 = StepSmem<real, TX, TY>::bytes;
    size_t smem_tma = 0;
    if constexpr (HasTma<S, TX, TY, NT>::value) smem_tma = TmaSmem<S, TX, TY>::bytes;
    if constexpr (HasTmaPair<S, TX, TY, NT>::value)
        smem_tma = TmaPairSmem<typename S::pop_t, TX, TY, NT>::bytes;
    const size_t smem_max = smem_v4 > smem_tma ? smem_v4 : smem_tma;
    TmaMaps m{};
    if (maps && maps->valid && maps->tx == TX && maps->ty == TY) m = *maps;
    // kernels of periodic (index 0) and walled (1) lattices, by parity
    void (*const kern[2][2])(const Lattice, int, int, const TmaMaps) = {
        {step_kernel<S, TX, TY, NT, 0, false>, step_kernel<S, TX, TY, NT, 1, false>},
        {step_kernel<S, TX, TY, NT, 0, true>, step_kernel<S, TX, TY, NT, 1, true>}};
    static int configured = -1;  // device the attributes were set on
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (configured != dev) {
        for (int w = 0; w < 2 && e == cudaSuccess; ++w)
            for (int p = 0; p < 2 && e == cudaSuccess; ++p)
                e = cudaFuncSetAttribute(kern[w][p],
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_max);
        if (e != cudaSuccess) return e;
        configured = dev;
    }
    // Tile classes (tile_kind): the TMA paths also take the seam tiles of
    // periodic edges.
    const int ntx = (L.nx + TX - 1) / TX, nty = (L.nyf + TY - 1) / TY;
    const int seams = HasTma<S, TX, TY, NT>::value || HasTmaPair<S, TX, TY, NT>::value
                          ? seam_bits(L, TX, TY) : 0;
    // When every tile is interior or an edge tile and the maps are valid,
    // every tile takes the TMA path (step_kernel has no general fallback on
    // it), so the launch needs only that path's shared memory, and more CTAs
    // fit: x periodic seams over full tiles, and in y either periodic seams
    // over full tiles or walls whose top tile is full or at least 4 rows
    // high (otherwise the tile below it is general).
    const int ry = L.nyf % TY;
    const bool all_tma = m.valid && (seams & 1) && L.nx % TX == 0 &&
                         (L.walls ? ((seams & 4) && (ry == 0 || ry >= 4))
                                  : ((seams & 2) && ry == 0));
    const size_t smem = (all_tma && smem_tma > 0) ? smem_tma : smem_max;
    dim3 grid(ntx, nty);
    kern[L.walls ? 1 : 0][parity & 1]<<<grid, NT, smem, s>>>(L, cur, seams, m);
    return cudaGetLastError();
}

// Tile shapes with a compiled kernel (all precisions).
#define CPLBM_STEP_SHAPES(X) X(32, 16) X(32, 24) X(32, 32) X(64, 16) X(64, 32)

// ---------------------------------------------------------------------------
// Batched step of lattices of one geometry: step_kernel's tile grid,
// flattened into grid x, with one grid row per lattice.  The descriptors and
// tensor maps come as the kernel parameter (UniformGroup), so a CTA starts
// its copies with no global read before them, and the tile class follows
// from the tile position as in step_kernel.  Only for groups whose every
// tile takes a TMA path; WALLS as for step_kernel.
// ---------------------------------------------------------------------------
template <class S, int TX, int TY, int NT, int PARITY, bool WALLS>
__global__ void __launch_bounds__(NT, HasTmaPair<S, TX, TY, NT>::value
                                          ? pair_min_ctas<S, TX, TY, NT>() : 0)
    step_uniform_kernel(int cur, int seams, int ntx, int nty,
                        const __grid_constant__ UniformGroup G)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long bar[2];
    // lattice by lattice, each in tile-grid order; odd steps walk the order
    // backwards (step_kernel)
    const int c = PARITY ? (int)gridDim.x - 1 - (int)blockIdx.x : (int)blockIdx.x;
    const int per = ntx * nty;  // tiles per lattice
    const int k = c / per;
    const int t = c - k * per;
    const int by = t / ntx, bx = t - by * ntx;
    const Lattice &L = G.L[k];
    const int X0 = bx * TX, Y0 = by * TY;
    const bool interior = tile_kind(L, TX, TY, bx, by, seams) == TILE_INTERIOR;
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
    }
    __syncthreads();
    const TileMaps tm{&G.pops[k], &G.rho[k]};
    if constexpr (HasTma<S, TX, TY, NT>::value) {
        if (interior)
            step_tile_tma<S, TX, TY, NT, PARITY, 0>(L, cur, X0, Y0, smem_raw, tm, bar, 0);
        else
            step_tile_tma<S, TX, TY, NT, PARITY, WALLS ? 2 : 1>(L, cur, X0, Y0, smem_raw,
                                                                tm, bar, 0);
    } else {
        if (interior)
            step_tile_tma_pair<S, TX, TY, NT, PARITY, 0>(L, cur, X0, Y0, smem_raw, tm, bar,
                                                         0);
        else
            step_tile_tma_pair<S, TX, TY, NT, PARITY, WALLS ? 2 : 1>(L, cur, X0, Y0,
                                                                     smem_raw, tm, bar, 0);
    }
}

// ---------------------------------------------------------------------------
// Batched step: many independent lattices of different sizes and physics in
// one launch.  Each CTA takes `per_cta` consecutive work items (tiles of the
// work list, in list order, backwards on odd steps as step_kernel walks its
// grid); the hardware hands out the CTAs as others finish, so there is no
// work counter and no per-item wait on one.  The CTA stages its items in
// shared memory with one load, so no tile waits on a global read of the
// next item.  Consecutive items mostly belong to one lattice: its
// descriptor is copied to shared memory when the CTA's lattice changes, not
// per item, and per_cta
// (lbm_batch_autotune) trades that saving against the balance of the last
// CTAs.  The tensor maps come as a kernel parameter (BatchMaps, up to
// BATCH_LAUNCH_LATTICES lattices from inst0 on): a map in global memory,
// written by the host, would need a proxy fence and a fetch in every CTA
// before its first copy, which cost a sixth of the step time at one item
// per CTA.  Little state lives across the tile bodies (the
// item index, the mbarrier phase, the wait status).  GEN = false compiles
// the kernel without the general tile path, for work lists whose every item
// takes a TMA path: the general body is what makes the compiler spill, and
// its shared memory is the larger one for the FP16 storage.  Without it, a
// wait that gives up leaves the CTA's remaining tiles as they were (the
// error flag is raised), as step_kernel does.
// ---------------------------------------------------------------------------
template <class S, int TX, int TY, int NT, int PARITY, bool GEN>
__global__ void __launch_bounds__(NT, HasTmaPair<S, TX, TY, NT>::value
                                          ? pair_min_ctas<S, TX, TY, NT>()
                                          : (sizeof(typename S::real) == 8 ? 2 : 4))
    step_batch_kernel(const Lattice *__restrict__ lats,
                      const WorkItem *__restrict__ items, int n_items, int cur,
                      int per_cta, int inst0, const __grid_constant__ BatchMaps maps)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ Lattice sL;
    __shared__ __align__(8) unsigned long long bar[2];
    __shared__ int4 s_items[BATCH_MAX_PER_CTA];
    static_assert(sizeof(Lattice) % sizeof(int) == 0, "descriptor copy");
    static_assert(sizeof(WorkItem) == sizeof(int4), "work item staging");
    constexpr bool kTma = HasTma<S, TX, TY, NT>::value || HasTmaPair<S, TX, TY, NT>::value;
    const int w0 = (int)blockIdx.x * per_cta;
    const int cnt = min(per_cta, n_items - w0);
    for (int q = threadIdx.x; q < cnt; q += NT)
        s_items[q] = reinterpret_cast<const int4 *>(items)[PARITY ? n_items - 1 - (w0 + q)
                                                                   : w0 + q];
    if (kTma && threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
    }
    __syncthreads();
    unsigned phase = 0;    // next phase of the mbarriers
    bool tma_ok = true;    // a wait that gave up sends the rest to the general path
    for (int j = 0; j < cnt; ++j) {
        const int4 it = s_items[j];   // (inst, bx, by, kind)
        if (j == 0 || s_items[j - 1].x != it.x) {
            const int *src = reinterpret_cast<const int *>(lats + it.x);
            int *dst = reinterpret_cast<int *>(&sL);
            for (int q = threadIdx.x; q < (int)(sizeof(Lattice) / sizeof(int)); q += NT)
                dst[q] = src[q];
        }
        __syncthreads();
        const int kind = it.w & 3;
        const int x0 = it.y * TX, y0 = it.z * TY;
        bool done = false;
        if constexpr (kTma) {
            if (tma_ok && kind != TILE_GENERAL && !(it.w & ITEM_NO_TMA)) {
                const TileMaps m{&maps.pops[it.x - inst0], &maps.rho[it.x - inst0]};
                // lattices of a batch may or may not have walls: edge tiles
                // take the variant that handles both
                if constexpr (HasTma<S, TX, TY, NT>::value) {
                    if (kind == TILE_INTERIOR)
                        tma_ok = step_tile_tma<S, TX, TY, NT, PARITY, 0>(
                            sL, cur, x0, y0, smem_raw, m, bar, phase);
                    else
                        tma_ok = step_tile_tma<S, TX, TY, NT, PARITY, 2>(
                            sL, cur, x0, y0, smem_raw, m, bar, phase);
                } else {  // two nodes per lane (64-wide FP32-arithmetic shapes)
                    if (kind == TILE_INTERIOR)
                        tma_ok = step_tile_tma_pair<S, TX, TY, NT, PARITY, 0>(
                            sL, cur, x0, y0, smem_raw, m, bar, phase);
                    else
                        tma_ok = step_tile_tma_pair<S, TX, TY, NT, PARITY, 2>(
                            sL, cur, x0, y0, smem_raw, m, bar, phase);
                }
                phase ^= 1u;
                done = true;
            }
        }
        if constexpr (GEN) {
            if (!done) {
                if (kind == TILE_INTERIOR)
                    step_tile<S, TX, TY, NT, PARITY, true>(sL, cur, x0, y0, smem_raw);
                else
                    step_tile<S, TX, TY, NT, PARITY, false>(sL, cur, x0, y0, smem_raw);
            }
        } else {
            (void)done;
        }
        __syncthreads();  // smem and sL are reused by the next item
    }
}

template <class S, int TX, int TY>
static cudaError_t launch_batch_shape(const BatchList &w, int parity, int cur,
                                      cudaStream_t s)
{
    using real = typename S::real;
    constexpr int NT = step_threads<S, TX, TY>();
    constexpr bool kTma = HasTma<S, TX, TY, NT>::value || HasTmaPair<S, TX, TY, NT>::value;
    size_t smem_tma = 0;
    if constexpr (HasTma<S, TX, TY, NT>::value) smem_tma = TmaSmem<S, TX, TY>::bytes;
    if constexpr (HasTmaPair<S, TX, TY, NT>::value)
        smem_tma = TmaPairSmem<typename S::pop_t, TX, TY, NT>::bytes;
    const size_t smem_gen = StepSmem<real, TX, TY>::bytes > smem_tma
                                ? StepSmem<real, TX, TY>::bytes : smem_tma;
    // [general path compiled in][parity]
    void (*kern[2][2])(const Lattice *, const WorkItem *, int, int, int, int,
                       const BatchMaps) = {
        {step_batch_kernel<S, TX, TY, NT, 0, !kTma>, step_batch_kernel<S, TX, TY, NT, 1, !kTma>},
        {step_batch_kernel<S, TX, TY, NT, 0, true>, step_batch_kernel<S, TX, TY, NT, 1, true>}};
    static int configured = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (configured != dev) {
        for (int g = 0; g < 2 && e == cudaSuccess; ++g)
            for (int p = 0; p < 2 && e == cudaSuccess; ++p)
                e = cudaFuncSetAttribute(kern[g][p], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(g || !kTma ? smem_gen : smem_tma));
        if (e != cudaSuccess) return e;
        configured = dev;
    }
    if constexpr (kTma) {
        if (w.uniform) {
            void (*uk[2][2])(int, int, int, int, const UniformGroup) = {
                {step_uniform_kernel<S, TX, TY, NT, 0, false>,
                 step_uniform_kernel<S, TX, TY, NT, 1, false>},
                {step_uniform_kernel<S, TX, TY, NT, 0, true>,
                 step_uniform_kernel<S, TX, TY, NT, 1, true>}};
            static int uconfigured = -1;
            if (uconfigured != dev) {
                for (int q = 0; q < 4 && e == cudaSuccess; ++q)
                    e = cudaFuncSetAttribute(uk[q >> 1][q & 1],
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem_tma);
                if (e != cudaSuccess) return e;
                uconfigured = dev;
            }
            if (w.n_uniform <= 0) return cudaSuccess;
            const int grid = w.ntx * w.nty * w.n_uniform;
            uk[w.walls ? 1 : 0][parity & 1]<<<grid, NT, smem_tma, s>>>(cur, w.seams, w.ntx,
                                                                       w.nty, *w.uniform);
            return cudaGetLastError();
        }
    }
    if (w.n_items <= 0) return cudaSuccess;
    const int per_cta = w.per_cta < 1 ? 1 : w.per_cta;
    const int grid = (w.n_items + per_cta - 1) / per_cta;
    const int g = (kTma && w.tma_only) ? 0 : 1;
    const size_t smem = g || !kTma ? smem_gen : smem_tma;
    kern[g][parity & 1]<<<grid, NT, smem, s>>>(w.lats, w.items, w.n_items, cur, per_cta,
                                               w.inst0, *w.maps);
    return cudaGetLastError();
}

template <class S>
static cudaError_t launch_batch_t(const BatchList &w, int parity, int cur, int tx, int ty,
                                  cudaStream_t s)
{
#define CPLBM_CASE(a, b)                                                        \
    if (tx == a && ty == b) return launch_batch_shape<S, a, b>(w, parity, cur, s);
    CPLBM_STEP_SHAPES(CPLBM_CASE)
#undef CPLBM_CASE
    return cudaErrorInvalidValue;
}


// ---------------------------------------------------------------------------
// Baseline: the same step with the pressure-tensor force (Eq. 5, Eq. 9),
// the form the method avoids, for measuring what avoiding it saves.
// Periodic lattices, FP32 and FP64, on the same tile paths as the step
// kernel: TMA for interior and periodic-seam tiles (32-wide shapes, and the
// two-nodes-per-lane path of 64-wide FP32 shapes), the general path for the
// rest.
// ---------------------------------------------------------------------------
// Resident CTAs a pressure-tensor kernel asks for: three on the pair path,
// whose three tensor planes take the tile's shared memory to ~58 KB.
template <class S, int TX, int TY, int NT>
constexpr int pt_min_ctas()
{
    return HasTmaPair<S, TX, TY, NT>::value ? 3 : 0;
}

template <class S, int TX, int TY, int NT, int PARITY>
__global__ void __launch_bounds__(NT, pt_min_ctas<S, TX, TY, NT>())
    step_pt_kernel(const Lattice L, int cur, int seams, const __grid_constant__ TmaMaps maps)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int bx = PARITY ? gridDim.x - 1 - blockIdx.x : blockIdx.x;  // as step_kernel
    const int by = PARITY ? gridDim.y - 1 - blockIdx.y : blockIdx.y;
    const int kind = tile_kind(L, TX, TY, bx, by, seams);
    const bool interior = kind == TILE_INTERIOR;
    if constexpr (HasTma<S, TX, TY, NT>::value || HasTmaPair<S, TX, TY, NT>::value) {
        if (kind != TILE_GENERAL && maps.valid) {
            __shared__ __align__(8) unsigned long long bar[2];
            if (threadIdx.x == 0) {
                mbar_init(&bar[0], 1);
                mbar_init(&bar[1], 1);
            }
            __syncthreads();
            const TileMaps tm{&maps.pops, &maps.rho[cur]};
            if constexpr (HasTma<S, TX, TY, NT>::value) {
                if (interior)
                    step_tile_tma<S, TX, TY, NT, PARITY, 0, true>(L, cur, bx * TX, by * TY,
                                                                  smem_raw, tm, bar, 0);
                else
                    step_tile_tma<S, TX, TY, NT, PARITY, 1, true>(L, cur, bx * TX, by * TY,
                                                                  smem_raw, tm, bar, 0);
            } else {
                if (interior)
                    step_tile_tma_pair<S, TX, TY, NT, PARITY, 0, true>(
                        L, cur, bx * TX, by * TY, smem_raw, tm, bar, 0);
                else
                    step_tile_tma_pair<S, TX, TY, NT, PARITY, 1, true>(
                        L, cur, bx * TX, by * TY, smem_raw, tm, bar, 0);
            }
            return;
        }
    }
    if (interior)
        step_tile<S, TX, TY, NT, PARITY, true, true>(L, cur, bx * TX, by * TY,
                                                     smem_raw);
    else
        step_tile<S, TX, TY, NT, PARITY, false, true>(L, cur, bx * TX, by * TY,
                                                      smem_raw);
}

template <class S, int TX, int TY>
static cudaError_t launch_pt_shape(const Lattice &L, int parity, int cur,
                                   cudaStream_t s, const TmaMaps *maps)
{
    using real = typename S::real;
    using SM = StepSmem<real, TX, TY>;
    constexpr int NT = step_threads<S, TX, TY>();
    size_t smem = SM::bytes + 2 * sizeof(real) * SM::WM * SM::HM;
    if constexpr (HasTma<S, TX, TY, NT>::value)
        if (TmaSmem<S, TX, TY, 3>::bytes > smem) smem = TmaSmem<S, TX, TY, 3>::bytes;
    if constexpr (HasTmaPair<S, TX, TY, NT>::value) {
        using PS = TmaPairSmem<typename S::pop_t, TX, TY, NT, 3>;
        if (PS::bytes > smem) smem = PS::bytes;
    }
    TmaMaps m{};
    if (maps && maps->valid && maps->tx == TX && maps->ty == TY) m = *maps;
    auto k0 = step_pt_kernel<S, TX, TY, NT, 0>;
    auto k1 = step_pt_kernel<S, TX, TY, NT, 1>;
    static int configured = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (configured != dev) {
        e = cudaFuncSetAttribute(k0, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(
                k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = dev;
    }
    const int ntx = (L.nx + TX - 1) / TX, nty = (L.nyf + TY - 1) / TY;
    const int seams = HasTma<S, TX, TY, NT>::value || HasTmaPair<S, TX, TY, NT>::value
                          ? seam_bits(L, TX, TY) : 0;
    dim3 grid(ntx, nty);
    if (parity == 0)
        k0<<<grid, NT, smem, s>>>(L, cur, seams, m);
    else
        k1<<<grid, NT, smem, s>>>(L, cur, seams, m);
    return cudaGetLastError();
}

template <class S>
static cudaError_t launch_step_t(const Lattice &L, int parity, int cur,
                                 cudaStream_t s, const TmaMaps *maps)
{
#define CPLBM_CASE(a, b)                                           \
    if (L.tx == a && L.ty == b)                                    \
        return launch_shape<S, a, b>(L, parity, cur, s, maps);
    CPLBM_STEP_SHAPES(CPLBM_CASE)
#undef CPLBM_CASE
    return cudaErrorInvalidValue;
}

}  // namespace cplbm
