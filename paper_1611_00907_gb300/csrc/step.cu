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
// parts in a fixed order (load_rho): results do not depend on scheduling.
#include "device_common.cuh"

namespace cplbm {

template <class S, int TX, int TY, int NT>
__global__ void __launch_bounds__(NT)
    step_kernel(const Lattice L, int parity, int cur)
{
    using real = typename S::real;
    using pop_t = typename S::pop_t;
    using rho_t = typename S::rho_t;
    constexpr int WR = TX + 4;       // s_rho row width
    constexpr int WM = TX + 2;       // s_mu row width
    constexpr int NODES = TX * TY;
    constexpr int PER = NODES / NT;  // nodes per thread
    static_assert(NODES % NT == 0, "tile must split evenly over threads");

    extern __shared__ unsigned char smem_raw[];
    real *s_rho = reinterpret_cast<real *>(smem_raw);
    real *s_mu = s_rho + (TY + 4) * WR;
    real *s_post = s_mu + (TY + 2) * WM;  // [9][TY][TX] post-collision

    const int X0 = blockIdx.x * TX, Y0 = blockIdx.y * TY;
    const int wx = min(TX, L.nx - X0), wy = min(TY, L.nyf - Y0);
    const int nxt = cur ^ 1;

    load_rho_tile<S, TX, TY>(L, cur, X0, Y0, s_rho);
    __syncthreads();
    mu_tile<S, TX, TY>(L, X0, Y0, s_rho, s_mu);
    __syncthreads();

    const real omega = real(1) / (real)L.tau;
    const real tau = (real)L.tau;
    const real rho_ref = S::offset ? (real)L.rho_ref : real(0);
    pop_t *A = (pop_t *)L.pops;

#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int n = threadIdx.x + k * NT;
        const int lx = n % TX, ly = n / TX;
        if (lx >= wx || ly >= wy) continue;
        const int x = X0 + lx, r = Y0 + ly;

        // stored values (offset form for offset precisions)
        real f[9];
        real sum = real(0);
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            f[i] = ld_real(A + aa_read_index(L, parity, i, r, x));
            sum += f[i];
        }
        const int cr = (ly + 2) * WR + lx + 2, cm = (ly + 1) * WM + lx + 1;
        const real rho = s_rho[cr];
        f[0] = (rho - rho_ref) - sum;

        // Eq. 12: F = -rho grad(mu) + grad(cs^2 rho)
        real gmx, gmy, grx, gry;
        grad9<real, WM>(s_mu, cm, gmx, gmy);
        grad9<real, WR>(s_rho, cr, grx, gry);
        const real Fx = -rho * gmx + grx / real(3);
        const real Fy = -rho * gmy + gry / real(3);

        // u = sum f_i e_i / rho; u_eq = u + tau F / rho (Sec. II)
        const real jx = f[1] - f[3] + f[5] - f[6] - f[7] + f[8];
        const real jy = f[2] - f[4] + f[5] + f[6] - f[7] - f[8];
        const real inv_rho = real(1) / rho;
        const real ux = (jx + tau * Fx) * inv_rho;
        const real uy = (jy + tau * Fy) * inv_rho;
        const real usq = real(1.5) * (ux * ux + uy * uy);

        // BGK towards Eq. 14 (offset form: f_eq - w_i rho_ref)
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const real eu = real(ex(i)) * ux + real(ey(i)) * uy;
            const real poly = real(3) * eu + real(4.5) * eu * eu - usq;
            const real feq = wgt<real>(i) * ((rho - rho_ref) + rho * poly);
            const real fp = f[i] + omega * (feq - f[i]);
            s_post[(i * TY + ly) * TX + lx] = fp;
            if (i > 0) st_real(A + aa_write_index(L, parity, i, r, x), fp);
        }
    }
    __syncthreads();

    // Density hand-over: every node of the tile and of its one-node ring
    // receives the post-collision populations streaming to it from the tile.
    rho_t *Rn = (rho_t *)L.rho[nxt];
    rho_t *const *ring = (rho_t *const *)L.ring[nxt];
    constexpr int WO = TX + 2, HO = TY + 2;
    for (int k = threadIdx.x; k < WO * HO; k += NT) {
        const int ox = k % WO - 1, oy = k / WO - 1;
        if (ox > wx || oy > wy) continue;
        const int r = Y0 + oy;
        if (L.walls && (r < 0 || r >= L.nyf)) continue;  // solid: no density
        const bool in_x = ox >= 0 && ox < wx, in_y = oy >= 0 && oy < wy;
        const bool inside = in_x && in_y;
        real s = real(0);
        bool any = false;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int sx = ox - ex(i), sy = oy - ey(i);
            if (i > 0 && inside && L.walls &&
                row_is_solid(L, r - ey(i))) {
                // bounce-back: f*_opp(i) of this node comes back as f_i
                s += s_post[(opp(i) * TY + oy) * TX + ox];
                any = true;
            } else if (sx >= 0 && sx < wx && sy >= 0 && sy < wy) {
                s += s_post[(i * TY + sy) * TX + sx];
                any = true;
            }
        }
        if (!any) continue;
        const int x = wrapi(X0 + ox, L.nx);
        const int rw = row_wrap(L, r);
        if (inside) {
            Rn[fidx(L, rw, x)] = (rho_t)s;
        } else {
            int c;
            if (ox < 0) c = oy < 0 ? R_TR : (oy >= wy ? R_BR : R_R);
            else if (ox >= wx) c = oy < 0 ? R_TL : (oy >= wy ? R_BL : R_L);
            else c = oy < 0 ? R_T : R_B;
            const long long idx =
                (c == R_L || c == R_R) ? cidx(L, rw, x) : fidx(L, rw, x);
            ring[c][idx] = (rho_t)s;
        }
    }
}

template <class S>
static cudaError_t launch_step_t(const Lattice &L, int parity, int cur,
                                 cudaStream_t s)
{
    using real = typename S::real;
    constexpr int TX = TILE_X, TY = TILE_Y, NT = STEP_THREADS;
    const size_t smem = sizeof(real) * ((TY + 4) * (TX + 4) +
                                        (TY + 2) * (TX + 2) + 9 * TY * TX);
    auto kern = step_kernel<S, TX, TY, NT>;
    static bool configured = false;  // per template instance
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(
            kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    dim3 grid((L.nx + TX - 1) / TX, (L.nyf + TY - 1) / TY);
    kern<<<grid, NT, smem, s>>>(L, parity, cur);
    return cudaGetLastError();
}

cudaError_t launch_step(const Lattice &L, int parity, int cur, cudaStream_t s)
{
    switch (L.precision) {
    case P_F64: return launch_step_t<SF64>(L, parity, cur, s);
    case P_F32: return launch_step_t<SF32>(L, parity, cur, s);
    case P_F32_OFF: return launch_step_t<SF32Off>(L, parity, cur, s);
    case P_F16_OFF: return launch_step_t<SF16Off>(L, parity, cur, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace cplbm
