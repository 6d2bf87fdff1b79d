/*
 * Plain FP64 CPU oracle of the chemical-potential lattice Boltzmann method
 * (Wen, Zhou, He, Zhang, Fang, "Chemical-potential-based lattice Boltzmann
 * method for nonideal fluids", arXiv 1611.00907).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * statement of what one time step computes; it exists so that the CUDA
 * library can be checked against it.  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header or
 * constant table with the CUDA library.
 *
 * Layout: every field is row-major [ny][nx]; populations are [9][ny][nx].
 * Two population arrays and push streaming are used (the CUDA path keeps one
 * array in place), so the two implementations also differ in how they move
 * data.
 *
 * Geometry: x is always periodic.  walls == 0: y periodic.  walls == 1: rows
 * y = 0 and y = ny-1 are solid (Sec. IV); fluid rows are 1..ny-2.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* D2Q9 lattice (Eq. 13-14): speeds e_i, weights w_i, opposite directions.   */
/* ------------------------------------------------------------------------ */
static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double WGT[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
                              1.0 / 9.0,  1.0 / 9.0,  1.0 / 36.0,
                              1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const double CS2 = 1.0 / 3.0; /* lattice sound speed squared */

enum { EOS_VDW = 0, EOS_CS = 1, EOS_PR = 2, EOS_RKS = 3 };

typedef struct {
    int eos;      /* EOS_* */
    double a, b;  /* attraction and volume parameters */
    double R, T;  /* gas constant and absolute temperature */
    double alpha; /* alpha(T) of PR / RKS (ignored by vdW and CS) */
} orc_eos;

typedef struct {
    int nx, ny;
    int walls;        /* 0 periodic, 1 solid rows y=0 and y=ny-1 */
    double tau;       /* BGK relaxation time, Eq. 13 */
    double kappa;     /* square-gradient coefficient, Eq. 1 and Eq. 8 */
    orc_eos eos;
    double mu_bottom; /* surface chemical potential of row y=0, Sec. IV */
    int top_mode;     /* 0: top solid mu copies its fluid neighbour (Sec. V) */
    double mu_top;    /* used when top_mode == 1 */
} orc_params;

static int g_threads = 1;

void orc_set_threads(int n) { g_threads = n > 0 ? n : 1; }

int orc_get_threads(void) { return g_threads; }

/* ------------------------------------------------------------------------ */
/* Free-energy density psi, bulk chemical potential psi'(rho) and EOS p0.    */
/* Each is the paper's printed formula.                                      */
/* ------------------------------------------------------------------------ */

/* psi(rho): Eq. 17 (vdW), Eq. 20 (RK/RKS), Eq. 23 (PR), Eq. 26 (CS). */
double orc_psi(const orc_eos *e, double rho)
{
    const double a = e->a, b = e->b, RT = e->R * e->T;
    switch (e->eos) {
    case EOS_VDW:
        return rho * RT * log(rho / (1.0 - b * rho)) - a * rho * rho;
    case EOS_RKS:
        return RT * rho * log(rho / (1.0 - b * rho)) -
               a * e->alpha / b * rho * log(1.0 + b * rho);
    case EOS_PR: {
        const double s2 = sqrt(2.0);
        return RT * rho * log(rho / (1.0 - b * rho)) -
               a * e->alpha * rho / (2.0 * s2 * b) *
                   log((s2 - 1.0 + b * rho) / (s2 + 1.0 - b * rho));
    }
    case EOS_CS: {
        const double q = 1.0 - b * rho / 4.0;
        return RT * rho * ((3.0 - b * rho / 2.0) / (q * q) + log(rho)) -
               a * rho * rho;
    }
    }
    return NAN;
}

/* psi'(rho): the bulk part of Eq. 18 (vdW), Eq. 21 (RK/RKS), Eq. 24 (PR),
 * Eq. 27 (CS), i.e. the printed chemical potential without -kappa lap(rho). */
double orc_mu_bulk(const orc_eos *e, double rho)
{
    const double a = e->a, b = e->b, RT = e->R * e->T;
    switch (e->eos) {
    case EOS_VDW:
        return RT * (log(rho / (1.0 - b * rho)) + 1.0 / (1.0 - b * rho)) -
               2.0 * a * rho;
    case EOS_RKS:
        return RT * log(rho / (1.0 - b * rho)) + RT / (1.0 - b * rho) -
               a * e->alpha / b * log(1.0 + b * rho) -
               a * e->alpha * rho / (1.0 + b * rho);
    case EOS_PR: {
        const double s2 = sqrt(2.0);
        return RT * log(rho / (1.0 - b * rho)) -
               a * e->alpha / (2.0 * s2 * b) *
                   log((s2 - 1.0 + b * rho) / (s2 + 1.0 - b * rho)) +
               RT / (1.0 - b * rho) -
               a * e->alpha * rho / (1.0 + 2.0 * b * rho - b * b * rho * rho);
    }
    case EOS_CS: {
        const double q = 1.0 - b * rho / 4.0;
        return RT * ((3.0 - b * rho / 4.0) / (q * q * q) + log(rho) + 1.0) -
               2.0 * a * rho;
    }
    }
    return NAN;
}

/* p0(rho): Eq. 16 (vdW), Eq. 19 (RK/RKS), Eq. 22 (PR), Eq. 25 (CS). */
double orc_p0(const orc_eos *e, double rho)
{
    const double a = e->a, b = e->b, RT = e->R * e->T;
    switch (e->eos) {
    case EOS_VDW:
        return rho * RT / (1.0 - b * rho) - a * rho * rho;
    case EOS_RKS:
        return rho * RT / (1.0 - b * rho) -
               a * e->alpha * rho * rho / (1.0 + b * rho);
    case EOS_PR:
        return rho * RT / (1.0 - b * rho) -
               a * e->alpha * rho * rho /
                   (1.0 + 2.0 * b * rho - b * b * rho * rho);
    case EOS_CS: {
        const double h = b * rho / 4.0;
        return rho * RT * (1.0 + h + h * h - h * h * h) /
                   ((1.0 - h) * (1.0 - h) * (1.0 - h)) -
               a * rho * rho;
    }
    }
    return NAN;
}

/* Vectorised evaluation for the Python thermodynamics helpers. */
void orc_eos_eval(const orc_eos *e, const double *rho, long n, double *psi,
                  double *mu, double *p0)
{
    for (long k = 0; k < n; ++k) {
        if (psi) psi[k] = orc_psi(e, rho[k]);
        if (mu) mu[k] = orc_mu_bulk(e, rho[k]);
        if (p0) p0[k] = orc_p0(e, rho[k]);
    }
}

/* ------------------------------------------------------------------------ */
/* Geometry helpers.                                                         */
/* ------------------------------------------------------------------------ */
static int is_solid_row(const orc_params *p, int y)
{
    return p->walls && (y == 0 || y == p->ny - 1);
}

static int wrap(int v, int n) { return ((v % n) + n) % n; }

/* Neighbour of (x, y) along e_i: x periodic; y periodic only without walls.
 * With walls, a fluid node's neighbours stay inside rows 0..ny-1. */
static long nbr(const orc_params *p, int x, int y, int i)
{
    const int xn = wrap(x + EX[i], p->nx);
    const int yn = p->walls ? y + EY[i] : wrap(y + EY[i], p->ny);
    return (long)yn * p->nx + xn;
}

/* ------------------------------------------------------------------------ */
/* Step pieces.                                                              */
/* ------------------------------------------------------------------------ */

/* rho = sum_i f_i at fluid nodes (zeroth moment of the distributions). */
void orc_density(const orc_params *p, const double *f, double *rho)
{
    const long N = (long)p->nx * p->ny;
#pragma omp parallel for num_threads(g_threads)
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            const long n = (long)y * p->nx + x;
            if (is_solid_row(p, y)) { rho[n] = 0.0; continue; }
            double s = 0.0;
            for (int i = 0; i < 9; ++i) s += f[i * N + n];
            rho[n] = s;
        }
}

/* Solid-row density by the weighted average of Eq. 28.  The bottom row uses
 * fluid row 1; the top row (walls on both sides) mirrors it from row ny-2. */
void orc_wall_density(const orc_params *p, double *rho)
{
    if (!p->walls) return;
    const int nx = p->nx;
    const double *r1 = rho + (long)1 * nx;
    const double *rt = rho + (long)(p->ny - 2) * nx;
    double *r0 = rho;
    double *rN = rho + (long)(p->ny - 1) * nx;
    for (int x = 0; x < nx; ++x) {
        const int xm = wrap(x - 1, nx), xp = wrap(x + 1, nx);
        r0[x] = 2.0 / 3.0 * r1[x] + 1.0 / 6.0 * r1[xm] + 1.0 / 6.0 * r1[xp];
        rN[x] = 2.0 / 3.0 * rt[x] + 1.0 / 6.0 * rt[xm] + 1.0 / 6.0 * rt[xp];
    }
}

/* Isotropic D2Q9 Laplacian: 6 sum_i w_i (phi(x+e_i) - phi(x)). */
double orc_laplacian_at(const orc_params *p, const double *phi, int x, int y)
{
    const double c = phi[(long)y * p->nx + x];
    double s = 0.0;
    for (int i = 1; i < 9; ++i) s += WGT[i] * (phi[nbr(p, x, y, i)] - c);
    return 6.0 * s;
}

/* Isotropic D2Q9 gradient: 3 sum_i w_i phi(x+e_i) e_i. */
void orc_gradient_at(const orc_params *p, const double *phi, int x, int y,
                     double *gx, double *gy)
{
    double sx = 0.0, sy = 0.0;
    for (int i = 1; i < 9; ++i) {
        const double v = phi[nbr(p, x, y, i)];
        sx += WGT[i] * v * EX[i];
        sy += WGT[i] * v * EY[i];
    }
    *gx = 3.0 * sx;
    *gy = 3.0 * sy;
}

/* Whole-field Laplacian and gradient at fluid nodes (solid rows get 0). */
void orc_laplacian(const orc_params *p, const double *phi, double *out)
{
#pragma omp parallel for num_threads(g_threads)
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x)
            out[(long)y * p->nx + x] =
                is_solid_row(p, y) ? 0.0 : orc_laplacian_at(p, phi, x, y);
}

void orc_gradient(const orc_params *p, const double *phi, double *gx,
                  double *gy)
{
#pragma omp parallel for num_threads(g_threads)
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            const long n = (long)y * p->nx + x;
            if (is_solid_row(p, y)) { gx[n] = gy[n] = 0.0; continue; }
            orc_gradient_at(p, phi, x, y, gx + n, gy + n);
        }
}

/* mu = psi'(rho) - kappa lap(rho) at fluid nodes (Eq. 8).  The solid rows
 * carry the surface chemical potential (Sec. IV); the top row copies its
 * fluid neighbour (Sec. V) unless a value is given.  rho must already hold
 * the Eq. 28 solid-row densities. */
void orc_chem_potential(const orc_params *p, const double *rho, double *mu)
{
#pragma omp parallel for num_threads(g_threads)
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            const long n = (long)y * p->nx + x;
            if (is_solid_row(p, y)) { mu[n] = 0.0; continue; }
            mu[n] = orc_mu_bulk(&p->eos, rho[n]) -
                    p->kappa * orc_laplacian_at(p, rho, x, y);
        }
    if (p->walls) {
        const int nx = p->nx, ny = p->ny;
        for (int x = 0; x < nx; ++x) {
            mu[x] = p->mu_bottom;
            mu[(long)(ny - 1) * nx + x] =
                p->top_mode == 0 ? mu[(long)(ny - 2) * nx + x] : p->mu_top;
        }
    }
}

/* Nonideal force F = -rho grad(mu) + grad(cs^2 rho) at fluid nodes (Eq. 12,
 * with the ideal-gas tensor P0 = cs^2 rho I of Eq. 5). */
void orc_force(const orc_params *p, const double *rho, const double *mu,
               double *Fx, double *Fy)
{
#pragma omp parallel for num_threads(g_threads)
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            const long n = (long)y * p->nx + x;
            if (is_solid_row(p, y)) { Fx[n] = Fy[n] = 0.0; continue; }
            double mx, my, rx, ry;
            orc_gradient_at(p, mu, x, y, &mx, &my);
            orc_gradient_at(p, rho, x, y, &rx, &ry);
            Fx[n] = -rho[n] * mx + CS2 * rx;
            Fy[n] = -rho[n] * my + CS2 * ry;
        }
}

/* Nonideal force from the pressure tensor instead (Eq. 5 with Eq. 9), the
 * form the method replaces: P = [p0 - kappa rho lap(rho) - kappa/2 |grad
 * rho|^2] I + kappa grad(rho) grad(rho), F = -div(P) + grad(cs^2 rho), with
 * the same isotropic stencils for every derivative.  Periodic lattices only
 * (the paper gives no wall rule for this form).  rho must hold the density
 * at every node. */
void orc_force_pressure_tensor(const orc_params *p, const double *rho,
                               double *Fx, double *Fy)
{
    const long N = (long)p->nx * p->ny;
    double *pxx = malloc(sizeof(double) * N);
    double *pxy = malloc(sizeof(double) * N);
    double *pyy = malloc(sizeof(double) * N);
    if (!pxx || !pxy || !pyy) {
        free(pxx); free(pxy); free(pyy);
        for (long n = 0; n < N; ++n) Fx[n] = Fy[n] = NAN;
        return;
    }
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            const long n = (long)y * p->nx + x;
            double gx, gy;
            orc_gradient_at(p, rho, x, y, &gx, &gy);
            const double lap = orc_laplacian_at(p, rho, x, y);
            const double iso = orc_p0(&p->eos, rho[n]) -
                               p->kappa * rho[n] * lap -
                               0.5 * p->kappa * (gx * gx + gy * gy);
            pxx[n] = iso + p->kappa * gx * gx;
            pyy[n] = iso + p->kappa * gy * gy;
            pxy[n] = p->kappa * gx * gy;
        }
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            const long n = (long)y * p->nx + x;
            double dxx, dxy_x, dxy_y, dyy, rx, ry, unused;
            orc_gradient_at(p, pxx, x, y, &dxx, &unused);
            orc_gradient_at(p, pxy, x, y, &dxy_x, &dxy_y);
            orc_gradient_at(p, pyy, x, y, &unused, &dyy);
            orc_gradient_at(p, rho, x, y, &rx, &ry);
            Fx[n] = -(dxx + dxy_y) + CS2 * rx;
            Fy[n] = -(dxy_x + dyy) + CS2 * ry;
        }
    free(pxx); free(pxy); free(pyy);
}

/* Second-order equilibrium of Eq. 14 for density rho and velocity (ux, uy). */
void orc_equilibrium(double rho, double ux, double uy, double *feq)
{
    const double uu = ux * ux + uy * uy;
    for (int i = 0; i < 9; ++i) {
        const double eu = EX[i] * ux + EY[i] * uy;
        feq[i] = rho * WGT[i] * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
    }
}

/* BGK collision of one node (Eq. 13) with the force entering through the
 * equilibrium velocity u_eq = u + tau F / rho (Sec. II, ref. [36]). */
void orc_collide_node(const double *f, double Fx, double Fy, double tau,
                      double *fout)
{
    double rho = 0.0, jx = 0.0, jy = 0.0;
    for (int i = 0; i < 9; ++i) {
        rho += f[i];
        jx += f[i] * EX[i];
        jy += f[i] * EY[i];
    }
    const double ux = jx / rho, uy = jy / rho;
    const double uex = ux + tau * Fx / rho, uey = uy + tau * Fy / rho;
    double feq[9];
    orc_equilibrium(rho, uex, uey, feq);
    for (int i = 0; i < 9; ++i) fout[i] = f[i] - (f[i] - feq[i]) / tau;
}

/* Push streaming of post-collision populations with halfway bounce-back on
 * links into solid rows (Sec. IV): f_i(x + e_i) <- f*_i(x), or, when x + e_i
 * is solid, f_opp(i)(x) <- f*_i(x). */
void orc_stream(const orc_params *p, const double *fpost, double *fnext)
{
    const long N = (long)p->nx * p->ny;
    memset(fnext, 0, sizeof(double) * 9 * N);
#pragma omp parallel for num_threads(g_threads)
    for (int y = 0; y < p->ny; ++y) {
        if (is_solid_row(p, y)) continue;
        for (int x = 0; x < p->nx; ++x) {
            const long n = (long)y * p->nx + x;
            for (int i = 0; i < 9; ++i) {
                const int yt = p->walls ? y + EY[i] : wrap(y + EY[i], p->ny);
                if (is_solid_row(p, yt))
                    fnext[OPP[i] * N + n] = fpost[i * N + n];
                else
                    fnext[i * N + nbr(p, x, y, i)] = fpost[i * N + n];
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Whole step and moments.                                                   */
/* ------------------------------------------------------------------------ */

/* The macroscopic fields of the current state, as the step uses them:
 * rho (solid rows by Eq. 28), mu (solid rows by the wall rule), F. */
static void fields(const orc_params *p, const double *f, double *rho,
                   double *mu, double *Fx, double *Fy)
{
    orc_density(p, f, rho);
    orc_wall_density(p, rho);
    orc_chem_potential(p, rho, mu);
    orc_force(p, rho, mu, Fx, Fy);
}

static int step_impl(const orc_params *p, double *f, int nsteps, int model);

/* Advance f by nsteps time steps.  Returns 0, or -1 on allocation failure. */
int orc_step(const orc_params *p, double *f, int nsteps)
{
    return step_impl(p, f, nsteps, 0);
}

/* The same step with the pressure-tensor force (Eq. 5); periodic only.
 * Returns -2 for a lattice with walls. */
int orc_step_pressure_tensor(const orc_params *p, double *f, int nsteps)
{
    if (p->walls) return -2;
    return step_impl(p, f, nsteps, 1);
}

static int step_impl(const orc_params *p, double *f, int nsteps, int model)
{
    const long N = (long)p->nx * p->ny;
    double *rho = malloc(sizeof(double) * N);
    double *mu = malloc(sizeof(double) * N);
    double *Fx = malloc(sizeof(double) * N);
    double *Fy = malloc(sizeof(double) * N);
    double *fpost = malloc(sizeof(double) * 9 * N);
    double *fnext = malloc(sizeof(double) * 9 * N);
    int rc = 0;
    if (!rho || !mu || !Fx || !Fy || !fpost || !fnext) { rc = -1; goto out; }
    for (int s = 0; s < nsteps; ++s) {
        if (model == 0) {
            fields(p, f, rho, mu, Fx, Fy);
        } else {
            orc_density(p, f, rho);
            orc_force_pressure_tensor(p, rho, Fx, Fy);
        }
#pragma omp parallel for num_threads(g_threads)
        for (int y = 0; y < p->ny; ++y) {
            if (is_solid_row(p, y)) continue;
            for (int x = 0; x < p->nx; ++x) {
                const long n = (long)y * p->nx + x;
                double fi[9], fo[9];
                for (int i = 0; i < 9; ++i) fi[i] = f[i * N + n];
                orc_collide_node(fi, Fx[n], Fy[n], p->tau, fo);
                for (int i = 0; i < 9; ++i) fpost[i * N + n] = fo[i];
            }
        }
        orc_stream(p, fpost, fnext);
        memcpy(f, fnext, sizeof(double) * 9 * N);
    }
out:
    free(rho); free(mu); free(Fx); free(Fy); free(fpost); free(fnext);
    return rc;
}

/* Macroscopic fields of the state f: rho and mu (including the solid-row
 * values the step uses), the force F, and the fluid velocity
 * v = u + F / (2 rho) (Sec. II).  Any output pointer may be NULL.  Velocity,
 * force and u are zero on solid rows. */
int orc_moments(const orc_params *p, const double *f, double *rho_out,
                double *vx, double *vy, double *mu_out, double *Fx_out,
                double *Fy_out)
{
    const long N = (long)p->nx * p->ny;
    double *rho = malloc(sizeof(double) * N);
    double *mu = malloc(sizeof(double) * N);
    double *Fx = malloc(sizeof(double) * N);
    double *Fy = malloc(sizeof(double) * N);
    if (!rho || !mu || !Fx || !Fy) {
        free(rho); free(mu); free(Fx); free(Fy);
        return -1;
    }
    fields(p, f, rho, mu, Fx, Fy);
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            const long n = (long)y * p->nx + x;
            double jx = 0.0, jy = 0.0;
            if (!is_solid_row(p, y))
                for (int i = 0; i < 9; ++i) {
                    jx += f[i * N + n] * EX[i];
                    jy += f[i * N + n] * EY[i];
                }
            const double r = rho[n];
            const int solid = is_solid_row(p, y);
            if (vx) vx[n] = solid ? 0.0 : (jx + 0.5 * Fx[n]) / r;
            if (vy) vy[n] = solid ? 0.0 : (jy + 0.5 * Fy[n]) / r;
        }
    if (rho_out) memcpy(rho_out, rho, sizeof(double) * N);
    if (mu_out) memcpy(mu_out, mu, sizeof(double) * N);
    if (Fx_out) memcpy(Fx_out, Fx, sizeof(double) * N);
    if (Fy_out) memcpy(Fy_out, Fy, sizeof(double) * N);
    free(rho); free(mu); free(Fx); free(Fy);
    return 0;
}

/* Equilibrium populations for given density and velocity fields at fluid
 * nodes (solid rows are left zero): the usual initial state f = f_eq. */
void orc_init_equilibrium(const orc_params *p, const double *rho,
                          const double *ux, const double *uy, double *f)
{
    const long N = (long)p->nx * p->ny;
    memset(f, 0, sizeof(double) * 9 * N);
    for (int y = 0; y < p->ny; ++y) {
        if (is_solid_row(p, y)) continue;
        for (int x = 0; x < p->nx; ++x) {
            const long n = (long)y * p->nx + x;
            double feq[9];
            orc_equilibrium(rho[n], ux ? ux[n] : 0.0, uy ? uy[n] : 0.0, feq);
            for (int i = 0; i < 9; ++i) f[i * N + n] = feq[i];
        }
    }
}
