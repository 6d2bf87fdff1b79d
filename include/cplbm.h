/*
 * cplbm: chemical-potential lattice Boltzmann method for nonideal fluids on
 * one GPU (sm_103a), after Wen, Zhou, He, Zhang, Fang, arXiv 1611.00907.
 *
 * C ABI of the D2Q9 time step.  One call of lbm_step advances the
 * distributions by the paper's update:
 *   density             rho = sum_i f_i                        (Sec. II)
 *   solid-row density    weighted average of Eq. 28              (Sec. IV)
 *   chemical potential   mu = psi'(rho) - kappa lap(rho)         (Eq. 8; psi'
 *                        from Eq. 18 vdW, Eq. 21 RK/RKS, Eq. 24 PR,
 *                        Eq. 27 CS); solid rows carry the surface value
 *                        (Sec. IV, Sec. V)
 *   nonideal force       F = -rho grad(mu) + grad(cs^2 rho)      (Eq. 12)
 *   collision            BGK, Eq. 13, towards Eq. 14 with the equilibrium
 *                        velocity u + tau F / rho                (Sec. II)
 *   streaming            with halfway bounce-back on solid rows  (Sec. IV)
 * Gradients and Laplacians are the isotropic D2Q9 stencils
 *   grad(phi) = 3 sum_i w_i phi(x + e_i) e_i,
 *   lap(phi)  = 6 sum_i w_i (phi(x + e_i) - phi(x)).
 *
 * Conventions.
 *  - Fields passed in or out are double, row-major [ny][nx], node (x, y) at
 *    index y * nx + x, lattice directions e_0 = (0,0), e_1..4 = (1,0),
 *    (0,1), (-1,0), (0,-1), e_5..8 = (1,1), (-1,1), (-1,-1), (1,-1).
 *  - x is always periodic.  walls == 0: y periodic.  walls == 1: rows y = 0
 *    and y = ny - 1 are solid; fluid rows are 1..ny-2.
 *  - The caller owns every buffer it passes; the library never keeps a
 *    caller pointer past the call.  `on_device` != 0 means the pointer is
 *    device memory of the context's GPU, else host memory.
 *  - Every function returns a status and never aborts or throws.  After an
 *    error, lbm_last_error() describes it.  Calls on one context are not
 *    thread-safe; separate contexts are independent.
 *  - Work is queued on the context's CUDA stream.  lbm_step returns without
 *    waiting; lbm_moments, lbm_reduce, lbm_get_populations and the state
 *    calls wait for the stream.
 */
#ifndef CPLBM_H
#define CPLBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

typedef enum {
    LBM_OK = 0,
    LBM_ERR_ARG = -1,     /* invalid argument or configuration */
    LBM_ERR_CUDA = -2,    /* a CUDA runtime call failed */
    LBM_ERR_OOM = -3,     /* device or host allocation failed */
    LBM_ERR_NUMERIC = -4, /* non-finite value found by lbm_reduce */
    LBM_ERR_STATE = -5    /* call out of order (e.g. step before init) */
} lbm_status;

typedef enum {
    LBM_EOS_VDW = 0, /* van der Waals, Eqs. 16-18 */
    LBM_EOS_CS = 1,  /* Carnahan-Starling, Eqs. 25-27 */
    LBM_EOS_PR = 2,  /* Peng-Robinson, Eqs. 22-24 */
    LBM_EOS_RKS = 3  /* Redlich-Kwong-Soave, Eqs. 19-21 */
} lbm_eos;

/* Storage and arithmetic of the distributions.
 *  LBM_F64:        FP64 storage and arithmetic.
 *  LBM_F32:        FP32 storage and arithmetic.
 *  LBM_F32_OFFSET: FP32 arithmetic; each f_i is stored as f_i - w_i rho_ref
 *                  and the density as rho - rho_ref.
 *  LBM_F16_OFFSET: FP32 arithmetic; offsets stored as FP16, density as FP32.
 * The global reductions of lbm_reduce always accumulate in FP64. */
typedef enum {
    LBM_F64 = 0,
    LBM_F32 = 1,
    LBM_F32_OFFSET = 2,
    LBM_F16_OFFSET = 3
} lbm_precision;

typedef struct {
    int nx, ny;     /* lattice size, solid rows included; nx >= 5, ny >= 5 */
    int walls;      /* 0 periodic in y, 1 solid rows y = 0 and y = ny - 1 */
    double tau;     /* BGK relaxation time (Eq. 13), > 0.5 */
    double kappa;   /* square-gradient coefficient (Eq. 1, Eq. 8), >= 0 */
    double rho_ref; /* reference density of the offset precisions */
    int precision;  /* lbm_precision */
    void *stream;   /* cudaStream_t to queue work on; NULL: legacy stream */
    int device;     /* CUDA device ordinal */
} lbm_config;

/* Allocate a context and its device state for cfg.  *out receives the
 * context (NULL on error).  Device memory per lattice node: 8 distributions
 * in the storage type plus three densities. */
lbm_status lbm_create(const lbm_config *cfg, lbm_ctx **out);

/* Select the equation of state (Sec. III): a, b, R as in Eqs. 16, 19, 22,
 * 25; T = T_over_Tc * T_c, where T_c is the EOS's critical temperature with
 * alpha = 1, found by the library; omega is the acentric factor of the
 * alpha(T) of PR (Eq. 22 text) and RKS (Eq. 19 text) and is ignored by vdW
 * and CS.  Must be called before lbm_init. */
lbm_status lbm_set_eos(lbm_ctx *ctx, int eos, double a, double b, double R,
                       double T_over_Tc, double omega);

/* Surface chemical potentials of the solid rows (Sec. IV, Sec. V).  The
 * bottom row y = 0 carries mu_bottom.  top_mode 0: the top row copies the
 * chemical potential of its fluid neighbour (Sec. V); top_mode 1: it
 * carries mu_top.  Ignored when walls == 0.  Default: 0, mode 0. */
lbm_status lbm_set_wall_mu(lbm_ctx *ctx, double mu_bottom, int top_mode,
                           double mu_top);

/* Tile shape of the fused step kernel: tx x ty fluid nodes per CTA, one of
 * 32x16, 32x24, 32x32, 64x16, 64x32 (LBM_ERR_ARG otherwise).  The shape
 * changes speed, and in FP32 arithmetic the rounding order of some sums,
 * not the method.  May be called at any time.  Default: 64x16 (two nodes
 * per lane) for FP32 arithmetic, 32x32 for FP64. */
lbm_status lbm_set_tile(lbm_ctx *ctx, int tx, int ty);
lbm_status lbm_get_tile(const lbm_ctx *ctx, int *tx, int *ty);

/* Time nsteps (rounded up to an even count >= 2) steps of each compiled
 * tile shape of the force model in use (lbm_set_force_model) on the
 * context's own lattice, keep the fastest, and restore
 * the state exactly as it was (the step counter included).  Allocates one
 * temporary copy of the state.  *tx, *ty (may be NULL) receive the shape. */
lbm_status lbm_autotune(lbm_ctx *ctx, int nsteps, int *tx, int *ty);

/* Force model of lbm_step.  0 (default): the chemical-potential force of
 * Eq. 12.  1: the pressure-tensor force it replaces, F = -div(P) +
 * grad(cs^2 rho) with P of Eq. 9 (Eq. 5), same stencils - a baseline for
 * measuring the cost the method avoids; periodic lattices, LBM_F64 or
 * LBM_F32.  Model 1 has kernels for tiles 64x16 (FP32, set by this call;
 * the same two-nodes-per-lane path as the default step) and 32x32 (FP32),
 * and 32x16 (FP64, set by this call); lbm_set_tile refuses other shapes
 * while it is in use, and lbm_autotune times its step over those shapes.
 * lbm_moments reports v and mu with the chemical-potential definitions in
 * both models. */
lbm_status lbm_set_force_model(lbm_ctx *ctx, int model);

/* Set the state to equilibrium populations f_i = f_i^eq(rho, u) (Eq. 14)
 * at every fluid node, and the step counter to 0.  rho must be positive and
 * below the EOS's repulsive pole at fluid nodes; ux and uy may be NULL
 * (zero velocity).  Values on solid rows are ignored. */
lbm_status lbm_init(lbm_ctx *ctx, const double *rho, const double *ux,
                    const double *uy, int on_device);

/* Queue nsteps (>= 0) time steps (Sec. II: density, Eq. 8, Eq. 12, the
 * BGK collision of Eq. 13-14 and streaming, with the wall rule of Sec. IV)
 * on the context's stream.  Returns without waiting for the GPU.  Blocks of
 * 16 steps replay a CUDA graph captured on a private stream at the first
 * such call (and again after any change of tile shape, physics, force
 * model or wait limit); while the context's stream is being captured by
 * the caller, every step is a plain launch that joins the caller's graph. */
lbm_status lbm_step(lbm_ctx *ctx, int nsteps);

/* Macroscopic fields of the current state: rho (solid rows: Eq. 28), the
 * fluid velocity v = u + F / (2 rho) (Sec. II; zero on solid rows) and mu
 * (solid rows: the wall values the step uses).  Any pointer may be NULL. */
lbm_status lbm_moments(lbm_ctx *ctx, double *rho, double *vx, double *vy,
                       double *mu, int on_device);

/* Distributions of the current state in natural order, FP64
 * [9][ny][nx] (solid rows zero). */
lbm_status lbm_get_populations(lbm_ctx *ctx, double *f, int on_device);

/* FP64 global reductions over fluid nodes: out[0] = sum rho,
 * out[1], out[2] = sum rho v, out[3] = max |rho - rho at the previous
 * lbm_reduce call| (the first call after lbm_init reports the change since
 * the initial state).  LBM_ERR_NUMERIC if a non-finite value is found.
 * out is host memory. */
lbm_status lbm_reduce(lbm_ctx *ctx, double out[4]);

/* Checkpoint: the raw device state (distributions, current density, step
 * parity) copied to or from host memory, for a bitwise resume in the same
 * precision and geometry.  lbm_state_size() gives the byte count. */
size_t lbm_state_size(const lbm_ctx *ctx);
lbm_status lbm_get_state(lbm_ctx *ctx, void *buf, size_t bytes);
lbm_status lbm_set_state(lbm_ctx *ctx, const void *buf, size_t bytes);

/* Steps taken since lbm_init or lbm_set_state's saved counter. */
long long lbm_step_count(const lbm_ctx *ctx);

/* Absolute temperature, alpha(T) and critical point of the selected EOS. */
lbm_status lbm_eos_info(const lbm_ctx *ctx, double *T, double *alpha,
                        double *Tc, double *rhoc);

/* Critical point (T_c, rho_c) of an EOS with alpha = 1: both the first and
 * the second density derivative of p0 vanish (Sec. III's reduced
 * variables).  Host-only helper. */
lbm_status lbm_eos_critical(int eos, double a, double b, double R,
                            double *Tc, double *rhoc);

/* ------------------------------------------------------------------------
 * Batches: many independent lattices (different sizes, EOS, temperatures,
 * relaxation times, wall chemical potentials; one precision) advanced
 * together by one kernel launch per step over all their tiles,
 * with blocks of 16 steps replayed from a captured CUDA graph.  Every
 * lattice follows the same update as lbm_step.  Lattice i is addressed by
 * its index in the array given to lbm_batch_create.
 * ------------------------------------------------------------------------ */
typedef struct lbm_batch lbm_batch;

typedef struct {
    int nx, ny, walls;      /* as lbm_config */
    double tau, kappa, rho_ref;
    int eos;                /* as lbm_set_eos */
    double a, b, R, T_over_Tc, omega;
    double mu_bottom;       /* as lbm_set_wall_mu */
    int top_mode;
    double mu_top;
} lbm_instance;

/* Create count lattices on one device.  stream NULL: the batch creates its
 * own (graph capture needs one); else all work goes to that stream.  On
 * error *out is NULL and lbm_batch_last_error(NULL) explains. */
lbm_status lbm_batch_create(const lbm_instance *inst, int count, int precision,
                            void *stream, int device, lbm_batch **out);
/* lbm_init for lattice `index`; allowed while the batch has taken an even
 * number of steps (the in-place order is then the natural one). */
lbm_status lbm_batch_init(lbm_batch *b, int index, const double *rho,
                          const double *ux, const double *uy, int on_device);
/* Queue nsteps steps of every active lattice; all must be initialised. */
lbm_status lbm_batch_step(lbm_batch *b, int nsteps);
/* Take lattice `index` out of the batched launch (active = 0) or put it
 * back (active = 1).  An inactive lattice keeps its state and step count and
 * the per-lattice calls below still work on it: a sweep drops the lattices
 * that have converged so that the launch carries only the rest.  Allowed
 * after an even number of batch steps (the in-place order is then the
 * natural one); the next lbm_batch_step re-captures its graph. */
lbm_status lbm_batch_set_active(lbm_batch *b, int index, int active);
/* Per-lattice lbm_moments, lbm_get_populations and lbm_reduce. */
lbm_status lbm_batch_moments(lbm_batch *b, int index, double *rho, double *vx,
                             double *vy, double *mu, int on_device);
lbm_status lbm_batch_populations(lbm_batch *b, int index, double *f,
                                 int on_device);
lbm_status lbm_batch_reduce(lbm_batch *b, int index, double out[4]);
/* Tile shape of the batched kernel (as lbm_set_tile; default 32x32), or
 * the fastest configuration measured over nsteps steps (every tile shape
 * with each schedule of lbm_batch_schedule: 0 when some group of lattices
 * qualifies, 1, 2 and 4) with the state restored afterwards; *tx, *ty
 * receive the shape kept. */
lbm_status lbm_batch_set_tile(lbm_batch *b, int tx, int ty);
lbm_status lbm_batch_autotune(lbm_batch *b, int nsteps, int *tx, int *ty);
/* Schedule of the batched kernel.  The lattices go to the GPU in groups of
 * 32 (by index), one launch per group and step; the groups run on parallel
 * branches of the captured graph.  items_per_cta in 1 .. 64: each CTA takes
 * that many consecutive tiles of the group's work list, which mostly belong
 * to one lattice, so its descriptor is loaded once for them; more items per
 * CTA save that set-up, fewer balance the end of a step better.  0 (the
 * default): a group whose active lattices share nx, ny and walls and whose
 * every tile takes a TMA path (a sweep of physical parameters on one
 * geometry) is launched as a grid of one row of tiles per lattice, with the
 * descriptors passed as a kernel parameter and no work list; the other
 * groups take one item per CTA.  Speed only, results are unchanged.  -1
 * leaves the setting; *current (may be NULL) receives the value in use.
 * LBM_ERR_ARG outside -1 .. 64. */
lbm_status lbm_batch_schedule(lbm_batch *b, int items_per_cta, int *current);
/* Lattice count, total nodes, steps taken, tile shape (any may be NULL). */
lbm_status lbm_batch_info(const lbm_batch *b, int *count, long long *nodes,
                          long long *steps, int *tx, int *ty);
void lbm_batch_destroy(lbm_batch *b);
const char *lbm_batch_last_error(const lbm_batch *b);

/* ------------------------------------------------------------------------
 * Learned warm start: a small BF16 multilayer perceptron with FP32
 * accumulation (tensor-core kernels) that maps a case's parameters to its
 * converged observables, used to start a simulation near equilibrium.  The
 * paper has no counterpart; the simulation it initialises is the paper's.
 * Network: up to 16 inputs -> 3 x 128 tanh -> up to 16 linear outputs.
 * Parameters are FP32 in one array of lbm_mlp_param_count() values: per
 * layer the weights [k][n] (k inputs, n outputs; 16, 128, 128, 128 by
 * 128, 128, 128, 16), then the biases of the four layers.
 * ------------------------------------------------------------------------ */
typedef struct lbm_mlp lbm_mlp;
int lbm_mlp_param_count(void);
/* init: host array of the initial parameters. */
lbm_status lbm_mlp_create(int device, const float *init, lbm_mlp **out);
/* iters full-batch Adam steps (lr; betas 0.9, 0.999) minimising the mean
 * squared error between the first nout outputs and T.  X [B][nin] and
 * T [B][nout] are device FP32 arrays; *loss (may be NULL) receives the mean
 * squared error of the last step's forward pass. */
lbm_status lbm_mlp_train(lbm_mlp *m, const float *X, int nin, const float *T,
                         int nout, int B, int iters, float lr, float *loss);
/* The full-batch gradient of the loss of lbm_mlp_train (mean squared
 * error of the first nout outputs against T) with respect to the FP32
 * parameters, from one forward and backward pass of the training kernels
 * (BF16 weights, activations and layer deltas, FP32 accumulation); the
 * parameters and the optimiser state are left unchanged.  X, T as for
 * lbm_mlp_train (device); grad: host array of lbm_mlp_param_count()
 * values; *loss (may be NULL) receives the mean squared error. */
lbm_status lbm_mlp_gradient(lbm_mlp *m, const float *X, int nin, const float *T,
                            int nout, int B, float *grad, float *loss);
/* Y [B][nout] = the network's first nout outputs for X [B][nin] (device). */
lbm_status lbm_mlp_predict(lbm_mlp *m, const float *X, int nin, float *Y,
                           int nout, int B);
lbm_status lbm_mlp_get_params(lbm_mlp *m, float *out);  /* host FP32 */
void lbm_mlp_destroy(lbm_mlp *m);
const char *lbm_mlp_last_error(const lbm_mlp *m);

/* Allocation-free FP64 step, for callers that may not allocate device
 * memory: for example a host application whose own allocator owns the GPU
 * and forbids other code from calling cudaMalloc, or one that cannot accept
 * the device-wide synchronisation cudaMalloc and cudaFree can cause while
 * other work shares the GPU.  The paper has no counterpart: this is an
 * interface variant of lbm_step, not part of the method.
 *
 * f is the caller's device array of natural-order FP64 populations
 * [9][ny][nx] (the layout lbm_get_populations returns; solid rows unused),
 * advanced in place by nsteps steps of the same update as lbm_step, with
 * the EOS and wall arguments of lbm_set_eos and lbm_set_wall_mu.  cfg gives
 * nx, ny, walls, tau, kappa, stream and device; precision must be LBM_F64.
 * nsteps must be even (f is in natural order only between step pairs).
 * Work is queued on cfg->stream and the call returns without waiting.
 *
 * The call allocates nothing: the density buffers a context would own live
 * in one fixed device array of LBM_NOALLOC_SCRATCH_BYTES, which every GPU
 * that loads the library holds until the process exits.  A lattice needs
 * two density fields (8 nx nyf bytes each, nyf = ny - 2 with walls, else ny)
 * and two generations of the partial sums that cross tile edges, about
 * 1.2 nx nyf bytes each (the sizes a context allocates), each part rounded
 * up to 256 bytes: about 19.2 bytes a node, so 702 x 702 periodic is the
 * largest square that fits; larger lattices are rejected with LBM_ERR_ARG
 * and a message naming the bytes needed.  The first call on a device (and
 * the first after a device reset, which makes a new context) looks up the
 * array's device address (cudaGetSymbolAddress) and caches it with the
 * context's ID; make that first call before any stream capture.  All calls
 * share the array and each clears what must start at zero: calls that
 * overlap on the GPU race on it and must be serialised by the caller.
 * Errors are reported through lbm_last_error(NULL) of the calling thread. */
#define LBM_NOALLOC_SCRATCH_BYTES (18u * 65536u * 8u)
lbm_status lbm_step_noalloc(const lbm_config *cfg, int eos, double a,
                            double b, double R, double T_over_Tc,
                            double omega, double mu_bottom, int top_mode,
                            double mu_top, double *f, int nsteps);

/* Coexisting vapour and liquid densities and their common chemical
 * potential psi' at T = T_over_Tc * T_c (0 < T_over_Tc < 1): the Maxwell
 * equal-area construction of Sec. III (equal p0 and equal psi').  Host-only
 * helper for initial states. */
lbm_status lbm_eos_coexistence(int eos, double a, double b, double R,
                               double T_over_Tc, double omega, double *rho_v,
                               double *rho_l, double *mu_coex);

/* Bulk pressure p0 of the EOS at T = T_over_Tc * T_c for n densities:
 * Eq. 16 (vdW), Eq. 19 (RKS), Eq. 22 (PR), Eq. 25 (CS).  rho[n] in, p[n]
 * out, host arrays.  Host-only helper for measurements such as the Laplace
 * pressure jump (Sec. III); a density outside (0, pole of the EOS) gives
 * LBM_ERR_ARG and leaves p unspecified. */
lbm_status lbm_eos_pressure(int eos, double a, double b, double R,
                            double T_over_Tc, double omega, const double *rho,
                            double *p, size_t n);

/* Path class of every tile of the fused step for an nx x ny lattice (ny
 * counts the two solid rows when walls != 0) at tile shape tx x ty, one of
 * the compiled shapes: kinds[by * ntx + bx] = 2 for an interior tile (the
 * TMA or cp.async interior path), 1 for an edge tile (the TMA paths only:
 * its halo wraps around a periodic edge or meets a wall, or, on 32-wide
 * shapes, it is the ragged last tile, at least 4 nodes wide, of a periodic
 * direction), 0 for a general tile, with ntx = ceil(nx / tx), nty =
 * ceil(fluid rows / ty) and max >= ntx * nty entries in kinds (a host
 * array).  seams != 0 gives the classes of a lattice (single or in a
 * batch) whose shape has a TMA path; seams == 0 those of a shape without
 * one (edge tiles general).  Host-only, no device work; for choosing
 * lattice sizes and for tests.  LBM_ERR_ARG on a bad size, shape or a
 * short array. */
lbm_status lbm_tile_kinds(int nx, int ny, int walls, int tx, int ty, int seams,
                          int *kinds, size_t max);

/* Release the context and its device memory.  NULL is ignored. */
void lbm_destroy(lbm_ctx *ctx);

/* Message of the last error on ctx (or, when ctx is NULL, of the last
 * failed call without a context made by the calling thread: lbm_create,
 * the host EOS helpers, lbm_step_noalloc).  Never NULL. */
const char *lbm_last_error(const lbm_ctx *ctx);

/* ------------------------------------------------------------------------
 * Test hooks: host-side fault injection.  They make the library's own
 * failure paths run without any fault on the GPU; they are not needed for
 * normal use.
 * ------------------------------------------------------------------------ */

/* Limit, in SM clock cycles, of the step kernels' first wait for a tile's
 * staged data (the TMA paths).  Default about 2e9 (one second at 2 GHz);
 * cycles < 0 restores it; 0 gives up at once, without polling.  A
 * tile whose wait gives up waits (with the default limit) for its copies
 * still in flight, leaves its nodes untouched and raises a flag that the
 * next synchronising call on ctx (lbm_moments, lbm_reduce,
 * lbm_get_populations) reports as LBM_ERR_CUDA with a message naming the
 * timeout; the flag is then cleared.  The lattice is
 * then inconsistent: re-initialise it (lbm_init or lbm_set_state). */
lbm_status lbm_test_set_wait_cycles(lbm_ctx *ctx, long long cycles);

/* Make the device allocation after the next `after` ones (counted over the
 * whole library and every thread) fail as if the device were out of
 * memory; after < 0 disarms a pending failure.  The call that meets the
 * failure returns LBM_ERR_OOM and frees whatever it had allocated. */
void lbm_test_fail_device_alloc(int after);

/* Device allocations the library currently holds (contexts, batches,
 * networks and their staging buffers), for leak checks. */
long long lbm_test_device_allocs(void);

/* Bounds-checked debug build only (libcplbm_checked.so, CPLBM_CHECK_BOUNDS):
 * make the device checks treat each density buffer of ctx as rho_bytes long
 * (0 .. its real size), so that in-bounds accesses beyond that count as out
 * of bounds: they are skipped and the next synchronising call reports
 * LBM_ERR_CUDA naming an access outside its buffer.  A negative control of
 * the checks that makes no real out-of-bounds access.  LBM_ERR_STATE in the
 * product build; LBM_ERR_ARG outside that range. */
lbm_status lbm_test_shrink_bounds(lbm_ctx *ctx, long long rho_bytes);

/* The FP64 natural logarithm and reciprocal the FP64 step evaluates the EOS
 * and the collision with (a table-driven logarithm and a Newton-refined
 * reciprocal, each within a few ulp of log(x) and 1/x), applied on the
 * current device to the n host values x into the host arrays log_out and
 * rcp_out; for accuracy tests.  Synchronous.  LBM_ERR_ARG on a NULL buffer
 * or n < 0; errors go to lbm_last_error(NULL). */
lbm_status lbm_test_fp64_math(const double *x, int n, double *log_out, double *rcp_out);

#ifdef __cplusplus
}
#endif

#endif /* CPLBM_H */
