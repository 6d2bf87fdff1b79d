// Internal declarations shared by the host side (capi.cu) and the kernels
// (step.cu, fields.cu) of the cplbm library.  Nothing here is public ABI.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda.h>  // CUtensorMap (tensor-map descriptors only)
#include <cuda_runtime.h>

namespace cplbm {

enum Precision { P_F64 = 0, P_F32 = 1, P_F32_OFF = 2, P_F16_OFF = 3 };
enum EosKind { EOS_VDW = 0, EOS_CS = 1, EOS_PR = 2, EOS_RKS = 3 };

// Tile of the field kernels (moments, reductions): independent of the step.
constexpr int FIELD_TILE_X = 64;
constexpr int FIELD_TILE_Y = 16;
// Threads of a step CTA.  The step's tile shape (tx x ty fluid nodes per
// CTA) is a property of the lattice: it also fixes the grid on which the
// step hands the next density over (see step.cu), so every kernel that reads
// the density uses the lattice's tx, ty.
constexpr int STEP_THREADS = 256;

// Classes of partial density sums that cross a tile boundary, named by the
// direction from the receiving node's tile to the tile that wrote them.
enum Ring { R_L = 0, R_R, R_B, R_T, R_BL, R_BR, R_TL, R_TR, R_COUNT };

// EOS constants as the context holds them (double).
struct EosParams {
    int kind;
    double a, b, RT;   // RT = R * T
    double aalpha;     // a * alpha(T) (PR, RKS); a otherwise
};

// The same constants in the arithmetic type T of a kernel, with the
// combinations the bulk chemical potentials use precomputed (set_consts):
//   quarter_b = b / 4 (CS), pr_c = a alpha / (2 sqrt2 b) (PR),
//   pr_s2m1 = sqrt2 - 1, pr_s2p1 = sqrt2 + 1 (PR), rks_c = a alpha / b (RKS).
template <class T> struct EosT {
    int kind;
    T a, b, RT, aalpha, quarter_b, pr_c, pr_s2m1, pr_s2p1, rks_c;
};

// Physical constants of one lattice in the arithmetic type T, filled on the
// host by set_consts: kernels do no double arithmetic and no double-to-float
// conversion (GB300's FP64 pipe is narrow enough that two double divisions
// per thread showed up as a busy FP64 pipe in the FP32 step).
template <class T> struct Consts {
    T tau, omega, kappa, rho_ref, mu_bottom, mu_top;   // omega = 1 / tau
    EosT<T> eos;
};

// Geometry, storage and physics of one lattice as the kernels see it.
//
// Device layout (all row pitches are `pitch` elements, pitch >= nx):
//  pops   [8][nyf][pitch]   moving populations f_1..f_8 in the AA-pattern
//                           in-place order (see step.cu), storage type;
//  rho[k] [nyf][pitch]      k = 0, 1: density of the current / next step
//                           (offset precisions: rho - rho_ref), where a
//                           node on a tile's edge holds only the part
//                           summed inside its own tile;
//  ring[k][c]               k = 0, 1: the partial sums of class c written
//                           by the neighbouring tile, compact: a class
//                           holds one entry per tile along the axis it
//                           crosses (ring_index in device_common.cuh).
//                           L, R: [ceil(nx / 32)][nyf_pad], one column per
//                           tile column; B, T: [ceil(nyf / 16)][pitch], one
//                           row per tile row; corners: [ceil(nyf / 16)]
//                           [ceil(nx / 32)].  The strides fit the smallest
//                           compiled tile (32 x 16), so every tile shape
//                           uses the same buffers.
// nyf is the number of fluid rows: ny - 2 with walls, ny otherwise; fluid
// row r is lattice row r + 1 with walls.
struct Lattice {
    void *pops;
    void *rho[2];
    void *ring[2][R_COUNT];
    int nx, ny, nyf, pitch, nyf_pad;
    int tx, ty;          // step tile shape
    int walls;
    long long plane;     // nyf * pitch
    double tau, kappa, rho_ref;
    EosParams eos;
    double mu_bottom, mu_top;
    int top_mode;
    int precision;
    int *err;            // device flag: a bounded wait in a kernel gave up
    long long wait_cycles;  // SM clocks a tile waits for its staged data
                            // before it gives up (WAIT_CYCLES_DEFAULT)
    Consts<float> cf;    // tau .. mu_top and eos as float (set_consts)
    Consts<double> cd;   // ... and as double
#ifdef CPLBM_CHECK_BOUNDS
    // bounds-checked build: bytes of pops, of each density buffer and of
    // each partial-sum class (set_bounds)
    long long b_pops, b_rho, b_ring[R_COUNT];
#endif
};

// Refresh L.cf and L.cd from the double fields; call after any change of
// tau, kappa, rho_ref, eos, mu_bottom or mu_top.
void set_consts(Lattice &L);

template <class T> __host__ __device__ __forceinline__ const Consts<T> &consts(const Lattice &L);
template <> __host__ __device__ __forceinline__ const Consts<float> &consts<float>(const Lattice &L)
{
    return L.cf;
}
template <> __host__ __device__ __forceinline__ const Consts<double> &consts<double>(const Lattice &L)
{
    return L.cd;
}

// Tensor-map descriptors for the TMA loads of the step's interior tiles:
// the population array (3-D: x, fluid row, plane) and the two density
// buffers (2-D), with boxes sized for the tile shape (tx, ty).
struct TmaMaps {
    CUtensorMap pops;
    CUtensorMap rho[2];
    int valid;
    int tx, ty;
};

// tma.cu: build the maps for lattice L and its current tile shape; false
// (with a message) when the layout does not allow TMA.
bool build_tma_maps(const Lattice &L, TmaMaps *m, char *err, size_t errlen);

// Bits of Lattice::err.  ERR_BOUNDS: a global access outside its buffer,
// caught (and skipped) by the bounds-checked build.
enum { ERR_WAIT_TIMEOUT = 1, ERR_BOUNDS = 2 };
// Limit of the step kernels' first wait for a tile's staged data: about a
// second at the 2 GHz SM clock, far beyond any copy's latency.  A wait
// that reaches it raises ERR_WAIT_TIMEOUT, drains the tile's copies (with
// this same long limit, whatever Lattice::wait_cycles says) and leaves the
// tile untouched.
constexpr long long WAIT_CYCLES_DEFAULT = 2000000000LL;

// Entries of partial-sum class c (R_L .. R_TR) of one generation: one
// column per 32-wide tile column (L, R), one row per 16-high tile row
// (B, T), one entry per such tile (corners); see ring_index.
inline size_t ring_elems(const Lattice &L, int c)
{
    const size_t ncx = ((size_t)L.nx + 31) / 32, ncy = ((size_t)L.nyf + 15) / 16;
    if (c == R_L || c == R_R) return ncx * L.nyf_pad;
    if (c == R_B || c == R_T) return ncy * L.pitch;
    return ncy * ncx;
}

// Every device allocation of the library goes through these two (capi.cu),
// which count the live allocations and can be told to fail one on purpose
// (lbm_test_fail_device_alloc): the host-side fault injection of the tests.
cudaError_t dev_alloc(void **p, size_t bytes);
void dev_free(void *p);

// Sizes of the storage types per precision.
inline size_t pop_bytes(int prec)
{
    return prec == P_F64 ? 8 : prec == P_F16_OFF ? 2 : 4;
}
inline size_t rho_bytes(int prec) { return prec == P_F64 ? 8 : 4; }

#ifdef CPLBM_CHECK_BOUNDS
// Bounds-checked build: record the extents the device checks compare with;
// pops_bytes counts from L.pops to the end of the population storage,
// rho_buf_bytes is the size of each density buffer.
inline void set_bounds(Lattice &L, long long pops_bytes, long long rho_buf_bytes)
{
    const long long rb = (long long)rho_bytes(L.precision);
    L.b_pops = pops_bytes;
    L.b_rho = rho_buf_bytes;
    for (int c = 0; c < R_COUNT; ++c) L.b_ring[c] = (long long)ring_elems(L, c) * rb;
}
#endif

// Launchers (step.cu).  `cur` selects rho[cur] / ring[cur] as the current
// density and `parity` the AA phase of the step being taken.
cudaError_t launch_step(const Lattice &L, int parity, int cur,
                        cudaStream_t s, const TmaMaps *maps = nullptr);
// Whether the step has a kernel for tile shape tx x ty in precision prec,
// and the default shape of a precision.
bool step_shape_supported(int prec, int tx, int ty);
void step_default_shape(int prec, int *tx, int *ty);
// The compiled tile shapes, in a fixed order: returns how many, fills up to
// `max` pairs.
int step_shapes(int *tx, int *ty, int max);

// Baseline step with the pressure-tensor force (Eq. 5): FP32 (tiles 64x16,
// two nodes per lane, and 32x32) and FP64 (32x16), periodic lattices;
// pt_shape gives the default tile, pt_shape_supported the others.
// maps: the TMA maps of that tile (interior and seam tiles take the TMA
// path), or nullptr for the general path only.
cudaError_t launch_step_pt(const Lattice &L, int parity, int cur, cudaStream_t s,
                           const TmaMaps *maps = nullptr);
void pt_shape(int prec, int *tx, int *ty);
bool pt_shape_supported(int prec, int tx, int ty);

// Edge tiles the TMA tile paths may take (bit 0: periodic left and right,
// bit 1: periodic bottom and top, bit 2: the bottom and top wall rows, bit
// 3: the ragged last tile of a periodic direction).  Periodic edges: at
// least three full tiles span the lattice, and the last tile across the
// edge is full or at least 4 nodes wide, so the halo that wraps around the
// edge has the layout of an interior halo.  That ragged last tile takes the
// TMA path too on 32-wide tiles (bit 3), whose tile function places the
// right and top tile edges at the tile's own width and height; the
// two-nodes-per-lane path leaves it to the general path.  Walls: at least
// two tile rows, the bottom one full and the one above it full or at least
// 4 rows high, so the bottom wall tile's halo above sees interior tile
// edges; the top wall tile may be ragged down to two rows (tile_kind).
__host__ __device__ inline int seam_bits(const Lattice &L, int tx, int ty)
{
    int s = 0;
    const int rx = L.nx % tx, ry = L.nyf % ty, nfy = L.nyf / ty;
    if (L.nx / tx >= 3 && (rx == 0 || rx >= 4)) s |= 1;
    if (!L.walls && nfy >= 3 && (ry == 0 || ry >= 4)) s |= 2;
    if (L.walls && (nfy >= 2 || (nfy == 1 && ry >= 4))) s |= 4;
    if (tx == 32) s |= 8;
    return s;
}

// Path class of tile (bx, by): TILE_INTERIOR when the tile is full, its
// halo neither wraps nor meets a wall, and its halo's tile edges sit where
// they sit between full tiles: every neighbour is full, except that the
// last (ragged) tile of a row or column may be the right or top neighbour
// when it is at least 4 nodes wide (its far edge then lies beyond the
// 2-node halo, and the halo's staged rows and columns stay inside the
// arrays); TILE_SEAM (an edge tile of the TMA paths) when the same holds
// along each direction except that the halo wraps around a periodic edge
// allowed by `seams` (the ragged last tile there too when `seams` allows
// it), or the tile is a bottom or top wall tile allowed by `seams`
// (seam_bits); TILE_GENERAL otherwise.  A top wall tile of one
// fluid row stays general: that row is then also the tile's bottom edge,
// which holds partial sums from the tile below, and the Eq. 28 average of
// the halo's outermost columns reads it one column beyond the halo, where
// the TMA paths add no partial sums.
enum { TILE_GENERAL = 0, TILE_SEAM = 1, TILE_INTERIOR = 2 };
__host__ __device__ inline int tile_kind(const Lattice &L, int tx, int ty, int bx, int by,
                                         int seams)
{
    const int nfx = L.nx / tx, nfy = L.nyf / ty;
    const int xhi = L.nx - nfx * tx >= 4 ? nfx - 1 : nfx - 2;
    const int yhi = L.nyf - nfy * ty >= 4 ? nfy - 1 : nfy - 2;
    const bool ix = bx >= 1 && bx <= xhi, iy = by >= 1 && by <= yhi;
    if (ix && iy) return TILE_INTERIOR;
    const int nty = (L.nyf + ty - 1) / ty;
    const bool wall = (seams & 4) && (by == 0 || (by == nty - 1 && L.nyf - by * ty >= 2));
    const bool ragged = (seams & 8) != 0;
    const bool sx = ix || ((seams & 1) && (bx < nfx || ragged));
    const bool sy = iy || ((seams & 2) && (by < nfy || ragged)) || wall;
    return sx && sy ? TILE_SEAM : TILE_GENERAL;
}

// A tile of one lattice of a batch: the batched step walks a list of these
// (step.cu).
struct WorkItem {
    int inst;      // index into the batch's Lattice array
    int bx, by;    // tile position
    int kind;      // tile_kind of the tile, | ITEM_NO_TMA when the lattice
                   // has no usable tensor maps
};
enum { ITEM_NO_TMA = 4 };
// Most work items one CTA of the batched step takes (lbm_batch_schedule).
constexpr int BATCH_MAX_PER_CTA = 64;
// Tensor maps of the lattices of one batched launch, a kernel parameter:
// for lattice inst0 + k, the population map and the map of the density
// buffer the step reads.  Batches of more lattices take one launch per
// group of BATCH_LAUNCH_LATTICES.
constexpr int BATCH_LAUNCH_LATTICES = 32;
struct BatchMaps {
    CUtensorMap pops[BATCH_LAUNCH_LATTICES];
    CUtensorMap rho[BATCH_LAUNCH_LATTICES];
};
// A group of lattices of one geometry (nx, ny, walls; the physics may
// differ) whose every tile takes a TMA path, as one kernel parameter of
// 24 KB: descriptors and the maps of the step's density buffer.  Lattice k
// of the launch is grid row k.
struct UniformGroup {
    CUtensorMap pops[BATCH_LAUNCH_LATTICES];
    CUtensorMap rho[BATCH_LAUNCH_LATTICES];
    Lattice L[BATCH_LAUNCH_LATTICES];
};
// One launch of a batch's work list (batch.cu builds it).
struct BatchList {
    const Lattice *lats = nullptr;    // device: descriptors of all lattices
    const WorkItem *items = nullptr;  // device: tiles of this launch's lattices
    int n_items = 0;
    int per_cta = 1;                  // consecutive items per CTA
    bool tma_only = false;            // every item takes a TMA path
    int inst0 = 0;                    // first lattice of this launch
    const BatchMaps *maps = nullptr;  // host: their maps for the step's density
    // Set for a group of one geometry (instead of the work list): the
    // launch is one grid row of ntx * nty tiles per lattice.
    const UniformGroup *uniform = nullptr;  // host
    int n_uniform = 0, ntx = 0, nty = 0, seams = 0;
    bool walls = false;
};
// One step of a group of lattices of a batch in one launch: each CTA takes
// per_cta consecutive items of the work list.  All lattices share
// precision, tile shape and step parity.  With tma_only the kernel holds
// no general tile path (fewer registers live, less shared memory).
cudaError_t launch_step_batch(const BatchList &w, int parity, int cur, int precision,
                              int tx, int ty, cudaStream_t s);

// fields.cu
// The FP64 logarithm and reciprocal of the step kernels (log_tab, rcp_nr)
// on n device values, into lg and rc (device).
cudaError_t launch_fp64_math(const double *x, int n, double *lg, double *rc,
                             cudaStream_t s);
// Equilibrium initial state from double fields [ny][nx] on the device:
// fills pops (parity 0 order) and rho[0]/ring[0]; counts invalid densities
// into *bad (device int, zeroed by the caller).
cudaError_t launch_init(const Lattice &L, const double *rho, const double *ux,
                        const double *uy, int *bad, cudaStream_t s);

// Macroscopic fields of the state (any output may be NULL; [ny][nx]), and
// optional FP64 reductions into red[0..3] (sum rho, sum rho vx, sum rho vy,
// max |rho - prev| as ordered bits) with `prev` the snapshot density
// [ny][nx] that is then updated; nonfinite counts into *bad.
cudaError_t launch_macro(const Lattice &L, int parity, int cur, double *rho,
                         double *vx, double *vy, double *mu, double *red,
                         double *prev, int *bad, cudaStream_t s);

// Natural-order FP64 populations [9][ny][nx].
cudaError_t launch_populations(const Lattice &L, int parity, int cur,
                               double *f, cudaStream_t s);

// Re-sum the current density of every node into rho[dst] (all nodes full,
// ring classes zero): used when restoring a checkpoint.
cudaError_t launch_gather_rho(const Lattice &L, int cur, void *dst,
                              cudaStream_t s);

// capi.cu: host helpers for entry points outside it.
bool host_critical(int kind, double a, double b, double R, double *Tc,
                   double *rhoc);
double host_alpha(int kind, double Tr, double omega);
void set_global_error(const char *msg);

}  // namespace cplbm
