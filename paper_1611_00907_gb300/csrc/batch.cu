// Batched lattices (lbm_batch_* in include/cplbm.h): many independent
// lattices of different sizes, EOS, temperatures, relaxation times and wall
// chemical potentials advanced together, one kernel launch per step over a
// work list of tiles (a few consecutive tiles per CTA), with blocks of steps
// replayed from a captured CUDA graph.  Each lattice is a full context (its
// own device state), so the per-lattice calls (moments, reductions) are the
// single-lattice ones.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "context.h"
#include "trace.h"

using namespace cplbm;

namespace {

// The lattices [inst0, inst0 + BATCH_LAUNCH_LATTICES) of a batch: one
// launch per step over their segment of the work list.
struct Group {
    int inst0 = 0;
    int item0 = 0, n_items = 0;    // segment of the device work list
    bool tma_only = false;         // no item takes the general path
    std::unique_ptr<BatchMaps> maps[2];  // by the density buffer a step reads
    // active lattices of one geometry, every tile on a TMA path: the
    // grid-per-lattice launch (step_uniform_kernel) can take the group
    std::unique_ptr<UniformGroup> uniform[2];
    int n_uniform = 0, ntx = 0, nty = 0, seams = 0;
    bool walls = false;
};

}  // namespace

struct lbm_batch {
    std::vector<lbm_ctx *> inst;
    std::vector<char> active;  // lattices in the launch
    int precision = 0, device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int tx = 32, ty = 32;
    Lattice *d_lats = nullptr;
    WorkItem *d_items = nullptr;
    // work items per CTA of the batched kernel; 0: a grid row per lattice
    // for the groups of one geometry (lbm_batch_schedule), one item per CTA
    // for the others
    int per_cta = 0;
    int n_items = 0;            // all groups
    std::vector<Group> groups;
    // graph branches: the groups after the first run on their own streams
    // inside the captured graph (their lattices are independent)
    std::vector<cudaStream_t> aux;
    std::vector<cudaEvent_t> joins;
    cudaEvent_t fork = nullptr;
    long long t = 0;
    long long nodes = 0;
    cudaGraphExec_t exec = nullptr;  // GRAPH_STEPS steps from an even step
    std::string err;
};

namespace {

constexpr int GRAPH_STEPS = 16;
thread_local std::string g_batch_err;  // message of the last failed create

lbm_status bfail(lbm_batch *b, lbm_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    b->err = buf;
    return s;
}

#define BCUDA(b, call)                                                       \
    do {                                                                     \
        cudaError_t e_ = (call);                                             \
        if (e_ != cudaSuccess)                                               \
            return bfail((b), e_ == cudaErrorMemoryAllocation ? LBM_ERR_OOM  \
                                                              : LBM_ERR_CUDA, \
                         "%s: %s", #call, cudaGetErrorString(e_));           \
    } while (0)

void drop_graph(lbm_batch *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
}

// Apply the batch tile shape to every lattice and rebuild the device copies
// of the descriptors, the work list and the groups' tensor maps.
lbm_status rebuild(lbm_batch *b)
{
    drop_graph(b);
    const int n = (int)b->inst.size();
    std::vector<Lattice> lats;
    std::vector<WorkItem> items;
    // edge tiles (periodic seams, wall rows) take the TMA paths too: the
    // 32-wide one, and for FP32 arithmetic the 64-wide pair path
    // (step_batch_kernel); FP64 64-wide tiles have no TMA path
    const bool tma_shape = b->tx == 32 || (b->tx == 64 && b->precision != LBM_F64);
    b->groups.clear();
    for (int g0 = 0; g0 < n; g0 += BATCH_LAUNCH_LATTICES) {
        Group grp;
        grp.inst0 = g0;
        grp.item0 = (int)items.size();
        for (int p = 0; p < 2; ++p) {
            grp.maps[p].reset(new (std::nothrow) BatchMaps);
            if (!grp.maps[p]) return bfail(b, LBM_ERR_OOM, "host allocation failed");
            std::memset(grp.maps[p].get(), 0, sizeof(BatchMaps));
        }
        std::vector<WorkItem> gen, edge, inner;
        for (int i = g0; i < n && i < g0 + BATCH_LAUNCH_LATTICES; ++i) {
            lbm_ctx *c = b->inst[i];
            c->L.tx = b->tx;
            c->L.ty = b->ty;
            ctx_refresh_maps(c);
            lats.push_back(c->L);
            const bool maps_ok = tma_shape && c->use_tma && c->maps.valid;
            if (maps_ok)
                for (int p = 0; p < 2; ++p) {
                    grp.maps[p]->pops[i - g0] = c->maps.pops;
                    grp.maps[p]->rho[i - g0] = c->maps.rho[p];
                }
            if (!b->active[i]) continue;
            const Lattice &L = c->L;
            const int ntx = (L.nx + b->tx - 1) / b->tx, nty = (L.nyf + b->ty - 1) / b->ty;
            const int seams = tma_shape ? seam_bits(L, b->tx, b->ty) : 0;
            const int no_tma = maps_ok ? 0 : ITEM_NO_TMA;
            for (int by = 0; by < nty; ++by)
                for (int bx = 0; bx < ntx; ++bx) {
                    const int kind = tile_kind(L, b->tx, b->ty, bx, by, seams);
                    (kind == TILE_GENERAL ? gen : kind == TILE_SEAM ? edge : inner)
                        .push_back({i, bx, by, kind | no_tma});
                }
        }
        // General tiles cost a few interior tiles each, edge tiles (seams,
        // walls) somewhat more than one.  CTAs take items in list order,
        // backwards on odd steps: the interior tiles go in two halves at the
        // ends, so that in either direction a step ends on short items and
        // the CTAs finish close together, and the edge and general tiles
        // between them, each class in one run, so that the CTAs of an SM
        // mostly run the same code path at a time (the batched kernel holds
        // three large ones and the instruction cache does not hold them all).
        const size_t h = inner.size() / 2;
        items.insert(items.end(), inner.begin(), inner.begin() + h);
        items.insert(items.end(), edge.begin(), edge.end());
        items.insert(items.end(), gen.begin(), gen.end());
        items.insert(items.end(), inner.begin() + h, inner.end());
        grp.n_items = (int)items.size() - grp.item0;
        grp.tma_only = tma_shape;
        for (int k = grp.item0; k < (int)items.size(); ++k)
            if ((items[k].kind & 3) == TILE_GENERAL || (items[k].kind & ITEM_NO_TMA))
                grp.tma_only = false;
        // one geometry among the active lattices: the grid-per-lattice launch
        int first = -1;
        bool same = grp.tma_only && grp.n_items > 0;
        for (int i = g0; same && i < n && i < g0 + BATCH_LAUNCH_LATTICES; ++i) {
            if (!b->active[i]) continue;
            const Lattice &L = b->inst[i]->L;
            if (first < 0) first = i;
            const Lattice &F = b->inst[first]->L;
            same = L.nx == F.nx && L.ny == F.ny && L.walls == F.walls;
        }
        if (same && first >= 0) {
            const Lattice &F = b->inst[first]->L;
            grp.ntx = (F.nx + b->tx - 1) / b->tx;
            grp.nty = (F.nyf + b->ty - 1) / b->ty;
            grp.seams = seam_bits(F, b->tx, b->ty);
            grp.walls = F.walls != 0;
            for (int p = 0; p < 2; ++p) {
                grp.uniform[p].reset(new (std::nothrow) UniformGroup);
                if (!grp.uniform[p]) return bfail(b, LBM_ERR_OOM, "host allocation failed");
                std::memset(grp.uniform[p].get(), 0, sizeof(UniformGroup));
            }
            int k = 0;
            for (int i = g0; i < n && i < g0 + BATCH_LAUNCH_LATTICES; ++i) {
                if (!b->active[i]) continue;
                const lbm_ctx *c = b->inst[i];
                for (int p = 0; p < 2; ++p) {
                    grp.uniform[p]->pops[k] = c->maps.pops;
                    grp.uniform[p]->rho[k] = c->maps.rho[p];
                    grp.uniform[p]->L[k] = c->L;
                }
                ++k;
            }
            grp.n_uniform = k;
        }
        b->groups.push_back(std::move(grp));
    }
    dev_free(b->d_lats);
    dev_free(b->d_items);
    b->d_lats = nullptr;
    b->d_items = nullptr;
    BCUDA(b, dev_alloc((void **)&b->d_lats, lats.size() * sizeof(Lattice)));
    BCUDA(b, dev_alloc((void **)&b->d_items, (items.size() + 1) * sizeof(WorkItem)));
    BCUDA(b, cudaMemcpy(b->d_lats, lats.data(), lats.size() * sizeof(Lattice),
                        cudaMemcpyHostToDevice));
    if (!items.empty())
        BCUDA(b, cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(WorkItem),
                            cudaMemcpyHostToDevice));
    b->n_items = (int)items.size();
    // one stream and join event per group after the first, for the graph
    while (b->aux.size() + 1 < b->groups.size()) {
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr;
        BCUDA(b, cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        b->aux.push_back(st);
        BCUDA(b, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        b->joins.push_back(ev);
    }
    if (!b->fork && b->groups.size() > 1)
        BCUDA(b, cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
    return LBM_OK;
}

BatchList work_list(const lbm_batch *b, const Group &g, int cur)
{
    BatchList w;
    w.lats = b->d_lats;
    w.items = b->d_items + g.item0;
    w.n_items = g.n_items;
    w.per_cta = b->per_cta > 0 ? b->per_cta : 1;
    w.tma_only = g.tma_only;
    w.inst0 = g.inst0;
    w.maps = g.maps[cur].get();
    if (b->per_cta == 0 && g.n_uniform > 0) {
        w.uniform = g.uniform[cur].get();
        w.n_uniform = g.n_uniform;
        w.ntx = g.ntx;
        w.nty = g.nty;
        w.seams = g.seams;
        w.walls = g.walls;
    }
    return w;
}

// One step of every group; group k on streams[k] (the batch stream for the
// direct launches).
cudaError_t launch_groups(const lbm_batch *b, int p, const cudaStream_t *streams)
{
    for (size_t k = 0; k < b->groups.size(); ++k) {
        const Group &g = b->groups[k];
        if (g.n_items == 0) continue;
        cudaError_t e = launch_step_batch(work_list(b, g, p), p, p, b->precision, b->tx,
                                          b->ty, streams[k]);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

lbm_status launch_one(lbm_batch *b)
{
    const int p = (int)(b->t & 1);
    std::vector<cudaStream_t> streams(b->groups.size(), b->stream);
    BCUDA(b, launch_groups(b, p, streams.data()));
    ++b->t;
    return LBM_OK;
}

lbm_status ensure_graph(lbm_batch *b)
{
    if (b->exec) return LBM_OK;
    std::vector<cudaStream_t> streams(b->groups.size(), b->stream);
    for (size_t k = 1; k < b->groups.size(); ++k) streams[k] = b->aux[k - 1];
    cudaGraph_t g = nullptr;
    BCUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    if (b->groups.size() > 1) {  // fork: the branches start after the batch stream
        e = cudaEventRecord(b->fork, b->stream);
        for (size_t k = 1; k < b->groups.size() && e == cudaSuccess; ++k)
            e = cudaStreamWaitEvent(streams[k], b->fork, 0);
    }
    for (int k = 0; k < GRAPH_STEPS && e == cudaSuccess; ++k)
        e = launch_groups(b, k & 1, streams.data());
    for (size_t k = 1; k < b->groups.size() && e == cudaSuccess; ++k) {  // join
        e = cudaEventRecord(b->joins[k - 1], streams[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->joins[k - 1], 0);
    }
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return bfail(b, LBM_ERR_CUDA, "graph capture: %s",
                     cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->exec = nullptr;
        return bfail(b, LBM_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
    return LBM_OK;
}

lbm_status check_index(lbm_batch *b, int index)
{
    if (index < 0 || index >= (int)b->inst.size())
        return bfail(b, LBM_ERR_ARG, "lattice index %d out of range", index);
    return LBM_OK;
}

lbm_status forward(lbm_batch *b, lbm_ctx *c, lbm_status st)
{
    if (st != LBM_OK) b->err = lbm_last_error(c);
    return st;
}

}  // namespace

extern "C" {

lbm_status lbm_batch_create(const lbm_instance *inst, int count, int precision,
                            void *stream, int device, lbm_batch **out)
{
    if (out) *out = nullptr;
    if (!inst || !out || count <= 0) {
        g_batch_err = "need at least one instance and an output pointer";
        return LBM_ERR_ARG;
    }
    if (precision < LBM_F64 || precision > LBM_F16_OFFSET) {
        g_batch_err = "unknown precision";
        return LBM_ERR_ARG;
    }
    lbm_batch *b = new (std::nothrow) lbm_batch();
    if (!b) {
        g_batch_err = "host allocation failed";
        return LBM_ERR_OOM;
    }
    b->precision = precision;
    b->device = device;
    lbm_status st = LBM_OK;
    if (cudaSetDevice(device) != cudaSuccess) {
        g_batch_err = "cudaSetDevice failed";
        delete b;
        return LBM_ERR_CUDA;
    }
    if (stream) {
        b->stream = (cudaStream_t)stream;
    } else {  // graph capture needs a stream other than the legacy one
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            g_batch_err = "cudaStreamCreate failed";
            delete b;
            return LBM_ERR_CUDA;
        }
        b->own_stream = true;
    }
    // the default shape (lbm_batch_autotune picks among all of them)
    b->tx = 32;
    b->ty = 32;
    for (int i = 0; i < count && st == LBM_OK; ++i) {
        const lbm_instance &q = inst[i];
        lbm_config cfg{q.nx, q.ny, q.walls, q.tau, q.kappa, q.rho_ref, precision,
                       (void *)b->stream, device};
        lbm_ctx *c = nullptr;
        st = lbm_create(&cfg, &c);
        if (st != LBM_OK) {
            bfail(b, st, "lattice %d: %s", i, lbm_last_error(nullptr));
            break;
        }
        b->inst.push_back(c);
        b->active.push_back(1);
        st = lbm_set_eos(c, q.eos, q.a, q.b, q.R, q.T_over_Tc, q.omega);
        if (st == LBM_OK) st = lbm_set_wall_mu(c, q.mu_bottom, q.top_mode, q.mu_top);
        if (st != LBM_OK) bfail(b, st, "lattice %d: %s", i, lbm_last_error(c));
        b->nodes += (long long)q.nx * q.ny;
    }
    if (st == LBM_OK) st = rebuild(b);
    if (st != LBM_OK) {
        g_batch_err = b->err;
        lbm_batch_destroy(b);
        return st;
    }
    *out = b;
    return LBM_OK;
}

lbm_status lbm_batch_init(lbm_batch *b, int index, const double *rho,
                          const double *ux, const double *uy, int on_device)
{
    CPLBM_TRACE("lbm_batch_init");
    if (!b) return LBM_ERR_ARG;
    lbm_status st = check_index(b, index);
    if (st != LBM_OK) return st;
    if (b->t & 1)
        return bfail(b, LBM_ERR_STATE, "lattices can be initialised only after "
                     "an even number of batch steps (now %lld)", b->t);
    lbm_ctx *c = b->inst[index];
    st = forward(b, c, lbm_init(c, rho, ux, uy, on_device));
    if (st == LBM_OK) c->t = b->t;  // same in-place phase as the batch
    return st;
}

lbm_status lbm_batch_step(lbm_batch *b, int nsteps)
{
    CPLBM_TRACE("lbm_batch_step");
    if (!b) return LBM_ERR_ARG;
    if (nsteps < 0) return bfail(b, LBM_ERR_ARG, "nsteps must be >= 0");
    for (size_t i = 0; i < b->inst.size(); ++i)
        if (!b->inst[i]->initialized)
            return bfail(b, LBM_ERR_STATE, "lattice %zu is not initialised", i);
    BCUDA(b, cudaSetDevice(b->device));
    const long long t0 = b->t;
    int left = b->n_items > 0 ? nsteps : 0;  // nothing to launch: time only
    lbm_status st = LBM_OK;
    if (left > 0 && (b->t & 1)) {
        st = launch_one(b);
        --left;
    }
    if (st == LBM_OK && left >= GRAPH_STEPS) st = ensure_graph(b);
    while (st == LBM_OK && left >= GRAPH_STEPS) {
        cudaError_t e = cudaGraphLaunch(b->exec, b->stream);
        if (e != cudaSuccess) {
            st = bfail(b, LBM_ERR_CUDA, "graph launch: %s", cudaGetErrorString(e));
            break;
        }
        b->t += GRAPH_STEPS;
        left -= GRAPH_STEPS;
    }
    while (st == LBM_OK && left > 0) {
        st = launch_one(b);
        --left;
    }
    if (b->n_items == 0) b->t += nsteps;
    for (size_t i = 0; i < b->inst.size(); ++i)
        if (b->active[i]) b->inst[i]->t += b->t - t0;
    return st;
}

lbm_status lbm_batch_set_active(lbm_batch *b, int index, int active)
{
    if (!b) return LBM_ERR_ARG;
    lbm_status st = check_index(b, index);
    if (st != LBM_OK) return st;
    if (b->t & 1)
        return bfail(b, LBM_ERR_STATE, "lattices can leave or join the launch "
                     "only after an even number of batch steps (now %lld)", b->t);
    const char want = active ? 1 : 0;
    if (b->active[index] == want) return LBM_OK;
    b->active[index] = want;
    BCUDA(b, cudaSetDevice(b->device));
    return rebuild(b);
}

lbm_status lbm_batch_moments(lbm_batch *b, int index, double *rho, double *vx,
                             double *vy, double *mu, int on_device)
{
    CPLBM_TRACE("lbm_batch_moments");
    if (!b) return LBM_ERR_ARG;
    lbm_status st = check_index(b, index);
    if (st != LBM_OK) return st;
    lbm_ctx *c = b->inst[index];
    return forward(b, c, lbm_moments(c, rho, vx, vy, mu, on_device));
}

lbm_status lbm_batch_populations(lbm_batch *b, int index, double *f, int on_device)
{
    if (!b) return LBM_ERR_ARG;
    lbm_status st = check_index(b, index);
    if (st != LBM_OK) return st;
    lbm_ctx *c = b->inst[index];
    return forward(b, c, lbm_get_populations(c, f, on_device));
}

lbm_status lbm_batch_reduce(lbm_batch *b, int index, double out[4])
{
    CPLBM_TRACE("lbm_batch_reduce");
    if (!b) return LBM_ERR_ARG;
    lbm_status st = check_index(b, index);
    if (st != LBM_OK) return st;
    lbm_ctx *c = b->inst[index];
    return forward(b, c, lbm_reduce(c, out));
}

lbm_status lbm_batch_set_tile(lbm_batch *b, int tx, int ty)
{
    CPLBM_TRACE("lbm_batch_set_tile");
    if (!b) return LBM_ERR_ARG;
    if (!step_shape_supported(b->precision, tx, ty))
        return bfail(b, LBM_ERR_ARG, "no step kernel for tile %d x %d", tx, ty);
    BCUDA(b, cudaSetDevice(b->device));
    // re-split each lattice's current density for the new tile grid
    for (lbm_ctx *c : b->inst) {
        lbm_status st = forward(b, c, lbm_set_tile(c, tx, ty));
        if (st != LBM_OK) return st;
    }
    b->tx = tx;
    b->ty = ty;
    return rebuild(b);
}

lbm_status lbm_batch_schedule(lbm_batch *b, int items_per_cta, int *current)
{
    if (!b) return LBM_ERR_ARG;
    if (items_per_cta < -1 || items_per_cta > BATCH_MAX_PER_CTA)
        return bfail(b, LBM_ERR_ARG, "items per CTA must be 0 .. %d, or -1 (got %d)",
                     BATCH_MAX_PER_CTA, items_per_cta);
    if (items_per_cta >= 0 && items_per_cta != b->per_cta) {
        b->per_cta = items_per_cta;
        drop_graph(b);  // the captured launches carry the old grid
    }
    if (current) *current = b->per_cta;
    return LBM_OK;
}

lbm_status lbm_batch_autotune(lbm_batch *b, int nsteps, int *tx, int *ty)
{
    CPLBM_TRACE("lbm_batch_autotune");
    if (!b) return LBM_ERR_ARG;
    for (size_t i = 0; i < b->inst.size(); ++i)
        if (!b->inst[i]->initialized)
            return bfail(b, LBM_ERR_STATE, "lattice %zu is not initialised", i);
    if (nsteps < 2) nsteps = 2;
    nsteps &= ~1;
    BCUDA(b, cudaSetDevice(b->device));
    std::vector<char *> snaps(b->inst.size(), nullptr);
    lbm_status st = LBM_OK;
    for (size_t i = 0; i < b->inst.size() && st == LBM_OK; ++i) {
        cudaError_t e = dev_alloc((void **)&snaps[i], ctx_state_bytes(b->inst[i]));
        if (e != cudaSuccess) st = bfail(b, LBM_ERR_OOM, "autotune snapshot");
        else st = ctx_snapshot(b->inst[i], snaps[i], true);
    }
    int sx[16], sy[16];
    const int n = step_shapes(sx, sy, 16);
    const long long t0 = b->t;
    std::vector<long long> tsave;  // inactive lattices may lag the batch
    for (lbm_ctx *c : b->inst) tsave.push_back(c->t);
    int best = -1;
    float best_ms = 0.f;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (st == LBM_OK && (cudaEventCreate(&e0) != cudaSuccess ||
                         cudaEventCreate(&e1) != cudaSuccess))
        st = bfail(b, LBM_ERR_CUDA, "event create");
    // configurations: every tile shape with a grid row per lattice (groups of
    // one geometry) or 1, 2 or 4 work items per CTA
    const int per[4] = {0, 1, 2, 4};
    auto restore = [&](int k) -> lbm_status {
        b->tx = sx[k / 4];
        b->ty = sy[k / 4];
        b->per_cta = per[k % 4];
        lbm_status s2 = rebuild(b);
        for (size_t i = 0; i < b->inst.size() && s2 == LBM_OK; ++i)
            s2 = ctx_snapshot(b->inst[i], snaps[i], false);
        b->t = t0;
        for (size_t i = 0; i < b->inst.size(); ++i) b->inst[i]->t = tsave[i];
        return s2;
    };
    for (int k = 0; k < 4 * n && st == LBM_OK; ++k) {
        if (!step_shape_supported(b->precision, sx[k / 4], sy[k / 4])) continue;
        st = restore(k);
        if (st != LBM_OK) break;
        if (per[k % 4] == 0) {  // the same launches as one item per CTA otherwise
            bool any = false;
            for (const Group &g : b->groups) any = any || g.n_uniform > 0;
            if (!any) continue;
        }
        for (int w = 0; w < 2 && st == LBM_OK; ++w) st = launch_one(b);
        if (st != LBM_OK) break;
        if (cudaEventRecord(e0, b->stream) != cudaSuccess) {
            st = bfail(b, LBM_ERR_CUDA, "event record");
            break;
        }
        for (int s = 0; s < nsteps && st == LBM_OK; ++s) st = launch_one(b);
        float ms = 0.f;
        if (st == LBM_OK && (cudaEventRecord(e1, b->stream) != cudaSuccess ||
                             cudaEventSynchronize(e1) != cudaSuccess ||
                             cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            st = bfail(b, LBM_ERR_CUDA, "event timing");
        if (st == LBM_OK && (best < 0 || ms < best_ms)) {
            best = k;
            best_ms = ms;
        }
    }
    if (st == LBM_OK && best >= 0) {
        st = restore(best);
        if (st == LBM_OK && cudaStreamSynchronize(b->stream) != cudaSuccess)
            st = bfail(b, LBM_ERR_CUDA, "synchronize");
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    for (char *p : snaps) dev_free(p);
    if (st != LBM_OK) return st;
    if (tx) *tx = b->tx;
    if (ty) *ty = b->ty;
    return LBM_OK;
}

lbm_status lbm_batch_info(const lbm_batch *b, int *count, long long *nodes,
                          long long *steps, int *tx, int *ty)
{
    if (!b) return LBM_ERR_ARG;
    if (count) *count = (int)b->inst.size();
    if (nodes) *nodes = b->nodes;
    if (steps) *steps = b->t;
    if (tx) *tx = b->tx;
    if (ty) *ty = b->ty;
    return LBM_OK;
}

void lbm_batch_destroy(lbm_batch *b)
{
    if (!b) return;
    cudaSetDevice(b->device);
    drop_graph(b);
    for (lbm_ctx *c : b->inst) lbm_destroy(c);
    dev_free(b->d_lats);
    dev_free(b->d_items);
    for (cudaStream_t st : b->aux) cudaStreamDestroy(st);
    for (cudaEvent_t ev : b->joins) cudaEventDestroy(ev);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
}

const char *lbm_batch_last_error(const lbm_batch *b)
{
    return b ? b->err.c_str() : g_batch_err.c_str();
}

}  // extern "C"
