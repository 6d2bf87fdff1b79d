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
#include <new>
#include <string>
#include <vector>

#include "context.h"

using namespace cplbm;

struct lbm_batch {
    std::vector<lbm_ctx *> inst;
    std::vector<char> active;  // lattices in the launch
    int precision = 0, device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int tx = 32, ty = 32;
    Lattice *d_lats = nullptr;
    WorkItem *d_items = nullptr;
    TmaMaps *d_maps = nullptr;  // per-lattice tensor maps, or null (no TMA)
    int per_cta = 1;            // work items per CTA of the batched kernel
    int n_items = 0;
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
// of the descriptors and the work list.
lbm_status rebuild(lbm_batch *b)
{
    drop_graph(b);
    std::vector<Lattice> lats;
    std::vector<WorkItem> items;
    std::vector<TmaMaps> maps;
    bool any_maps = false;
    for (size_t i = 0; i < b->inst.size(); ++i) {
        lbm_ctx *c = b->inst[i];
        c->L.tx = b->tx;
        c->L.ty = b->ty;
        ctx_refresh_maps(c);
        lats.push_back(c->L);
        maps.push_back(c->maps);
        if (!c->use_tma) maps.back().valid = 0;
        any_maps = any_maps || maps.back().valid;
        if (!b->active[i]) continue;
        const Lattice &L = c->L;
        const int ntx = (L.nx + b->tx - 1) / b->tx, nty = (L.nyf + b->ty - 1) / b->ty;
        // edge tiles (periodic seams, wall rows) take the TMA paths too: the
        // 32-wide one, and for FP32 arithmetic the 64-wide pair path
        // (step_batch_kernel)
        const bool tma_shape = b->tx == 32 || (b->tx == 64 && b->precision != LBM_F64);
        const int seams = tma_shape ? seam_bits(L, b->tx, b->ty) : 0;
        for (int by = 0; by < nty; ++by)
            for (int bx = 0; bx < ntx; ++bx)
                items.push_back({(int)i, bx, by, tile_kind(L, b->tx, b->ty, bx, by, seams)});
    }
    // General tiles cost a few interior tiles each, edge tiles (seams,
    // walls) somewhat more than one.  CTAs take items in list order,
    // backwards on odd steps: the interior tiles go in two halves at the
    // ends, so that in either direction a step ends on short items and the
    // CTAs finish close together, and the edge and general tiles between
    // them, each class in one run, so that the CTAs of an SM mostly run the
    // same code path at a time (the batched kernel holds three large ones
    // and the instruction cache does not hold them all).
    {
        std::vector<WorkItem> gen, edge, inner;
        for (const WorkItem &it : items)
            (it.kind == TILE_GENERAL ? gen : it.kind == TILE_SEAM ? edge : inner).push_back(it);
        const size_t h = inner.size() / 2;
        items.clear();
        items.insert(items.end(), inner.begin(), inner.begin() + h);
        items.insert(items.end(), edge.begin(), edge.end());
        items.insert(items.end(), gen.begin(), gen.end());
        items.insert(items.end(), inner.begin() + h, inner.end());
    }
    dev_free(b->d_lats);
    dev_free(b->d_items);
    dev_free(b->d_maps);
    b->d_lats = nullptr;
    b->d_items = nullptr;
    b->d_maps = nullptr;
    if (any_maps) {
        BCUDA(b, dev_alloc((void **)&b->d_maps, maps.size() * sizeof(TmaMaps)));
        BCUDA(b, cudaMemcpy(b->d_maps, maps.data(), maps.size() * sizeof(TmaMaps),
                            cudaMemcpyHostToDevice));
    }
    BCUDA(b, dev_alloc((void **)&b->d_lats, lats.size() * sizeof(Lattice)));
    BCUDA(b, dev_alloc((void **)&b->d_items, items.size() * sizeof(WorkItem)));
    BCUDA(b, cudaMemcpy(b->d_lats, lats.data(), lats.size() * sizeof(Lattice),
                        cudaMemcpyHostToDevice));
    BCUDA(b, cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(WorkItem),
                        cudaMemcpyHostToDevice));
    b->n_items = (int)items.size();
    return LBM_OK;
}

lbm_status launch_one(lbm_batch *b)
{
    const int p = (int)(b->t & 1);
    BCUDA(b, launch_step_batch(b->d_lats, b->d_items, b->d_maps, b->n_items, p, p,
                               b->precision, b->tx, b->ty, b->per_cta, b->stream));
    ++b->t;
    return LBM_OK;
}

lbm_status ensure_graph(lbm_batch *b)
{
    if (b->exec) return LBM_OK;
    cudaGraph_t g = nullptr;
    BCUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < GRAPH_STEPS && e == cudaSuccess; ++k)
        e = launch_step_batch(b->d_lats, b->d_items, b->d_maps, b->n_items, k & 1, k & 1,
                              b->precision, b->tx, b->ty, b->per_cta, b->stream);
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
    if (!b) return LBM_ERR_ARG;
    lbm_status st = check_index(b, index);
    if (st != LBM_OK) return st;
    lbm_ctx *c = b->inst[index];
    return forward(b, c, lbm_reduce(c, out));
}

lbm_status lbm_batch_set_tile(lbm_batch *b, int tx, int ty)
{
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
    if (items_per_cta > 64)
        return bfail(b, LBM_ERR_ARG, "items per CTA must be 1 .. 64 (got %d)",
                     items_per_cta);
    if (items_per_cta > 0 && items_per_cta != b->per_cta) {
        b->per_cta = items_per_cta;
        drop_graph(b);  // the captured launches carry the old grid
    }
    if (current) *current = b->per_cta;
    return LBM_OK;
}

lbm_status lbm_batch_autotune(lbm_batch *b, int nsteps, int *tx, int *ty)
{
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
    // configurations: every tile shape with 1, 2 or 4 work items per CTA
    const int per[3] = {1, 2, 4};
    auto restore = [&](int k) -> lbm_status {
        b->tx = sx[k / 3];
        b->ty = sy[k / 3];
        b->per_cta = per[k % 3];
        lbm_status s2 = rebuild(b);
        for (size_t i = 0; i < b->inst.size() && s2 == LBM_OK; ++i)
            s2 = ctx_snapshot(b->inst[i], snaps[i], false);
        b->t = t0;
        for (size_t i = 0; i < b->inst.size(); ++i) b->inst[i]->t = tsave[i];
        return s2;
    };
    for (int k = 0; k < 3 * n && st == LBM_OK; ++k) {
        if (!step_shape_supported(b->precision, sx[k / 3], sy[k / 3])) continue;
        st = restore(k);
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
    dev_free(b->d_maps);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
}

const char *lbm_batch_last_error(const lbm_batch *b)
{
    return b ? b->err.c_str() : g_batch_err.c_str();
}

}  // extern "C"
