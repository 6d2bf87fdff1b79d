// Internal definition of the context behind the opaque lbm_ctx of the C ABI,
// shared by the translation units that implement the ABI (capi.cu,
// batch.cu).  Not public.
#pragma once

#include <string>

#include "../../include/cplbm.h"
#include "cplbm_internal.h"

struct lbm_ctx {
    cplbm::Lattice L{};
    int device = 0;
    cudaStream_t stream = nullptr;
    long long t = 0;
    bool eos_set = false, initialized = false;
    double T = 0, alpha = 1, Tc = 0, rhoc = 0;
    double *d_red = nullptr;   // 4 reduction slots
    int *d_bad = nullptr;      // error counter
    double *d_prev = nullptr;  // density snapshot of lbm_reduce [ny][nx]
    double *d_tmp = nullptr;   // staging for host-side field transfers
    size_t tmp_bytes = 0;
    int *d_err = nullptr;      // kernel error flags (Lattice::err)
    cplbm::TmaMaps maps{};            // tensor maps of the TMA interior path
    bool use_tma = true;
    int force_model = 0;       // 0 chemical potential (Eq. 12), 1 Eq. 5
    // lbm_step replays blocks of steps from a captured CUDA graph (capi.cu,
    // step_graph): the graph, the stream it was captured on, and the launch
    // parameters it holds, compared before each replay
    cudaGraphExec_t graph = nullptr;
    cudaStream_t capture_stream = nullptr;
    cplbm::Lattice graph_L{};
    cplbm::TmaMaps graph_maps{};
    int graph_force = -1;
    bool graph_failed = false;  // capture refused: direct launches only
    std::string err;
};

namespace cplbm {
// capi.cu: copy a context's state (populations, whole density) to a device
// buffer of ctx_state_bytes(), or back (partial sums cleared).
size_t ctx_state_bytes(const lbm_ctx *c);
lbm_status ctx_snapshot(lbm_ctx *c, char *snap, bool save);
// capi.cu: rebuild the TMA maps after a tile-shape change.
void ctx_refresh_maps(lbm_ctx *c);
}  // namespace cplbm
