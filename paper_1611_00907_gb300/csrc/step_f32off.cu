// Step kernels of one storage precision (SF32Off); the templates live in
// step_impl.cuh and the dispatch in step.cu.  One translation unit per
// precision keeps the build parallel.
#include "step_impl.cuh"

namespace cplbm {

cudaError_t launch_step_f32off(const Lattice &L, int parity, int cur,
                            cudaStream_t s, const TmaMaps *maps)
{
    return launch_step_t<SF32Off>(L, parity, cur, s, maps);
}

cudaError_t launch_batch_f32off(const Lattice *d_lats, const WorkItem *d_items,
                             const TmaMaps *d_maps, int *d_counter, int n_items, int parity, int cur, int tx, int ty,
                             int grid, cudaStream_t s)
{
    return launch_batch_t<SF32Off>(d_lats, d_items, d_maps, d_counter, n_items, parity, cur, tx, ty, grid, s);
}

}  // namespace cplbm
