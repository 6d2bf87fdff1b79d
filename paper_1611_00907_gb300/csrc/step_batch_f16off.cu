// Batched step kernels of one storage precision (SF16Off); the templates live
// in step_impl.cuh and the dispatch in step.cu.  Apart from the
// single-lattice kernels (step_f16off.cu) so that the two compile in parallel.
#include "step_impl.cuh"

namespace cplbm {

cudaError_t launch_batch_f16off(const Lattice *d_lats, const WorkItem *d_items,
                             const TmaMaps *d_maps, int *d_counter, int n_items, int parity, int cur, int tx, int ty,
                             int grid, cudaStream_t s)
{
    return launch_batch_t<SF16Off>(d_lats, d_items, d_maps, d_counter, n_items, parity, cur, tx, ty, grid, s);
}

}  // namespace cplbm
