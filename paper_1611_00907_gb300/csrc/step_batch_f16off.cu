// Batched step kernels of one storage precision (SF16Off); the templates live
// in step_impl.cuh and the dispatch in step.cu.  Apart from the
// single-lattice kernels (step_f16off.cu) so that the two compile in parallel.
#include "step_impl.cuh"

namespace cplbm {

cudaError_t launch_batch_f16off(const Lattice *d_lats, const WorkItem *d_items,
                             const TmaMaps *d_maps, int n_items, int parity, int cur,
                             int tx, int ty, int per_cta, cudaStream_t s)
{
    return launch_batch_t<SF16Off>(d_lats, d_items, d_maps, n_items, parity, cur, tx, ty,
                              per_cta, s);
}

}  // namespace cplbm
