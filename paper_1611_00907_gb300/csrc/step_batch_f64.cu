// Batched step kernels of one storage precision (SF64); the templates live
// in step_impl.cuh and the dispatch in step.cu.  Apart from the
// single-lattice kernels (step_f64.cu) so that the two compile in parallel.
#include "step_impl.cuh"

namespace cplbm {

cudaError_t launch_batch_f64(const BatchList &w, int parity, int cur, int tx,
                             int ty, cudaStream_t s)
{
    return launch_batch_t<SF64>(w, parity, cur, tx, ty, s);
}

}  // namespace cplbm
