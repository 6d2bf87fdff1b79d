// Single-lattice step kernels of one storage precision (SF16Off); the templates live in
// step_impl.cuh and the dispatch in step.cu.  One translation unit per
// precision keeps the build parallel.
#include "step_impl.cuh"

namespace cplbm {

cudaError_t launch_step_f16off(const Lattice &L, int parity, int cur,
                            cudaStream_t s, const TmaMaps *maps)
{
    return launch_step_t<SF16Off>(L, parity, cur, s, maps);
}


}  // namespace cplbm
