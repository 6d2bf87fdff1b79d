// Single-lattice step kernels of one storage precision (SF64); the templates live in
// step_impl.cuh and the dispatch in step.cu.  One translation unit per
// precision keeps the build parallel.
#include "step_impl.cuh"

namespace cplbm {

cudaError_t launch_step_f64(const Lattice &L, int parity, int cur,
                            cudaStream_t s, const TmaMaps *maps)
{
    return launch_step_t<SF64>(L, parity, cur, s, maps);
}


cudaError_t launch_pt_f64(const Lattice &L, int parity, int cur, cudaStream_t s,
                          const TmaMaps *maps)
{
    return launch_pt_shape<SF64, 32, 16>(L, parity, cur, s, maps);
}

}  // namespace cplbm
