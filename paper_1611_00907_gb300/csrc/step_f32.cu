// Single-lattice step kernels of one storage precision (SF32); the templates live in
// step_impl.cuh and the dispatch in step.cu.  One translation unit per
// precision keeps the build parallel.
#include "step_impl.cuh"

namespace cplbm {

cudaError_t launch_step_f32(const Lattice &L, int parity, int cur,
                            cudaStream_t s, const TmaMaps *maps)
{
    return launch_step_t<SF32>(L, parity, cur, s, maps);
}


cudaError_t launch_pt_f32(const Lattice &L, int parity, int cur, cudaStream_t s,
                          const TmaMaps *maps)
{
    if (L.tx == 64 && L.ty == 16) return launch_pt_shape<SF32, 64, 16>(L, parity, cur, s, maps);
    return launch_pt_shape<SF32, 32, 32>(L, parity, cur, s, maps);
}

}  // namespace cplbm
