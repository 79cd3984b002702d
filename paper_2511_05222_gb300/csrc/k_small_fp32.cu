// Mixed-mode (FP32 arithmetic, FP64 inversion and sums) instantiations of the small-system kernels.
#include "kernels_small.cuh"

namespace vmcf {
template <>
cudaError_t launch_move_small<float>(const DevSys& S, int nm, int lpw, int W, size_t smem,
                                   const SmallMoveParams& P, cudaStream_t st) {
  return launch_move_small_impl<float>(S, nm, lpw, W, smem, P, st);
}
template <>
cudaError_t launch_propose_small<float>(const DevSys& S, int nm, int grid, int warps, size_t smem,
                                        const SmallProposeParams& P, cudaStream_t st) {
  if (S.MJ > 0) return launch_propose_small_jb<float>(S, nm, grid, warps, smem, P, st);
  return launch_propose_small_impl<float, false>(S, nm, grid, warps, smem, P, st);
}
template <>
cudaError_t launch_measure_small<float>(const DevSys& S, int nm, const SmallLayout& L, int grid, int warps,
                                      const SmallMeasParams& P, cudaStream_t st) {
  if (S.MJ > 0) return launch_measure_small_jb<float>(S, nm, L, grid, warps, P, st);
  return launch_measure_small_impl<float, false>(S, nm, L, grid, warps, P, st);
}
template <>
cudaError_t set_smem_limits_small<float>() {
  cudaError_t e = set_smem_limits_small_impl<float, false>();
  return e == cudaSuccess ? set_smem_limits_small_jb<float>() : e;
}
}  // namespace vmcf
