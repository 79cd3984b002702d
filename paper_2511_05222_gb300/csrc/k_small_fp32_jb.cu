// Mixed-mode instances of the small-system proposal and measurement kernels with the AO-expanded Jastrow
// terms (their own translation unit: compile time, and the instances without the terms stay free of them).
#include "kernels_small.cuh"

namespace vmcf {
template <>
cudaError_t launch_propose_small_jb<float>(const DevSys& S, int nm, int grid, int warps, size_t smem,
                                           const SmallProposeParams& P, cudaStream_t st) {
  return launch_propose_small_impl<float, true>(S, nm, grid, warps, smem, P, st);
}
template <>
cudaError_t launch_measure_small_jb<float>(const DevSys& S, int nm, const SmallLayout& L, int grid, int warps,
                                           const SmallMeasParams& P, cudaStream_t st) {
  return launch_measure_small_impl<float, true>(S, nm, L, grid, warps, P, st);
}
template <>
cudaError_t set_smem_limits_small_jb<float>() {
  return set_smem_limits_small_impl<float, true>();
}
}  // namespace vmcf
