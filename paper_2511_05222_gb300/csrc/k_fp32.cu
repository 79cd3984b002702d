// Mixed-mode (FP32 arithmetic, FP64 inversion and sums) instantiations of the walker-group kernels; the
// instances with the AO-expanded Jastrow terms are in k_fp32_jb.cu.
#include "kernels.cuh"

namespace vmcf {
extern template cudaError_t set_smem_limits_impl<float, true>();
extern template cudaError_t launch_move_impl<float, true>(const DevSys&, const Launch&, const MoveParams&, cudaStream_t);
extern template cudaError_t launch_measure_impl<float, true>(const DevSys&, const Launch&, const MeasParams&, cudaStream_t);

template <>
cudaError_t launch_refresh<float>(const DevSys& S, const Launch& lc, const double* pos, void* B, int W,
                                   unsigned long long* counters, cudaStream_t st) {
  return launch_refresh_impl<float>(S, lc, pos, B, W, counters, st);
}
template <>
cudaError_t launch_propose_group<float>(const DevSys& S, const GroupProposeParams& P, cudaStream_t st) {
  return launch_propose_group_impl<float>(S, P, st);
}
template <>
cudaError_t launch_move<float>(const DevSys& S, const Launch& lc, const MoveParams& P, cudaStream_t st) {
  return S.MJ > 0 ? launch_move_impl<float, true>(S, lc, P, st) : launch_move_impl<float, false>(S, lc, P, st);
}
template <>
cudaError_t launch_measure<float>(const DevSys& S, const Launch& lc, const MeasParams& P, cudaStream_t st) {
  return S.MJ > 0 ? launch_measure_impl<float, true>(S, lc, P, st) : launch_measure_impl<float, false>(S, lc, P, st);
}
template <>
cudaError_t set_smem_limits<float>(int) {
  cudaError_t e = set_smem_limits_impl<float, false>();
  return e != cudaSuccess ? e : set_smem_limits_impl<float, true>();
}
}  // namespace vmcf
