// Mixed-mode (FP32 arithmetic, FP64 inversion and sums) instantiations of the hot-path kernels.
#include "kernels.cuh"

namespace vmcf {
template <>
cudaError_t launch_refresh<float>(const DevSys& S, const Launch& lc, const double* pos, void* B, int W,
                                   unsigned long long* counters, cudaStream_t st) {
  return launch_refresh_impl<float>(S, lc, pos, B, W, counters, st);
}
template <>
cudaError_t launch_move<float>(const DevSys& S, const Launch& lc, const MoveParams& P, cudaStream_t st) {
  return launch_move_impl<float>(S, lc, P, st);
}
template <>
cudaError_t launch_measure<float>(const DevSys& S, const Launch& lc, const MeasParams& P, cudaStream_t st) {
  return launch_measure_impl<float>(S, lc, P, st);
}
template <>
cudaError_t set_smem_limits<float>(int) {
  return set_smem_limits_impl<float>();
}
}  // namespace vmcf
