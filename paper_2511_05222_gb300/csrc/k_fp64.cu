// FP64-mode instantiations of the hot-path kernels.
#include <algorithm>

#include "kernels.cuh"

namespace vmcf {
template <>
cudaError_t launch_refresh<double>(const DevSys& S, const Launch& lc, const double* pos, void* B, int W,
                                   unsigned long long* counters, cudaStream_t st) {
  return launch_refresh_impl<double>(S, lc, pos, B, W, counters, st);
}
template <>
cudaError_t launch_move<double>(const DevSys& S, const Launch& lc, const MoveParams& P, cudaStream_t st) {
  return launch_move_impl<double>(S, lc, P, st);
}
template <>
cudaError_t launch_measure<double>(const DevSys& S, const Launch& lc, const MeasParams& P, cudaStream_t st) {
  return launch_measure_impl<double>(S, lc, P, st);
}
template <>
cudaError_t set_smem_limits<double>(int) {
  return set_smem_limits_impl<double>();
}
}  // namespace vmcf
