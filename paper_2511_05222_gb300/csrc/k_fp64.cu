// FP64 instantiations of the walker-group kernels; the instances with the AO-expanded
// Jastrow terms are in k_fp64_jb.cu.
#include "kernels.cuh"

namespace vmcf {
extern template cudaError_t set_smem_limits_impl<double, true>();
extern template cudaError_t launch_move_impl<double, true>(const DevSys&, const Launch&, const MoveParams&, cudaStream_t);
extern template cudaError_t launch_measure_impl<double, true>(const DevSys&, const Launch&, const MeasParams&, cudaStream_t);

template <>
cudaError_t launch_refresh<double>(const DevSys& S, const Launch& lc, const double* pos, void* B, int W,
                                   unsigned long long* counters, cudaStream_t st) {
  return launch_refresh_impl<double>(S, lc, pos, B, W, counters, st);
}
template <>
cudaError_t launch_propose_group<double>(const DevSys& S, const GroupProposeParams& P, cudaStream_t st) {
  return launch_propose_group_impl<double>(S, P, st);
}
template <>
cudaError_t launch_move<double>(const DevSys& S, const Launch& lc, const MoveParams& P, cudaStream_t st) {
  return S.MJ > 0 ? launch_move_impl<double, true>(S, lc, P, st) : launch_move_impl<double, false>(S, lc, P, st);
}
template <>
cudaError_t launch_measure<double>(const DevSys& S, const Launch& lc, const MeasParams& P, cudaStream_t st) {
  return S.MJ > 0 ? launch_measure_impl<double, true>(S, lc, P, st) : launch_measure_impl<double, false>(S, lc, P, st);
}
template <>
cudaError_t set_smem_limits<double>(int) {
  cudaError_t e = set_smem_limits_impl<double, false>();
  return e != cudaSuccess ? e : set_smem_limits_impl<double, true>();
}
}  // namespace vmcf
