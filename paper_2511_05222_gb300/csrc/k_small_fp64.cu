// FP64-mode instantiations of the small-system kernels.
#include "kernels_small.cuh"

namespace vmcf {
template <>
cudaError_t launch_move_small<double>(const DevSys& S, int nm, int lpw, int W, size_t smem,
                                   const SmallMoveParams& P, cudaStream_t st) {
  return launch_move_small_impl<double>(S, nm, lpw, W, smem, P, st);
}
template <>
cudaError_t launch_propose_small<double>(const DevSys& S, int nm, int grid, int warps, size_t smem,
                                        const SmallProposeParams& P, cudaStream_t st) {
  if (S.MJ > 0) return launch_propose_small_jb<double>(S, nm, grid, warps, smem, P, st);
  return launch_propose_small_impl<double, false>(S, nm, grid, warps, smem, P, st);
}
template <>
cudaError_t launch_measure_small<double>(const DevSys& S, int nm, const SmallLayout& L, int grid, int warps,
                                      const SmallMeasParams& P, cudaStream_t st) {
  if (S.MJ > 0) return launch_measure_small_jb<double>(S, nm, L, grid, warps, P, st);
  return launch_measure_small_impl<double, false>(S, nm, L, grid, warps, P, st);
}
template <>
cudaError_t set_smem_limits_small<double>() {
  cudaError_t e = set_smem_limits_small_impl<double, false>();
  return e == cudaSuccess ? set_smem_limits_small_jb<double>() : e;
}
cudaError_t launch_to_interleaved(const double* src, double* dst, float2* dstf, int W, int n3, cudaStream_t st) {
  to_interleaved<<<std::min(4096, (int)(((long long)W * n3 + 255) / 256)), 256, 0, st>>>(src, dst, dstf, W, n3);
  return cudaGetLastError();
}
cudaError_t launch_from_interleaved(const double* src, double* dst, int W, int n3, cudaStream_t st) {
  from_interleaved<<<std::min(4096, (int)(((long long)W * n3 + 255) / 256)), 256, 0, st>>>(src, dst, W, n3);
  return cudaGetLastError();
}
}  // namespace vmcf
