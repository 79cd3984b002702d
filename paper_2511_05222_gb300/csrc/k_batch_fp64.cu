// Ragged batches: the FP64 persistent batch kernels (the instances for batches with AO-expanded Jastrow
// terms are in k_batch_fp64_jb.cu).
#include "batch_kernels.cuh"

namespace vmcf {
extern template cudaError_t launch_batch_impl<double, true>(int, int, int, int, size_t, const BatchArgs&, cudaStream_t);
extern template cudaError_t batch_occupancy_impl<double, true>(int, int, int, size_t, int*);

template <>
cudaError_t launch_batch<double>(int phase, int GS, int groups, int grid, size_t smem, const BatchArgs& A, bool jb,
                                 cudaStream_t st) {
  return jb ? launch_batch_impl<double, true>(phase, GS, groups, grid, smem, A, st)
            : launch_batch_impl<double, false>(phase, GS, groups, grid, smem, A, st);
}
template <>
cudaError_t batch_occupancy<double>(int phase, int GS, int groups, size_t smem, bool jb, int* ctas) {
  return jb ? batch_occupancy_impl<double, true>(phase, GS, groups, smem, ctas)
            : batch_occupancy_impl<double, false>(phase, GS, groups, smem, ctas);
}
}  // namespace vmcf
