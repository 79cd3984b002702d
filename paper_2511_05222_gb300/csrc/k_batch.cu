// Ragged batches: the batch-clock kernel and the mixed-mode (FP32) persistent batch kernels (the instances
// for batches with AO-expanded Jastrow terms are in k_batch_jb.cu).
#include "batch_kernels.cuh"

namespace vmcf {

// After a sweep of the whole batch: advance every geometry's clock and rewind the queues.
__global__ void batch_advance_kernel(BatchClock* clk, int G, int mode, int kref, int* queues, int nq) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
    BatchClock c = clk[g];
    c.sweep += 1;
    c.c = mode != 0 ? 0 : (int)((c.c + c.Ne) % kref);  // a measurement rebuilds the inverses
    clk[g] = c;
  }
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) queues[q] = 0;
}

cudaError_t launch_batch_advance(BatchClock* clk, int G, int mode, int kref, int* queues, int nq, cudaStream_t st) {
  batch_advance_kernel<<<1, 128, 0, st>>>(clk, G, mode, kref, queues, nq);
  return cudaGetLastError();
}

extern template cudaError_t launch_batch_impl<float, true>(int, int, int, int, size_t, const BatchArgs&, cudaStream_t);
extern template cudaError_t batch_occupancy_impl<float, true>(int, int, int, size_t, int*);

template <>
cudaError_t launch_batch<float>(int phase, int GS, int groups, int grid, size_t smem, const BatchArgs& A, bool jb,
                                cudaStream_t st) {
  return jb ? launch_batch_impl<float, true>(phase, GS, groups, grid, smem, A, st)
            : launch_batch_impl<float, false>(phase, GS, groups, grid, smem, A, st);
}
template <>
cudaError_t batch_occupancy<float>(int phase, int GS, int groups, size_t smem, bool jb, int* ctas) {
  return jb ? batch_occupancy_impl<float, true>(phase, GS, groups, smem, ctas)
            : batch_occupancy_impl<float, false>(phase, GS, groups, smem, ctas);
}

}  // namespace vmcf
