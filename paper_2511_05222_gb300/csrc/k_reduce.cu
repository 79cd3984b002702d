// Per-block sums of the per-CTA FP64 accumulator slots, in a fixed order (deterministic).
#include "vmcf_internal.h"

namespace vmcf {

__global__ void block_reduce_kernel(const double* __restrict__ acc, int cpb, int accL, double* __restrict__ out) {
  const int b = blockIdx.y;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < accL; i += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < cpb; ++c) s += acc[((size_t)b * cpb + c) * accL + i];
    out[(size_t)b * accL + i] = s;
  }
}

cudaError_t launch_block_reduce(const double* acc, int grid, int cpb, int accL, double* out, int nblocks,
                                cudaStream_t st) {
  (void)grid;
  const int threads = 256;
  const int gx = (accL + threads - 1) / threads;
  block_reduce_kernel<<<dim3(gx, nblocks), threads, 0, st>>>(acc, cpb, accL, out);
  return cudaGetLastError();
}

}  // namespace vmcf
