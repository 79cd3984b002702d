// Ragged batches: the FP64 persistent batch kernels.
#include "batch_kernels.cuh"

namespace vmcf {
template cudaError_t launch_batch<double>(int, int, int, int, size_t, const BatchArgs&, cudaStream_t);
template cudaError_t batch_occupancy<double>(int, int, int, size_t, int*);
}  // namespace vmcf
