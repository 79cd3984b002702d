// Ragged batches: the mixed-mode (FP32) persistent batch kernels for batches with AO-expanded Jastrow terms.
#include "batch_kernels.cuh"

namespace vmcf {
template cudaError_t launch_batch_impl<float, true>(int, int, int, int, size_t, const BatchArgs&, cudaStream_t);
template cudaError_t batch_occupancy_impl<float, true>(int, int, int, size_t, int*);
}  // namespace vmcf
