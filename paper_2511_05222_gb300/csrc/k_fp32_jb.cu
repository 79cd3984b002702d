// Mixed-mode (FP32 arithmetic, FP64 inversion and sums) instantiations of the walker-group kernels for systems with the AO-expanded Jastrow terms.
#include "kernels.cuh"

namespace vmcf {
template cudaError_t set_smem_limits_impl<float, true>();
template cudaError_t launch_move_impl<float, true>(const DevSys&, const Launch&, const MoveParams&, cudaStream_t);
template cudaError_t launch_measure_impl<float, true>(const DevSys&, const Launch&, const MeasParams&, cudaStream_t);
}  // namespace vmcf
