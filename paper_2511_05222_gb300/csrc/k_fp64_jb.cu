// FP64 instantiations of the walker-group kernels for systems with the AO-expanded Jastrow terms.
#include "kernels.cuh"

namespace vmcf {
template cudaError_t set_smem_limits_impl<double, true>();
template cudaError_t launch_move_impl<double, true>(const DevSys&, const Launch&, const MoveParams&, cudaStream_t);
template cudaError_t launch_measure_impl<double, true>(const DevSys&, const Launch&, const MeasParams&, cudaStream_t);
}  // namespace vmcf
