/*
 * vmcf_diag — measurement diagnostics of libvmcf. They are not part of the method's interface
 * (the paper has no counterpart): the benchmark uses them to split a step's device time by
 * kernel and to measure the ALU peaks its roofline fractions are quoted against. They live in
 * libvmcf.so beside the entry points of vmcf.h.
 */
#ifndef VMCF_DIAG_H
#define VMCF_DIAG_H

#include "vmcf.h"

#ifdef __cplusplus
extern "C" {
#endif

/* vmcf_profile: record a CUDA event pair around every kernel this walker set launches from
 * now on (enable != 0) or stop recording (0). Recording adds host work to every launch: time
 * a step without it and use it only to split a step's time by kernel.
 * vmcf_kernel_times: synchronise on the recorded events and return the summed device time
 * in ms and the launch count per kernel kind: [0] Metropolis sweep kernel, [1] measurement
 * kernel, [2] refresh kernel, [3] tensor-core walker-sum kernel, [4] proposal pass of a sweep
 * (host arrays of 5; either may be NULL); reset != 0 zeroes the totals afterwards.
 * vmcf_probe_pipes: measure this GPU's FP64 FMA and FP32 FMA throughput (TFLOP/s) and FP32
 * expf throughput (G/s) with short register-only kernels on `stream` (synchronises; about
 * 30 ms). Used as the measured ALU peaks of the roofline. */
int vmcf_profile(vmcf_walkers_t wk, int enable);
int vmcf_kernel_times(vmcf_walkers_t wk, double* ms, long long* count, int reset);
int vmcf_probe_pipes(double* fp64_tflops, double* fp32_tflops, double* exp_gops, void* stream);

/* vmcf_diag_group_proposals: run the proposal pass of the walker set's next sweep (walker-group kernels only,
 * VMCF_EINVAL for a small-system walker set) from its current positions with step `step_sigma`, exactly as
 * vmcf_sample would (the same Philox counters and kernel: the tensor-core orbital rows in mixed precision unless
 * vmcf_set_tuning(s, "tensor_core_rows", 0) switched them off), and copy its buffers to host arrays: rnew
 * [W][Ne][3] proposed positions, rows [W][Ne][nmax] orbital rows of each electron's spin at its proposal (the
 * system's largest spin block nmax; entries beyond the spin's orbital count are not written), u [W][Ne] acceptance
 * uniforms, dchi [W][Ne] changes of the electron-nucleus Jastrow terms (mixed-precision values widened to double).
 * Does not advance the chain. Synchronises `stream`. The rows are the orbital values
 * phi = psi C of App. A ("Computing derivatives") at the proposals of the Metropolis sweep. */
int vmcf_diag_group_proposals(vmcf_walkers_t wk, double step_sigma, double* rnew, double* rows, double* u,
                              double* dchi, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* VMCF_DIAG_H */
