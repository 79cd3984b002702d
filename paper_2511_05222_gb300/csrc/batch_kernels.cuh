// Ragged batch of geometries: per sweep, a Metropolis phase and (when measuring) an evaluation
// phase, each made of one persistent kernel per launch shape (threads per walker GS, walker
// groups per CTA) over the geometries assigned to that shape. Each walker group pulls work
// items (geometry g, accumulator slot c) from a device queue; item (g, c) covers the walkers
// of g whose walker sums go to slot c, so a slot is only ever touched by the group that holds
// its item and is updated without atomics. The phases keep their own shapes because their
// working sets differ (a sweep needs the inverses; an evaluation needs the adjoint matrices).
#pragma once
#include "kernels.cuh"

namespace vmcf {

// JB: some geometry of the batch has AO-expanded Jastrow terms (else their code is compiled out).
template <typename T, int GS, int PHASE, bool JB>
__global__ void __launch_bounds__(256) batch_kernel(BatchArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int gid = threadIdx.x / GS, t = threadIdx.x % GS;
  unsigned char* region = smem + (size_t)gid * A.region;
  BatchGeom* G = reinterpret_cast<BatchGeom*>(region);
  int* cur = reinterpret_cast<int*>(region + A.hdr - 16);  // [0] geometry held, [1] item taken
  unsigned char* base = region + A.hdr;
  if (t == 0) cur[0] = -1;
  for (;;) {
    if (t == 0) cur[1] = atomicAdd(A.queue, 1);
    gsync<GS>();
    const int it = cur[1];
    if (it >= A.n_items) break;  // uniform over the group
    const int2 item = A.items[it];
    if (item.x != cur[0]) {
      gsync<GS>();  // every thread has read cur[0]
      const int* src = reinterpret_cast<const int*>(A.geo + item.x);
      int* dst = reinterpret_cast<int*>(G);
      for (int i = t; i < (int)(sizeof(BatchGeom) / 4); i += GS) dst[i] = src[i];
      gsync<GS>();
      if (t == 0) {
        cur[0] = item.x;
        const BatchClock ck = A.clk[item.x];
        G->P.sweep0 = ck.sweep;
        G->P.c0 = ck.c;
        G->P.nsweeps = 1;
        G->P.kref = A.kref;
        G->P.sigma = A.sigma;
        G->P.skip_final_refresh = A.mode != 0;
        G->Mp.acc_in_smem = 0;
      }
      gsync<GS>();
    }
    const int W = G->P.W;
    const long long w0 = (long long)W * item.y / G->grid_meas, w1 = (long long)W * (item.y + 1) / G->grid_meas;
    if constexpr (PHASE == 0) {
      for (long long w = w0; w < w1; ++w) move_walker<T, GS, JB>(G->S, G->Lrm, G->P, base, (int)w, G->P.c0, G->P.sweep0);
    } else {
      double* slot = A.mode == 1 ? G->Mp.acc + (size_t)item.y * G->Mp.accL : nullptr;
      for (long long w = w0; w < w1; ++w) measure_walker<T, GS, JB>(G->S, G->Lmeas, G->Mp, base, nullptr, slot, (int)w);
    }
    gsync<GS>();  // cur[1] is read by every thread before it is overwritten
  }
}

template <typename T, int PHASE, bool JB>
const void* batch_fn(int GS) {
  switch (GS) {
    case 32: return reinterpret_cast<const void*>(batch_kernel<T, 32, PHASE, JB>);
    case 128: return reinterpret_cast<const void*>(batch_kernel<T, 128, PHASE, JB>);
    case 256: return reinterpret_cast<const void*>(batch_kernel<T, 256, PHASE, JB>);
    default: return nullptr;
  }
}

template <typename T, bool JB>
cudaError_t launch_batch_impl(int phase, int GS, int groups, int grid, size_t smem, const BatchArgs& A,
                              cudaStream_t st) {
  const void* fn = phase == 0 ? batch_fn<T, 0, JB>(GS) : batch_fn<T, 1, JB>(GS);
  if (!fn || GS * groups > 256) return cudaErrorInvalidValue;
  BatchArgs a = A;
  void* args[] = {&a};
  return cudaLaunchKernel(fn, dim3(grid), dim3(GS * groups), args, smem, st);
}

template <typename T, bool JB>
cudaError_t batch_occupancy_impl(int phase, int GS, int groups, size_t smem, int* ctas_per_sm) {
  const void* fn = phase == 0 ? batch_fn<T, 0, JB>(GS) : batch_fn<T, 1, JB>(GS);
  if (!fn || GS * groups > 256) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, fn, GS * groups, smem);
}

}  // namespace vmcf
