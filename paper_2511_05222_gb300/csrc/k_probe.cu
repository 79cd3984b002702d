// Pipe-throughput probes (FP64 FMA, FP32 FMA, FP32 exp) used as the measured ALU peaks of
// the roofline. Independent FMA chains in registers; one store per thread.
#include <cuda_runtime.h>

#include "vmcf_internal.h"

namespace vmcf {

template <typename T, int NCH>
__global__ void fma_probe(T* out, int iters, T a, T b) {
  T x[NCH];
#pragma unroll
  for (int c = 0; c < NCH; ++c) x[c] = (T)(threadIdx.x * 1e-3) + (T)c;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < NCH; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < NCH; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int NCH>
__global__ void exp_probe(float* out, int iters) {
  float x[NCH];
#pragma unroll
  for (int c = 0; c < NCH; ++c) x[c] = -(float)(threadIdx.x % 7) * 1e-3f - c * 1e-4f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < NCH; ++c) x[c] = -0.5f * expf(x[c]);
  }
  float s = 0;
#pragma unroll
  for (int c = 0; c < NCH; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

cudaError_t run_probes(double* fp64_tflops, double* fp32_tflops, double* exp_gops, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev))) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))) return e;
  const int blocks = sms * 8, threads = 256, n = blocks * threads;
  void* buf = nullptr;
  if ((e = cudaMalloc(&buf, sizeof(double) * n))) return e;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  float ms = 0.f;
  auto timed = [&](auto launch) -> float {
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      cudaEventRecord(a, st);
      launch();
      cudaEventRecord(b, st);
      cudaEventSynchronize(b);
      cudaEventElapsedTime(&ms, a, b);
      best = ms < best ? ms : best;
    }
    return best;
  };
  const int i64 = 400, i32 = 8000, iex = 2000;
  float t64 = timed([&] { fma_probe<double, 8><<<blocks, threads, 0, st>>>((double*)buf, i64, 0.999999, 1e-7); });
  float t32 = timed([&] { fma_probe<float, 8><<<blocks, threads, 0, st>>>((float*)buf, i32, 0.999999f, 1e-7f); });
  float tex = timed([&] { exp_probe<8><<<blocks, threads, 0, st>>>((float*)buf, iex); });
  e = cudaGetLastError();
  if (fp64_tflops) *fp64_tflops = 2.0 * 8 * i64 * (double)n / (t64 * 1e-3) / 1e12;
  if (fp32_tflops) *fp32_tflops = 2.0 * 8 * i32 * (double)n / (t32 * 1e-3) / 1e12;
  if (exp_gops) *exp_gops = 8.0 * iex * (double)n / (tex * 1e-3) / 1e9;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(buf);
  return e;
}

}  // namespace vmcf
