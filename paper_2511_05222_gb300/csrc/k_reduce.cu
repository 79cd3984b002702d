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

// Add the tensor-core slots [2 spins][tiles][nblocks * cpb][128][32] of each jackknife block into
// its block sums: the O section takes columns j < n_s of D, the (E_L - E_ref) O section columns
// n_s + j; D[mu][j] sits in tile (mu / 128, j / 32) at (mu % 128, j % 32).
__global__ void tc_fold_kernel(const double* __restrict__ slots, int cpb, int Nt, int tiles, int M, int n_up,
                               int n_dn, int oo, int nO, int accL, double* __restrict__ blocks) {
  const int b = blockIdx.y, G = gridDim.y * cpb;
  const int tot = M * (n_up + n_dn);
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < tot; idx += gridDim.x * blockDim.x) {
    const int sg = idx < M * n_up ? 0 : 1;
    const int n = sg == 0 ? n_up : n_dn, loc = idx - (sg == 0 ? 0 : M * n_up);
    const int mu = loc / n, i = loc - mu * n;
    const int mt = mu >> 7, row = mu & 127;
    const int jo = i, jc = n + i;
    const int zo = mt * Nt + (jo >> 5), zc = mt * Nt + (jc >> 5);
    double so = 0.0, sc = 0.0;
    for (int c = 0; c < cpb; ++c) {
      const size_t cta = (size_t)b * cpb + c;
      so += slots[((((size_t)sg * tiles + zo) * G + cta) * 128 + row) * 32 + (jo & 31)];
      sc += slots[((((size_t)sg * tiles + zc) * G + cta) * 128 + row) * 32 + (jc & 31)];
    }
    blocks[(size_t)b * accL + oo + idx] += so;
    blocks[(size_t)b * accL + oo + nO + idx] += sc;
  }
}

cudaError_t launch_tc_fold(const double* slots, int nblocks, int cpb, int Mf, int Nf, int M, int n_up, int n_dn,
                           int oo, int nO, int accL, double* blocks, cudaStream_t st) {
  const int tot = M * (n_up + n_dn);
  const int Nt = (Nf + 31) / 32, tiles = ((Mf + 127) / 128) * Nt;
  tc_fold_kernel<<<dim3((tot + 255) / 256, nblocks), 256, 0, st>>>(slots, cpb, Nt, tiles, M, n_up, n_dn, oo, nO,
                                                                   accL, blocks);
  return cudaGetLastError();
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
