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

// The estimators of the walker sums and their delete-one-block jackknife errors from the block sums blk [nb][L]
// (App. A: E = <E_L>; F = -(<dE_L/dR> + 2 (<E_L dlnPsi/dR> - E <dlnPsi/dR>)), Eqs. hf, pulay; B = dE/dC =
// 2 (<E_L O> - E <O>), Eq. fc-vmc-eval; E_ref cancels), with the arithmetic of the host routine
// vmcf_finish_estimators: every sum over the blocks in block order, the leave-one-out estimate of block b from
// the totals minus that block's row, the error sqrt((nb - 1)/nb sum_b (theta_b - mean)^2). One thread per
// component c of (E, F [3K], B [nO]); out: [0] E, [1] E_err, then F [3K], F_err [3K], B [nO], B_err [nO].
// Each CTA first forms the per-block scalars (leave-one-out sample count, mean E_L - E_ref, reciprocal count) in
// shared memory ([2 nb + 2] doubles). The loops over the blocks are unrolled so that their loads overlap; the sums
// keep their order. status |= 1 when there are no samples, |= 2 when one block holds all of them.
__global__ void finish_kernel(const double* __restrict__ blk, int nb, int L, int K3, int nO, double er,
                              double* __restrict__ out, int* status) {
  extern __shared__ double fin_s[];
  double* inb = fin_s;            // 1 / (leave-one-out sample count) of block b
  double* emb = fin_s + nb;       // leave-one-out mean E_L of block b
  double* tots = fin_s + 2 * nb;  // [0] total count, [1] total E_L sum
  if (threadIdx.x == 0) {
    double t0 = 0.0, t1 = 0.0;
#pragma unroll 8
    for (int b = 0; b < nb; ++b) {
      t0 += blk[(size_t)b * L];
      t1 += blk[(size_t)b * L + 1];
    }
    tots[0] = t0;
    tots[1] = t1;
  }
  __syncthreads();
  const double n = tots[0];
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    const double nl = n - blk[(size_t)b * L];
    inb[b] = 1.0 / nl;
    emb[b] = (tots[1] - blk[(size_t)b * L + 1]) / nl;
    if (!(nl > 0.0) && status) atomicOr(status, 2);
  }
  if (!(n > 0.0)) {
    if (threadIdx.x == 0 && blockIdx.x == 0 && status) atomicOr(status, 1);
    return;  // CTA-uniform
  }
  __syncthreads();
  const double in = 1.0 / n, Em = tots[1] / n, c = Em - er;
  const int o_dEL = 3, o_d = 3 + K3, o_Ed = 3 + 2 * K3, o_O = 3 + 3 * K3, o_EO = 3 + 3 * K3 + nO;
  const int nc = 1 + K3 + nO;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nc; q += gridDim.x * blockDim.x) {
    // the component's fields: kind 0 E, 1 F_i, 2 B_i
    const int kind = q == 0 ? 0 : (q <= K3 ? 1 : 2), i = kind == 1 ? q - 1 : q - 1 - K3;
    const int a0 = kind == 1 ? o_dEL + i : o_EO + i, a1 = kind == 1 ? o_Ed + i : o_O + i, a2 = o_d + i;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    if (kind != 0)
#pragma unroll 8
      for (int b = 0; b < nb; ++b) {
        const double* v = blk + (size_t)b * L;
        s0 += v[a0];
        s1 += v[a1];
        if (kind == 1) s2 += v[a2];
      }
    auto est = [&](double v0, double v1, double v2, double ib, double cc, double Eb) {
      if (kind == 0) return Eb;
      if (kind == 1) return -(v0 * ib + 2.0 * (v1 * ib - cc * (v2 * ib)));
      return 2.0 * (v0 * ib - cc * (v1 * ib));
    };
    const double full = est(s0, s1, s2, in, c, Em);
    double m = 0.0;
#pragma unroll 8
    for (int b = 0; b < nb; ++b) {
      const double* v = blk + (size_t)b * L;
      m += est(s0 - v[a0], s1 - v[a1], kind == 1 ? s2 - v[a2] : 0.0, inb[b], emb[b] - er, emb[b]);
    }
    m /= nb;
    double var = 0.0;
#pragma unroll 8
    for (int b = 0; b < nb; ++b) {
      const double* v = blk + (size_t)b * L;
      const double d = est(s0 - v[a0], s1 - v[a1], kind == 1 ? s2 - v[a2] : 0.0, inb[b], emb[b] - er, emb[b]) - m;
      var += d * d;
    }
    const double err = sqrt((nb - 1.0) / nb * var);
    if (kind == 0) {
      out[0] = full;
      out[1] = err;
    } else if (kind == 1) {
      out[2 + i] = full;
      out[2 + K3 + i] = err;
    } else {
      out[2 + 2 * K3 + i] = full;
      out[2 + 2 * K3 + nO + i] = err;
    }
  }
}

cudaError_t launch_finish(const double* blk, int nb, int L, int K3, int nO, double er, double* out, int* status,
                          cudaStream_t st) {
  // one warp per CTA: each thread's loops carry FP64 work (about 3 x nb estimates), which takes the SM's FP64 pipe
  // for a whole warp instruction per operation, so the components are spread over as many SMs as they fill
  const int nc = 1 + K3 + nO, threads = 32;
  const int grid = (nc + threads - 1) / threads;
  finish_kernel<<<grid, threads, (size_t)(2 * nb + 2) * sizeof(double), st>>>(blk, nb, L, K3, nO, er, out, status);
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
