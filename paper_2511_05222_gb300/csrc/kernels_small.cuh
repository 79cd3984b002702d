// Small-system kernels (at most 32 electrons, 16 orbitals per spin): the VMC hot path of
// arXiv:2511.05222, App. A, laid out so that every lane does independent work.
//
//  move_small     LPW lanes per walker (1, 2, 4 or 8): a run of single-electron Metropolis
//                 moves with the MO row in registers and the CTA's inverses and positions
//                 staged walker-interleaved in shared memory (read from and written back to
//                 walker-interleaved global memory once per launch)
//  measure_small  one warp per walker, one lane per electron: two sweeps over the AOs, shell
//                 by shell, contracted straight into register rows (C rows broadcast from
//                 shared memory): the Slater row and the row of P = lap(phi) + 2 grad J .
//                 grad(phi), then (after the FP64 Gauss-Jordan inversion and B P B,
//                 cooperatively in the warp) the adjoint nuclear derivatives, the determinant
//                 drift and O; E_L and the walker sums
//
// Walker state on this path: positions [3 Ne][W] (double, plus a float-float copy in mixed
// mode) and inverses [n_up^2 + n_dn^2][W], walker index fastest.
#pragma once
#include <cuda_bf16.h>

#include <type_traits>

#include "vmcf_device.cuh"
#include "vmcf_internal.h"

namespace vmcf {

// Radial sums of a shell at displacement (x, y, z): R0 = sum e_k, R1 = sum -2a_k e_k,
// R2 = sum 4a_k^2 e_k, LF = sum -2a_k e_k ((2l+3) - 2a_k r^2), T3 = sum 4a_k^2 e_k ((2l+5) - 2a_k r^2).
template <typename T>
struct Radial {
  T R0, R1, R2, LF, T3;
};

template <typename T, int LEVEL>
__device__ __forceinline__ Radial<T> radial_sums(const DevSys& S, int s, int l, int np, T r2, int smask, R2FF r2ff) {
  Radial<T> o{T(0), T(0), T(0), T(0), T(0)};
  for (int k = 0; k < np; ++k) {
    const T a = prim_alpha<T>(S, s, k);
    T e, f3, f5;
    if (sizeof(T) == 4 && ((smask >> k) & 1)) {
      // a r^2 in float-float: (ah + al)(r2h + r2l)
      const float ah = __ldg(S.alpha_f + s * kMaxPrim + k), al = __ldg(S.alpha_lo + s * kMaxPrim + k);
      const float xh = ah * r2ff.h;
      const float xl = fmaf(ah, r2ff.h, -xh) + (ah * r2ff.l + al * r2ff.h);
      e = (T)(prim_coef<float>(S, s, k) * expf(-xh) * (1.0f - xl));
      f3 = (T)((float(2 * l + 3) - 2.0f * xh) - 2.0f * xl);
      f5 = (T)((float(2 * l + 5) - 2.0f * xh) - 2.0f * xl);
    } else {
      const T xa = a * r2;
      e = prim_coef<T>(S, s, k) * dexp<T>(-xa);
      f3 = T(2 * l + 3) - T(2) * xa;
      f5 = T(2 * l + 5) - T(2) * xa;
    }
    o.R0 += e;
    if (LEVEL >= 1) {
      const T m2ae = T(-2) * a * e;
      o.R1 += m2ae;
      o.LF += m2ae * f3;
      if (LEVEL >= 2) {
        const T a4e = T(4) * a * a * e;
        o.R2 += a4e;
        o.T3 += a4e * f5;
      }
    }
  }
  return o;
}

// Displacement of the electron from nucleus c (double in FP64 mode; float from the
// float-float positions in mixed mode), and for shells with sharp primitives (mixed mode)
// the squared distance as a float-float pair; returns the shell's sharp mask (0 if none).
template <typename T>
__device__ __forceinline__ int shell_disp(const DevSys& S, int s, int c, const double p[3], const float ph[3],
                                          const float pl[3], T d[3], R2FF& r2ff) {
  if constexpr (sizeof(T) == 8) {
#pragma unroll
    for (int k = 0; k < 3; ++k) d[k] = p[k] - __ldg(S.R + 3 * c + k);
    return 0;
  } else {
    const int smask = __ldg(S.sharp + s);
    if (!smask) {
#pragma unroll
      for (int k = 0; k < 3; ++k) d[k] = (ph[k] - __ldg(S.Rh + 3 * c + k)) + (pl[k] - __ldg(S.Rl + 3 * c + k));
      return 0;
    }
    float hsum = 0.f, lsum = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float dh, dl, sdiff, eh;
      two_sum(ph[k], -__ldg(S.Rh + 3 * c + k), sdiff, eh);
      fast_two_sum(sdiff, (pl[k] - __ldg(S.Rl + 3 * c + k)) + eh, dh, dl);
      d[k] = dh;
      const float pp = dh * dh, pe = fmaf(dh, dh, -pp);
      float t;
      two_sum(hsum, pp, hsum, t);
      lsum += t + pe + 2.0f * dh * dl;
    }
    fast_two_sum(hsum, lsum, r2ff.h, r2ff.l);
    return smask;
  }
}

__device__ __forceinline__ void split_ff(double v, float& h, float& l) {
  h = (float)v;
  l = (float)(v - (double)h);
}

// a r / (1 + F r) at r = |d| for the Metropolis ratio: in mixed mode with the approximate
// reciprocal square root and division (a few ulp; the ratio feeds an acceptance test only).
template <typename T>
__device__ __forceinline__ T pade_at(T a, T F, const T d[3]) {
  const T r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  if constexpr (sizeof(T) == 4) {
    const float r = r2 * rsqrtf(fmaxf(r2, 1e-30f));
    return __fdividef(a * r, 1.0f + F * r);
  } else {
    const double r = sqrt(r2);
    return a * r / (1.0 + F * r);
  }
}

// The two-body term of a pair at r = |d| for the Metropolis ratio, in the system's form.
template <typename T>
__device__ __forceinline__ T pair_at(const DevSys& S, bool par, const T d[3]) {
  if (!S.j2exp) return pade_at<T>((T)(par ? S.ap : S.aa), (T)(par ? S.Fp : S.Fa), d);
  const T r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  return expo_value<T>((T)(par ? S.ap : S.aa), (T)(par ? S.Fp : S.Fa), dsqrt<T>(r2));
}

template <typename T, int NM>
__device__ __forceinline__ void axpy_row(T (&acc)[NM], T a, const T* __restrict__ crow) {
#pragma unroll
  for (int i = 0; i < NM; ++i) acc[i] += a * crow[i];
}

template <typename T, int NM>
__device__ __forceinline__ T dot_row(const T (&x)[NM], const T* __restrict__ crow) {
  T s0 = 0, s1 = 0;  // two chains for instruction-level parallelism
#pragma unroll
  for (int i = 0; i < NM; i += 2) {
    s0 += x[i] * crow[i];
    if (i + 1 < NM) s1 += x[i + 1] * crow[i + 1];
  }
  return s0 + s1;
}

// Row stride of the staged coefficients for register rows of NM orbitals: a multiple of 4, so that
// every row starts on 16 bytes.
template <int NM>
__host__ __device__ constexpr int c_stride() { return (NM + 3) / 4 * 4; }

// Stage C^up and C^dn into shared memory as [2][M][c_stride<NM>()], zero-padded beyond n_s.
template <typename T, int NM>
__device__ __forceinline__ void stage_C(const DevSys& S, T* Cs) {
  constexpr int NMS = c_stride<NM>();
  for (int idx = threadIdx.x; idx < 2 * S.M * NMS; idx += blockDim.x) {
    const int sg = idx / (S.M * NMS), r = idx - sg * S.M * NMS, mu = r / NMS, i = r - mu * NMS;
    const int n = sg == 0 ? S.nup : S.ndn;
    Cs[idx] = (i < n) ? __ldg(coefC<T>(S, sg) + mu * n + i) : T(0);
  }
}


// ---------------------------------------------------------------- moves, LPW lanes per walker
// Sum over the LPW lanes of a walker (xor butterfly: every lane receives the same bits).
template <int LPW, typename V>
__device__ __forceinline__ V lane_group_sum(V v, unsigned mask) {
#pragma unroll
  for (int o = 1; o < LPW; o <<= 1) v += __shfl_xor_sync(mask, v, o);
  return v;
}

// A run of single-electron Metropolis moves. LPW lanes cooperate on one walker: shells, ratio
// terms, Jastrow pairs and Sherman-Morrison columns are split across them and combined with
// butterfly sums, so the accept decision is identical in all of a walker's lanes.
template <typename T, int NM, int LPW, bool GUIDE>
__global__ void __launch_bounds__(256) move_small(DevSys S, SmallMoveParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  // shared memory: C^up, C^dn [2][M][c_stride<NM>()]; the CTA's inverses walker-interleaved [nB][WPC]; its
  // positions [3 Ne][WPC] (float-float pairs in mixed mode, double in FP64 mode)
  T* Cs = reinterpret_cast<T*>(smem);
  const int WPC = P.wpc;
  T* Bs = Cs + 2 * S.M * c_stride<NM>();
  using PosT = typename std::conditional<sizeof(T) == 4, float2, double>::type;
  PosT* Ps = reinterpret_cast<PosT*>(Bs + (size_t)S.nB * WPC);
  stage_C<T, NM>(S, Cs);
  const int W = P.W, Ne = S.Ne, nup = S.nup, K = S.K, nB = S.nB;
  const int wbase = blockIdx.x * WPC;
  T* Bg = reinterpret_cast<T*>(P.B);
  for (int idx = threadIdx.x; idx < nB * WPC; idx += blockDim.x) {
    const int k = idx / WPC, ws = idx - k * WPC;
    if (wbase + ws < W) Bs[idx] = Bg[(size_t)k * W + wbase + ws];
  }
  for (int idx = threadIdx.x; idx < 3 * Ne * WPC; idx += blockDim.x) {
    const int k = idx / WPC, ws = idx - k * WPC;
    if (wbase + ws < W) {
      const double v = P.pos[(size_t)k * W + wbase + ws];
      if constexpr (sizeof(T) == 4) {
        float h, l;
        split_ff(v, h, l);
        Ps[idx] = make_float2(h, l);
      } else {
        Ps[idx] = v;
      }
    }
  }
  __syncthreads();
  const int ws = threadIdx.x / LPW, q = threadIdx.x % LPW, w = wbase + ws;
  // whole lane groups leave together (LPW divides 32)
  if (ws >= WPC || w >= P.W) return;
  // lanes of this walker only: barriers inside the accept branch must not wait for other
  // walkers' lanes, which take their own branch
  const unsigned mask = (LPW == 32) ? 0xffffffffu : (((1u << LPW) - 1u) << ((threadIdx.x & 31) & ~(LPW - 1)));
  T* B = Bs + ws;     // element k of this walker's inverses at B[k * WPC]
  PosT* pp = Ps + ws;  // coordinate k of this walker's electrons at pp[k * WPC]
  const uint64_t wid = P.wid0 + (uint64_t)w;
  uint32_t nacc = 0, nrej = 0;
  // reweighted sampling of |Psi_G|^2, Psi_G = Psi max(1, eps sqrt(S)): S of the current inverses
  constexpr bool guide = GUIDE;  // P.eps > 0
  double Sg = 0.0;
  if (guide) {
    for (int k = q; k < nB; k += LPW) Sg += (double)B[k * WPC] * (double)B[k * WPC];
    Sg = lane_group_sum<LPW>(Sg, mask);
  }
  for (int mv = 0; mv < P.nmoves; ++mv) {
    const uint64_t gm = P.move0 + (uint64_t)mv;
    const int e = (int)(gm % (uint64_t)Ne);
    const uint64_t sweep = gm / (uint64_t)Ne;
    const int sg = e < nup ? 0 : 1;
    const int n = sg == 0 ? nup : S.ndn, el = e - (sg == 0 ? 0 : nup);
    const int off = sg == 0 ? 0 : nup * nup;
    const T* Csg = Cs + sg * S.M * c_stride<NM>();
    uint64_t r[4] = {wid, sweep, (uint64_t)e, 0};
    philox4x64_10(r, P.k0, P.k1);
    double xi[3];
    normals3(r, xi, T(0));
    double po[3], rn[3];
    float nh[3], nl[3], oh[3], ol[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      po[k] = P.pos[(size_t)(3 * e + k) * W + w];
      rn[k] = po[k] + P.sigma * xi[k];
      split_ff(rn[k], nh[k], nl[k]);
      if constexpr (sizeof(T) == 4) {
        const float2 f = pp[(3 * e + k) * WPC];
        oh[k] = f.x;
        ol[k] = f.y;
      }
    }
    // new orbital row: this lane's shells, then the group sum
    T row[NM];
#pragma unroll
    for (int i = 0; i < NM; ++i) row[i] = T(0);
    for (int s = q; s < S.nshell; s += LPW) {
      const int4 sh = __ldg(S.shell + s);
      T d[3];
      if constexpr (sizeof(T) == 8) {
#pragma unroll
        for (int k = 0; k < 3; ++k) d[k] = rn[k] - __ldg(S.R + 3 * sh.x + k);
      } else {
#pragma unroll
        for (int k = 0; k < 3; ++k) d[k] = (nh[k] - __ldg(S.Rh + 3 * sh.x + k)) + (nl[k] - __ldg(S.Rl + 3 * sh.x + k));
      }
      const T r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      const Radial<T> rs = radial_sums<T, 0>(S, s, sh.y, sh.z, r2, 0, R2FF{0.f, 0.f});
      for (int m = 0; m < 2 * sh.y + 1; ++m) {
        T Pa, g[3], h[6];
        angular<T>(sh.y, m, d[0], d[1], d[2], Pa, g, h);
        axpy_row<T, NM>(row, Pa * rs.R0, Csg + (sh.w + m) * c_stride<NM>());
      }
    }
#pragma unroll
    for (int i = 0; i < NM; ++i) row[i] = lane_group_sum<LPW>(row[i], mask);
    // determinant ratio (FP64): this lane's orbitals i = q, q + LPW, ...
    double R = 0.0;
#pragma unroll
    for (int i = 0; i < NM; ++i)
      if (i % LPW == q && i < n) R += (double)row[i] * (double)B[(off + i * n + el) * WPC];
    R = lane_group_sum<LPW>(R, mask);
    // Jastrow ratio: this lane's partners j = q, q + LPW, ... and nuclei I = q, q + LPW, ...
    T jacc = 0;
    if (S.J2) {
      for (int j = q; j < Ne; j += LPW) {
        if (j == e) continue;
        const bool par = (j < nup) == (e < nup);
        T d1[3], d0[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          if constexpr (sizeof(T) == 8) {
            const double pj = pp[(3 * j + k) * WPC];
            d1[k] = rn[k] - pj;
            d0[k] = po[k] - pj;
          } else {
            const float2 f = pp[(3 * j + k) * WPC];
            d1[k] = (nh[k] - f.x) + (nl[k] - f.y);
            d0[k] = (oh[k] - f.x) + (ol[k] - f.y);
          }
        }
        jacc += pair_at<T>(S, par, d1) - pair_at<T>(S, par, d0);
      }
    }
    if (S.J1) {
      for (int I = q; I < K; I += LPW) {
        const T mz = (T)(-__ldg(S.Z + I)), b = (T)S.ben;
        T d1[3], d0[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          if constexpr (sizeof(T) == 8) {
            d1[k] = rn[k] - __ldg(S.R + 3 * I + k);
            d0[k] = po[k] - __ldg(S.R + 3 * I + k);
          } else {
            d1[k] = (nh[k] - __ldg(S.Rh + 3 * I + k)) + (nl[k] - __ldg(S.Rl + 3 * I + k));
            d0[k] = (oh[k] - __ldg(S.Rh + 3 * I + k)) + (ol[k] - __ldg(S.Rl + 3 * I + k));
          }
        }
        jacc += pade_at<T>(mz, b, d1) - pade_at<T>(mz, b, d0);
      }
    }
    const double dJ = (double)lane_group_sum<LPW>(jacc, mask);
    uint64_t r2[4] = {wid, sweep, (uint64_t)e, 1};
    philox4x64_10(r2, P.k0, P.k1);
    const double u = u01(r2[0]);
    double pr = R * R * (double)dexp<T>((T)(2.0 * dJ));
    // Sherman-Morrison: w_j = sum_i row_i B_ij - delta_j,el; B_kj <- B_kj - B_k,el w_j / R.
    // This lane owns columns j = q, q + LPW, ...; every lane reads the whole column el first.
    T wv[NM], col[NM];
    auto sm_vectors = [&]() {
#pragma unroll
      for (int j = 0; j < NM; ++j) {
        wv[j] = T(0);
        col[j] = (j < n) ? B[(off + j * n + el) * WPC] : T(0);
      }
#pragma unroll
      for (int i = 0; i < NM; ++i) {
        if (i >= n) continue;
        const T ri = row[i];
#pragma unroll
        for (int j = 0; j < NM; ++j)
          if (j % LPW == q && j < n) wv[j] += ri * B[(off + i * n + j) * WPC];
      }
    };
    double Sn = Sg;
    if constexpr (guide) if (R != 0.0) {
      // S after the update B' = B - c w^T / R (c = column el): S - (2/R) w.(B^T c) + |c|^2 |w|^2 / R^2
      sm_vectors();
      double tw = 0.0, ww = 0.0, cc = 0.0;
#pragma unroll
      for (int j = 0; j < NM; ++j) {
        if (j >= n) continue;
        cc += (double)col[j] * (double)col[j];
        if (j % LPW != q) continue;
        T tj = 0;
#pragma unroll
        for (int i = 0; i < NM; ++i)
          if (i < n) tj += col[i] * B[(off + i * n + j) * WPC];
        const double wj = (double)((j == el) ? wv[j] - T(1) : wv[j]);
        tw += wj * (double)tj;
        ww += wj * wj;
      }
      tw = lane_group_sum<LPW>(tw, mask);
      ww = lane_group_sum<LPW>(ww, mask);
      Sn = Sg - 2.0 * tw / R + cc * ww / (R * R);
      const double g0 = fmax(1.0, P.eps * sqrt(Sg)), g1 = fmax(1.0, P.eps * sqrt(fmax(Sn, 0.0)));
      pr *= (g1 / g0) * (g1 / g0);
    }
    const bool ok = isfinite(pr) && R != 0.0;
    if (!ok) ++nrej;
    if (ok && u < pr) {
      if constexpr (!guide) sm_vectors();
      Sg = Sn;
      if (LPW > 1) __syncwarp(mask);  // column el is read by all lanes before its owner rewrites it
      const T rinv = (T)(1.0 / R);
#pragma unroll
      for (int j = 0; j < NM; ++j) {
        if (j % LPW != q || j >= n) continue;
        const T wj = (j == el) ? wv[j] - T(1) : wv[j];
#pragma unroll
        for (int k = 0; k < NM; ++k) {
          if (k >= n) continue;
          T& bkj = B[(off + k * n + j) * WPC];
          bkj -= col[k] * rinv * wj;
        }
      }
      if (q == 0) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          P.pos[(size_t)(3 * e + k) * W + w] = rn[k];
          if constexpr (sizeof(T) == 4) pp[(3 * e + k) * WPC] = make_float2(nh[k], nl[k]);
          else pp[(3 * e + k) * WPC] = rn[k];
        }
      }
      ++nacc;
    }
    if (LPW > 1) __syncwarp(mask);  // the new position is visible to the group's next move
  }
  if (q == 0) {
    P.nacc[w] += nacc;
    P.nrej[w] += nrej;
  }
  // this walker's inverses back to global memory (its lanes share the copy)
  if (LPW > 1) __syncwarp(mask);
  for (int k = q; k < nB; k += LPW) Bg[(size_t)k * W + w] = B[k * WPC];
}

// ---------------------------------------------------------------- both spin blocks' FP64 inverses
// The two Slater matrices of a walker inverted at once by one warp, half-warp h (lanes 16h..16h+15)
// taking matrix h (A_h, n_h x n_h row-major, in place), with the steps of gj_inverse: partial row
// pivoting (largest |x|, lowest row on ties, found over the half-warp), the scaled pivot row, the row
// it displaces and column k copied, then every element updated once with the row swap folded in; the
// row permutation is undone as column swaps at the end. The pivot sequence and every operation on an
// element are those of gj_inverse, so the inverses are the same to the bit. piv: int[2][nmax];
// f: double[2][3 nmax + 1]. flag is set to 1 on a zero or non-finite pivot; with want_logdet the
// logarithm of |det A_0 det A_1| and the sign of the product are accumulated into logabs and sgn.
static __device__ __forceinline__ void gj_inverse_pair(double* A0, int n0, double* A1, int n1, int nmax, int* piv, double* f, int* flag,
                                double* logabs, double* sgn, bool want_logdet) {
  const int lane = threadIdx.x & 31, h = lane >> 4, hl = lane & 15;
  double* A = h ? A1 : A0;
  const int n = h ? n1 : n0;
  int* pv = piv + h * nmax;
  double* ff = f + h * (3 * nmax + 1);
  double* rs = ff + n + 1;      // scaled pivot row: the new row k
  double* rk = ff + 2 * n + 1;  // old row k: the new row p
  const int i0 = n > 0 ? hl / n : 0, j0 = n > 0 ? hl - i0 * n : 0;
  const int di = n > 0 ? 16 / n : 0, dj = n > 0 ? 16 - di * n : 0;
  double la = 0.0, sg = 1.0;
  const int nk = n0 > n1 ? n0 : n1;
  for (int k = 0; k < nk; ++k) {
    const bool act = k < n;
    long long best = -1;
    int bi = k;
    if (act)
      for (int i = k + hl; i < n; i += 16) {
        const long long v = __double_as_longlong(A[i * n + k]) & 0x7fffffffffffffffLL;
        if (v > best) { best = v; bi = i; }
      }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {  // within the half-warp
      const long long ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (act && hl == 0) {
      pv[k] = bi;
      const double p = A[bi * n + k];
      if (!(p != 0.0) || !isfinite(p)) *flag = 1;
      ff[n] = 1.0 / p;
      if (want_logdet) {
        la += log(fabs(p));
        if (p < 0) sg = -sg;
        if (bi != k) sg = -sg;
      }
    }
    __syncwarp();
    if (act) {
      const int p = pv[k];
      const double pinv = ff[n];
      for (int j = hl; j < n; j += 16) {
        rs[j] = (j == k ? 1.0 : A[p * n + j]) * pinv;
        rk[j] = A[k * n + j];
      }
      for (int i = hl; i < n; i += 16) ff[i] = A[i * n + k];
    }
    __syncwarp();
    if (act) {
      const int p = pv[k];
      const double fp = ff[k];
      for (int i = i0, j = j0; i < n;) {
        double v;
        if (i == k) {
          v = rs[j];
        } else {
          const double fi = i == p ? fp : ff[i];
          const double aij = i == p ? rk[j] : A[i * n + j];
          v = (j == k ? 0.0 : aij) - fi * rs[j];
        }
        A[i * n + j] = v;
        i += di;
        j += dj;
        if (j >= n) {
          j -= n;
          ++i;
        }
      }
    }
    __syncwarp();
  }
  for (int i = hl; i < n; i += 16)
    for (int k = n - 1; k >= 0; --k) {
      const int p = pv[k];
      if (p != k) {
        const double a = A[i * n + k];
        A[i * n + k] = A[i * n + p];
        A[i * n + p] = a;
      }
    }
  if (want_logdet) {
    const double la1 = __shfl_sync(0xffffffffu, la, 16), sg1 = __shfl_sync(0xffffffffu, sg, 16);
    if (lane == 0) {
      *logabs += la + la1;
      *sgn *= sg * sg1;
    }
  }
  __syncwarp();
}

// ---------------------------------------------------------------- measurement, one warp per walker


template <int NV>
__device__ __forceinline__ void warp_sum_f(float (&v)[NV]) {
#pragma unroll
  for (int k = 0; k < NV; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
}
template <int NV>
__device__ __forceinline__ void warp_sum_f(double (&v)[NV]) {
#pragma unroll
  for (int k = 0; k < NV; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
}

template <typename T, int NM>
__global__ void __launch_bounds__(256, 2) measure_small(DevSys S, SmallLayout L, SmallMeasParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  T* Cs = reinterpret_cast<T*>(smem + L.cta_C);
  T* acc_s = reinterpret_cast<T*>(smem + L.cta_acc);
  unsigned char* base = smem + L.cta_bytes + warp * L.bytes;
  double* pd = reinterpret_cast<double*>(base + L.pd);
  float* ph = reinterpret_cast<float*>(base + L.ph);
  float* pl = reinterpret_cast<float*>(base + L.pl);
  double* Ad = reinterpret_cast<double*>(base + L.Ad);
  T* Bf = reinterpret_cast<T*>(base + L.Bf);
  T* Pm = reinterpret_cast<T*>(base + L.Pm);
  T* Q = reinterpret_cast<T*>(base + L.Q);
  int* piv = reinterpret_cast<int*>(base + L.piv);
  double* f = reinterpret_cast<double*>(base + L.f);
  T* frc = reinterpret_cast<T*>(base + L.frc);
  T* phi = reinterpret_cast<T*>(base + L.phi);
  int* flag = reinterpret_cast<int*>(base + L.scal);
  double* la = reinterpret_cast<double*>(base + L.scal + 8);
  double* sgn = reinterpret_cast<double*>(base + L.scal + 16);

  const int Ne = S.Ne, nup = S.nup, ndn = S.ndn, K = S.K, M = S.M, W = P.W;
  const int nO = M * Ne;
  const bool accum = P.mode == 2;
  // mixed-mode walker sums of O through the tensor-core kernel: emit PhiT and YT tiles
  const bool tc = accum && sizeof(T) == 4 && P.phiT[0] != nullptr;
  stage_C<T, NM>(S, Cs);
  if (accum)
    for (int i = threadIdx.x; i < P.accL; i += blockDim.x) acc_s[i] = T(0);
  __syncthreads();

  const long long w0 = (long long)W * blockIdx.x / gridDim.x, w1 = (long long)W * (blockIdx.x + 1) / gridDim.x;
  const int e = lane;
  const bool has_e = e < Ne;
  const int sg = e < nup ? 0 : 1;
  const int n = sg == 0 ? nup : ndn, el = e - (sg == 0 ? 0 : nup), off = sg == 0 ? 0 : nup * nup;
  for (long long wl = w0 + warp; wl < w1; wl += nwarps) {
    const int w = (int)wl;
    // ---- positions
    double p[3] = {0.0, 0.0, 0.0};
    float hh[3] = {0.f, 0.f, 0.f}, ll[3] = {0.f, 0.f, 0.f};
    if (has_e) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        p[k] = P.pos[(long long)(3 * e + k) * P.pos_sk + (long long)w * P.pos_sw];
        split_ff(p[k], hh[k], ll[k]);
        pd[3 * e + k] = p[k];
        ph[3 * e + k] = hh[k];
        pl[3 * e + k] = ll[k];
        if (P.posf_out) P.posf_out[(size_t)(3 * e + k) * W + w] = make_float2(hh[k], ll[k]);
      }
    }
    if (lane == 0) {
      *flag = 0;
      *la = 0.0;
      *sgn = 1.0;
    }
    __syncwarp();  // every electron's position visible to the warp
    const bool full = P.mode != 0;  // mode 0 only rebuilds the inverses
    // ---- Jastrow and potentials (lane = electron)
    T jg[3] = {T(0), T(0), T(0)}, jl = T(0);
    double vpart[4] = {0.0, 0.0, 0.0, 0.0};  // kinetic, V_ee, V_en, J
    if (full && has_e) {
      T vee = 0, ven = 0, jv = 0;
      for (int j = 0; j < Ne; ++j) {
        if (j == e) continue;
        T d[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          if constexpr (sizeof(T) == 8) d[k] = p[k] - pd[3 * j + k];
          else d[k] = (hh[k] - ph[3 * j + k]) + (ll[k] - pl[3 * j + k]);
        }
        const T r = dsqrt<T>(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]), ri = T(1) / r;
        if (j > e) vee += ri;
        if (S.J2) {
          const bool par = (j < nup) == (e < nup);
          const Rad3<T> u = pair_rad<T>(S, par, r);
          const T gr = u.h1 * ri;
#pragma unroll
          for (int k = 0; k < 3; ++k) jg[k] += gr * d[k];
          jl += u.h2 + T(2) * gr;
          if (j > e) jv += u.h;
        }
      }
      for (int I = 0; I < K; ++I) {
        T d[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          if constexpr (sizeof(T) == 8) d[k] = p[k] - __ldg(S.R + 3 * I + k);
          else d[k] = (hh[k] - __ldg(S.Rh + 3 * I + k)) + (ll[k] - __ldg(S.Rl + 3 * I + k));
        }
        const T r = dsqrt<T>(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]), ri = T(1) / r;
        const T Z = (T)__ldg(S.Z + I);
        ven -= Z * ri;
        if (S.J1) {
          const Rad3<T> c = pade<T>(-Z, (T)S.ben, r);
          const T gr = c.h1 * ri;
#pragma unroll
          for (int k = 0; k < 3; ++k) jg[k] += gr * d[k];
          jl += c.h2 + T(2) * gr;
          jv += c.h;
        }
      }
      vpart[1] = (double)vee;
      vpart[2] = (double)ven;
      vpart[3] = (double)jv;
    }

    // ---- pass 1: the Slater row (one per lane) -> FP64 -> Gauss-Jordan per spin; when measuring, in
    // the same sweep over the AOs, the row of P = lap(phi) + 2 grad(J) . grad(phi) that the adjoint
    // weights B P B and the kinetic term need (linear in C, so one coefficient per AO:
    // P_{e i} = sum_mu C_{mu i} (lap psi_mu + 2 grad J . grad psi_mu))
    if (has_e) {
      T row[NM];
#pragma unroll
      for (int i = 0; i < NM; ++i) row[i] = T(0);
      const T* Csg = Cs + sg * M * c_stride<NM>();
      if (!full) {
        for (int s = 0; s < S.nshell; ++s) {
          const int4 sh = __ldg(S.shell + s);
          T d[3];
          R2FF r2ff{0.f, 0.f};
          const int smask = shell_disp<T>(S, s, sh.x, p, hh, ll, d, r2ff);
          const Radial<T> rs = radial_sums<T, 0>(S, s, sh.y, sh.z, d[0] * d[0] + d[1] * d[1] + d[2] * d[2], smask, r2ff);
          for (int m = 0; m < 2 * sh.y + 1; ++m) {
            T Pa, g[3], h[6];
            angular<T>(sh.y, m, d[0], d[1], d[2], Pa, g, h);
            axpy_row<T, NM>(row, Pa * rs.R0, Csg + (sh.w + m) * c_stride<NM>());
          }
        }
      } else {
        T prow[NM];
#pragma unroll
        for (int i = 0; i < NM; ++i) prow[i] = T(0);
        for (int s = 0; s < S.nshell; ++s) {
          const int4 sh = __ldg(S.shell + s);
          T d[3];
          R2FF r2ff{0.f, 0.f};
          const int smask = shell_disp<T>(S, s, sh.x, p, hh, ll, d, r2ff);
          const Radial<T> rs = radial_sums<T, 1>(S, s, sh.y, sh.z, d[0] * d[0] + d[1] * d[1] + d[2] * d[2], smask, r2ff);
          const T xjR1 = T(2) * (d[0] * jg[0] + d[1] * jg[1] + d[2] * jg[2]) * rs.R1;
          for (int m = 0; m < 2 * sh.y + 1; ++m) {
            T Pa, g[3], h[6];
            angular<T>(sh.y, m, d[0], d[1], d[2], Pa, g, h);
            const T* cr = Csg + (sh.w + m) * c_stride<NM>();
            axpy_row<T, NM>(row, Pa * rs.R0, cr);
            // lap psi = P LF; grad psi = g R0 + P d R1
            const T gj2 = T(2) * (g[0] * jg[0] + g[1] * jg[1] + g[2] * jg[2]);
            axpy_row<T, NM>(prow, Pa * (rs.LF + xjR1) + gj2 * rs.R0, cr);
          }
        }
#pragma unroll
        for (int i = 0; i < NM; ++i)
          if (i < n) Pm[off + el * n + i] = prow[i];
      }
#pragma unroll
      for (int i = 0; i < NM; ++i)
        if (i < n) Ad[off + el * n + i] = (double)row[i];
    }
    __syncwarp();
    gj_inverse_pair(Ad, nup, Ad + nup * nup, ndn, S.nmax, piv, f, flag, la, sgn, P.logpsi != nullptr);
    if (static_cast<void*>(Bf) != static_cast<void*>(Ad))
      for (int i = lane; i < S.nB; i += 32) Bf[i] = (T)Ad[i];
    __syncwarp();
    if (P.Bout && P.mode != 1) {
      T* Bg = reinterpret_cast<T*>(P.Bout);
      for (int i = lane; i < S.nB; i += 32) Bg[(size_t)i * W + w] = Bf[i];
    }
    if (lane == 0 && *flag) atomicAdd(&P.counters[0], 1ull);
    // reweighting factor |Psi / Psi_G|^2 = 1 / g^2 of a guided chain (g = max(1, eps sqrt(S)), S the
    // sum of the squared entries of the fresh inverses); every walker sum below carries it
    double wt = 1.0;
    if (accum && P.eps > 0.0) {
      double sq = 0.0;
      for (int i = lane; i < S.nB; i += 32) sq += (double)Bf[i] * (double)Bf[i];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
      const double g = fmax(1.0, P.eps * sqrt(sq));
      wt = 1.0 / (g * g);
    }
    if (P.mode == 0) {
      __syncwarp();
      continue;
    }

    // ---- kinetic term: -1/2 (lap Psi / Psi) of electron e = -1/2 (sum_i P_{e i} B_{i e} + lap J + |grad J|^2)
    T bc[NM];  // column el of B^s: B_{i, el}
#pragma unroll
    for (int i = 0; i < NM; ++i) bc[i] = (has_e && i < n) ? Bf[off + i * n + el] : T(0);
    if (has_e) {
      T ps = 0;
#pragma unroll
      for (int i = 0; i < NM; ++i)
        if (i < n) ps += Pm[off + el * n + i] * bc[i];
      const T te = ps + jl + (jg[0] * jg[0] + jg[1] * jg[1] + jg[2] * jg[2]);
      vpart[0] = -0.5 * (double)te;
    }
    warp_sum_f<4>(vpart);
    const double EL = vpart[0] + vpart[1] + vpart[2] + S.Vnn;
    const double cw = EL - P.e_ref;
    if (P.mode == 1 && !P.dlnpsi && !P.dEL && !P.O) {  // E_L and ln|Psi| only: no adjoint pass
      if (lane == 0) {
        if (P.EL) P.EL[w] = EL;
        if (P.logpsi) P.logpsi[w] = *la + vpart[3];
      }
      __syncwarp();
      continue;
    }
    __syncwarp();

    // ---- adjoint weights per spin: Q = B P, X = Q B (X[e][i] = (B P B)_{i e}, over P)
    for (int s2 = 0; s2 < 2; ++s2) {
      const int ns = s2 == 0 ? nup : ndn, o2 = s2 == 0 ? 0 : nup * nup;
      if (ns == 0) continue;
      const T* Bs = Bf + o2;
      T* Ps = Pm + o2;
      for (int idx = lane; idx < ns * ns; idx += 32) {
        const int i = idx / ns, j = idx - i * ns;
        T v = 0;
        for (int k = 0; k < ns; ++k) v += Bs[i * ns + k] * Ps[k * ns + j];
        Q[idx] = v;
      }
      __syncwarp();
      for (int idx = lane; idx < ns * ns; idx += 32) {
        const int ee = idx / ns, i = idx - ee * ns;
        T v = 0;
        for (int j = 0; j < ns; ++j) v += Q[i * ns + j] * Bs[j * ns + ee];
        Ps[idx] = v;
      }
      __syncwarp();
    }
    for (int i = lane; i < 6 * K; i += 32) frc[i] = T(0);
    __syncwarp();

    // ---- pass 3: nuclear derivatives (lane = electron) and O in AO chunks
    T xr[NM];
#pragma unroll
    for (int i = 0; i < NM; ++i) xr[i] = (has_e && i < n) ? Pm[off + el * n + i] : T(0);
    T fl[3] = {T(0), T(0), T(0)}, fe[3] = {T(0), T(0), T(0)};
    T fr[3] = {T(0), T(0), T(0)};  // sum over every AO of the dE_L terms of this electron (space warp): fe summed over nuclei
    // determinant drift grad_e D / D = sum_i grad phi_i(r_e) B_{i e} = sum_mu grad psi_mu(r_e) (C B)_{mu e}:
    // the sum over every AO of the products that fl collects per nucleus (with the opposite sign)
    T gd[3] = {T(0), T(0), T(0)};
    int cur = -1;
    int chunk0 = 0, chunk_n = 0;  // AOs [chunk0, chunk0 + chunk_n) pending in phi
    const T* Csg = Cs + sg * M * c_stride<NM>();
    auto flush_centre = [&](int I) {
      float v6f[6];
      double v6d[6];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        gd[k] -= fl[k];
        fr[k] += fe[k];
      }
      if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          v6f[k] = fl[k];
          v6f[3 + k] = fe[k];
        }
        warp_sum_f<6>(v6f);
        if (lane == 0)
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            frc[3 * I + k] += v6f[k];
            frc[3 * K + 3 * I + k] += v6f[3 + k];
          }
      } else {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          v6d[k] = fl[k];
          v6d[3 + k] = fe[k];
        }
        warp_sum_f<6>(v6d);
        if (lane == 0)
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            frc[3 * I + k] += v6d[k];
            frc[3 * K + 3 * I + k] += v6d[3 + k];
          }
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) fl[k] = fe[k] = T(0);
    };
    // O^s[mu][i] = sum over electrons e of spin s of psi_mu(r_e) B_{i, el(e)}; lanes 0..15 take
    // spin up, 16..31 spin down, one orbital i each.
    auto flush_chunk = [&]() {
      if (tc) {
        chunk0 += chunk_n;
        chunk_n = 0;
        return;
      }
      __syncwarp();
      const int g = lane >> 4, i = lane & 15;
      const int ng = g == 0 ? nup : ndn, og = g == 0 ? 0 : nup * nup, e0 = g == 0 ? 0 : nup;
      const int ooff = g == 0 ? 0 : M * nup;
      if (i < ng) {
        T brow[NM];
#pragma unroll
        for (int k = 0; k < NM; ++k) brow[k] = (k < ng) ? Bf[og + i * ng + k] : T(0);
        for (int c = 0; c < chunk_n; ++c) {
          T s = 0;
#pragma unroll
          for (int k = 0; k < NM; ++k)
            if (k < ng) s += phi[(e0 + k) * L.chunk + c] * brow[k];
          const int mu = chunk0 + c;
          if (P.O) P.O[(size_t)w * nO + ooff + mu * ng + i] = (double)s;
          if (accum) {
            atomicAdd(&acc_s[3 + 9 * K + ooff + mu * ng + i], (T)wt * s);
            atomicAdd(&acc_s[3 + 9 * K + nO + ooff + mu * ng + i], (T)(wt * cw) * s);
          }
        }
      }
      __syncwarp();
      chunk0 += chunk_n;
      chunk_n = 0;
    };
    for (int s = 0; s < S.nshell; ++s) {
      const int4 sh = __ldg(S.shell + s);
      const int ncomp = 2 * sh.y + 1;
      if (chunk_n + ncomp > L.chunk) flush_chunk();
      if (sh.x != cur) {
        if (cur >= 0) flush_centre(cur);
        cur = sh.x;
      }
      if (has_e) {
        T d[3];
        R2FF r2ff{0.f, 0.f};
        const int smask = shell_disp<T>(S, s, sh.x, p, hh, ll, d, r2ff);
        const Radial<T> rs = radial_sums<T, 2>(S, s, sh.y, sh.z, d[0] * d[0] + d[1] * d[1] + d[2] * d[2], smask, r2ff);
        const T xj = d[0] * jg[0] + d[1] * jg[1] + d[2] * jg[2];
        for (int m = 0; m < ncomp; ++m) {
          T Pa, g[3], h[6];
          angular<T>(sh.y, m, d[0], d[1], d[2], Pa, g, h);
          const T* cr = Csg + (sh.w + m) * c_stride<NM>();
          const T yA = dot_row<T, NM>(xr, cr), yL = dot_row<T, NM>(bc, cr);
          // Hessian of the AO contracted with grad J without forming it:
          // (H j)_a = (h j)_a R0 + g_a (x.j) R1 + (g.j) x_a R1 + P x_a (x.j) R2 + P j_a R1
          const T hj0 = h[0] * jg[0] + h[3] * jg[1] + h[4] * jg[2];
          const T hj1 = h[3] * jg[0] + h[1] * jg[1] + h[5] * jg[2];
          const T hj2 = h[4] * jg[0] + h[5] * jg[1] + h[2] * jg[2];
          const T hjv[3] = {hj0, hj1, hj2};
          const T gj = g[0] * jg[0] + g[1] * jg[1] + g[2] * jg[2];
          const T PxjR2 = Pa * xj * rs.R2, gjR1 = gj * rs.R1, PR1 = Pa * rs.R1, xjR1 = xj * rs.R1;
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const T gv = g[k] * rs.R0 + Pa * d[k] * rs.R1;
            const T gl = g[k] * rs.LF + Pa * d[k] * rs.T3;
            const T hj = hjv[k] * rs.R0 + g[k] * xjR1 + d[k] * (gjR1 + PxjR2) + jg[k] * PR1;
            fl[k] -= gv * yL;
            const T cde = T(-0.5) * (gv * yA - yL * (gl + T(2) * hj));
            fe[k] += cde;
          }
          if (tc)
            reinterpret_cast<__nv_bfloat16*>(P.phiT[sg])[((size_t)w * P.Mp + sh.w + m) * 16 + el] =
                __float2bfloat16_rn((float)(Pa * rs.R0));
          else
            phi[e * L.chunk + chunk_n + m] = Pa * rs.R0;
        }
      }
      chunk_n += ncomp;
    }
    if (cur >= 0) flush_centre(cur);
    flush_chunk();
    if (tc && has_e) {  // Y rows: B_{i, el} and (E_L - E_ref) B_{i, el}
      __nv_bfloat16* y = reinterpret_cast<__nv_bfloat16*>(P.yT[sg]) + (size_t)w * P.Np * 16;
#pragma unroll
      for (int i = 0; i < NM; ++i)
        if (i < n) {
          y[i * 16 + el] = __float2bfloat16_rn((float)((T)wt * bc[i]));
          y[(n + i) * 16 + el] = __float2bfloat16_rn((float)((T)(wt * cw) * bc[i]));
        }
    }
    // e-n Jastrow and V_en derivatives, one nucleus at a time; an electron moving is the
    // negative of the nucleus moving, so dE_L/dr_e collects minus every term
    T dr[3] = {-fr[0], -fr[1], -fr[2]};
    for (int I = 0; I < K; ++I) {
      T c6[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
      if (has_e) {
        T sd[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          if constexpr (sizeof(T) == 8) sd[k] = p[k] - __ldg(S.R + 3 * I + k);
          else sd[k] = (hh[k] - __ldg(S.Rh + 3 * I + k)) + (ll[k] - __ldg(S.Rl + 3 * I + k));
        }
        const T r = dsqrt<T>(sd[0] * sd[0] + sd[1] * sd[1] + sd[2] * sd[2]), ri = T(1) / r;
        const T Z = (T)__ldg(S.Z + I);
        const T nn[3] = {sd[0] * ri, sd[1] * ri, sd[2] * ri};
        const T ven = -Z * ri * ri * ri;
#pragma unroll
        for (int k = 0; k < 3; ++k) c6[3 + k] = ven * sd[k];
        if (S.J1) {
          const Rad3<T> c = pade<T>(-Z, (T)S.ben, r);
          const T gs[3] = {gd[0] + jg[0], gd[1] + jg[1], gd[2] + jg[2]};
          const T dl = c.h3 + T(2) * c.h2 * ri - T(2) * c.h1 * ri * ri;
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            T hs = 0;
#pragma unroll
            for (int cc = 0; cc < 3; ++cc)
              hs += (c.h2 * nn[k] * nn[cc] + c.h1 * ri * ((k == cc ? T(1) : T(0)) - nn[k] * nn[cc])) * gs[cc];
            c6[k] = -c.h1 * nn[k];
            c6[3 + k] += hs + T(0.5) * dl * nn[k];
          }
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) dr[k] -= c6[3 + k];
      }
      if constexpr (sizeof(T) == 4) {
        float v6[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) v6[k] = c6[k];
        warp_sum_f<6>(v6);
        if (lane == 0)
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            frc[3 * I + k] += v6[k];
            frc[3 * K + 3 * I + k] += v6[3 + k];
          }
      } else {
        double v6[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) v6[k] = c6[k];
        warp_sum_f<6>(v6);
        if (lane == 0)
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            frc[3 * I + k] += v6[k];
            frc[3 * K + 3 * I + k] += v6[3 + k];
          }
      }
    }
    __syncwarp();
    // ---- space warp (force expression with omega_a(r) = kappa(|r - R_a|) / sum_b kappa(|r - R_b|),
    // kappa(r) = r^-4): e-e pair terms of dE_L/dr_e, then per nucleus
    //   dE_L^sw/dR_a = dE_L/dR_a + sum_e omega_a(r_e) dE_L/dr_e,
    //   d ln Psi^sw/dR_a = d ln Psi/dR_a + sum_e [omega_a(r_e) d ln Psi/dr_e + 1/2 grad omega_a(r_e)].
    if (accum && P.swct_off > 0) {
      const T ge[3] = {gd[0] + jg[0], gd[1] + jg[1], gd[2] + jg[2]};
      for (int j = 0; j < Ne; ++j) {  // every lane takes part in the shuffles
        T gj[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) gj[k] = __shfl_sync(0xffffffffu, ge[k], j);
        if (!has_e || j == e) continue;
        T sv[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          if constexpr (sizeof(T) == 8) sv[k] = p[k] - pd[3 * j + k];
          else sv[k] = (hh[k] - ph[3 * j + k]) + (ll[k] - pl[3 * j + k]);
        }
        const T r = dsqrt<T>(sv[0] * sv[0] + sv[1] * sv[1] + sv[2] * sv[2]), ri = T(1) / r;
        const T ri3 = ri * ri * ri;
#pragma unroll
        for (int k = 0; k < 3; ++k) dr[k] -= sv[k] * ri3;
        if (S.J2) {
          const bool par = (j < nup) == (e < nup);
          const Rad3<T> u = pair_rad<T>(S, par, r);
          const T nn[3] = {sv[0] * ri, sv[1] * ri, sv[2] * ri};
          const T dl = u.h3 + T(2) * u.h2 * ri - T(2) * u.h1 * ri * ri;
          const T vec[3] = {ge[0] - gj[0], ge[1] - gj[1], ge[2] - gj[2]};
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            T hs = 0;
#pragma unroll
            for (int c = 0; c < 3; ++c)
              hs += (u.h2 * nn[k] * nn[c] + u.h1 * ri * ((k == c ? T(1) : T(0)) - nn[k] * nn[c])) * vec[c];
            dr[k] -= dl * nn[k] + hs;
          }
        }
      }
      T k0 = T(0), gk[3] = {T(0), T(0), T(0)};
      if (has_e)
        for (int I = 0; I < K; ++I) {
          T sv[3];
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            if constexpr (sizeof(T) == 8) sv[k] = p[k] - __ldg(S.R + 3 * I + k);
            else sv[k] = (hh[k] - __ldg(S.Rh + 3 * I + k)) + (ll[k] - __ldg(S.Rl + 3 * I + k));
          }
          const T r2 = sv[0] * sv[0] + sv[1] * sv[1] + sv[2] * sv[2], kap = T(1) / (r2 * r2);
          k0 += kap;
#pragma unroll
          for (int k = 0; k < 3; ++k) gk[k] += T(-4) * sv[k] * kap / r2;
        }
      const int so = P.swct_off;
      for (int a = 0; a < K; ++a) {
        T v6[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
        if (has_e) {
          T sv[3];
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            if constexpr (sizeof(T) == 8) sv[k] = p[k] - __ldg(S.R + 3 * a + k);
            else sv[k] = (hh[k] - __ldg(S.Rh + 3 * a + k)) + (ll[k] - __ldg(S.Rl + 3 * a + k));
          }
          const T r2 = sv[0] * sv[0] + sv[1] * sv[1] + sv[2] * sv[2];
          const T kap = T(1) / (r2 * r2), kinv = T(1) / k0, om = kap * kinv;
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            v6[k] = om * dr[k];
            v6[3 + k] = om * ge[k] + T(0.5) * (T(-4) * sv[k] * kap / r2 - om * gk[k]) * kinv;
          }
        }
        warp_sum_f<6>(v6);
        if (lane == 0)
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const double sE = (double)v6[k] + (double)frc[3 * K + 3 * a + k] + __ldg(S.dVnn + 3 * a + k);
            const double sL = (double)v6[3 + k] + (double)frc[3 * a + k];
            atomicAdd(&acc_s[so + 3 * a + k], (T)(wt * sE));
            atomicAdd(&acc_s[so + 3 * K + 3 * a + k], (T)(wt * sL));
            atomicAdd(&acc_s[so + 6 * K + 3 * a + k], (T)(wt * cw * sL));
          }
      }
    }
    // ---- outputs and walker sums
    for (int i = lane; i < 3 * K; i += 32) {
      const double dl = (double)frc[i];
      const double de = (double)frc[3 * K + i] + __ldg(S.dVnn + i);
      if (P.dlnpsi) P.dlnpsi[(size_t)w * 3 * K + i] = dl;
      if (P.dEL) P.dEL[(size_t)w * 3 * K + i] = de;
      if (accum) {
        atomicAdd(&acc_s[3 + i], (T)(wt * de));
        atomicAdd(&acc_s[3 + 3 * K + i], (T)(wt * dl));
        atomicAdd(&acc_s[3 + 6 * K + i], (T)(wt * cw * dl));
      }
    }
    if (lane == 0) {
      if (P.EL) P.EL[w] = EL;
      if (P.logpsi) P.logpsi[w] = *la + vpart[3];
      if (accum) {
        atomicAdd(&acc_s[0], (T)wt);
        atomicAdd(&acc_s[1], (T)(wt * cw));
        atomicAdd(&acc_s[2], (T)(wt * cw * cw));
      }
    }
    __syncwarp();
  }
  if (accum) {
    __syncthreads();
    double* slot = P.acc + (size_t)blockIdx.x * P.accL;
    const double cnt = (double)acc_s[0];
    for (int i = threadIdx.x; i < P.accL; i += blockDim.x) {
      double v = (double)acc_s[i];
      if (i == 2) v = v + 2.0 * P.e_ref * (double)acc_s[1] + cnt * P.e_ref * P.e_ref;
      if (i == 1) v = v + cnt * P.e_ref;
      slot[i] += v;
    }
  }
}

// Layout conversion between the ABI's [W][Ne][3] and the walker-interleaved [3 Ne][W].
static __global__ void to_interleaved(const double* __restrict__ src, double* __restrict__ dst, float2* __restrict__ dstf,
                               int W, int n3) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < (long long)W * n3;
       idx += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(idx / W), w = (int)(idx - (long long)k * W);
    const double v = src[(size_t)w * n3 + k];
    dst[idx] = v;
    if (dstf) {
      float h, l;
      split_ff(v, h, l);
      dstf[idx] = make_float2(h, l);
    }
  }
}
static __global__ void from_interleaved(const double* __restrict__ src, double* __restrict__ dst, int W, int n3) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < (long long)W * n3;
       idx += (long long)gridDim.x * blockDim.x) {
    const int w = (int)(idx / n3), k = (int)(idx - (long long)w * n3);
    dst[idx] = src[(size_t)k * W + w];
  }
}

template <typename T, int NM>
cudaError_t launch_move_small_lpw(int lpw, const DevSys& S, int W, size_t smem, const SmallMoveParams& P,
                                  cudaStream_t st) {
  const int threads = (P.wpc * lpw + 31) / 32 * 32;
  smem += (sizeof(T) * (size_t)S.nB + (sizeof(T) == 4 ? 8 : 8) * (size_t)(3 * S.Ne)) * P.wpc;
  const dim3 grid((unsigned)((W + P.wpc - 1) / P.wpc));
  if (P.eps > 0.0) {  // guided sampling: one lane-group width (the launch planned it with lpw = 2)
    if (lpw != 2) return cudaErrorInvalidValue;
    move_small<T, NM, 2, true><<<grid, threads, smem, st>>>(S, P);
    return cudaGetLastError();
  }
  switch (lpw) {
    case 1: move_small<T, NM, 1, false><<<grid, threads, smem, st>>>(S, P); break;
    case 2: move_small<T, NM, 2, false><<<grid, threads, smem, st>>>(S, P); break;
    case 4: move_small<T, NM, 4, false><<<grid, threads, smem, st>>>(S, P); break;
    default: move_small<T, NM, 8, false><<<grid, threads, smem, st>>>(S, P); break;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_move_small_impl(const DevSys& S, int nm, int lpw, int W, size_t smem, const SmallMoveParams& P,
                                   cudaStream_t st) {
  if (nm <= 8) return launch_move_small_lpw<T, 8>(lpw, S, W, smem, P, st);
  if (nm <= 14) return launch_move_small_lpw<T, 14>(lpw, S, W, smem, P, st);
  return launch_move_small_lpw<T, 16>(lpw, S, W, smem, P, st);
}

template <typename T>
cudaError_t launch_measure_small_impl(const DevSys& S, int nm, const SmallLayout& L, int grid, int warps,
                                      const SmallMeasParams& P, cudaStream_t st) {
  const size_t smem = (size_t)L.cta_bytes + (size_t)warps * L.bytes;
  if (nm <= 8)
    measure_small<T, 8><<<grid, 32 * warps, smem, st>>>(S, L, P);
  else if (nm <= 14)
    measure_small<T, 14><<<grid, 32 * warps, smem, st>>>(S, L, P);
  else
    measure_small<T, 16><<<grid, 32 * warps, smem, st>>>(S, L, P);
  return cudaGetLastError();
}

template <typename T>
cudaError_t set_smem_limits_small_impl() {
  const int lim = 227 * 1024;
  cudaError_t e;
#define VMCF_MOVE_ATTR(NM, L, G)                                                                                  \
  if ((e = cudaFuncSetAttribute(move_small<T, NM, L, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  VMCF_MOVE_ATTR(8, 1, false) VMCF_MOVE_ATTR(8, 2, false) VMCF_MOVE_ATTR(8, 4, false) VMCF_MOVE_ATTR(8, 8, false)
  VMCF_MOVE_ATTR(14, 1, false) VMCF_MOVE_ATTR(14, 2, false) VMCF_MOVE_ATTR(14, 4, false) VMCF_MOVE_ATTR(14, 8, false)
  VMCF_MOVE_ATTR(16, 1, false) VMCF_MOVE_ATTR(16, 2, false) VMCF_MOVE_ATTR(16, 4, false) VMCF_MOVE_ATTR(16, 8, false)
  VMCF_MOVE_ATTR(8, 2, true) VMCF_MOVE_ATTR(14, 2, true) VMCF_MOVE_ATTR(16, 2, true)
#undef VMCF_MOVE_ATTR
  if ((e = cudaFuncSetAttribute(measure_small<T, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(measure_small<T, 14>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(measure_small<T, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  return cudaSuccess;
}

}  // namespace vmcf
