// Small-system kernels (at most 32 electrons, 16 orbitals per spin): the VMC hot path of
// arXiv:2511.05222, App. A, laid out so that every lane does independent work.
//
//  propose_small  one warp per walker, one lane per electron: everything of a sweep's moves that
//                 depends only on the electron's own start-of-sweep position and its proposal
//                 (the Philox draws, the orbital row at the proposal, the electron-nucleus Jastrow
//                 change), for all electrons at once
//  move_small     LPW lanes per walker (1, 2, 4 or 8): the sequential part of a run of
//                 single-electron Metropolis moves (determinant ratio, electron-electron Jastrow
//                 change, acceptance, Sherman-Morrison update) with the CTA's inverses and
//                 positions staged walker-interleaved in shared memory (read from and written back
//                 to walker-interleaved global memory once per launch)
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
#include "kernels_small_jb.cuh"

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

// Displacement of the electron from nucleus c (double in FP64 mode; float from the float-float
// positions in mixed mode) and, in mixed mode when ff is set, the squared distance as a float-float
// pair (for the shells of a group with sharp primitives).
template <typename T>
__device__ __forceinline__ void centre_disp(const DevSys& S, int c, const double p[3], const float ph[3],
                                            const float pl[3], bool ff, T d[3], R2FF& r2ff) {
  if constexpr (sizeof(T) == 8) {
#pragma unroll
    for (int k = 0; k < 3; ++k) d[k] = p[k] - __ldg(S.R + 3 * c + k);
  } else if (!ff) {
#pragma unroll
    for (int k = 0; k < 3; ++k) d[k] = (ph[k] - __ldg(S.Rh + 3 * c + k)) + (pl[k] - __ldg(S.Rl + 3 * c + k));
  } else {
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
  }
}

// Runs f(std::integral_constant<int, l>, group, d, r2ff) for every shell group, with the displacement
// from the group's centre taken once per group and the angular momentum a compile-time constant.
template <typename T, typename F>
__device__ __forceinline__ void for_each_group(const DevSys& S, const double p[3], const float ph[3], const float pl[3],
                                               F&& f) {
  for (int gi = 0; gi < S.ngrp; ++gi) {
    const int4 gr = __ldg(S.shgrp + gi);
    T d[3];
    R2FF r2ff{0.f, 0.f};
    centre_disp<T>(S, gr.w, p, ph, pl, (gr.z & 256) != 0, d, r2ff);
    const int l = gr.z & 255;
    if (l == 0) f(std::integral_constant<int, 0>{}, gr, d, r2ff);
    else if (l == 1) f(std::integral_constant<int, 1>{}, gr, d, r2ff);
    else f(std::integral_constant<int, 2>{}, gr, d, r2ff);
  }
}

__device__ __forceinline__ void split_ff(double v, float& h, float& l) { split_ff_bits(v, h, l); }

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
  if (!S.j2exp) return pade_at<T>(jas_a<T>(S, par), jas_F<T>(S, par), d);
  const T r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  return expo_value<T>(jas_a<T>(S, par), jas_F<T>(S, par), dsqrt<T>(r2));
}

// A staged coefficient row (16-byte aligned, padded to a multiple of 4 entries) into registers with
// 16-byte shared-memory loads.
template <typename T, int NM>
__device__ __forceinline__ void crow_load(const T* __restrict__ crow, T (&c)[NM]) {
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int i = 0; i < NM; i += 4) {
      const float4 v = *reinterpret_cast<const float4*>(crow + i);
      c[i] = v.x;
      if (i + 1 < NM) c[i + 1] = v.y;
      if (i + 2 < NM) c[i + 2] = v.z;
      if (i + 3 < NM) c[i + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < NM; i += 2) {
      const double2 v = *reinterpret_cast<const double2*>(crow + i);
      c[i] = v.x;
      if (i + 1 < NM) c[i + 1] = v.y;
    }
  }
}

template <typename T, int NM>
__device__ __forceinline__ void axpy_row(T (&acc)[NM], T a, const T* __restrict__ crow) {
  T c[NM];
  crow_load<T, NM>(crow, c);
#pragma unroll
  for (int i = 0; i < NM; ++i) acc[i] += a * c[i];
}

// Two rows updated from one coefficient row: acc0 += a0 c, acc1 += a1 c.
template <typename T, int NM>
__device__ __forceinline__ void axpy2_row(T (&acc0)[NM], T a0, T (&acc1)[NM], T a1, const T* __restrict__ crow) {
  T c[NM];
  crow_load<T, NM>(crow, c);
#pragma unroll
  for (int i = 0; i < NM; ++i) {
    acc0[i] += a0 * c[i];
    acc1[i] += a1 * c[i];
  }
}

// Two dot products with one coefficient row: (x0 . c, x1 . c).
template <typename T, int NM>
__device__ __forceinline__ void dot2_row(const T (&x0)[NM], const T (&x1)[NM], const T* __restrict__ crow, T& d0,
                                         T& d1) {
  T c[NM];
  crow_load<T, NM>(crow, c);
  T s0 = 0, s1 = 0, t0 = 0, t1 = 0;
#pragma unroll
  for (int i = 0; i < NM; i += 2) {
    s0 += x0[i] * c[i];
    t0 += x1[i] * c[i];
    if (i + 1 < NM) {
      s1 += x0[i + 1] * c[i + 1];
      t1 += x1[i + 1] * c[i + 1];
    }
  }
  d0 = s0 + s1;
  d1 = t0 + t1;
}

template <typename T, int NM>
__device__ __forceinline__ T dot_row(const T (&x)[NM], const T* __restrict__ crow) {
  T c[NM];
  crow_load<T, NM>(crow, c);
  T s0 = 0, s1 = 0;  // two chains for instruction-level parallelism
#pragma unroll
  for (int i = 0; i < NM; i += 2) {
    s0 += x[i] * c[i];
    if (i + 1 < NM) s1 += x[i + 1] * c[i + 1];
  }
  return s0 + s1;
}

// Row stride of the staged coefficients for register rows of NM orbitals: a multiple of 4, so that
// every row starts on 16 bytes.
template <int NM>
__host__ __device__ constexpr int c_stride() { return (NM + 3) / 4 * 4; }

// A row of c_stride<NM>() values (16-byte aligned) into NM registers with vector loads.
template <typename T, int NM>
__device__ __forceinline__ void load_row(const T* __restrict__ src, T (&row)[NM]) {
  constexpr int NMS = c_stride<NM>();
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int i = 0; i < NMS; i += 4) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(src + i));
      const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (i + k < NM) row[i + k] = vv[k];
    }
  } else {
#pragma unroll
    for (int i = 0; i < NMS; i += 2) {
      const double2 v = __ldg(reinterpret_cast<const double2*>(src + i));
      if (i < NM) row[i] = v.x;
      if (i + 1 < NM) row[i + 1] = v.y;
    }
  }
}

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


// ---------------------------------------------------------------- sweep schedule in a batch graph
// The moves of one sweep, in the order vmcf_sample issues them: runs of at most k moves separated by
// the FP64 re-inversion every k attempted moves (none after the sweep's last move when the sweep is
// measured, because the measurement re-inverts). c0 = moves since the last re-inversion at the start
// of the sweep (< k). Segment s: its first move (start) and count (0 if the sweep has fewer segments),
// and whether a re-inversion follows it.
__device__ __forceinline__ void sweep_segment(int c0, int Ne, int kref, int measure, int s, int& start, int& count,
                                              bool& refresh_after) {
  int done = 0, c = c0;
  start = 0;
  count = 0;
  refresh_after = false;
  for (int k = 0; k <= s && done < Ne; ++k) {
    const int chunk = min(Ne - done, kref - c);
    done += chunk;
    c += chunk;
    bool ref = false;
    if (c >= kref) {
      ref = !(measure && done == Ne);
      c = 0;
    }
    if (k == s) {
      start = done - chunk;
      count = chunk;
      refresh_after = ref;
    }
  }
}

// ---------------------------------------------------------------- proposals of one sweep
// In sweep s electron e of walker w is proposed r'_e = r_e + sigma xi, xi from the Philox counter
// (wid, s, e, 0), and accepted against the uniform of counter (wid, s, e, 1) (App. A, MCMC). Every
// electron moves once per sweep, so r_e is its position at the start of the sweep, and whatever
// depends only on r_e and r'_e is the same however the sweep's earlier moves went: the draws, the
// orbital row phi^s(r'_e) = sum_mu psi_mu(r'_e) C^s_mu of the electron's spin, and the change of the
// electron-nucleus Jastrow terms. With AO-expanded Jastrow terms (JB) also their change, which depends on
// the earlier moves only through which of them were accepted: the part that does not (added to the
// electron-nucleus change) and a pair term for each accepted earlier electron. This kernel computes them
// for every electron of every walker at once (one warp per walker, one lane per electron); the move kernel
// keeps only what depends on the order of the moves.
template <typename T, int NM, bool JB>
__global__ void __launch_bounds__(256) propose_small(DevSys S, SmallProposeParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  T* Cs = reinterpret_cast<T*>(smem);  // C^up, C^dn [2][M][c_stride<NM>()]
  stage_C<T, NM>(S, Cs);
  __syncthreads();
  constexpr int NMS = c_stride<NM>();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int Ne = S.Ne, W = P.W, e = lane;
  if (!JB && e >= Ne) return;  // no warp-wide operation follows
  const bool has_e = e < Ne;
  // with the Jastrow-basis terms: Xi's rows [MJ][MJp] staged once, then this warp's rows dphi [Ne][JS] and
  // vectors s and t0 [2][MJp]
  const int JS = P.jJS;
  T* jXs = reinterpret_cast<T*>(smem + propose_c_bytes(S.M, NMS, sizeof(T)));
  T* jD = reinterpret_cast<T*>(reinterpret_cast<unsigned char*>(jXs) + propose_xi_bytes(S.MJ, sizeof(T)) +
                               warp * propose_jb_bytes(Ne, S.MJ, JS, sizeof(T)));
  if constexpr (JB) {
    const T* Xr = jas_Xr<T>(S);
    for (int i = threadIdx.x; i < S.MJ * S.MJp; i += blockDim.x) jXs[i] = __ldg(Xr + i);
    __syncthreads();
  }
  const int sg = e < S.nup ? 0 : 1;
  const T* Csg = Cs + sg * S.M * NMS;
  for (long long w = (long long)blockIdx.x * nwarps + warp; w < W; w += (long long)gridDim.x * nwarps) {
   EPos epo{}, epn{};  // start-of-sweep position and proposal (Jastrow-basis terms)
   T dchi = T(0);
   size_t pe = 0;
   if (has_e) {
    const uint64_t wid = P.wid0 + (uint64_t)w, sweep = P.clk ? P.clk->sweep : P.sweep;
    uint64_t r[4] = {wid, sweep, (uint64_t)e, 0};
    philox4x64_10(r, P.k0, P.k1);
    uint64_t r2[4] = {wid, sweep, (uint64_t)e, 1};
    philox4x64_10(r2, P.k0, P.k1);
    // r'_e = r_e + sigma xi: in double in FP64 mode; in mixed mode a float-float sum of the float-float
    // position and a float step, so that no FP64 instruction is needed
    double po[3] = {0.0, 0.0, 0.0}, rn[3] = {0.0, 0.0, 0.0};
    float nh[3], nl[3], oh[3], ol[3];
    if constexpr (sizeof(T) == 8) {
      double xi[3];
      normals3(r, xi, 0.0);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        po[k] = P.pos[(size_t)(3 * e + k) * W + w];
        rn[k] = po[k] + P.sigma * xi[k];
      }
    } else {
      float xi[3];
      normals3_f(r, xi);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float2 f = P.posf[(size_t)(3 * e + k) * W + w];
        oh[k] = f.x;
        ol[k] = f.y;
        float sh, se;
        two_sum(oh[k], P.sigma_f * xi[k], sh, se);
        fast_two_sum(sh, se + ol[k], nh[k], nl[k]);
      }
    }
    T row[NM];
#pragma unroll
    for (int i = 0; i < NM; ++i) row[i] = T(0);
    // the row at r'_e; a move's row takes no float-float a r^2 for sharp primitives (its error enters only
    // the acceptance ratio, and the measurement rebuilds every row)
    for_each_group<T>(S, rn, nh, nl, [&](auto Lc, const int4 gr, const T (&d)[3], const R2FF) {
      constexpr int LA = decltype(Lc)::value;
      const T r2s = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      for (int s = gr.x; s < gr.x + gr.y; ++s) {
        const int4 sh = __ldg(S.shell + s);
        const Radial<T> rs = radial_sums<T, 0>(S, s, LA, sh.z, r2s, 0, R2FF{0.f, 0.f});
#pragma unroll
        for (int m = 0; m < 2 * LA + 1; ++m) {
          T Pa, g[3], h[6];
          angular<T>(LA, m, d[0], d[1], d[2], Pa, g, h);
          axpy_row<T, NM>(row, Pa * rs.R0, Csg + (sh.w + m) * NMS);
        }
      }
    });
    if (S.J1) {
      for (int I = 0; I < S.K; ++I) {
        const T mz = -nuc_Z<T>(S, I), b = jas_b<T>(S);
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
        dchi += pade_at<T>(mz, b, d1) - pade_at<T>(mz, b, d0);
      }
    }
    pe = (size_t)w * Ne + e;
    T* rw = reinterpret_cast<T*>(P.pr.rows) + pe * NMS;
#pragma unroll
    for (int i = 0; i < NMS; ++i) rw[i] = i < NM ? row[i] : T(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if constexpr (sizeof(T) == 8) P.pr.rnew[pe * 3 + k] = rn[k];
      else reinterpret_cast<float2*>(P.pr.rnew)[pe * 3 + k] = make_float2(nh[k], nl[k]);
    }
    P.pr.u[pe] = u01_bits(r2[0]);
    if constexpr (JB) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        epo.d[k] = po[k];
        epn.d[k] = rn[k];
        if constexpr (sizeof(T) == 4) {
          epo.h[k] = oh[k];
          epo.l[k] = ol[k];
          epn.h[k] = nh[k];
          epn.l[k] = nl[k];
        }
      }
    }
   }
    if constexpr (JB) {
      T* js = jD + Ne * JS;
      jb_propose_small<T>(S, JS, jXs, jD, js, js + S.MJp, lane, has_e, epo, epn, P.pr.npair,
                          reinterpret_cast<T*>(P.pr.dpair) + (size_t)w * P.pr.npair, dchi);
    }
    if (has_e) reinterpret_cast<T*>(P.pr.dchi)[pe] = dchi;
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
  // shared memory: the CTA's inverses walker-interleaved [nB][WPC]; its positions [3 Ne][WPC]
  // (float-float pairs in mixed mode, double in FP64 mode)
  const int WPC = P.wpc;
  uint64_t move0 = P.move0;
  int nmoves = P.nmoves;
  if (P.clk) {  // batch graph: this launch's segment of the sweep (uniform over the grid)
    int start, count;
    bool ref;
    sweep_segment(P.clk->c, S.Ne, P.kref, P.measure, P.seg, start, count, ref);
    if (count == 0) return;
    move0 = P.clk->sweep * (uint64_t)S.Ne + (uint64_t)start;
    nmoves = count;
  }
  T* Bs = reinterpret_cast<T*>(smem);
  using PosT = typename std::conditional<sizeof(T) == 4, float2, double>::type;
  PosT* Ps = reinterpret_cast<PosT*>(smem + (sizeof(T) * (size_t)S.nB * WPC + 7) / 8 * 8);  // move_small_smem
  const int W = P.W, Ne = S.Ne, nup = S.nup, nB = S.nB;
  const int wbase = blockIdx.x * WPC;
  T* Bg = reinterpret_cast<T*>(P.B);
  for (int idx = threadIdx.x; idx < nB * WPC; idx += blockDim.x) {
    const int k = idx / WPC, ws = idx - k * WPC;
    if (wbase + ws < W) Bs[idx] = Bg[(size_t)k * W + wbase + ws];
  }
  for (int idx = threadIdx.x; idx < 3 * Ne * WPC; idx += blockDim.x) {
    const int k = idx / WPC, ws = idx - k * WPC;
    if (wbase + ws < W) {
      if constexpr (sizeof(T) == 4) Ps[idx] = P.posf[(size_t)k * W + wbase + ws];
      else Ps[idx] = P.pos[(size_t)k * W + wbase + ws];
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
  uint32_t nacc = 0, nrej = 0;
  // reweighted sampling of |Psi_G|^2, Psi_G = Psi max(1, eps sqrt(S)): S of the current inverses
  constexpr bool guide = GUIDE;  // P.eps > 0
  double Sg = 0.0;
  if (guide) {
    for (int k = q; k < nB; k += LPW) Sg += (double)B[k * WPC] * (double)B[k * WPC];
    Sg = lane_group_sum<LPW>(Sg, mask);
  }
  // a launch never crosses a sweep: its moves are electrons e0, e0 + 1, ... of one sweep
  const int e0 = (int)(move0 % (uint64_t)Ne);
  // AO-expanded Jastrow pair terms: which of the sweep's earlier moves were accepted (a run after a
  // re-inversion continues the sweep's mask)
  const bool jbp = P.pr.npair > 0;
  uint32_t am = (jbp && e0 > 0) ? P.pr.amask[w] : 0u;
  // this sweep's proposals, one move ahead: the loads of move mv + 1 are in flight while move mv runs
  T rowc[NM], rown[NM];
  double rnc[3], rnn[3], uc = 0.0, un = 0.0;
  T dcc = T(0), dcn = T(0);
  auto fetch = [&](int mv) {
    const size_t pe = (size_t)w * Ne + e0 + mv;
    load_row<T, NM>(reinterpret_cast<const T*>(P.pr.rows) + pe * c_stride<NM>(), rown);
#pragma unroll
    for (int k = 0; k < 3; ++k) rnn[k] = __ldg(P.pr.rnew + pe * 3 + k);
    un = __ldg(P.pr.u + pe);
    dcn = __ldg(reinterpret_cast<const T*>(P.pr.dchi) + pe);
  };
  if (nmoves > 0) fetch(0);
  for (int mv = 0; mv < nmoves; ++mv) {
    const int e = e0 + mv;
    const int sg = e < nup ? 0 : 1;
    const int n = sg == 0 ? nup : S.ndn, el = e - (sg == 0 ? 0 : nup);
    const int off = sg == 0 ? 0 : nup * nup;
#pragma unroll
    for (int i = 0; i < NM; ++i) rowc[i] = rown[i];
#pragma unroll
    for (int k = 0; k < 3; ++k) rnc[k] = rnn[k];
    uc = un;
    dcc = dcn;
    if (mv + 1 < nmoves) fetch(mv + 1);
    const T (&row)[NM] = rowc;
    double po[3] = {0.0, 0.0, 0.0}, rn[3] = {0.0, 0.0, 0.0};
    float nh[3], nl[3], oh[3], ol[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if constexpr (sizeof(T) == 8) {
        po[k] = P.pos[(size_t)(3 * e + k) * W + w];
        rn[k] = rnc[k];
      } else {  // r'_e as a float-float pair in the proposal's bytes; r_e from shared memory
        nh[k] = __int_as_float(__double2loint(rnc[k]));
        nl[k] = __int_as_float(__double2hiint(rnc[k]));
        const float2 f = pp[(3 * e + k) * WPC];
        oh[k] = f.x;
        ol[k] = f.y;
      }
    }
    // determinant ratio (FP64): this lane's orbitals i = q, q + LPW, ...; the lane's row entry is picked
    // by selects so that each FP64 FMA is issued once per LPW orbitals (the FP64 pipe charges a whole
    // warp instruction whatever the number of active lanes)
    double R = 0.0;
#pragma unroll
    for (int ii = 0; ii < (NM + LPW - 1) / LPW; ++ii) {
      T rv = row[ii * LPW];
#pragma unroll
      for (int k = 1; k < LPW; ++k)
        if (ii * LPW + k < NM && q == k) rv = row[ii * LPW + k];
      const int i = ii * LPW + q;
      if (i < n) {
        if constexpr (sizeof(T) == 8) R += rv * B[(off + i * n + el) * WPC];
        else R += f2d_bits(rv) * f2d_bits(B[(off + i * n + el) * WPC]);
      }
    }
    R = lane_group_sum<LPW>(R, mask);
    // electron-electron Jastrow ratio: this lane's partners j = q, q + LPW, ... at their current
    // positions; the electron-nucleus change came with the proposal
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
    if (jbp) {  // the Jastrow-basis pair terms of the accepted earlier electrons j = q, q + LPW, ... < e
      const T* dpe = reinterpret_cast<const T*>(P.pr.dpair) + (size_t)w * P.pr.npair + e * (e - 1) / 2;
      for (int j = q; j < e; j += LPW)
        if ((am >> j) & 1u) jacc += __ldg(dpe + j);
    }
    const double u = uc;
    // |R exp(dJ)|^2 with R in FP64; in mixed mode the Jastrow factor is formed in float
    double pr;
    if constexpr (sizeof(T) == 8) {
      const double dJ = lane_group_sum<LPW>(jacc, mask) + dcc;
      pr = R * R * exp(2.0 * dJ);
    } else {
      const float dJ = lane_group_sum<LPW>(jacc, mask) + dcc;
      pr = R * R * f2d_bits(expf(2.0f * dJ));
    }
    // Sherman-Morrison: w_j = sum_i row_i B_ij - delta_j,el; B_kj <- B_kj - B_k,el w_j / R.
    // This lane owns columns j = q, q + LPW, ...; every lane reads the whole column el first.
    // This lane owns columns j = jj LPW + q; its vector entries sit at wv[jj] (compile-time index).
    constexpr int NJ = (NM + LPW - 1) / LPW;
    T wv[NJ], col[NM];
    auto sm_vectors = [&]() {
#pragma unroll
      for (int j = 0; j < NM; ++j) col[j] = (j < n) ? B[(off + j * n + el) * WPC] : T(0);
#pragma unroll
      for (int jj = 0; jj < NJ; ++jj) wv[jj] = T(0);
#pragma unroll
      for (int i = 0; i < NM; ++i) {
        if (i >= n) continue;
        const T ri = row[i];
#pragma unroll
        for (int jj = 0; jj < NJ; ++jj) {
          const int j = jj * LPW + q;
          if (j < n) wv[jj] += ri * B[(off + i * n + j) * WPC];
        }
      }
    };
    double Sn = Sg;
    if constexpr (guide) if (R != 0.0) {
      // S after the update B' = B - c w^T / R (c = column el): S - (2/R) w.(B^T c) + |c|^2 |w|^2 / R^2
      sm_vectors();
      double tw = 0.0, ww = 0.0, cc = 0.0;
#pragma unroll
      for (int j = 0; j < NM; ++j)
        if (j < n) cc += (double)col[j] * (double)col[j];
#pragma unroll
      for (int jj = 0; jj < NJ; ++jj) {
        const int j = jj * LPW + q;
        if (j >= n) continue;
        T tj = 0;
#pragma unroll
        for (int i = 0; i < NM; ++i)
          if (i < n) tj += col[i] * B[(off + i * n + j) * WPC];
        const double wj = (double)((j == el) ? wv[jj] - T(1) : wv[jj]);
        tw += wj * (double)tj;
        ww += wj * wj;
      }
      tw = lane_group_sum<LPW>(tw, mask);
      ww = lane_group_sum<LPW>(ww, mask);
      Sn = Sg - 2.0 * tw / R + cc * ww / (R * R);
      const double g0 = fmax(1.0, P.eps * sqrt(Sg)), g1 = fmax(1.0, P.eps * sqrt(fmax(Sn, 0.0)));
      pr *= (g1 / g0) * (g1 / g0);
    }
    // finite and non-zero, tested on the bits (no FP64 compare)
    const bool ok = ((__double2hiint(pr) >> 20) & 0x7ff) != 0x7ff && (__double_as_longlong(R) << 1) != 0;
    if (!ok) ++nrej;
    if (ok && u < pr) {
      if constexpr (!guide) sm_vectors();
      Sg = Sn;
      if (LPW > 1) __syncwarp(mask);  // column el is read by all lanes before its owner rewrites it
      T rinv;
      if constexpr (sizeof(T) == 8) rinv = 1.0 / R;
      else rinv = __frcp_rn(d2f_trunc(R));  // the update itself is FP32
#pragma unroll
      for (int jj = 0; jj < NJ; ++jj) {
        const int j = jj * LPW + q;
        if (j >= n) continue;
        const T wj = (j == el) ? wv[jj] - T(1) : wv[jj];
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
          if constexpr (sizeof(T) == 4) {
            pp[(3 * e + k) * WPC] = make_float2(nh[k], nl[k]);
            P.pos[(size_t)(3 * e + k) * W + w] = f2d_bits(nh[k]) + f2d_bits(nl[k]);  // exact
          } else {
            pp[(3 * e + k) * WPC] = rn[k];
            P.pos[(size_t)(3 * e + k) * W + w] = rn[k];
          }
        }
      }
      ++nacc;
      am |= 1u << e;
    }
    if (LPW > 1) __syncwarp(mask);  // the new position is visible to the group's next move
  }
  if (q == 0) {
    P.nacc[w] += nacc;
    P.nrej[w] += nrej;
    if (jbp) P.pr.amask[w] = am;
  }
  // this walker's inverses (and, in mixed mode, float-float positions) back to global memory (its lanes
  // share the copy)
  if (LPW > 1) __syncwarp(mask);
  for (int k = q; k < nB; k += LPW) Bg[(size_t)k * W + w] = B[k * WPC];
  if constexpr (sizeof(T) == 4)
    for (int k = q; k < 3 * Ne; k += LPW) P.posf[(size_t)k * W + w] = pp[k * WPC];
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
      const long long pb = __double_as_longlong(p);  // zero or not finite: tested on the bits
      if ((pb << 1) == 0 || ((pb >> 52) & 0x7ff) == 0x7ff) *flag = 1;
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

template <typename T, int NM, bool JB>
__global__ void __launch_bounds__(256, 2) measure_small(DevSys S, SmallLayout L, SmallMeasParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  T* Cs = reinterpret_cast<T*>(smem + L.cta_C);
  T* acc_s = reinterpret_cast<T*>(smem + L.cta_acc);
  // mixed-mode walker sums of O through the tensor-core kernel: the kernel emits PhiT and YT tiles, and the
  // CTA's accumulator leaves out the O range [3 + 9K, 3 + 9K + 2 nO) of the slot (which stays zero): accumulator
  // entry k is slot entry k < oskip ? k : k + olen
  const bool tc = P.mode == 2 && sizeof(T) == 4 && P.phiT[0] != nullptr;
  const int olen = tc ? 2 * S.M * S.Ne : 0, oskip = 3 + 9 * S.K, accn = P.accL - olen;
  unsigned char* base = smem + (tc ? L.cta_bytes_tc : L.cta_bytes) + warp * L.bytes;
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
  if (P.mode == 0 && P.clk) {  // batch graph: re-invert only where the sweep's schedule has a re-inversion
    int start, count;
    bool ref;
    sweep_segment(P.clk->c, S.Ne, P.kref, P.measure, P.seg, start, count, ref);
    if (!ref) return;  // uniform over the grid
  }
  stage_C<T, NM>(S, Cs);
  if (accum)
    for (int k = threadIdx.x; k < accn; k += blockDim.x) acc_s[k] = T(0);
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
    // ---- Jastrow and potentials (lane = electron). E_L takes the 1/r parts of -1/2 lap J per pair and per
    // nucleus together with the Coulomb terms they cancel at coalescence (the cusps), in forms without
    // that cancellation. With q = 1/(1 + F r): a nucleus of charge Z with chi = -Z r q gives
    //   -1/2 (2 chi'/r) - Z/r = -Z (1 - q^2)/r = -Z F q (q + 1);
    // a pair with u = a r q gives, per electron (half the pair's 1/r),
    //   -1/2 (2 u'/r) + 1/(2 r) = (1/2 - a)/r + a F q (q + 1)
    // (exponential form u = (a/F)(1 - exp(-F r)): (1/2 - a)/r - a expm1(-F r)/r). The remaining Jastrow
    // Laplacian terms u'', chi'' go to jl.
    T jg[3] = {T(0), T(0), T(0)}, jl = T(0);
    T vee = 0, ven = 0, jv = 0, te = 0;  // pair and nucleus terms as above, J, and the kinetic term of this electron
    if (full && has_e) {
      for (int j = 0; j < Ne; ++j) {
        if (j == e) continue;
        T d[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          if constexpr (sizeof(T) == 8) d[k] = p[k] - pd[3 * j + k];
          else d[k] = (hh[k] - ph[3 * j + k]) + (ll[k] - pl[3 * j + k]);
        }
        T r, ri;
        dist_inv<T>(d[0] * d[0] + d[1] * d[1] + d[2] * d[2], r, ri);
        if (S.J2) {
          const bool par = (j < nup) == (e < nup);
          const T a = jas_a<T>(S, par), F = jas_F<T>(S, par);
          T h, h1, h2, reg;
          if (!S.j2exp) {
            const T q = fast_rcp<T>(T(1) + F * r), q2 = q * q;
            h = a * r * q;
            h1 = a * q2;
            h2 = T(-2) * a * F * q2 * q;
            reg = a * F * q * (q + T(1));
          } else {
            const T ex = dexp<T>(-F * r), em1 = dexpm1<T>(-F * r);
            h = -(a / F) * em1;
            h1 = a * ex;
            h2 = -a * F * ex;
            reg = -a * em1 * ri;
          }
          const T gr = h1 * ri;
#pragma unroll
          for (int k = 0; k < 3; ++k) jg[k] += gr * d[k];
          jl += h2;
          vee += (T(0.5) - a) * ri + reg;
          if (j > e) jv += h;
        } else {
          vee += T(0.5) * ri;
        }
      }
      for (int I = 0; I < K; ++I) {
        T d[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          if constexpr (sizeof(T) == 8) d[k] = p[k] - __ldg(S.R + 3 * I + k);
          else d[k] = (hh[k] - __ldg(S.Rh + 3 * I + k)) + (ll[k] - __ldg(S.Rl + 3 * I + k));
        }
        T r, ri;
        dist_inv<T>(d[0] * d[0] + d[1] * d[1] + d[2] * d[2], r, ri);
        const T Z = nuc_Z<T>(S, I);
        if (S.J1) {
          const T b = jas_b<T>(S), q = fast_rcp<T>(T(1) + b * r), q2 = q * q;
          const T gr = -Z * q2 * ri;  // chi'/r
#pragma unroll
          for (int k = 0; k < 3; ++k) jg[k] += gr * d[k];
          jl += T(2) * Z * b * q2 * q;  // chi''
          ven -= Z * b * q * (q + T(1));
          jv -= Z * r * q;
        } else {
          ven -= Z * ri;
        }
      }
    }

    // ---- AO-expanded Jastrow terms (JB): their shares of grad J, lap J and J; t0 stays in the vector region
    EPos jep{};
    if constexpr (JB) {
      jep = make_epos(p);
      if (full) {
        T* jv0 = reinterpret_cast<T*>(base + L.jv);
        jb_eval_small<T>(S, L.JS, reinterpret_cast<T*>(base + L.jA), jv0, jv0 + S.MJp, lane, has_e, jep, jg, jl, jv);
        __syncwarp();  // the rows are in the work space of the passes below
      }
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
        for_each_group<T>(S, p, hh, ll, [&](auto Lc, const int4 gr, const T (&d)[3], const R2FF r2ff) {
          constexpr int LA = decltype(Lc)::value;
          const T r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
          for (int s = gr.x; s < gr.x + gr.y; ++s) {
            const int4 sh = __ldg(S.shell + s);
            const int smask = sizeof(T) == 4 ? __ldg(S.sharp + s) : 0;
            const Radial<T> rs = radial_sums<T, 0>(S, s, LA, sh.z, r2, smask, r2ff);
#pragma unroll
            for (int m = 0; m < 2 * LA + 1; ++m) {
              T Pa, g[3], h[6];
              angular<T>(LA, m, d[0], d[1], d[2], Pa, g, h);
              axpy_row<T, NM>(row, Pa * rs.R0, Csg + (sh.w + m) * c_stride<NM>());
            }
          }
        });
      } else {
        T prow[NM];
#pragma unroll
        for (int i = 0; i < NM; ++i) prow[i] = T(0);
        for_each_group<T>(S, p, hh, ll, [&](auto Lc, const int4 gr, const T (&d)[3], const R2FF r2ff) {
          constexpr int LA = decltype(Lc)::value;
          const T r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
          const T xj2 = T(2) * (d[0] * jg[0] + d[1] * jg[1] + d[2] * jg[2]);
          for (int s = gr.x; s < gr.x + gr.y; ++s) {
            const int4 sh = __ldg(S.shell + s);
            const int smask = sizeof(T) == 4 ? __ldg(S.sharp + s) : 0;
            const Radial<T> rs = radial_sums<T, 1>(S, s, LA, sh.z, r2, smask, r2ff);
            const T xjR1 = xj2 * rs.R1;
#pragma unroll
            for (int m = 0; m < 2 * LA + 1; ++m) {
              T Pa, g[3], h[6];
              angular<T>(LA, m, d[0], d[1], d[2], Pa, g, h);
              // lap psi = P LF; grad psi = g R0 + P d R1
              const T gj2 = T(2) * (g[0] * jg[0] + g[1] * jg[1] + g[2] * jg[2]);
              axpy2_row<T, NM>(row, Pa * rs.R0, prow, Pa * (rs.LF + xjR1) + gj2 * rs.R0,
                               Csg + (sh.w + m) * c_stride<NM>());
            }
          }
        });
#pragma unroll
        for (int i = 0; i < NM; ++i)
          if (i < n) Pm[off + el * n + i] = prow[i];
      }
#pragma unroll
      for (int i = 0; i < NM; ++i)
        if (i < n) {
          if constexpr (sizeof(T) == 8) Ad[off + el * n + i] = row[i];
          else Ad[off + el * n + i] = f2d_bits(row[i]);  // exact, no FP64 conversion instruction
        }
    }
    __syncwarp();
    gj_inverse_pair(Ad, nup, Ad + nup * nup, ndn, S.nmax, piv, f, flag, la, sgn, P.logpsi != nullptr);
    if (static_cast<void*>(Bf) != static_cast<void*>(Ad))
      for (int i = lane; i < S.nB; i += 32) Bf[i] = to_T<T>(Ad[i]);
    __syncwarp();
    if (P.Bout && P.mode != 1) {
      T* Bg = reinterpret_cast<T*>(P.Bout);
      for (int i = lane; i < S.nB; i += 32) Bg[(size_t)i * W + w] = Bf[i];
    }
    if (lane == 0 && *flag) atomicAdd(&P.counters[0], 1ull);
    if (lane == 0 && P.mode == 0) atomicAdd(&P.counters[1], 1ull);  // a re-inversion between moves
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
      te = ps + jl + (jg[0] * jg[0] + jg[1] * jg[1] + jg[2] * jg[2]);
    }
    // E_L = sum over electrons of -te/2 + V_ee + V_en, plus V_nn: summed in FP64 (in mixed mode as
    // float-float pairs, about 44 bits, on the FP32 pipe)
    double EL;
    if constexpr (sizeof(T) == 8) {
      EL = warp_sum(-0.5 * te + vee + ven) + S.Vnn;
    } else {
      float h, l;
      two_sum(-0.5f * te, vee, h, l);
      ff_add(h, l, ven, 0.0f, h, l);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(0xffffffffu, h, o), l2 = __shfl_xor_sync(0xffffffffu, l, o);
        ff_add(h, l, h2, l2, h, l);
      }
      EL = (f2d_bits(h) + f2d_bits(l)) + S.Vnn;
    }
    const double jsum = P.logpsi ? warp_sum((double)jv) : 0.0;  // ln|Psi| wanted (evaluation only)
    const double cw = EL - P.e_ref;
    // the weights of this walker's sums in the working precision
    const T wtT = to_T<T>(wt), wcwT = to_T<T>(wt * cw), wcw2T = to_T<T>(wt * cw * cw);
    if (P.mode == 1 && !P.dlnpsi && !P.dEL && !P.O) {  // E_L and ln|Psi| only: no adjoint pass
      if (lane == 0) {
        if (P.EL) P.EL[w] = EL;
        if (P.logpsi) P.logpsi[w] = *la + jsum;
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
            atomicAdd(&acc_s[3 + 9 * K + ooff + mu * ng + i], wtT * s);
            atomicAdd(&acc_s[3 + 9 * K + nO + ooff + mu * ng + i], wcwT * s);
          }
        }
      }
      __syncwarp();
      chunk0 += chunk_n;
      chunk_n = 0;
    };
    for_each_group<T>(S, p, hh, ll, [&](auto Lc, const int4 gr, const T (&d)[3], const R2FF r2ff) {
      constexpr int LA = decltype(Lc)::value, ncomp = 2 * LA + 1;
      if (gr.w != cur) {
        if (cur >= 0) flush_centre(cur);
        cur = gr.w;
      }
      const T r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      const T xj = d[0] * jg[0] + d[1] * jg[1] + d[2] * jg[2];
      for (int s = gr.x; s < gr.x + gr.y; ++s) {
        const int4 sh = __ldg(S.shell + s);
        if (chunk_n + ncomp > L.chunk) flush_chunk();
        if (has_e) {
          const int smask = sizeof(T) == 4 ? __ldg(S.sharp + s) : 0;
          const Radial<T> rs = radial_sums<T, 2>(S, s, LA, sh.z, r2, smask, r2ff);
          // Every force term of an AO is linear in its harmonic P_m, its gradient g_m and its constant Hessian
          // h_m, so the weights y_A, y_L (back-projected adjoint weights C X and C B of this electron) are folded
          // over the shell's components first, and the radial factors applied once per shell:
          //   sum_m y_m grad psi_m = R0 G + d R1 S, sum_m y_m grad lap psi_m = LF G + d T3 S,
          //   sum_m y_m (Hess psi_m) j = R0 H + G (d.j) R1 + d (G.j) R1 + S d (d.j) R2 + S j R1,
          // with S = sum_m y_m P_m, G = sum_m y_m g_m, H = sum_m y_m h_m j.
          T SA = T(0), SL = T(0), GA[3] = {T(0), T(0), T(0)}, GL[3] = {T(0), T(0), T(0)}, HL[3] = {T(0), T(0), T(0)};
#pragma unroll
          for (int m = 0; m < ncomp; ++m) {
            T Pa, g[3], h[6];
            angular<T>(LA, m, d[0], d[1], d[2], Pa, g, h);
            T yA, yL;
            dot2_row<T, NM>(xr, bc, Csg + (sh.w + m) * c_stride<NM>(), yA, yL);
            SA += yA * Pa;
            SL += yL * Pa;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
              GA[k] += yA * g[k];
              GL[k] += yL * g[k];
            }
            HL[0] += yL * (h[0] * jg[0] + h[3] * jg[1] + h[4] * jg[2]);
            HL[1] += yL * (h[3] * jg[0] + h[1] * jg[1] + h[5] * jg[2]);
            HL[2] += yL * (h[4] * jg[0] + h[5] * jg[1] + h[2] * jg[2]);
            if (tc)
              reinterpret_cast<__nv_bfloat16*>(P.phiT[sg])[(size_t)w * P.Mp * 16 + tc_tile_index(sh.w + m, el)] =
                  __float2bfloat16_rn((float)(Pa * rs.R0));
            else
              phi[e * L.chunk + chunk_n + m] = Pa * rs.R0;
          }
          const T GLj = GL[0] * jg[0] + GL[1] * jg[1] + GL[2] * jg[2];
          const T xjR1 = xj * rs.R1, SLR1 = SL * rs.R1, cR = GLj * rs.R1 + SL * xj * rs.R2;
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const T gvL = GL[k] * rs.R0 + d[k] * SLR1;
            const T gvA = GA[k] * rs.R0 + d[k] * (SA * rs.R1);
            const T glL = GL[k] * rs.LF + d[k] * (SL * rs.T3);
            const T hjL = HL[k] * rs.R0 + GL[k] * xjR1 + d[k] * cR + jg[k] * SLR1;
            fl[k] -= gvL;
            fe[k] += T(-0.5) * (gvA - (glL + T(2) * hjL));
          }
        }
        chunk_n += ncomp;
      }
    });
    if (cur >= 0) flush_centre(cur);
    flush_chunk();
    if (tc && has_e) {  // Y rows: B_{i, el} and (E_L - E_ref) B_{i, el}
      __nv_bfloat16* y = reinterpret_cast<__nv_bfloat16*>(P.yT[sg]) + (size_t)w * P.Np * 16;
#pragma unroll
      for (int i = 0; i < NM; ++i)
        if (i < n) {
          y[tc_tile_index(i, el)] = __float2bfloat16_rn((float)(wtT * bc[i]));
          y[tc_tile_index(n + i, el)] = __float2bfloat16_rn((float)(wcwT * bc[i]));
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
        T r, ri;
        dist_inv<T>(sd[0] * sd[0] + sd[1] * sd[1] + sd[2] * sd[2], r, ri);
        const T Z = nuc_Z<T>(S, I);
        const T nn[3] = {sd[0] * ri, sd[1] * ri, sd[2] * ri};
        const T ven = -Z * ri * ri * ri;
#pragma unroll
        for (int k = 0; k < 3; ++k) c6[3 + k] = ven * sd[k];
        if (S.J1) {
          const Rad3<T> c = pade_fast<T>(-Z, jas_b<T>(S), r);
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
    // AO-expanded Jastrow terms (JB): their shares of the nuclear derivatives and of dE_L/dr_e, with
    // h = grad ln D + grad J of this electron
    if constexpr (JB) {
      const T h[3] = {gd[0] + jg[0], gd[1] + jg[1], gd[2] + jg[2]};
      T* jv0 = reinterpret_cast<T*>(base + L.jv);
      jb_force_small<T>(S, L.JS, reinterpret_cast<T*>(base + L.jA), jv0, jv0 + 2 * S.MJp, jv0 + S.MJp, lane, has_e, jep,
                        h, frc, dr);
    }
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
      const int so = P.swct_off - olen;  // in the accumulator
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
      if (P.dlnpsi) P.dlnpsi[(size_t)w * 3 * K + i] = (double)frc[i];
      if (P.dEL) P.dEL[(size_t)w * 3 * K + i] = (double)frc[3 * K + i] + __ldg(S.dVnn + i);
      if (accum) {  // the CTA's accumulator is in the working precision
        const T dl = frc[i], de = frc[3 * K + i] + to_T<T>(__ldg(S.dVnn + i));
        atomicAdd(&acc_s[3 + i], wtT * de);
        atomicAdd(&acc_s[3 + 3 * K + i], wtT * dl);
        atomicAdd(&acc_s[3 + 6 * K + i], wcwT * dl);
      }
    }
    if (lane == 0) {
      if (P.EL) P.EL[w] = EL;
      if (P.logpsi) P.logpsi[w] = *la + jsum;
      if (accum) {
        atomicAdd(&acc_s[0], wtT);
        atomicAdd(&acc_s[1], wcwT);
        atomicAdd(&acc_s[2], wcw2T);
      }
    }
    __syncwarp();
  }
  if (accum) {
    __syncthreads();
    double* slot = P.acc + (size_t)blockIdx.x * P.accL;
    const double cnt = (double)acc_s[0];
    for (int k = threadIdx.x; k < accn; k += blockDim.x) {
      const int i = k < oskip ? k : k + olen;
      double v = (double)acc_s[k];
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

// Shared memory of the move kernel for wpc walkers per CTA: inverses (padded to 8 bytes) and positions.
template <typename T>
size_t move_small_smem(const DevSys& S, int wpc) {
  return ((sizeof(T) * (size_t)S.nB * wpc + 7) / 8 * 8) + 8 * (size_t)(3 * S.Ne) * wpc;
}

template <typename T, int NM>
cudaError_t launch_move_small_lpw(int lpw, const DevSys& S, int W, size_t smem, const SmallMoveParams& P,
                                  cudaStream_t st) {
  const int threads = (P.wpc * lpw + 31) / 32 * 32;
  smem += move_small_smem<T>(S, P.wpc);
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

template <typename T, bool JB>
cudaError_t launch_propose_small_impl(const DevSys& S, int nm, int grid, int warps, size_t smem,
                                      const SmallProposeParams& P, cudaStream_t st) {
  if (nm <= 8)
    propose_small<T, 8, JB><<<grid, 32 * warps, smem, st>>>(S, P);
  else if (nm <= 14)
    propose_small<T, 14, JB><<<grid, 32 * warps, smem, st>>>(S, P);
  else
    propose_small<T, 16, JB><<<grid, 32 * warps, smem, st>>>(S, P);
  return cudaGetLastError();
}

template <typename T, bool JB>
cudaError_t launch_measure_small_impl(const DevSys& S, int nm, const SmallLayout& L, int grid, int warps,
                                      const SmallMeasParams& P, cudaStream_t st) {
  const bool tc = P.mode == 2 && sizeof(T) == 4 && P.phiT[0] != nullptr;
  const size_t smem = (size_t)(tc ? L.cta_bytes_tc : L.cta_bytes) + (size_t)warps * L.bytes;
  if (nm <= 8)
    measure_small<T, 8, JB><<<grid, 32 * warps, smem, st>>>(S, L, P);
  else if (nm <= 14)
    measure_small<T, 14, JB><<<grid, 32 * warps, smem, st>>>(S, L, P);
  else
    measure_small<T, 16, JB><<<grid, 32 * warps, smem, st>>>(S, L, P);
  return cudaGetLastError();
}

// Shared-memory limits of the proposal and measurement instances of one Jastrow flag (and, without the
// terms, of the move kernels).
template <typename T, bool JB>
cudaError_t set_smem_limits_small_impl() {
  const int lim = 227 * 1024;
  cudaError_t e;
  if constexpr (!JB) {
#define VMCF_MOVE_ATTR(NM, L, G)                                                                                  \
  if ((e = cudaFuncSetAttribute(move_small<T, NM, L, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
    VMCF_MOVE_ATTR(8, 1, false) VMCF_MOVE_ATTR(8, 2, false) VMCF_MOVE_ATTR(8, 4, false) VMCF_MOVE_ATTR(8, 8, false)
    VMCF_MOVE_ATTR(14, 1, false) VMCF_MOVE_ATTR(14, 2, false) VMCF_MOVE_ATTR(14, 4, false) VMCF_MOVE_ATTR(14, 8, false)
    VMCF_MOVE_ATTR(16, 1, false) VMCF_MOVE_ATTR(16, 2, false) VMCF_MOVE_ATTR(16, 4, false) VMCF_MOVE_ATTR(16, 8, false)
    VMCF_MOVE_ATTR(8, 2, true) VMCF_MOVE_ATTR(14, 2, true) VMCF_MOVE_ATTR(16, 2, true)
#undef VMCF_MOVE_ATTR
  }
  if ((e = cudaFuncSetAttribute(propose_small<T, 8, JB>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(propose_small<T, 14, JB>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(propose_small<T, 16, JB>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(measure_small<T, 8, JB>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(measure_small<T, 14, JB>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(measure_small<T, 16, JB>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  return cudaSuccess;
}

}  // namespace vmcf
