// AO-expanded Jastrow terms in the one-warp-per-walker kernels (arXiv:2511.05222, App., Eqs.
// onebody_J_inhom and threebody_jas), one lane per electron. The exponent's terms
//   U = sum_e xi . psi^J(r_e) + sum_{i<j} psi^J(r_i)^T Xi psi^J(r_j)
// are handled through s = sum_e psi^J(r_e), t0 = xi + Xi s and t_e = t0 - Xi psi^J(r_e) = dU/d psi^J(r_e):
//   grad_e U = sum_mu t_e,mu grad psi^J_mu(r_e),   lap_e U = sum_mu t_e,mu lap psi^J_mu(r_e),
//   U = sum_e psi^J(r_e) . (xi + t_e) / 2.
// Nuclear derivatives (with h_e = grad ln D + grad J at r_e, w_e = h_e . grad psi^J(r_e) + lap psi^J(r_e) / 2 and
// P = Xi sum_e w_e): function mu of nucleus a at electron e adds -d_d psi^J_mu t_e,mu to d ln Psi / dR_a,d and
// c = (h_e . d_d grad psi^J_mu + d_d lap psi^J_mu / 2) t_e,mu + (P - Xi w_e)_mu d_d psi^J_mu to dE_L / dR_a,d, and
// -c to dE_L / dr_e,d. A move of electron e by dphi = psi^J(r'_e) - psi^J(r_e) changes U by dphi . (t0 - Xi psi^J(r_e)).
//
// Each lane keeps its electron's MJ-vector as a row of a per-warp shared-memory block [Ne][JS] (JS: a row stride
// whose 16-byte loads by the warp's lanes fall in distinct banks; entries MJ..MJp-1 zero), and the products with Xi
// are formed one output at a time from Xi's rows (padded to MJp, read through the L1 cache as warp-wide broadcasts).
#pragma once
#include "jastrow_basis.cuh"

namespace vmcf {

template <typename T> __device__ __forceinline__ const T* jas_Xr(const DevSys& S);
template <> __device__ __forceinline__ const double* jas_Xr<double>(const DevSys& S) { return S.jXr; }
template <> __device__ __forceinline__ const float* jas_Xr<float>(const DevSys& S) { return S.jXr_f; }

// sum_nu a[nu] x[nu] over nu < MJp (a multiple of 4): a in global memory (a padded row of Xi), x in shared
// memory, both 16-byte aligned; four partial sums in a fixed order.
template <typename T>
__device__ __forceinline__ T jas_dot(const T* __restrict__ a, const T* x, int MJp) {
  T v0 = T(0), v1 = T(0), v2 = T(0), v3 = T(0);
  if constexpr (sizeof(T) == 4) {
#pragma unroll 4
    for (int nu = 0; nu < MJp; nu += 4) {
      const float4 p = __ldg(reinterpret_cast<const float4*>(a + nu));
      const float4 q = *reinterpret_cast<const float4*>(x + nu);
      v0 += p.x * q.x;
      v1 += p.y * q.y;
      v2 += p.z * q.z;
      v3 += p.w * q.w;
    }
  } else {
#pragma unroll 2
    for (int nu = 0; nu < MJp; nu += 4) {
      const double2 p0 = __ldg(reinterpret_cast<const double2*>(a + nu));
      const double2 p1 = __ldg(reinterpret_cast<const double2*>(a + nu + 2));
      const double2 q0 = *reinterpret_cast<const double2*>(x + nu);
      const double2 q1 = *reinterpret_cast<const double2*>(x + nu + 2);
      v0 += p0.x * q0.x;
      v1 += p0.y * q0.y;
      v2 += p1.x * q1.x;
      v3 += p1.y * q1.y;
    }
  }
  return (v0 + v1) + (v2 + v3);
}

// The same with both vectors in shared memory (16-byte aligned).
template <typename T>
__device__ __forceinline__ T jas_dot_s(const T* a, const T* x, int MJp) {
  T v0 = T(0), v1 = T(0), v2 = T(0), v3 = T(0);
  if constexpr (sizeof(T) == 4) {
#pragma unroll 4
    for (int nu = 0; nu < MJp; nu += 4) {
      const float4 p = *reinterpret_cast<const float4*>(a + nu);
      const float4 q = *reinterpret_cast<const float4*>(x + nu);
      v0 += p.x * q.x;
      v1 += p.y * q.y;
      v2 += p.z * q.z;
      v3 += p.w * q.w;
    }
  } else {
#pragma unroll 2
    for (int nu = 0; nu < MJp; nu += 4) {
      const double2 p0 = *reinterpret_cast<const double2*>(a + nu);
      const double2 p1 = *reinterpret_cast<const double2*>(a + nu + 2);
      const double2 q0 = *reinterpret_cast<const double2*>(x + nu);
      const double2 q1 = *reinterpret_cast<const double2*>(x + nu + 2);
      v0 += p0.x * q0.x;
      v1 += p0.y * q0.y;
      v2 += p1.x * q1.x;
      v3 += p1.y * q1.y;
    }
  }
  return (v0 + v1) + (v2 + v3);
}

// psi^J at p (level-0 values) into row, entries MJ..MJp-1 zeroed.
template <typename T>
__device__ __forceinline__ void jas_values_row(const DevSys& S, const EPos& p, T* row) {
  for (int sh = 0; sh < S.nJs; ++sh) jas_shell<T, 0>(S, sh, p, [&](int mu, const T* v) { row[mu] = v[0]; });
  for (int mu = S.MJ; mu < S.MJp; ++mu) row[mu] = T(0);
}

// out[mu] = sum_e rows[e][mu] for mu < MJp, the warp's lanes taking mu = lane, lane + 32, ...; rows are summed
// in order of e.
template <typename T>
__device__ __forceinline__ void jas_colsum(const DevSys& S, const T* rows, int JS, int lane, T* out) {
  for (int mu = lane; mu < S.MJp; mu += 32) {
    T v = T(0);
    for (int k = 0; k < S.Ne; ++k) v += rows[k * JS + mu];
    out[mu] = v;
  }
}

// t0 = xi + Xi s (entries past MJ zero), the warp's lanes taking mu = lane, lane + 32, ...
template <typename T>
__device__ __forceinline__ void jas_t0(const DevSys& S, const T* s, int lane, T* t0) {
  const T* xi = jas_xi<T>(S);
  const T* Xr = jas_Xr<T>(S);
  for (int mu = lane; mu < S.MJp; mu += 32) t0[mu] = mu < S.MJ ? __ldg(xi + mu) + jas_dot<T>(Xr + mu * S.MJp, s, S.MJp) : T(0);
}

// Evaluation: adds the terms to this lane's grad J (jg), lap J (jl) and J value share (jv); leaves t0 in jt0 for the
// force pass. rows: the warp's [Ne][JS] block; js, jt0: [MJp] vectors. Every lane of the warp calls it.
template <typename T>
__device__ void jb_eval_small(const DevSys& S, int JS, T* rows, T* js, T* jt0, int lane, bool has_e, const EPos& p,
                              T (&jg)[3], T& jl, T& jv) {
  T* row = rows + lane * JS;
  if (has_e) jas_values_row<T>(S, p, row);
  __syncwarp();
  jas_colsum<T>(S, rows, JS, lane, js);
  __syncwarp();
  jas_t0<T>(S, js, lane, jt0);
  __syncwarp();
  if (!has_e) return;
  const T* xi = jas_xi<T>(S);
  const T* Xr = jas_Xr<T>(S);
  const int MJp = S.MJp;
  for (int sh = 0; sh < S.nJs; ++sh)
    jas_shell<T, 1>(S, sh, p, [&](int mu, const T* v) {
      const T t = jt0[mu] - jas_dot<T>(Xr + mu * MJp, row, MJp);
      jg[0] += t * v[1];
      jg[1] += t * v[2];
      jg[2] += t * v[3];
      jl += t * v[4];
      jv += T(0.5) * v[0] * (__ldg(xi + mu) + t);
    });
}

// Nuclear derivatives: adds the terms to d ln Psi/dR (frc[0, 3K)), dE_L/dR (frc[3K, 6K)) and this lane's dE_L/dr_e
// (dr). h: grad ln D + grad J at this lane's electron; jt0: t0 from the evaluation (kept since); rows, jw, jP: the
// [Ne][JS] block and two [MJp] vectors. Every lane of the warp calls it.
template <typename T>
__device__ void jb_force_small(const DevSys& S, int JS, T* rows, T* jw, T* jP, const T* jt0, int lane, bool has_e,
                               const EPos& p, const T (&h)[3], T* frc, T (&dr)[3]) {
  const int K = S.K, MJp = S.MJp;
  const T* Xr = jas_Xr<T>(S);
  T* row = rows + lane * JS;
  T fl[3] = {T(0), T(0), T(0)}, fe[3] = {T(0), T(0), T(0)}, cr[3] = {T(0), T(0), T(0)};
  int cur = -1;
  // a nucleus' partial sums over the warp's electrons, added by lane 0 (every lane takes part)
  auto flush = [&](int I) {
    T v6[6] = {fl[0], fl[1], fl[2], fe[0], fe[1], fe[2]};
#pragma unroll
    for (int k = 0; k < 6; ++k)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v6[k] += __shfl_xor_sync(0xffffffffu, v6[k], o);
    if (lane == 0)
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        frc[3 * I + d] += v6[d];
        frc[3 * K + 3 * I + d] += v6[3 + d];
      }
#pragma unroll
    for (int d = 0; d < 3; ++d) fl[d] = fe[d] = T(0);
  };
  // psi^J(r_e) into this lane's row; t_e = t0 - Xi psi^J(r_e) from it, one function at a time
  if (has_e) jas_values_row<T>(S, p, row);
  __syncwarp();
  for (int sh = 0; sh < S.nJs; ++sh) {
    const int I = __ldg(S.jshell + sh).x;
    if (I != cur) {
      if (cur >= 0) flush(cur);
      cur = I;
    }
    if (has_e)
      jas_shell<T, 2>(S, sh, p, [&](int mu, const T* v) {
        const T t = jt0[mu] - jas_dot<T>(Xr + mu * MJp, row, MJp);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          T hh = T(0);
#pragma unroll
          for (int c = 0; c < 3; ++c) hh += h[c] * v[jas_hidx(d, c)];
          const T cd = (hh + T(0.5) * v[11 + d]) * t;
          fl[d] -= v[1 + d] * t;
          fe[d] += cd;
          cr[d] += cd;
        }
      });
  }
  if (cur >= 0) flush(cur);
  __syncwarp();  // every lane is done with the rows of psi^J
  // w_e into this lane's row, P = Xi sum_e w_e
  if (has_e) {
    for (int sh = 0; sh < S.nJs; ++sh)
      jas_shell<T, 1>(S, sh, p, [&](int mu, const T* v) {
        row[mu] = h[0] * v[1] + h[1] * v[2] + h[2] * v[3] + T(0.5) * v[4];
      });
    for (int mu = S.MJ; mu < MJp; ++mu) row[mu] = T(0);
  }
  __syncwarp();
  jas_colsum<T>(S, rows, JS, lane, jw);
  __syncwarp();
  for (int mu = lane; mu < MJp; mu += 32) jP[mu] = mu < S.MJ ? jas_dot<T>(Xr + mu * MJp, jw, MJp) : T(0);
  __syncwarp();
  // (P - Xi w_e)_mu d_d psi^J_mu
  cur = -1;
  for (int sh = 0; sh < S.nJs; ++sh) {
    const int I = __ldg(S.jshell + sh).x;
    if (I != cur) {
      if (cur >= 0) flush(cur);
      cur = I;
    }
    if (has_e)
      jas_shell<T, 1>(S, sh, p, [&](int mu, const T* v) {
        const T pd = jP[mu] - jas_dot<T>(Xr + mu * MJp, row, MJp);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          fe[d] += pd * v[1 + d];
          cr[d] += pd * v[1 + d];
        }
      });
  }
  if (cur >= 0) flush(cur);
#pragma unroll
  for (int d = 0; d < 3; ++d) dr[d] -= cr[d];
  __syncwarp();
}

// sum over the warp's lanes (xor butterfly: every lane receives the same bits)
template <typename T>
__device__ __forceinline__ T jas_warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Proposals: with old = psi^J(r_e) and dphi_e = psi^J(r'_e) - old, adds dphi_e . (t0 - Xi old) to dchi (this
// lane's electron) and writes dphi_a . Xi dphi_b for every pair b < a of the walker to dp (lane a writes its row
// of pairs). Xs: Xi's rows [MJ][MJp] in shared memory; D: the warp's [Ne][JS] rows dphi_e; js, jt0: [MJp]
// vectors. Per function mu, lane a forms (Xi dphi_a)_mu once and adds its products with dphi_b,mu to register
// accumulators for all b < a. Every lane of the warp calls it.
template <typename T>
__device__ void jb_propose_small(const DevSys& S, int JS, const T* Xs, T* D, T* js, T* jt0, int lane, bool has_e,
                                 const EPos& po, const EPos& pn, int npair, T* dp, T& dchi) {
  const int MJ = S.MJ, MJp = S.MJp, Ne = S.Ne;
  T* d = D + lane * JS;
  // dphi into this lane's row; s = sum_e old over the warp
  for (int sh = 0; sh < S.nJs; ++sh) {
    T vo[7] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
    const int4 sd = __ldg(S.jshell + sh);
    const int nf = 2 * sd.y + 1;
    if (has_e) {
      jas_shell<T, 0>(S, sh, po, [&](int mu, const T* v) { vo[mu - sd.w] = v[0]; });
      jas_shell<T, 0>(S, sh, pn, [&](int mu, const T* v) { d[mu] = v[0] - vo[mu - sd.w]; });
    }
#pragma unroll
    for (int m = 0; m < 7; ++m)
      if (m < nf) {
        const T sm = jas_warp_sum<T>(vo[m]);
        if (lane == 0) js[sd.w + m] = sm;
      }
  }
  if (has_e)
    for (int mu = MJ; mu < MJp; ++mu) d[mu] = T(0);
  if (lane == 0)
    for (int mu = MJ; mu < MJp; ++mu) js[mu] = T(0);
  __syncwarp();
  {  // t0 = xi + Xi s
    const T* xi = jas_xi<T>(S);
    for (int mu = lane; mu < MJp; mu += 32) jt0[mu] = mu < MJ ? __ldg(xi + mu) + jas_dot_s<T>(Xs + mu * MJp, js, MJp) : T(0);
  }
  __syncwarp();
  T acc[32];
#pragma unroll
  for (int b = 0; b < 32; ++b) acc[b] = T(0);
  T a1 = T(0), bsum = T(0);
  if (has_e) {
    a1 = jas_dot_s<T>(d, jt0, MJp);
    for (int sh = 0; sh < S.nJs; ++sh)
      jas_shell<T, 0>(S, sh, po, [&](int mu, const T* v) {
        const T g = jas_dot_s<T>(Xs + mu * MJp, d, MJp);  // (Xi dphi_a)_mu
        bsum += v[0] * g;
#pragma unroll
        for (int b = 0; b < 32; ++b)
          if (b < lane && b < Ne) acc[b] += g * D[b * JS + mu];
      });
    dchi += a1 - bsum;
    T* row = dp + lane * (lane - 1) / 2;
#pragma unroll
    for (int b = 0; b < 32; ++b)
      if (b < lane && b < Ne) row[b] = acc[b];
  }
  (void)npair;
  __syncwarp();  // the rows are reused for the warp's next walker
}

}  // namespace vmcf
