// AO-expanded Jastrow terms over a separate Jastrow basis psi^J (arXiv:2511.05222, App.,
// Eqs. onebody_J_inhom and threebody_jas), read as terms of the Jastrow exponent:
//   U = sum_e sum_mu xi_mu psi^J_mu(r_e) + sum_{i<j} sum_{mu,nu} Xi_{mu nu} psi^J_mu(r_i) psi^J_nu(r_j)
// with Xi symmetric. With s = sum_e psi^J(r_e), t0 = xi + Xi s and u_e = Xi psi^J(r_e):
//   t_e = t0 - u_e = dU / d psi^J(r_e),  grad_e U = sum_mu t_{e mu} grad psi^J_mu(r_e),
//   lap_e U = sum_mu t_{e mu} lap psi^J_mu(r_e),  U = sum_e psi^J(r_e) . (xi + t0 - u_e) / 2.
// A move of electron e by dphi = psi^J(r') - psi^J(r_e) changes U by dphi . t0 - psi^J(r_e) . (Xi dphi).
#pragma once
#include <type_traits>

#include "vmcf_device.cuh"

namespace vmcf {

template <typename T> __device__ __forceinline__ const T* jas_xi(const DevSys& S);
template <> __device__ __forceinline__ const double* jas_xi<double>(const DevSys& S) { return S.jxi; }
template <> __device__ __forceinline__ const float* jas_xi<float>(const DevSys& S) { return S.jxi_f; }
template <typename T> __device__ __forceinline__ const T* jas_Xi(const DevSys& S);
template <> __device__ __forceinline__ const double* jas_Xi<double>(const DevSys& S) { return S.jXi; }
template <> __device__ __forceinline__ const float* jas_Xi<float>(const DevSys& S) { return S.jXi_f; }
template <typename T> __device__ __forceinline__ T jas_alpha(const DevSys& S, int s, int k);
template <> __device__ __forceinline__ double jas_alpha<double>(const DevSys& S, int s, int k) { return __ldg(S.jalpha + s * kMaxPrim + k); }
template <> __device__ __forceinline__ float jas_alpha<float>(const DevSys& S, int s, int k) { return __ldg(S.jalpha_f + s * kMaxPrim + k); }
template <typename T> __device__ __forceinline__ T jas_coef(const DevSys& S, int s, int k);
template <> __device__ __forceinline__ double jas_coef<double>(const DevSys& S, int s, int k) { return __ldg(S.jcoef + s * kMaxPrim + k); }
template <> __device__ __forceinline__ float jas_coef<float>(const DevSys& S, int s, int k) { return __ldg(S.jcoef_f + s * kMaxPrim + k); }

// Index of the Hessian component (d, c) in the LEVEL-2 component layout below.
__device__ __forceinline__ int jas_hidx(int d, int c) {
  return d == c ? 5 + d : (d + c == 1 ? 8 : (d + c == 2 ? 9 : 10));
}

// The functions of Jastrow shell s at p, handed one by one to f(mu, v) with v[0] the value and,
// for LEVEL >= 1, v[1..3] the gradient and v[4] the Laplacian; for LEVEL 2 also v[5..10] the
// Hessian (xx yy zz xy xz yz) and v[11..13] the gradient of the Laplacian. Same radial sums as
// the determinant basis: with e_k = c_k exp(-a_k r^2), R0 = sum e_k, R1 = sum -2 a_k e_k,
// R2 = sum 4 a_k^2 e_k, lap F = sum -2 a_k e_k ((2l+3) - 2 a_k r^2), T3 = sum 4 a_k^2 e_k ((2l+5) - 2 a_k r^2).
template <typename T, int LEVEL, typename F>
__device__ __forceinline__ void jas_shell(const DevSys& S, int s, const EPos& p, F&& f) {
  const int4 sh = __ldg(S.jshell + s);
  const int l = sh.y, np = sh.z;
  T d[3];
  disp_nuc<T>(S, p, sh.x, d);
  const T x = d[0], y = d[1], z = d[2];
  const T r2 = x * x + y * y + z * z;
  T R0 = 0, R1 = 0, R2 = 0, LF = 0, T3 = 0;
  for (int k = 0; k < np; ++k) {
    const T a = jas_alpha<T>(S, s, k);
    const T xa = a * r2;
    const T e = jas_coef<T>(S, s, k) * dexp<T>(-xa);
    R0 += e;
    if (LEVEL >= 1) {
      const T m2ae = T(-2) * a * e;
      R1 += m2ae;
      LF += m2ae * (T(2 * l + 3) - T(2) * xa);
      if (LEVEL >= 2) {
        const T a4e = T(4) * a * a * e;
        R2 += a4e;
        T3 += a4e * (T(2 * l + 5) - T(2) * xa);
      }
    }
  }
  const T xs[3] = {x, y, z};
  for (int m = 0; m < 2 * l + 1; ++m) {
    T P, g[3], h[6];
    angular<T>(l, m, x, y, z, P, g, h);
    T v[LEVEL == 0 ? 1 : (LEVEL == 1 ? 5 : 14)];
    v[0] = P * R0;
    if (LEVEL >= 1) {
#pragma unroll
      for (int i = 0; i < 3; ++i) v[1 + i] = g[i] * R0 + P * xs[i] * R1;
      v[4] = P * LF;
    }
    if constexpr (LEVEL >= 2) {
      const int hi[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        const int i = hi[k][0], j = hi[k][1];
        v[5 + k] = h[k] * R0 + (g[i] * xs[j] + g[j] * xs[i]) * R1 + P * (xs[i] * xs[j] * R2 + (i == j ? R1 : T(0)));
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) v[11 + k] = g[k] * LF + P * xs[k] * T3;
    }
    f(sh.w + m, v);
  }
}

// sum_nu Xi_{nu mu} x[nu] in order of nu; consecutive threads read consecutive entries of a row of Xi
// (Xi is symmetric). The loads are issued eight rows ahead of their use: the rows come from L2, and
// a product per move is latency-bound with one load in flight.
template <typename T>
__device__ __forceinline__ T jas_column(const T* __restrict__ Xi, int MJ, int mu, const T* x) {
  T v = T(0);
  int nu = 0;
  for (; nu + 8 <= MJ; nu += 8) {
    T a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = __ldg(Xi + (size_t)(nu + k) * MJ + mu);
#pragma unroll
    for (int k = 0; k < 8; ++k) v += a[k] * x[nu + k];
  }
  for (; nu < MJ; ++nu) v += __ldg(Xi + (size_t)nu * MJ + mu) * x[nu];
  return v;
}

// y[mu] = b[mu] + sum_nu Xi_{nu mu} x[nu] for the group's functions mu (b may be NULL).
template <typename T, int GS>
__device__ __forceinline__ void jas_matvec(const DevSys& S, const T* x, const T* b, T* y) {
  const int t = threadIdx.x % GS, MJ = S.MJ;
  const T* Xi = jas_Xi<T>(S);
  for (int mu = t; mu < MJ; mu += GS) y[mu] = (b ? __ldg(b + mu) : T(0)) + jas_column<T>(Xi, MJ, mu, x);
}

// out[r][col] = sum_mu rows[r][mu] Xi_{mu col} for R rows row0, row0 + ng, ... of nrows rows with
// row stride MJp (entries MJ..MJp-1 zero, as are the rows of Xi past MJ): four inputs of a row per
// vector load, each output summed in order of mu. Rows past nrows are computed from a valid row and not
// stored.
template <typename T, int R>
__device__ __forceinline__ void jas_rows(const T* rows, const T* __restrict__ Xi, int MJp, int MJ, int col, int row0,
                                         int ng, int nrows, T* out, int out_stride) {
  T v[R];
  const T* a[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    v[r] = T(0);
    const int row = row0 + r * ng;
    a[r] = rows + (row < nrows ? row : nrows - 1) * MJp;
  }
  for (int mu = 0; mu < MJp; mu += 4) {
    T c[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) c[k] = __ldg(Xi + (size_t)(mu + k) * MJ + col);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      T x[4];
      if constexpr (sizeof(T) == 4) {
        const float4 q = *reinterpret_cast<const float4*>(a[r] + mu);
        x[0] = q.x; x[1] = q.y; x[2] = q.z; x[3] = q.w;
      } else {
        const double2 q0 = *reinterpret_cast<const double2*>(a[r] + mu);
        const double2 q1 = *reinterpret_cast<const double2*>(a[r] + mu + 2);
        x[0] = q0.x; x[1] = q0.y; x[2] = q1.x; x[3] = q1.y;
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) v[r] += x[k] * c[k];
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int row = row0 + r * ng;
    if (row < nrows) out[row * out_stride + col] = v[r];
  }
}

// All MJ columns of nrows (<= 8 per thread) rows times Xi over the group, the thread mapping of
// orbital_block: with GS >= MJ thread t owns column t % MJ and rows t / MJ + k ng (ng = GS / MJ); with
// GS < MJ it owns columns t, t + GS, ... and every row.
template <typename T, int GS>
__device__ __forceinline__ void jas_block(const DevSys& S, const T* rows, int nrows, T* out, int out_stride) {
  const int t = threadIdx.x % GS, MJ = S.MJ, MJp = S.MJp;
  const T* Xi = jas_Xi<T>(S);
  const bool wide = GS >= MJ;
  const int ng = wide ? GS / MJ : 1;
  const int col0 = wide ? t % MJ : t, rg = wide ? t / MJ : 0, dcol = wide ? MJ : GS;
  for (int col = col0; col < MJ && rg < ng && rg < nrows; col += dcol) {
    switch ((nrows - rg + ng - 1) / ng) {
      case 1: jas_rows<T, 1>(rows, Xi, MJp, MJ, col, rg, ng, nrows, out, out_stride); break;
      case 2: jas_rows<T, 2>(rows, Xi, MJp, MJ, col, rg, ng, nrows, out, out_stride); break;
      case 3: jas_rows<T, 3>(rows, Xi, MJp, MJ, col, rg, ng, nrows, out, out_stride); break;
      case 4: jas_rows<T, 4>(rows, Xi, MJp, MJ, col, rg, ng, nrows, out, out_stride); break;
      case 5: jas_rows<T, 5>(rows, Xi, MJp, MJ, col, rg, ng, nrows, out, out_stride); break;
      case 6: jas_rows<T, 6>(rows, Xi, MJp, MJ, col, rg, ng, nrows, out, out_stride); break;
      case 7: jas_rows<T, 7>(rows, Xi, MJp, MJ, col, rg, ng, nrows, out, out_stride); break;
      default: jas_rows<T, 8>(rows, Xi, MJp, MJ, col, rg, ng, nrows, out, out_stride); break;
    }
  }
}

// t0 = xi + Xi s with s = sum_e psi^J(r_e), by jng subgroups of GS / jng threads (whole warps): subgroup
// g sums the electrons e = g, g + jng, ... into part[g][MJ], a thread covering whole shells; then the
// parts are added in order of g. Every thread of the group calls it.
template <typename T, int GS>
__device__ void jas_refresh_t0_sub(const DevSys& S, const double* pos, int jng, T* part, T* s, T* t0) {
  const int t = threadIdx.x % GS, MJ = S.MJ, gsz = GS / jng, g = t / gsz, tt = t - g * gsz;
  T* pg = part + g * MJ;
  for (int sh = tt; sh < S.nJs; sh += gsz) {
    const int4 d = __ldg(S.jshell + sh);
    for (int m = 0; m < 2 * d.y + 1; ++m) pg[d.w + m] = T(0);
    for (int e = g; e < S.Ne; e += jng)
      jas_shell<T, 0>(S, sh, make_epos(pos + 3 * e), [&](int mu, const T* v) { pg[mu] += v[0]; });
  }
  gsync<GS>();
  for (int mu = t; mu < MJ; mu += GS) {
    T v = T(0);
    for (int k = 0; k < jng; ++k) v += part[k * MJ + mu];
    s[mu] = v;
  }
  gsync<GS>();
  jas_matvec<T, GS>(S, s, jas_xi<T>(S), t0);
  gsync<GS>();
}

// t0 = xi + Xi s with s = sum_e psi^J(r_e) for the walker at pos (every thread of the group
// calls it). s: [MJ] scratch; a thread sums the functions of its shells over all electrons.
template <typename T, int GS>
__device__ void jas_refresh_t0(const DevSys& S, const double* pos, T* s, T* t0) {
  const int t = threadIdx.x % GS;
  for (int sh = t; sh < S.nJs; sh += GS) {
    const int4 d = __ldg(S.jshell + sh);
    for (int m = 0; m < 2 * d.y + 1; ++m) s[d.w + m] = T(0);
    for (int e = 0; e < S.Ne; ++e)
      jas_shell<T, 0>(S, sh, make_epos(pos + 3 * e), [&](int mu, const T* v) { s[mu] += v[0]; });
  }
  gsync<GS>();
  jas_matvec<T, GS>(S, s, jas_xi<T>(S), t0);
  gsync<GS>();
}

}  // namespace vmcf
