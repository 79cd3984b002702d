// Kernels of the VMC hot path (arXiv:2511.05222, App. A), templated on the arithmetic type
// T (double: FP64 mode; float: mixed mode) and the walker-group size GS.
//
//  refresh_kernel  fresh FP64 Slater inverses from positions
//  move_kernel     Metropolis sweeps with Sherman-Morrison updates and periodic refresh
//  measure_kernel  fresh inverse, E_L, adjoint nuclear derivatives, O = dlnPsi/dC, and
//                  either per-walker outputs or the walker sums behind E, F and dE/dC
#pragma once
#include <cuda_bf16.h>

#include "jastrow_basis.cuh"
#include "vmcf_device.cuh"
#include "vmcf_internal.h"

namespace vmcf {

template <typename T>
__device__ __forceinline__ T* sm_ptr(unsigned char* base, int off) {
  return reinterpret_cast<T*>(base + off);
}

// Positions to shared memory: double, plus the float-float split used by mixed mode.
template <int GS>
__device__ __forceinline__ void load_positions(const double* src, int n3, double* pos, float* ph, float* pl) {
  const int t = threadIdx.x % GS;
  for (int i = t; i < n3; i += GS) {
    const double v = src[i];
    pos[i] = v;
    split_ff_bits(v, ph[i], pl[i]);
  }
}

// Sum over both spin blocks of the squared entries of the inverses (the S of the guiding
// function g = max(1, eps sqrt(S)) of reweighted sampling); identical in every thread.
template <typename T, int GS>
__device__ __forceinline__ double inverse_frob2(const DevSys& S, const T* B, double* red) {
  const int t = threadIdx.x % GS;
  double v[1] = {0.0};
  for (int i = t; i < S.nB; i += GS) v[0] += (double)B[i] * (double)B[i];
  group_sum<GS, 1>(v, red);
  return v[0];
}

// Rebuild the inverses of both spin blocks of one walker into B (T) from positions.
template <typename T, int GS>
__device__ void refresh_walker(const DevSys& S, const double* pos, T* B, double* A, T* ao, int ao_rows, int* piv,
                               double* f, int* flag) {
  const int t = threadIdx.x % GS;
  for (int sg = 0; sg < 2; ++sg) {
    const int n = sg == 0 ? S.nup : S.ndn;
    if (n == 0) continue;
    build_slater<T, GS>(S, pos, sg, A, ao, ao_rows);
    double la = 0.0, sgn = 1.0;
    gj_inverse<GS>(A, n, piv, f, flag, &la, &sgn, false);
    T* Bs = B + (sg == 0 ? 0 : S.nup * S.nup);
    for (int idx = t; idx < n * n; idx += GS) Bs[idx] = (T)A[idx];
    gsync<GS>();
  }
}

// ---------------------------------------------------------------- refresh
template <typename T, int GS>
__global__ void __launch_bounds__(256) refresh_kernel(DevSys S, GroupLayout L, const double* __restrict__ pos_g,
                                                      T* __restrict__ B_g, int W, unsigned long long* counters) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int gpb = blockDim.x / GS, gid = threadIdx.x / GS, t = threadIdx.x % GS;
  unsigned char* base = smem + gid * L.bytes;
  double* pos = sm_ptr<double>(base, L.pos);
  double* A = sm_ptr<double>(base, L.Bd);
  T* ao = sm_ptr<T>(base, L.ao);
  T* B = sm_ptr<T>(base, L.Bt);
  int* piv = sm_ptr<int>(base, L.piv);
  double* f = sm_ptr<double>(base, L.f);
  int* flag = sm_ptr<int>(base, L.scal);
  const int w = blockIdx.x * gpb + gid;
  if (w >= W) return;  // the whole group leaves together; only group barriers are used
  const int Ne = S.Ne;
  for (int i = t; i < 3 * Ne; i += GS) pos[i] = pos_g[(size_t)w * 3 * Ne + i];
  if (t == 0) *flag = 0;
  gsync<GS>();
  refresh_walker<T, GS>(S, pos, B, A, ao, L.ao_rows, piv, f, flag);
  for (int i = t; i < S.nB; i += GS) B_g[(size_t)w * S.nB + i] = B[i];
  if (t == 0) {
    if (*flag) atomicAdd(&counters[0], 1ull);
    atomicAdd(&counters[1], 1ull);
  }
}

// ---------------------------------------------------------------- Metropolis sweeps
// All sweeps of one walker (index w of P's arrays) by one group. c0: attempted moves since
// the last refresh when the launch starts; sweep0: global sweep index of the first sweep.
// Change of the electron-nucleus Jastrow terms when an electron moves from po to pn, summed over the nuclei by
// one whole warp: lane l takes nuclei l, l + 32, ... in order, then an xor butterfly, so every lane holds the same
// bits whichever kernel calls it (the sweep kernel or the proposal pass).
template <typename T>
__device__ __forceinline__ T en_change_warp(const DevSys& S, const EPos& pn, const EPos& po, int lane) {
  T v = T(0);
  if (S.J1) {
    const T b = jas_b<T>(S);
    for (int I = lane; I < S.K; I += 32) {
      const T mz = -nuc_Z<T>(S, I);
      T d1[3], d0[3];
      disp_nuc<T>(S, pn, I, d1);
      disp_nuc<T>(S, po, I, d0);
      v += pade_value<T>(mz, b, dsqrt<T>(d1[0] * d1[0] + d1[1] * d1[1] + d1[2] * d1[2])) -
           pade_value<T>(mz, b, dsqrt<T>(d0[0] * d0[0] + d0[1] * d0[1] + d0[2] * d0[2]));
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// sum_{mu in [m0, m1)} ao[mu] C[mu][i], in order of mu: one half of an orbital-row entry (the entry is the sum of
// the halves [0, M/2) and [M/2, M), in that order, in every kernel that forms it).
template <typename T>
__device__ __forceinline__ T orbital_half(const T* ao, const T* __restrict__ C, int n, int i, int m0, int m1) {
  T v = T(0);
  for (int mu = m0; mu < m1; ++mu) v += ao[mu] * __ldg(C + mu * n + i);
  return v;
}

// JB: the system has AO-expanded Jastrow terms; without them the terms' code is compiled out.
template <typename T, int GS, bool JB>
__device__ void move_walker(const DevSys& S, const GroupLayout& L, const MoveParams& P, unsigned char* base, int w,
                            int c0, uint64_t sweep0) {
  const int t = threadIdx.x % GS;
  double* pos = sm_ptr<double>(base, L.pos);
  float* ph = sm_ptr<float>(base, L.ph);
  float* pl = sm_ptr<float>(base, L.pl);
  double* A = sm_ptr<double>(base, L.Bd);
  T* B = sm_ptr<T>(base, L.Bt);
  T* ao = sm_ptr<T>(base, L.ao);
  T* row = sm_ptr<T>(base, L.row);
  T* wv = sm_ptr<T>(base, L.wv);
  T* col = sm_ptr<T>(base, L.col);
  int* piv = sm_ptr<int>(base, L.piv);
  double* f = sm_ptr<double>(base, L.f);
  double* red = sm_ptr<double>(base, L.red);
  int* flag = sm_ptr<int>(base, L.scal);
  const int Ne = S.Ne, nup = S.nup, K = S.K;
  double* posg = P.pos + (size_t)w * 3 * Ne;
  T* Bg = reinterpret_cast<T*>(P.B) + (size_t)w * S.nB;
  load_positions<GS>(posg, 3 * Ne, pos, ph, pl);
  for (int i = t; i < S.nB; i += GS) B[i] = Bg[i];
  if (t == 0) *flag = 0;
  gsync<GS>();
  // AO-expanded Jastrow terms: t0 = xi + Xi s, the Jastrow-basis values at r' and r_e, and
  // y = Xi (psi^J(r') - psi^J(r_e)); t0 is rebuilt here and at every re-inversion, and moves by y
  // on acceptance
  const int MJ = JB ? S.MJ : 0;
  T* jt0 = MJ ? sm_ptr<T>(base, L.jw) : nullptr;
  T* jpn = jt0 + MJ;
  T* jpo = jpn + MJ;
  T* jy = jpo + MJ;
  if (MJ) jas_refresh_t0<T, GS>(S, pos, jy, jt0);
  const uint64_t wid = P.wid0 + (uint64_t)w;
  int c = c0;
  uint32_t nacc = 0, nrej = 0, nref = 0;
  // reweighted sampling of |Psi_G|^2, Psi_G = Psi max(1, eps sqrt(S)): S of the current inverses
  const bool guide = P.eps > 0.0;
  double Sg = guide ? inverse_frob2<T, GS>(S, B, red) : 0.0;
  for (int sw = 0; sw < P.nsweeps; ++sw) {
    const uint64_t sweep = sweep0 + (uint64_t)sw;
    for (int e = 0; e < Ne; ++e) {
      const int sg = e < nup ? 0 : 1;
      const int n = sg == 0 ? nup : S.ndn, el = e - (sg == 0 ? 0 : nup);
      T* Bs = B + (sg == 0 ? 0 : nup * nup);
      const T* C = coefC<T>(S, sg);
      // the proposal: from the proposal pass when given, else drawn here (the same arithmetic)
      const bool pre = P.prn != nullptr;
      const size_t pidx = (size_t)w * Ne + e;
      double rn[3];
      if (pre) {
#pragma unroll
        for (int k = 0; k < 3; ++k) rn[k] = __ldg(P.prn + 3 * pidx + k);
      } else {
        uint64_t r[4] = {wid, sweep, (uint64_t)e, 0};
        philox4x64_10(r, P.k0, P.k1);
        double xi[3];
        normals3(r, xi, T(0));
#pragma unroll
        for (int k = 0; k < 3; ++k) rn[k] = pos[3 * e + k] + P.sigma * xi[k];
      }
      const EPos pn = make_epos(rn);
      const EPos po = make_epos(pos + 3 * e);
      if (!pre) ao_point<T, GS, 0, false>(S, pn, ao, 0);
      for (int sh = t; sh < (JB ? S.nJs : 0); sh += GS) {
        jas_shell<T, 0>(S, sh, pn, [&](int mu, const T* v) { jpn[mu] = v[0]; });
        jas_shell<T, 0>(S, sh, po, [&](int mu, const T* v) { jpo[mu] = v[0]; });
      }
      gsync<GS>();
      double part[1] = {0.0};  // determinant ratio (FP64)
      T dJ = T(0);              // Jastrow exponent difference
      // new orbital row phi_i(r'), each entry the sum of its halves over [0, M/2) and [M/2, M); with GS >= 2n
      // the halves go to different threads (the second through wv)
      const int mh = S.M / 2;
      if (pre) {
        const T* pr = reinterpret_cast<const T*>(P.prow) + pidx * S.nmax;
        for (int i = t; i < n; i += GS) {
          const T v = __ldg(pr + i);
          row[i] = v;
          part[0] += (double)v * (double)Bs[i * n + el];
        }
      } else if (GS < 2 * n) {
        for (int i = t; i < n; i += GS) {
          const T v = orbital_half<T>(ao, C, n, i, 0, mh) + orbital_half<T>(ao, C, n, i, mh, S.M);
          row[i] = v;
          part[0] += (double)v * (double)Bs[i * n + el];
        }
      } else {
        T v = 0;
        const int i = t % n, pp = t / n;
        if (pp < 2) {
          v = orbital_half<T>(ao, C, n, i, pp == 0 ? 0 : mh, pp == 0 ? mh : S.M);
          if (pp == 1) wv[i] = v;
        }
        gsync<GS>();
        if (pp == 0) {
          v = v + wv[i];
          row[i] = v;
          part[0] += (double)v * (double)Bs[i * n + el];
        }
      }
      // the electron-nucleus change: from the proposal pass, else from the group's first warp (into f[0], which
      // is free between re-inversions)
      if (!pre && t < 32) {
        const T en = en_change_warp<T>(S, pn, po, t);
        if (t == 0) f[0] = (double)en;
      }
      // Jastrow ratio: pairs with every other electron
      for (int q = t; q < Ne; q += GS) {
        {
          if (q == e || !S.J2) continue;
          const bool par = (q < nup) == (e < nup);

          T d1[3], d0[3];
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            if constexpr (sizeof(T) == 8) {
              d1[k] = rn[k] - pos[3 * q + k];
              d0[k] = pos[3 * e + k] - pos[3 * q + k];
            } else {
              d1[k] = (pn.h[k] - ph[3 * q + k]) + (pn.l[k] - pl[3 * q + k]);
              d0[k] = (po.h[k] - ph[3 * q + k]) + (po.l[k] - pl[3 * q + k]);
            }
          }
          dJ += pair_value<T>(S, par, dsqrt<T>(d1[0] * d1[0] + d1[1] * d1[1] + d1[2] * d1[2])) -
                pair_value<T>(S, par, dsqrt<T>(d0[0] * d0[0] + d0[1] * d0[1] + d0[2] * d0[2]));
        }
      }
      if (MJ) {  // AO-expanded terms: dphi . t0 - psi^J(r_e) . (Xi dphi), dphi = psi^J(r') - psi^J(r_e)
        for (int mu = t; mu < MJ; mu += GS) jpn[mu] -= jpo[mu];  // dphi in place of psi^J(r')
        gsync<GS>();
        for (int mu = t; mu < MJ; mu += GS) {
          const T y = jas_column<T>(jas_Xi<T>(S), MJ, mu, jpn);
          dJ += jpn[mu] * jt0[mu] - jpo[mu] * y;
          jy[mu] = y;
        }
      }
      gsync<GS>();
      group_sum_dt<GS>(part[0], dJ, red);
      dJ += pre ? __ldg(reinterpret_cast<const T*>(P.pdchi) + pidx) : (T)f[0];
      const double R = part[0];
      double u;
      if (pre) {
        u = __ldg(P.pu + pidx);
      } else {
        uint64_t r2[4] = {wid, sweep, (uint64_t)e, 1};
        philox4x64_10(r2, P.k0, P.k1);
        u = u01(r2[0]);
      }
      double pr = R * R * (double)dexp<T>(T(2) * dJ);
      double Sn = Sg;
      if (guide && R != 0.0) {
        // S after the Sherman-Morrison update B' = B - c w^T / R (c = column el of B):
        // S' = S - (2/R) sum_j w_j (B^T c)_j + |c|^2 |w|^2 / R^2
        double gs[3] = {0.0, 0.0, 0.0};
        for (int j = t; j < n; j += GS) {
          T v = 0, tj = 0;
          for (int i = 0; i < n; ++i) {
            v += row[i] * Bs[i * n + j];
            tj += Bs[i * n + el] * Bs[i * n + j];
          }
          const T wj = v - (j == el ? T(1) : T(0));
          wv[j] = wj;
          col[j] = Bs[j * n + el];
          gs[0] += (double)wj * (double)tj;
          gs[1] += (double)wj * (double)wj;
          gs[2] += (double)col[j] * (double)col[j];
        }
        group_sum<GS, 3>(gs, red);
        Sn = Sg - 2.0 * gs[0] / R + gs[2] * gs[1] / (R * R);
        const double g0 = fmax(1.0, P.eps * sqrt(Sg)), g1 = fmax(1.0, P.eps * sqrt(fmax(Sn, 0.0)));
        pr *= (g1 / g0) * (g1 / g0);
      }
      const bool ok = isfinite(pr) && R != 0.0;
      if (!ok) ++nrej;
      if (ok && u < pr) {
        // Sherman-Morrison: row el of A becomes `row`; with w_j = sum_i row_i B_ij - delta_j,el,
        // B_kj <- B_kj - B_k,el w_j / R.
        if (!guide) {
          for (int j = t; j < n; j += GS) {
            T v = 0;
            for (int i = 0; i < n; ++i) v += row[i] * Bs[i * n + j];
            wv[j] = v - (j == el ? T(1) : T(0));
            col[j] = Bs[j * n + el];
          }
        }
        Sg = Sn;
        gsync<GS>();
        const T rinv = (T)(1.0 / R);
        for (int idx = t; idx < n * n; idx += GS) {
          const int k = idx / n, j = idx - k * n;
          Bs[idx] -= col[k] * wv[j] * rinv;
        }
        if (t < 3) {
          pos[3 * e + t] = rn[t];
          ph[3 * e + t] = pn.h[t];
          pl[3 * e + t] = pn.l[t];
        }
        for (int mu = t; mu < MJ; mu += GS) jt0[mu] += jy[mu];  // s moves by dphi
        ++nacc;
        gsync<GS>();
      }
      if (++c == P.kref) {
        const bool last = (sw == P.nsweeps - 1) && (e == Ne - 1);
        if (!(last && P.skip_final_refresh)) {
          refresh_walker<T, GS>(S, pos, B, A, ao, L.ao_rows, piv, f, flag);
          ++nref;
          if (guide) Sg = inverse_frob2<T, GS>(S, B, red);
          if (MJ) jas_refresh_t0<T, GS>(S, pos, jy, jt0);
        }
        c = 0;
      }
    }
  }
  gsync<GS>();
  for (int i = t; i < 3 * Ne; i += GS) posg[i] = pos[i];
  for (int i = t; i < S.nB; i += GS) Bg[i] = B[i];
  if (t == 0) {
    P.nacc[w] += nacc;
    P.nrej[w] += nrej;
    if (*flag) atomicAdd(&P.counters[0], 1ull);
    if (nref) atomicAdd(&P.counters[1], (unsigned long long)nref);
  }
  gsync<GS>();
}

template <typename T, int GS, bool JB>
__global__ void __launch_bounds__(256) move_kernel(DevSys S, GroupLayout L, MoveParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int gpb = blockDim.x / GS, gid = threadIdx.x / GS;
  const int w = blockIdx.x * gpb + gid;
  if (w >= P.W) return;  // the whole group leaves together; only group barriers are used
  move_walker<T, GS, JB>(S, L, P, smem + gid * L.bytes, w, P.c0, P.sweep0);
}


// ---------------------------------------------------------------- measurement
template <typename T, int GS, bool JB>
__device__ void measure_walker(const DevSys& S, const GroupLayout& L, const MeasParams& P, unsigned char* base,
                               T* acc_s, double* acc_g, int w) {
  const int t = threadIdx.x % GS;
  const int Ne = S.Ne, nup = S.nup, K = S.K, M = S.M;
  double* pos = sm_ptr<double>(base, L.pos);
  float* ph = sm_ptr<float>(base, L.ph);
  float* pl = sm_ptr<float>(base, L.pl);
  double* Bd = sm_ptr<double>(base, L.Bd);
  T* Bt = sm_ptr<T>(base, L.Bt);
  T* Pm = sm_ptr<T>(base, L.P);
  T* Q = sm_ptr<T>(base, L.Q);
  T* Jg = sm_ptr<T>(base, L.Jg);
  T* Jl = sm_ptr<T>(base, L.Jl);
  T* gd = sm_ptr<T>(base, L.gd);
  T* ao = sm_ptr<T>(base, L.ao);
  T* frc = sm_ptr<T>(base, L.frc);  // [0,3K) d ln Psi/dR, [3K,6K) dE_L/dR
  T* Ow = sm_ptr<T>(base, L.Ow);
  T* D = sm_ptr<T>(base, L.D);
  int* piv = sm_ptr<int>(base, L.piv);
  double* f = sm_ptr<double>(base, L.f);
  double* red = sm_ptr<double>(base, L.red);
  int* flag = sm_ptr<int>(base, L.scal);
  double* la = sm_ptr<double>(base, L.scal + 8);
  double* sgn = sm_ptr<double>(base, L.scal + 16);
  const bool want_dC = P.dELdC != nullptr;

  load_positions<GS>(P.pos + (size_t)w * 3 * Ne, 3 * Ne, pos, ph, pl);
  for (int i = t; i < 6 * K; i += GS) frc[i] = T(0);
  if (t == 0) {
    *flag = 0;
    *la = 0.0;
    *sgn = 1.0;
  }
  gsync<GS>();

  // Jastrow gradient/Laplacian per electron, Jastrow value and potentials. The 1/r parts of -1/2 lap J
  // per pair and per nucleus are taken together with the Coulomb terms they cancel at coalescence, in
  // forms without that cancellation: with q = 1/(1 + F r), -1/2 (2 chi'/r) - Z/r = -Z F q (q + 1) for
  // chi = -Z r q, and per electron of a pair with u = a r q, -1/2 (2 u'/r) + 1/(2 r) = (1/2 - a)/r +
  // a F q (q + 1) (exponential form: (1/2 - a)/r - a expm1(-F r)/r); jl keeps u'' and chi''.
  double vs[3] = {0.0, 0.0, 0.0};  // pair terms, nucleus terms, J
  for (int e = t; e < Ne; e += GS) {
    T jg0 = 0, jg1 = 0, jg2 = 0, jl = 0;
    const bool up = e < nup;
    for (int j = 0; j < Ne; ++j) {
      if (j == e) continue;
      const T dx = edisp<T>(pos, ph, pl, e, j, 0), dy = edisp<T>(pos, ph, pl, e, j, 1),
              dz = edisp<T>(pos, ph, pl, e, j, 2);
      const T r = dsqrt<T>(dx * dx + dy * dy + dz * dz), ri = T(1) / r;
      if (S.J2) {
        const bool par = (j < nup) == up;
        const T a = jas_a<T>(S, par), F = jas_F<T>(S, par);
        T h, h1, h2, reg;
        if (!S.j2exp) {
          const T q = T(1) / (T(1) + F * r), q2 = q * q;
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
        jg0 += gr * dx;
        jg1 += gr * dy;
        jg2 += gr * dz;
        jl += h2;
        vs[0] += (double)((T(0.5) - a) * ri + reg);
        if (j > e) vs[2] += (double)h;
      } else {
        vs[0] += (double)(T(0.5) * ri);
      }
    }
    const EPos pe = make_epos(pos + 3 * e);
    for (int I = 0; I < K; ++I) {
      T dd[3];
      disp_nuc<T>(S, pe, I, dd);
      const T dx = dd[0], dy = dd[1], dz = dd[2];
      const T r = dsqrt<T>(dx * dx + dy * dy + dz * dz), ri = T(1) / r;
      const T Z = nuc_Z<T>(S, I);
      if (S.J1) {
        const T b = jas_b<T>(S), q = T(1) / (T(1) + b * r), q2 = q * q;
        const T gr = -Z * q2 * ri;  // chi'/r
        jg0 += gr * dx;
        jg1 += gr * dy;
        jg2 += gr * dz;
        jl += T(2) * Z * b * q2 * q;  // chi''
        vs[1] -= (double)(Z * b * q * (q + T(1)));
        vs[2] -= (double)(Z * r * q);
      } else {
        vs[1] -= (double)(Z * ri);
      }
    }
    Jg[3 * e] = jg0;
    Jg[3 * e + 1] = jg1;
    Jg[3 * e + 2] = jg2;
    Jl[e] = jl;
  }
  gsync<GS>();

  // AO-expanded Jastrow terms (Eqs. onebody_J_inhom, threebody_jas). Work space (free from here to
  // pass 1 and after pass 3): inputs of the products with Xi [2 jch][MJp] (jch electrons at a time),
  // their outputs [2 jch][MJ], t0 = xi + Xi s, s (later sum_e w_e), P, and the per-function force
  // shares [jng][6][MJ]. The per-electron loops run in jng subgroups of whole warps, each covering
  // every Jastrow-basis shell for its own electrons.
  const int MJ = JB ? S.MJ : 0, MJp = S.MJp, jch = L.jch, jng = L.jng > 0 ? L.jng : 1;
  T* jin = MJ ? sm_ptr<T>(base, L.jw) : nullptr;
  T* jout = jin + 2 * jch * MJp;
  T* jt0 = jout + 2 * jch * MJ;
  T* js = jt0 + MJ;
  T* jP = js + MJ;
  T* jfa = jP + MJ;
  const int jgsz = GS / jng, jg = t / jgsz, jt = t - jg * jgsz;
  if (MJ) {
    jas_refresh_t0_sub<T, GS>(S, pos, jng, jin, js, jt0);  // the input rows hold the partial sums meanwhile
    if (MJp > MJ)  // row padding of the inputs (the staging writes mu < MJ)
      for (int q = t; q < 2 * jch * (MJp - MJ); q += GS) jin[(q / (MJp - MJ)) * MJp + MJ + q % (MJp - MJ)] = T(0);
    const T* xi = jas_xi<T>(S);
    // with u_e = Xi psi^J(r_e) and t_e = t0 - u_e: grad_e J += sum_mu t_e grad psi^J, lap_e J +=
    // sum_mu t_e lap psi^J, J += sum_e psi^J(r_e) . (xi + t_e) / 2
    for (int c0 = 0; c0 < Ne; c0 += jch) {
      const int nc = Ne - c0 < jch ? Ne - c0 : jch;
      for (int q = t; q < nc * S.nJs; q += GS) {
        const int r = q / S.nJs, sh = q - r * S.nJs;
        jas_shell<T, 0>(S, sh, make_epos(pos + 3 * (c0 + r)), [&](int mu, const T* v) { jin[r * MJp + mu] = v[0]; });
      }
      gsync<GS>();
      jas_block<T, GS>(S, jin, nc, jout, MJ);
      gsync<GS>();
      for (int r0 = 0; r0 < nc; r0 += jng) {
        const int r = r0 + jg, e = c0 + r;
        T a[4] = {T(0), T(0), T(0), T(0)};
        if (r < nc)
          for (int sh = jt; sh < S.nJs; sh += jgsz)
            jas_shell<T, 1>(S, sh, make_epos(pos + 3 * e), [&](int mu, const T* v) {
              const T te = jt0[mu] - jout[r * MJ + mu];
              a[0] += v[1] * te;
              a[1] += v[2] * te;
              a[2] += v[3] * te;
              a[3] += v[4] * te;
              vs[2] += 0.5 * (double)(v[0] * (__ldg(xi + mu) + te));
            });
#pragma unroll
        for (int k = 0; k < 4; ++k) a[k] = warp_sum(a[k]);  // a warp belongs to one subgroup
        if ((t & 31) == 0 && r < nc) {
#pragma unroll
          for (int k = 0; k < 3; ++k) atomicAdd(&Jg[3 * e + k], a[k]);
          atomicAdd(&Jl[e], a[3]);
        }
      }
      gsync<GS>();
    }
  }
  group_sum<GS, 3>(vs, red);

  // Pass 1: Slater matrices (T) and their FP64 inverses. In FP64 mode Bt is Bd (both spin
  // blocks); in mixed mode Bd holds one block at a time and each inverse is rounded into Bt.
  for (int sg = 0; sg < 2; ++sg) {
    const int n = sg == 0 ? nup : S.ndn;
    if (n == 0) continue;
    const int off = sg == 0 ? 0 : nup * nup;
    double* A = sizeof(T) == 8 ? Bd + off : Bd;
    build_slater<T, GS, true>(S, pos, sg, A, ao, L.ao_rows);
    gj_inverse<GS>(A, n, piv, f, flag, la, sgn, P.logpsi != nullptr);
    if constexpr (sizeof(T) != 8) {
      for (int i = t; i < n * n; i += GS) Bt[off + i] = (T)A[i];
      gsync<GS>();
    }
  }

  // Reweighting factor |Psi / Psi_G|^2 = 1 / g^2 of a guided chain, from the fresh inverses;
  // every walker sum below carries it (the sample count included)
  double wt = 1.0;
  if (P.eps > 0.0) {
    const double g = fmax(1.0, P.eps * sqrt(inverse_frob2<T, GS>(S, Bt, red)));
    wt = 1.0 / (g * g);
  }

  // Pass 2: rows of P = lap(phi) + 2 grad J . grad(phi), a few electrons at a time. P is linear in
  // C, so each electron needs one AO row, lap psi_mu + 2 grad J_e . grad psi_mu, and one row of the
  // contraction with C. Kinetic term of electron e: -1/2 (sum_i P_ei B_ie + lap J_e + |grad J_e|^2).
  // (The determinant drift sum_i grad phi_i(r_e) B_ie is summed in pass 3, from the AO gradients
  // that the nuclear derivatives need.)
  double ekin = 0.0;  // this thread's share
  {
    const int ns = S.nshell;
    for (int sg = 0; sg < 2; ++sg) {
      const int n = sg == 0 ? nup : S.ndn;
      if (n == 0) continue;
      const int e0 = sg == 0 ? 0 : nup, off = sg == 0 ? 0 : nup * nup;
      const T* Bs = Bt + off;
      const T* C = coefC<T>(S, sg);
      const int ng = GS >= n ? GS / n : 1;
      const int ch = 4 * L.p2_chunk < 8 * ng ? 4 * L.p2_chunk : 8 * ng;  // one AO row each, at most 8 rows per thread
      for (int c0 = 0; c0 < n; c0 += ch) {
        const int nc = n - c0 < ch ? n - c0 : ch;
        for (int q = t; q < nc * ns; q += GS) {  // (electron, shell) pairs
          const int r = q / ns, sh = q - r * ns, e = e0 + c0 + r;
          shell_point<T, kAoLevelP, true>(S, make_epos(pos + 3 * e), sh, ao + r * M, 0, Jg + 3 * e);
        }
        gsync<GS>();
        orbital_block<T, GS>(ao, nc, C, M, n, Pm + off + c0 * n, n);
        gsync<GS>();
        if (t < nc) {
          const int el = c0 + t, e = e0 + el;
          const T* pr = Pm + off + el * n;
          double v = 0.0;
          for (int i = 0; i < n; ++i) v += (double)(pr[i] * Bs[i * n + el]);
          const double j0 = (double)Jg[3 * e], j1 = (double)Jg[3 * e + 1], j2 = (double)Jg[3 * e + 2];
          ekin += -0.5 * (v + (double)Jl[e] + j0 * j0 + j1 * j1 + j2 * j2);
        }
      }
    }
    double ek[1] = {ekin};
    group_sum<GS, 1>(ek, red);
    ekin = ek[0];
  }
  const double EL = ekin + vs[0] + vs[1] + S.Vnn;
  const double cw = EL - P.e_ref;

  // Pass 3, per spin: X = B P B (adjoint weight of A), Y = C X^T and C B back-projected
  // per AO; nuclear derivatives from the recomputed AO gradient, Hessian and gradient of
  // the Laplacian; O_{mu i} = sum_e psi_mu(r_e) B_ie.
  const int nO = M * (nup + S.ndn);
  // mixed accumulate with tensor-core O sums: AO values are staged as bf16 rows [Mf][8] (in place of O)
  const bool tcs = sizeof(T) == 4 && P.phiT[0] != nullptr;
  __nv_bfloat16* stg = reinterpret_cast<__nv_bfloat16*>(base + L.Ow);
  T* fa = sm_ptr<T>(base, L.fa);  // [6][M]: AO mu's share of the nuclear derivatives, owned by mu's thread
  for (int i = t; i < 6 * M; i += GS) fa[i] = T(0);
  // determinant drift grad_e D / D = sum_mu grad psi_mu(r_e) (C B)_{mu e}, summed with the AO terms below
  for (int i = t; i < 3 * Ne; i += GS) gd[i] = T(0);
  // space warp: the electron derivatives of E_L are wanted (walker sums or outputs)
  const bool warp = S.swct || P.dEL_dr || P.dEL_sw || P.dlnpsi_sw;
  T* er = sm_ptr<T>(base, L.ew);  // [3 Ne]: orbital part of dE_L/dr_e, then all of it (may share f)
  if (warp)
    for (int i = t; i < 3 * Ne; i += GS) er[i] = T(0);
  for (int sg = 0; sg < 2; ++sg) {
    const int n = sg == 0 ? nup : S.ndn;
    if (n == 0) continue;
    const int e0 = sg == 0 ? 0 : nup, off = sg == 0 ? 0 : nup * nup, ooff = sg == 0 ? 0 : M * nup;
    const T* Bs = Bt + off;
    T* Ps = Pm + off;
    const T* CT = coefCT<T>(S, sg);
    for (int idx = t; idx < n * n; idx += GS) {  // Q = B P
      const int i = idx / n, j = idx - i * n;
      T v = 0;
      for (int e = 0; e < n; ++e) v += Bs[i * n + e] * Ps[e * n + j];
      Q[idx] = v;
    }
    if (tcs) {  // the AO-value staging rows start empty: slots of absent electrons stay zero
      for (int mu = t; mu < P.Mf; mu += GS) *reinterpret_cast<uint4*>(stg + 8 * mu) = make_uint4(0, 0, 0, 0);
    } else {
      for (int idx = t; idx < M * n; idx += GS) {
        Ow[idx] = T(0);
        if (want_dC) D[idx] = T(0);
      }
    }
    gsync<GS>();
    for (int idx = t; idx < n * n; idx += GS) {  // X[e][i] = (B P B)_{i e}, over P
      const int e = idx / n, i = idx - e * n;
      T v = 0;
      for (int j = 0; j < n; ++j) v += Q[i * n + j] * Bs[j * n + e];
      Ps[idx] = v;
    }
    gsync<GS>();
    // one or two electrons per step (L.p3_chunk): their level-2 AO rows over (electron, shell) pairs,
    // then each AO's thread takes the electrons in order, sharing every coefficient load
    for (int el = 0; el < n; el += L.p3_chunk) {
      const int nr = n - el < L.p3_chunk ? n - el : L.p3_chunk;
      for (int q = t; q < nr * S.nshell; q += GS) {
        const int r = q / S.nshell, sh = q - r * S.nshell;
        shell_point<T, 2, true>(S, make_epos(pos + 3 * (e0 + el + r)), sh, ao + r * 14 * M, M);
      }
      gsync<GS>();
      T ce[2][3] = {{T(0), T(0), T(0)}, {T(0), T(0), T(0)}};  // this thread's share of sum_mu of the AO terms
      T gp[2][3] = {{T(0), T(0), T(0)}, {T(0), T(0), T(0)}};  // and of the determinant drift
      for (int mu = t; mu < M; mu += GS) {
        T yA[2] = {T(0), T(0)}, yL[2] = {T(0), T(0)};
        for (int i = 0; i < n; ++i) {
          const T cmi = __ldg(CT + i * M + mu);
          yA[0] += cmi * Ps[el * n + i];
          yL[0] += cmi * Bs[i * n + el];
          if (nr > 1) {
            yA[1] += cmi * Ps[(el + 1) * n + i];
            yL[1] += cmi * Bs[i * n + el + 1];
          }
        }
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          if (r >= nr) break;
          const int e = e0 + el + r;
          const T* a = ao + r * 14 * M;
          const T j0 = Jg[3 * e], j1 = Jg[3 * e + 1], j2 = Jg[3 * e + 2];
          const T v = a[mu], g0 = a[M + mu], g1 = a[2 * M + mu], g2 = a[3 * M + mu], lp = a[4 * M + mu];
          const T hxx = a[5 * M + mu], hyy = a[6 * M + mu], hzz = a[7 * M + mu];
          const T hxy = a[8 * M + mu], hxz = a[9 * M + mu], hyz = a[10 * M + mu];
          const T l0 = a[11 * M + mu], l1 = a[12 * M + mu], l2 = a[13 * M + mu];
          const T hj0 = hxx * j0 + hxy * j1 + hxz * j2;
          const T hj1 = hxy * j0 + hyy * j1 + hyz * j2;
          const T hj2 = hxz * j0 + hyz * j1 + hzz * j2;
          const T ya = r == 0 ? yA[0] : yA[1], yl = r == 0 ? yL[0] : yL[1];
          const T gy0 = g0 * yl, gy1 = g1 * yl, gy2 = g2 * yl;
          fa[0 * M + mu] -= gy0;
          fa[1 * M + mu] -= gy1;
          fa[2 * M + mu] -= gy2;
          gp[r][0] += gy0;
          gp[r][1] += gy1;
          gp[r][2] += gy2;
          const T c0 = T(-0.5) * (g0 * ya - yl * (l0 + T(2) * hj0));
          const T c1 = T(-0.5) * (g1 * ya - yl * (l1 + T(2) * hj1));
          const T c2 = T(-0.5) * (g2 * ya - yl * (l2 + T(2) * hj2));
          fa[3 * M + mu] += c0;
          fa[4 * M + mu] += c1;
          fa[5 * M + mu] += c2;
          ce[r][0] += c0;
          ce[r][1] += c1;
          ce[r][2] += c2;
          if (tcs) {
            stg[8 * mu + ((el + r) & 7)] = __float2bfloat16_rn((float)v);
          } else {
            const T tdc = lp + T(2) * (j0 * g0 + j1 * g1 + j2 * g2);
            for (int i = 0; i < n; ++i) {
              const T b = Bs[i * n + el + r];
              Ow[mu * n + i] += v * b;
              if (want_dC) D[mu * n + i] += b * tdc;
            }
          }
        }
      }
      const int ell = el + nr - 1;  // the step's last electron (steps start on even electrons)
      if (tcs && ((ell & 7) == 7 || ell == n - 1)) {
        // eight electron slots of psi_mu: one 16-byte row of the K-major PhiT tile (chunk ell / 16);
        // each staging row is written and flushed by the same thread
        __nv_bfloat16* dst = reinterpret_cast<__nv_bfloat16*>(P.phiT[sg]) + ((size_t)w * P.nch + (ell >> 4)) * P.Mf * 16;
        for (int mu = t; mu < M; mu += GS) {
          uint4* row = reinterpret_cast<uint4*>(stg + 8 * mu);
          *reinterpret_cast<uint4*>(dst + tc_tile_index(mu, ell & 8)) = *row;
          *row = make_uint4(0, 0, 0, 0);
        }
      }
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        if (r >= nr) break;
#pragma unroll
        for (int k = 0; k < 3; ++k) gp[r][k] = warp_sum(gp[r][k]);
        if ((t & 31) == 0)
#pragma unroll
          for (int k = 0; k < 3; ++k) atomicAdd(&gd[3 * (e0 + el + r) + k], gp[r][k]);
      }
      if (warp) {  // an AO moves with its nucleus as -d/dr_e: the same terms, summed over every AO
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          if (r >= nr) break;
#pragma unroll
          for (int k = 0; k < 3; ++k) ce[r][k] = warp_sum(ce[r][k]);
          if ((t & 31) == 0)
#pragma unroll
            for (int k = 0; k < 3; ++k) atomicAdd(&er[3 * (e0 + el + r) + k], ce[r][k]);
        }
      }
      gsync<GS>();
      // e-n Jastrow and V_en terms, one nucleus per thread, the step's electrons in order
      for (int I = t; I < K; I += GS) {
        for (int r = 0; r < nr; ++r) {
          const int e = e0 + el + r;
          const EPos pe = make_epos(pos + 3 * e);
          T sd[3];
          disp_nuc<T>(S, pe, I, sd);
          const T sx = sd[0], sy = sd[1], sz = sd[2];
          const T rr = dsqrt<T>(sx * sx + sy * sy + sz * sz), ri = T(1) / rr;
          const T Z = nuc_Z<T>(S, I);
          const T sv[3] = {sx, sy, sz};
          const T nn[3] = {sx * ri, sy * ri, sz * ri};
          const T ven = -Z * ri * ri * ri;
          for (int d = 0; d < 3; ++d) frc[3 * K + 3 * I + d] += ven * sv[d];
          if (S.J1) {
            const Rad3<T> c = pade<T>(-Z, jas_b<T>(S), rr);
            const T gsum[3] = {gd[3 * e] + Jg[3 * e], gd[3 * e + 1] + Jg[3 * e + 1], gd[3 * e + 2] + Jg[3 * e + 2]};
            const T dl = c.h3 + T(2) * c.h2 * ri - T(2) * c.h1 * ri * ri;
            for (int d = 0; d < 3; ++d) {
              T hs = 0;
              for (int cc = 0; cc < 3; ++cc)
                hs += (c.h2 * nn[d] * nn[cc] + c.h1 * ri * ((d == cc ? T(1) : T(0)) - nn[d] * nn[cc])) * gsum[cc];
              frc[3 * I + d] += -c.h1 * nn[d];
              frc[3 * K + 3 * I + d] += hs + T(0.5) * dl * nn[d];
            }
          }
        }
      }
      gsync<GS>();
    }
    if (tcs) {
      // Y rows of the tensor-core sums: wt B_{j, el} (j < n) and wt (E_L - E_ref) B_{j - n, el},
      // eight electron slots per 16-byte store
      __nv_bfloat16* y = reinterpret_cast<__nv_bfloat16*>(P.yT[sg]) + (size_t)w * P.nch * P.Nf * 16;
      for (int q = t; q < 2 * n * P.nch * 2; q += GS) {
        const int j = q / (2 * P.nch), r = q - j * 2 * P.nch, c = r >> 1, h = r & 1;
        const int i = j < n ? j : j - n;
        const float f = (float)(j < n ? wt : wt * cw);
        __align__(16) __nv_bfloat16 v8[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int e8 = 16 * c + 8 * h + k;
          v8[k] = __float2bfloat16_rn(e8 < n ? f * (float)Bs[i * n + e8] : 0.f);
        }
        *reinterpret_cast<uint4*>(y + (size_t)c * P.Nf * 16 + tc_tile_index(j, 8 * h)) =
            *reinterpret_cast<const uint4*>(v8);
      }
    }
    // this spin's O (and explicit dE_L/dC): outputs and walker sums
    const int oo = 3 + 9 * K;
    for (int idx = t; idx < (tcs ? 0 : M * n); idx += GS) {
      const T o = Ow[idx];
      if (P.O) P.O[(size_t)w * nO + ooff + idx] = (double)o;
      if (want_dC) {
        const int mu = idx / n, i = idx - mu * n;
        T q = 0;
        for (int j = 0; j < n; ++j) q += Ow[mu * n + j] * Q[i * n + j];
        P.dELdC[(size_t)w * nO + ooff + idx] = -0.5 * ((double)D[idx] - (double)q);
      }
      if (acc_s) {
        atomicAdd(&acc_s[oo + ooff + idx], (T)wt * o);
        atomicAdd(&acc_s[oo + nO + ooff + idx], (T)(wt * cw) * o);
      } else if (acc_g) {
        acc_g[oo + ooff + idx] += wt * (double)o;
        acc_g[oo + nO + ooff + idx] += wt * cw * (double)o;
      }
    }
    gsync<GS>();
  }

  // AO-expanded Jastrow terms: their shares of d ln Psi/dR, dE_L/dR and dE_L/dr_e. With
  // h_e = grad ln D + grad J at r_e, w_e = h_e . grad psi^J(r_e) + lap psi^J(r_e) / 2, p_e = Xi w_e and
  // P = sum_e p_e, function mu of nucleus a at electron e contributes -d_d psi^J_mu t_{e mu} to
  // d ln Psi/dR_{a,d}, and c = (h_e . d_d grad psi^J_mu + d_d lap psi^J_mu / 2) t_{e mu} +
  // (P - p_e)_mu d_d psi^J_mu to dE_L/dR_{a,d} and -c to dE_L/dr_{e,d}.
  if (MJ) {
    const int nJs = S.nJs;
    jas_refresh_t0_sub<T, GS>(S, pos, jng, jin, js, jt0);  // the work space may share the O buffer of pass 3
    if (MJp > MJ)
      for (int q = t; q < 2 * jch * (MJp - MJ); q += GS) jin[(q / (MJp - MJ)) * MJp + MJ + q % (MJp - MJ)] = T(0);
    for (int i = t; i < 6 * jng * MJ; i += GS) jfa[i] = T(0);
    T* wpart = jout;  // sum_e w_e by subgroup (electrons e = g, g + jng, ...) before the products
    for (int sh = jt; sh < nJs; sh += jgsz) {
      const int4 d4 = __ldg(S.jshell + sh);
      for (int m = 0; m < 2 * d4.y + 1; ++m) wpart[jg * MJ + d4.w + m] = T(0);
      for (int e = jg; e < Ne; e += jng) {
        const T h0 = gd[3 * e] + Jg[3 * e], h1 = gd[3 * e + 1] + Jg[3 * e + 1], h2 = gd[3 * e + 2] + Jg[3 * e + 2];
        jas_shell<T, 1>(S, sh, make_epos(pos + 3 * e), [&](int mu, const T* v) {
          wpart[jg * MJ + mu] += h0 * v[1] + h1 * v[2] + h2 * v[3] + T(0.5) * v[4];
        });
      }
    }
    gsync<GS>();
    for (int mu = t; mu < MJ; mu += GS) {
      T v = T(0);
      for (int k = 0; k < jng; ++k) v += wpart[k * MJ + mu];
      js[mu] = v;
    }
    gsync<GS>();
    jas_matvec<T, GS>(S, js, nullptr, jP);
    gsync<GS>();
    for (int c0 = 0; c0 < Ne; c0 += jch) {
      const int nc = Ne - c0 < jch ? Ne - c0 : jch;
      for (int q = t; q < nc * nJs; q += GS) {  // rows: psi^J at the chunk's electrons, then their w_e
        const int r = q / nJs, sh = q - r * nJs, e = c0 + r;
        const T h0 = gd[3 * e] + Jg[3 * e], h1 = gd[3 * e + 1] + Jg[3 * e + 1], h2 = gd[3 * e + 2] + Jg[3 * e + 2];
        jas_shell<T, 1>(S, sh, make_epos(pos + 3 * e), [&](int mu, const T* v) {
          jin[r * MJp + mu] = v[0];
          jin[(nc + r) * MJp + mu] = h0 * v[1] + h1 * v[2] + h2 * v[3] + T(0.5) * v[4];
        });
      }
      gsync<GS>();
      jas_block<T, GS>(S, jin, 2 * nc, jout, MJ);  // u_e, then p_e
      gsync<GS>();
      for (int r0 = 0; r0 < nc; r0 += jng) {
        const int r = r0 + jg, e = c0 + r;
        T ce[3] = {T(0), T(0), T(0)};
        if (r < nc) {
          const T h[3] = {gd[3 * e] + Jg[3 * e], gd[3 * e + 1] + Jg[3 * e + 1], gd[3 * e + 2] + Jg[3 * e + 2]};
          T* fa_g = jfa + jg * 6 * MJ;
          for (int sh = jt; sh < nJs; sh += jgsz)
            jas_shell<T, 2>(S, sh, make_epos(pos + 3 * e), [&](int mu, const T* v) {
              const T te = jt0[mu] - jout[r * MJ + mu];
              const T pd = jP[mu] - jout[(nc + r) * MJ + mu];
#pragma unroll
              for (int d = 0; d < 3; ++d) {
                T hh = T(0);
#pragma unroll
                for (int c = 0; c < 3; ++c) hh += h[c] * v[jas_hidx(d, c)];
                const T cd = (hh + T(0.5) * v[11 + d]) * te + pd * v[1 + d];
                fa_g[d * MJ + mu] -= v[1 + d] * te;
                fa_g[(3 + d) * MJ + mu] += cd;
                ce[d] += cd;
              }
            });
        }
        if (warp) {
#pragma unroll
          for (int k = 0; k < 3; ++k) ce[k] = warp_sum(ce[k]);
          if ((t & 31) == 0 && r < nc)
#pragma unroll
            for (int k = 0; k < 3; ++k) atomicAdd(&er[3 * e + k], ce[k]);
        }
      }
      gsync<GS>();
    }
    for (int mu = t; mu < MJ; mu += GS) {
      const int I = __ldg(S.jcenter + mu);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        T sl = T(0), se = T(0);
        for (int k = 0; k < jng; ++k) {
          sl += jfa[(k * 6 + d) * MJ + mu];
          se += jfa[(k * 6 + 3 + d) * MJ + mu];
        }
        atomicAdd(&frc[3 * I + d], sl);
        atomicAdd(&frc[3 * K + 3 * I + d], se);
      }
    }
  }

  // the AO shares of the nuclear derivatives, onto their centres
  for (int mu = t; mu < M; mu += GS) {
    const int I = __ldg(S.ao_center + mu);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      atomicAdd(&frc[3 * I + d], fa[d * M + mu]);
      atomicAdd(&frc[3 * K + 3 * I + d], fa[(3 + d) * M + mu]);
    }
  }
  gsync<GS>();

  // Space-warp force vectors (force expression with omega_a(r) = kappa(|r - R_a|) /
  // sum_b kappa(|r - R_b|), kappa(r) = r^-4): dE_L/dr_e, then per nucleus a
  //   dE_L^sw/dR_a = dE_L/dR_a + sum_e omega_a(r_e) dE_L/dr_e,
  //   d ln Psi^sw/dR_a = d ln Psi/dR_a + sum_e [omega_a(r_e) d ln Psi/dr_e + 1/2 grad omega_a(r_e)].
  if (warp) {
    T* ks = ao;            // [Ne] sum_b kappa_b(r_e) (the AO buffer is free after pass 3)
    T* gks = ao + Ne;      // [3 Ne] sum_b grad kappa_b(r_e)
    for (int e = t; e < Ne; e += GS) {
      const bool up = e < nup;
      const T ge[3] = {gd[3 * e] + Jg[3 * e], gd[3 * e + 1] + Jg[3 * e + 1], gd[3 * e + 2] + Jg[3 * e + 2]};
      T dr[3] = {-er[3 * e], -er[3 * e + 1], -er[3 * e + 2]};
      for (int j = 0; j < Ne; ++j) {  // e-e Jastrow pair terms and V_ee
        if (j == e) continue;
        const T sv[3] = {edisp<T>(pos, ph, pl, e, j, 0), edisp<T>(pos, ph, pl, e, j, 1), edisp<T>(pos, ph, pl, e, j, 2)};
        const T r = dsqrt<T>(sv[0] * sv[0] + sv[1] * sv[1] + sv[2] * sv[2]), ri = T(1) / r;
        const T ri3 = ri * ri * ri;
#pragma unroll
        for (int k = 0; k < 3; ++k) dr[k] -= sv[k] * ri3;
        if (S.J2) {
          const bool par = (j < nup) == up;
          const Rad3<T> u = pair_rad<T>(S, par, r);
          const T nn[3] = {sv[0] * ri, sv[1] * ri, sv[2] * ri};
          const T dl = u.h3 + T(2) * u.h2 * ri - T(2) * u.h1 * ri * ri;
          const T vec[3] = {ge[0] - gd[3 * j] - Jg[3 * j], ge[1] - gd[3 * j + 1] - Jg[3 * j + 1],
                            ge[2] - gd[3 * j + 2] - Jg[3 * j + 2]};
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
      const EPos pe = make_epos(pos + 3 * e);
      T k0 = T(0), gk[3] = {T(0), T(0), T(0)};
      for (int I = 0; I < K; ++I) {  // e-n Jastrow, V_en and the warp weights
        T sv[3];
        disp_nuc<T>(S, pe, I, sv);
        const T r2 = sv[0] * sv[0] + sv[1] * sv[1] + sv[2] * sv[2];
        const T r = dsqrt<T>(r2), ri = T(1) / r;
        const T Z = nuc_Z<T>(S, I);
#pragma unroll
        for (int k = 0; k < 3; ++k) dr[k] += Z * sv[k] * ri * ri * ri;
        if (S.J1) {
          const Rad3<T> c = pade<T>(-Z, jas_b<T>(S), r);
          const T nn[3] = {sv[0] * ri, sv[1] * ri, sv[2] * ri};
          const T dl = c.h3 + T(2) * c.h2 * ri - T(2) * c.h1 * ri * ri;
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            T hs = 0;
#pragma unroll
            for (int cc = 0; cc < 3; ++cc)
              hs += (c.h2 * nn[k] * nn[cc] + c.h1 * ri * ((k == cc ? T(1) : T(0)) - nn[k] * nn[cc])) * ge[cc];
            dr[k] -= T(0.5) * dl * nn[k] + hs;
          }
        }
        const T kap = T(1) / (r2 * r2);
        k0 += kap;
#pragma unroll
        for (int k = 0; k < 3; ++k) gk[k] += T(-4) * sv[k] * kap / r2;
      }
      ks[e] = k0;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        gks[3 * e + k] = gk[k];
        er[3 * e + k] = dr[k];
        if (P.dEL_dr) P.dEL_dr[((size_t)w * Ne + e) * 3 + k] = (double)dr[k];
      }
    }
    gsync<GS>();
    const int so = P.swct_off;  // offset of the warped sums in the accumulator (0: none)
    for (int a = t; a < K; a += GS) {
      double sE[3], sL[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        sE[k] = (double)frc[3 * K + 3 * a + k] + __ldg(S.dVnn + 3 * a + k);
        sL[k] = (double)frc[3 * a + k];
      }
      for (int e = 0; e < Ne; ++e) {
        T sv[3];
        disp_nuc<T>(S, make_epos(pos + 3 * e), a, sv);
        const T r2 = sv[0] * sv[0] + sv[1] * sv[1] + sv[2] * sv[2];
        const T kap = T(1) / (r2 * r2), kinv = T(1) / ks[e];
        const T om = kap * kinv;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const T gom = (T(-4) * sv[k] * kap / r2 - om * gks[3 * e + k]) * kinv;
          sE[k] += (double)(om * er[3 * e + k]);
          sL[k] += (double)(om * (gd[3 * e + k] + Jg[3 * e + k]) + T(0.5) * gom);
        }
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const int i = 3 * a + k;
        if (P.dEL_sw) P.dEL_sw[(size_t)w * 3 * K + i] = sE[k];
        if (P.dlnpsi_sw) P.dlnpsi_sw[(size_t)w * 3 * K + i] = sL[k];
        if (so > 0) {
          if (acc_s) {
            atomicAdd(&acc_s[so + i], (T)(wt * sE[k]));
            atomicAdd(&acc_s[so + 3 * K + i], (T)(wt * sL[k]));
            atomicAdd(&acc_s[so + 6 * K + i], (T)(wt * cw * sL[k]));
          } else if (acc_g) {
            acc_g[so + i] += wt * sE[k];
            acc_g[so + 3 * K + i] += wt * sL[k];
            acc_g[so + 6 * K + i] += wt * cw * sL[k];
          }
        }
      }
    }
    gsync<GS>();
  }

  // per-walker outputs and scalar / force sums
  for (int i = t; i < 3 * K; i += GS) {
    const double dl = (double)frc[i];
    const double de = (double)frc[3 * K + i] + __ldg(S.dVnn + i);
    if (P.dlnpsi) P.dlnpsi[(size_t)w * 3 * K + i] = dl;
    if (P.dEL) P.dEL[(size_t)w * 3 * K + i] = de;
    if (acc_s) {
      atomicAdd(&acc_s[3 + i], (T)(wt * de));
      atomicAdd(&acc_s[3 + 3 * K + i], (T)(wt * dl));
      atomicAdd(&acc_s[3 + 6 * K + i], (T)(wt * cw * dl));
    } else if (acc_g) {
      acc_g[3 + i] += wt * de;
      acc_g[3 + 3 * K + i] += wt * dl;
      acc_g[3 + 6 * K + i] += wt * cw * dl;
    }
  }
  if (t == 0) {
    if (P.EL) P.EL[w] = EL;
    if (P.logpsi) P.logpsi[w] = *la + vs[2];
    if (acc_s) {
      atomicAdd(&acc_s[0], (T)wt);
      atomicAdd(&acc_s[1], (T)(wt * cw));
      atomicAdd(&acc_s[2], (T)(wt * cw * cw));
    } else if (acc_g) {
      acc_g[0] += wt;
      acc_g[1] += wt * EL;
      acc_g[2] += wt * EL * EL;
    }
    if (*flag) atomicAdd(&P.counters[0], 1ull);
  }
  if (P.Bout) {
    T* Bg = reinterpret_cast<T*>(P.Bout) + (size_t)w * S.nB;
    for (int i = t; i < S.nB; i += GS) Bg[i] = Bt[i];
  }
  gsync<GS>();
}

// CTA c handles walkers [W c / grid, W (c+1) / grid); its groups take them in turn. Walker
// sums go to a CTA shared-memory accumulator (several groups per CTA) or straight to the
// CTA's FP64 slot (one group per CTA), and the slot is only ever touched by its CTA.
// In the shared accumulator, acc[1] and acc[2] hold sums of (E_L - E_ref) and its square;
// they are turned into sums of E_L and E_L^2 when the CTA flushes.
template <typename T, int GS, bool JB>
__global__ void __launch_bounds__(256, 2) measure_kernel(DevSys S, GroupLayout L, MeasParams P, int acc_off) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int gpb = blockDim.x / GS, gid = threadIdx.x / GS;
  unsigned char* base = smem + gid * L.bytes;
  T* acc_s = (P.acc && P.acc_in_smem) ? sm_ptr<T>(smem, acc_off) : nullptr;
  double* acc_g = (P.acc && !P.acc_in_smem) ? P.acc + (size_t)blockIdx.x * P.accL : nullptr;
  // with the tensor-core sums the O range [3 + 9K, 3 + 9K + 2 nO) of the accumulator stays zero and is
  // skipped: entry k < oskip is entry k, the rest entry k + olen
  const int olen = (sizeof(T) == 4 && P.phiT[0] != nullptr) ? 2 * S.M * S.Ne : 0, oskip = 3 + 9 * S.K;
  const int accn = P.accL - olen;
  if (acc_s) {
    for (int k = threadIdx.x; k < accn; k += blockDim.x) acc_s[k < oskip ? k : k + olen] = T(0);
    __syncthreads();
  }
  const long long w0 = (long long)P.W * blockIdx.x / gridDim.x;
  const long long w1 = (long long)P.W * (blockIdx.x + 1) / gridDim.x;
  for (long long w = w0 + gid; w < w1; w += gpb) measure_walker<T, GS, JB>(S, L, P, base, acc_s, acc_g, (int)w);
  if (acc_s) {
    __syncthreads();
    double* slot = P.acc + (size_t)blockIdx.x * P.accL;
    const double cnt = (double)acc_s[0];
    for (int k = threadIdx.x; k < accn; k += blockDim.x) {
      const int i = k < oskip ? k : k + olen;
      double v = (double)acc_s[i];
      if (i == 2) v = v + 2.0 * P.e_ref * (double)acc_s[1] + cnt * P.e_ref * P.e_ref;
      if (i == 1) v = v + cnt * P.e_ref;
      slot[i] += v;
    }
  }
}

// ---------------------------------------------------------------- proposals of a walker-group sweep
// Every electron moves once per sweep, from its position at the start of the sweep, so its proposal r'_e (Philox
// counter (wid, sweep, e, 0)), its acceptance uniform (counter (wid, sweep, e, 1)), the orbital row of its spin at
// r'_e and the change of the electron-nucleus Jastrow terms do not depend on the sweep's earlier moves and are
// formed here for every (walker, electron) at once (App. A, MCMC): one warp per pair, the AO values at r'_e in the
// warp's shared buffer. The arithmetic is that of move_walker's own path (orbital_half, en_change_warp), so the
// chain is the same bit for bit either way.
template <typename T>
__global__ void __launch_bounds__(256) propose_group(DevSys S, GroupProposeParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  T* ao = reinterpret_cast<T*>(smem) + (size_t)warp * ((S.M + 3) / 4 * 4);
  const int Ne = S.Ne, nup = S.nup, mh = S.M / 2;
  const long long nitem = (long long)P.W * Ne;
  for (long long it = (long long)blockIdx.x * nwarps + warp; it < nitem; it += (long long)gridDim.x * nwarps) {
    const int w = (int)(it / Ne), e = (int)(it - (long long)w * Ne);
    const uint64_t wid = P.wid0 + (uint64_t)w, sweep = P.clk ? P.clk->sweep : P.sweep;
    uint64_t r[4] = {wid, sweep, (uint64_t)e, 0};
    philox4x64_10(r, P.k0, P.k1);
    double xi[3];
    normals3(r, xi, T(0));
    double po3[3], rn[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      po3[k] = P.pos[(size_t)it * 3 + k];
      rn[k] = po3[k] + P.sigma * xi[k];
    }
    const EPos pn = make_epos(rn);
    const EPos po = make_epos(po3);
    ao_point<T, 32, 0, false>(S, pn, ao, 0);
    __syncwarp();
    const int sg = e < nup ? 0 : 1, n = sg == 0 ? nup : S.ndn;
    const T* C = coefC<T>(S, sg);
    T* prow = reinterpret_cast<T*>(P.prow) + (size_t)it * S.nmax;
    for (int i = lane; i < n; i += 32)
      prow[i] = orbital_half<T>(ao, C, n, i, 0, mh) + orbital_half<T>(ao, C, n, i, mh, S.M);
    const T en = en_change_warp<T>(S, pn, po, lane);
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < 3; ++k) P.prn[(size_t)it * 3 + k] = rn[k];
      reinterpret_cast<T*>(P.pdchi)[it] = en;
      uint64_t r2[4] = {wid, sweep, (uint64_t)e, 1};
      philox4x64_10(r2, P.k0, P.k1);
      P.pu[it] = u01(r2[0]);
    }
    __syncwarp();  // the AO buffer is reused for the warp's next pair
  }
}

template <typename T>
size_t propose_group_smem(const DevSys& S) {
  return (size_t)8 * ((S.M + 3) / 4 * 4) * sizeof(T);
}

template <typename T>
cudaError_t launch_propose_group_impl(const DevSys& S, const GroupProposeParams& P, cudaStream_t st) {
  const long long items = (long long)P.W * S.Ne;
  if (items == 0) return cudaSuccess;
  const int grid = (int)std::min<long long>((items + 7) / 8, 8192);
  propose_group<T><<<grid, 256, propose_group_smem<T>(S), st>>>(S, P);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- launchers
// Instances with the AO-expanded Jastrow terms (JB = true) live in their own translation units.
template <typename T, bool JB>
cudaError_t set_smem_limits_impl() {
  const int lim = 227 * 1024;
  cudaError_t e;
  if (!JB) {
    if ((e = cudaFuncSetAttribute(refresh_kernel<T, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
    if ((e = cudaFuncSetAttribute(refresh_kernel<T, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
    if ((e = cudaFuncSetAttribute(refresh_kernel<T, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
    if ((e = cudaFuncSetAttribute(propose_group<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  }
  if ((e = cudaFuncSetAttribute(move_kernel<T, 32, JB>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(move_kernel<T, 128, JB>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(move_kernel<T, 256, JB>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(measure_kernel<T, 32, JB>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(measure_kernel<T, 128, JB>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(measure_kernel<T, 256, JB>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  return cudaSuccess;
}

template <typename T>
cudaError_t launch_refresh_impl(const DevSys& S, const Launch& lc, const double* pos, void* B, int W,
                                unsigned long long* counters, cudaStream_t st) {
  const dim3 grid(lc.grid), block(lc.GS * lc.groups);
  if (lc.GS == 32)
    refresh_kernel<T, 32><<<grid, block, lc.smem, st>>>(S, lc.L, pos, reinterpret_cast<T*>(B), W, counters);
  else if (lc.GS == 128)
    refresh_kernel<T, 128><<<grid, block, lc.smem, st>>>(S, lc.L, pos, reinterpret_cast<T*>(B), W, counters);
  else if (lc.GS == 256)
    refresh_kernel<T, 256><<<grid, block, lc.smem, st>>>(S, lc.L, pos, reinterpret_cast<T*>(B), W, counters);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

template <typename T, bool JB>
cudaError_t launch_move_impl(const DevSys& S, const Launch& lc, const MoveParams& P, cudaStream_t st) {
  const dim3 grid(lc.grid), block(lc.GS * lc.groups);
  if (lc.GS == 32)
    move_kernel<T, 32, JB><<<grid, block, lc.smem, st>>>(S, lc.L, P);
  else if (lc.GS == 128)
    move_kernel<T, 128, JB><<<grid, block, lc.smem, st>>>(S, lc.L, P);
  else if (lc.GS == 256)
    move_kernel<T, 256, JB><<<grid, block, lc.smem, st>>>(S, lc.L, P);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

template <typename T, bool JB>
cudaError_t launch_measure_impl(const DevSys& S, const Launch& lc, const MeasParams& P, cudaStream_t st) {
  const dim3 grid(lc.grid), block(lc.GS * lc.groups);
  if (lc.GS == 32)
    measure_kernel<T, 32, JB><<<grid, block, lc.smem, st>>>(S, lc.L, P, lc.acc_off);
  else if (lc.GS == 128)
    measure_kernel<T, 128, JB><<<grid, block, lc.smem, st>>>(S, lc.L, P, lc.acc_off);
  else if (lc.GS == 256)
    measure_kernel<T, 256, JB><<<grid, block, lc.smem, st>>>(S, lc.L, P, lc.acc_off);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace vmcf
