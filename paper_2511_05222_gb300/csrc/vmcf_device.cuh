// Device building blocks of the VMC hot path (arXiv:2511.05222, App. A).
//
// Work is organised by walker groups: GS threads (one warp for small electron counts, a
// whole CTA for large ones) cooperate on one walker, with all its per-walker matrices in
// shared memory. T is the arithmetic type of AOs, MOs, Jastrow and adjoint work (double in
// FP64 mode, float in mixed mode); the Slater inversion, the determinant ratio and the walker
// sums are always double.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace vmcf {

// Position (in bf16 elements) of row r, electron slot k (0..15) in one chunk of the tensor-core
// walker-sum tiles: K-major 8-row x 16-byte core matrices without swizzle, slots 8..15 of a row
// group 128 bytes after slots 0..7, the next 8 rows 256 bytes on.
__host__ __device__ __forceinline__ int tc_tile_index(int r, int k) {
  return ((r >> 3) * 2 + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7);
}

constexpr int kMaxPrim = 8;

struct DevSys {
  int K, M, nup, ndn, Ne, nshell, nB, nmax;
  const double* R;       // [K][3]
  const double* Z;       // [K]
  const int4* shell;     // (center, l, nprim, ao0)
  const int4* shgrp;     // runs of consecutive shells with one centre and one l: (first shell, count,
                         // l + 256 if a shell of the run has sharp primitives, center)
  int ngrp;
  const double* alpha;   // [nshell][kMaxPrim]
  const double* coef;    // [nshell][kMaxPrim], normalised contraction coefficients
  const float* alpha_f;
  const float* coef_f;
  const int* ao_center;  // [M]
  const float* Rh;       // [K][3] nuclear positions as float-float pairs (mixed mode)
  const float* Rl;
  const int* sharp;      // [nshell] bit k set: primitive k is sharp (its a r^2 keeps extra precision)
  const float* alpha_lo; // [nshell][kMaxPrim] alpha - (float)alpha, for float-float a r^2
  const double* C[2];    // [M][n_s]
  const float* Cf[2];
  const double* CT[2];   // [n_s][M], the same coefficients transposed
  const float* CfT[2];
  double Fa, Fp, aa, ap, ben;
  float Fa_f, Fp_f, aa_f, ap_f, ben_f;  // the same in float (mixed mode reads these: no conversion per use)
  const float* Zf;                     // [K] nuclear charges in float
  int J1, J2;
  int swct;              // accumulate the space-warp force sums
  int j2exp;             // two-body form: 0 Pade, 1 exponential
  double Vnn;
  const double* dVnn;    // [K][3], derivative of V_nn
  // AO-expanded Jastrow terms over a separate Jastrow basis (nJs = MJ = 0: none):
  // U = sum_e sum_mu xi_mu psi^J_mu(r_e) + sum_{i<j} sum_{mu,nu} Xi_{mu nu} psi^J_mu(r_i) psi^J_nu(r_j)
  int nJs, MJ;           // Jastrow-basis shells and functions
  int MJp;               // MJ rounded up to a multiple of 4 (rows of the row-block products with Xi)
  const int4* jshell;    // (center, l, nprim, index of the shell's first function)
  const double* jalpha;  // [nJs][kMaxPrim]
  const double* jcoef;   // [nJs][kMaxPrim], normalised contraction coefficients
  const float* jalpha_f;
  const float* jcoef_f;
  const int* jcenter;    // [MJ] nucleus of each function
  const double* jxi;     // [MJ] one-body coefficients xi_mu
  const float* jxi_f;
  const double* jXi;     // [MJp][MJ] pair coefficients Xi_{mu nu}, symmetric; rows MJ..MJp-1 are zero
  const float* jXi_f;
  const double* jXr;     // [MJ][MJp] the same with rows padded to MJp (zero), 16-byte aligned rows
  const float* jXr_f;
};

template <typename T> __device__ __forceinline__ const T* coefC(const DevSys& S, int s);
template <> __device__ __forceinline__ const double* coefC<double>(const DevSys& S, int s) { return S.C[s]; }
template <> __device__ __forceinline__ const float* coefC<float>(const DevSys& S, int s) { return S.Cf[s]; }
template <typename T> __device__ __forceinline__ const T* coefCT(const DevSys& S, int s);
template <> __device__ __forceinline__ const double* coefCT<double>(const DevSys& S, int s) { return S.CT[s]; }
template <> __device__ __forceinline__ const float* coefCT<float>(const DevSys& S, int s) { return S.CfT[s]; }

// Jastrow parameters and nuclear charges in the working precision, read from the copy of that type:
// a conversion from double would take the FP64 pipe (a whole warp instruction) at every use.
template <typename T> __device__ __forceinline__ T jas_a(const DevSys& S, bool par) {
  if constexpr (sizeof(T) == 8) return par ? S.ap : S.aa;
  else return par ? S.ap_f : S.aa_f;
}
template <typename T> __device__ __forceinline__ T jas_F(const DevSys& S, bool par) {
  if constexpr (sizeof(T) == 8) return par ? S.Fp : S.Fa;
  else return par ? S.Fp_f : S.Fa_f;
}
template <typename T> __device__ __forceinline__ T jas_b(const DevSys& S) {
  if constexpr (sizeof(T) == 8) return S.ben;
  else return S.ben_f;
}
template <typename T> __device__ __forceinline__ T nuc_Z(const DevSys& S, int I) {
  if constexpr (sizeof(T) == 8) return __ldg(S.Z + I);
  else return __ldg(S.Zf + I);
}

template <typename T> __device__ __forceinline__ T dexp(T x);
template <> __device__ __forceinline__ double dexp<double>(double x) { return exp(x); }
template <> __device__ __forceinline__ float dexp<float>(float x) { return expf(x); }
template <typename T> __device__ __forceinline__ T dsqrt(T x);
template <> __device__ __forceinline__ double dsqrt<double>(double x) { return sqrt(x); }
template <> __device__ __forceinline__ float dsqrt<float>(float x) { return sqrtf(x); }

template <typename T> __device__ __forceinline__ T prim_alpha(const DevSys& S, int s, int k);
template <> __device__ __forceinline__ double prim_alpha<double>(const DevSys& S, int s, int k) { return __ldg(S.alpha + s * kMaxPrim + k); }
template <> __device__ __forceinline__ float prim_alpha<float>(const DevSys& S, int s, int k) { return __ldg(S.alpha_f + s * kMaxPrim + k); }
template <typename T> __device__ __forceinline__ T prim_coef(const DevSys& S, int s, int k);
template <> __device__ __forceinline__ double prim_coef<double>(const DevSys& S, int s, int k) { return __ldg(S.coef + s * kMaxPrim + k); }
template <> __device__ __forceinline__ float prim_coef<float>(const DevSys& S, int s, int k) { return __ldg(S.coef_f + s * kMaxPrim + k); }

// ---------------------------------------------------------------- group synchronisation
template <int GS>
__device__ __forceinline__ void gsync() {
  if constexpr (GS == 32) {
    __syncwarp();
  } else {
    // named barrier per group (id 1 + group index); GS threads take part
    asm volatile("bar.sync %0, %1;" ::"r"(1 + (int)(threadIdx.x / GS)), "r"(GS) : "memory");
  }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum of NV values over the group; every thread receives identical results (the xor
// butterfly adds the same operands in every lane). scratch: >= NV * GS/32 doubles.
template <int GS, int NV>
__device__ __forceinline__ void group_sum(double (&v)[NV], double* scratch) {
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
  if constexpr (GS > 32) {
    constexpr int NW = GS / 32;
    const int t = threadIdx.x % GS;
    if ((t & 31) == 0)
#pragma unroll
      for (int k = 0; k < NV; ++k) scratch[k * NW + (t >> 5)] = v[k];
    gsync<GS>();
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = 0.0;
      for (int w = 0; w < NW; ++w) s += scratch[k * NW + w];
      v[k] = s;
    }
    gsync<GS>();
  }
}

// Group sums of one double and one value of type T (identical results in every thread).
// scratch: >= 2 * GS/32 doubles.
template <int GS, typename T>
__device__ __forceinline__ void group_sum_dt(double& a, T& b, double* scratch) {
  a = warp_sum(a);
  b = warp_sum(b);
  if constexpr (GS > 32) {
    constexpr int NW = GS / 32;
    const int t = threadIdx.x % GS;
    if ((t & 31) == 0) {
      scratch[t >> 5] = a;
      scratch[NW + (t >> 5)] = (double)b;
    }
    gsync<GS>();
    double sa = 0.0;
    T sb = T(0);
    for (int w = 0; w < NW; ++w) {
      sa += scratch[w];
      sb += (T)scratch[NW + w];
    }
    a = sa;
    b = sb;
    gsync<GS>();
  }
}

// ---------------------------------------------------------------- Philox4x64-10
// Salmon et al., "Parallel random numbers: as easy as 1, 2, 3" (SC'11), 10 rounds.
__device__ __forceinline__ void philox4x64_10(uint64_t x[4], uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += W0;
      k1 += W1;
    }
    const uint64_t hi0 = __umul64hi(M0, x[0]), lo0 = M0 * x[0];
    const uint64_t hi1 = __umul64hi(M1, x[2]), lo1 = M1 * x[2];
    const uint64_t y0 = hi1 ^ x[1] ^ k0, y2 = hi0 ^ x[3] ^ k1;
    x[0] = y0;
    x[1] = lo1;
    x[2] = y2;
    x[3] = lo0;
  }
}
// 53 random bits -> [0, 1)
__device__ __forceinline__ double u01(uint64_t x) { return (double)(x >> 11) * 0x1.0p-53; }

// The same value as u01(x), (x >> 11) 2^-53, assembled from its bits with integer instructions: on
// this GPU every FP64 instruction (the integer-to-double conversion and the scaling of u01 included)
// takes the FP64 pipe for a whole warp, whatever the number of active lanes.
__device__ __forceinline__ double u01_bits(uint64_t x) {
  const uint64_t v = x >> 11;  // 53 bits
  if (v == 0) return 0.0;
  const int n = __clzll(v);   // 11 ... 63; v = 2^(63 - n) (1.f), value 2^(10 - n) (1.f)
  const uint64_t mant = ((v << n) << 1) >> 12;
  return __longlong_as_double((long long)(((uint64_t)(1033 - n) << 52) | mant));
}

// float -> double, exact, with integer instructions only (zeros, denormals, infinities and NaNs
// included), so that no conversion instruction reaches the FP64 pipe.
__device__ __forceinline__ double f2d_bits(float x) {
  const unsigned u = __float_as_uint(x), sgn = u & 0x80000000u, a = u & 0x7fffffffu;
  // normal numbers, infinities, NaNs: rebias the exponent (127 -> 1023; 255 -> 2047)
  const unsigned hn = sgn | ((a >> 3) + (a >= 0x7f800000u ? 0x70000000u : 0x38000000u)), ln = a << 29;
  // denormals a 2^-149, normalised (the leading bit of a at 31 - n); zeros keep their sign
  const int n = __clz(a | 1u);
  const unsigned m = (a << n) << 1;
  const unsigned hd = a ? (sgn | ((unsigned)(905 - n) << 20) | (m >> 12)) : sgn, ld = a ? (m << 20) : 0u;
  const bool normal = a >= 0x00800000u;
  return __hiloint2double((int)(normal ? hn : hd), (int)(normal ? ln : ld));
}

// double -> float, truncated toward zero, with integer instructions only: magnitudes below the
// normal floats give a signed zero, those beyond the float range a signed infinity (NaN: a NaN).
// Within the normal range the result is at most one float ulp from the rounded conversion.
__device__ __forceinline__ float d2f_trunc(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned sgn = hi & 0x80000000u, e = (hi >> 20) & 0x7ffu;
  const unsigned nrm = sgn | ((e - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  const bool nan = e == 0x7ffu && (((hi & 0xfffffu) | lo) != 0u);
  const unsigned big = nan ? 0x7fc00000u : (sgn | 0x7f800000u);
  return __uint_as_float(e < 897u ? sgn : (e > 1150u ? big : nrm));
}

// double -> float, rounded to nearest (ties to even), with integer instructions only; outside the
// normal float range as d2f_trunc (signed zero below, signed infinity above).
__device__ __forceinline__ float d2f_rn(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned sgn = hi & 0x80000000u, e = (hi >> 20) & 0x7ffu;
  unsigned nrm = sgn | ((e - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  const unsigned rest = lo & 0x1fffffffu;  // the 29 discarded bits
  nrm += (rest > 0x10000000u || (rest == 0x10000000u && (nrm & 1u))) ? 1u : 0u;  // a carry bumps the exponent
  const bool nan = e == 0x7ffu && (((hi & 0xfffffu) | lo) != 0u);
  const unsigned big = nan ? 0x7fc00000u : (sgn | 0x7f800000u);
  return __uint_as_float(e < 897u ? sgn : (e > 1150u ? big : nrm));
}

// v as a float-float pair (h + l, h the rounded float, l the rounded remainder) with one FP64
// instruction (the exact subtraction) instead of three; coordinates below the normal float range
// become zero.
__device__ __forceinline__ void split_ff_bits(double v, float& h, float& l) {
  h = d2f_rn(v);
  l = d2f_rn(v - f2d_bits(h));
}

// A double operand in the working precision: itself in FP64 mode, rounded to float with integer
// instructions in mixed mode (no FP64 conversion instruction).
template <typename T>
__device__ __forceinline__ T to_T(double x) {
  if constexpr (sizeof(T) == 8) return x;
  else return d2f_rn(x);
}

// Three standard normals (Box-Muller on 4 uniforms) for one proposal.
__device__ __forceinline__ void normals3(const uint64_t r[4], double xi[3], double) {
  const double twopi = 6.283185307179586;
  const double u1 = u01(r[0]), u2 = u01(r[1]), u3 = u01(r[2]), u4 = u01(r[3]);
  const double a = sqrt(-2.0 * log(1.0 - u1));
  const double b = sqrt(-2.0 * log(1.0 - u3));
  xi[0] = a * cos(twopi * u2);
  xi[1] = a * sin(twopi * u2);
  xi[2] = b * cos(twopi * u4);
}
__device__ __forceinline__ void normals3(const uint64_t r[4], double xi[3], float) {
  const float twopi = 6.2831853071795865f;
  const float a = sqrtf(-2.0f * logf((float)(1.0 - u01(r[0]))));
  const float b = sqrtf(-2.0f * logf((float)(1.0 - u01(r[2]))));
  float s, c;
  sincosf(twopi * (float)u01(r[1]), &s, &c);
  xi[0] = (double)(a * c);
  xi[1] = (double)(a * s);
  xi[2] = (double)(b * cosf(twopi * (float)u01(r[3])));
}

// Three standard normals in float (Box-Muller on 24-bit uniforms k 2^-24, 1 - u inside the log):
// the proposals of the mixed-precision chains, drawn from the same Philox outputs as normals3.
__device__ __forceinline__ void normals3_f(const uint64_t r[4], float xi[3]) {
  const float twopi = 6.2831853071795865f;
  const float v1 = 1.0f - (float)(unsigned)(r[0] >> 40) * 0x1.0p-24f;
  const float v3 = 1.0f - (float)(unsigned)(r[2] >> 40) * 0x1.0p-24f;
  const float a = sqrtf(-2.0f * logf(v1)), b = sqrtf(-2.0f * logf(v3));
  float sn, cs;
  sincosf(twopi * ((float)(unsigned)(r[1] >> 40) * 0x1.0p-24f), &sn, &cs);
  xi[0] = a * cs;
  xi[1] = a * sn;
  xi[2] = b * cosf(twopi * ((float)(unsigned)(r[3] >> 40) * 0x1.0p-24f));
}

// Error-free float transformations (Knuth two-sum; Dekker fast two-sum, |a| >= |b|).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  e = b - (s - a);
}

// Float-float addition (h1 + l1) + (h2 + l2) -> (h + l), about 44 significant bits.
__device__ __forceinline__ void ff_add(float h1, float l1, float h2, float l2, float& h, float& l) {
  float s, e;
  two_sum(h1, h2, s, e);
  e += l1 + l2;
  fast_two_sum(s, e, h, l);
}

// Squared distance of a shell's centre as a float-float pair (r2h + r2l), formed from the
// float-float positions; used for primitives whose a r^2 must keep more than float precision.
struct R2FF {
  float h, l;
};

// ---------------------------------------------------------------- AO shells
// Angular factor P (a real solid harmonic r^l Y_lm with its unit-sphere normalisation),
// its gradient g and its constant Hessian h (xx, yy, zz, xy, xz, yz).
template <typename T>
__device__ __forceinline__ void angular(int l, int m, T x, T y, T z, T& P, T g[3], T h[6]) {
  const T ns = T(0.28209479177387814);   // sqrt(1/(4 pi))
  const T np = T(0.48860251190291992);   // sqrt(3/(4 pi))
  const T nd = T(1.0925484305920792);    // sqrt(15/(4 pi))
  const T n0 = T(0.31539156525252005);   // sqrt(5/(16 pi))
  const T n2 = T(0.54627421529603959);   // sqrt(15/(16 pi))
#pragma unroll
  for (int k = 0; k < 6; ++k) h[k] = T(0);
  g[0] = g[1] = g[2] = T(0);
  if (l == 0) {
    P = ns;
  } else if (l == 1) {
    const T c[3] = {x, y, z};
    P = np * c[m];
    g[m] = np;
  } else {
    switch (m) {
      case 0: P = nd * x * y; g[0] = nd * y; g[1] = nd * x; h[3] = nd; break;          // xy
      case 1: P = nd * y * z; g[1] = nd * z; g[2] = nd * y; h[5] = nd; break;          // yz
      case 2: P = n0 * (T(2) * z * z - x * x - y * y);                                 // 3z^2 - r^2
        g[0] = T(-2) * n0 * x; g[1] = T(-2) * n0 * y; g[2] = T(4) * n0 * z;
        h[0] = T(-2) * n0; h[1] = T(-2) * n0; h[2] = T(4) * n0; break;
      case 3: P = nd * x * z; g[0] = nd * z; g[2] = nd * x; h[4] = nd; break;          // xz
      default: P = n2 * (x * x - y * y); g[0] = T(2) * n2 * x; g[1] = T(-2) * n2 * y;  // x^2 - y^2
        h[0] = T(2) * n2; h[1] = T(-2) * n2; break;
    }
  }
}

// Electron position in the two forms the AO and Jastrow code use: double, and a
// float-float pair (h + l) whose float differences keep full float relative precision.
struct EPos {
  double d[3];
  float h[3], l[3];
};
__device__ __forceinline__ EPos make_epos(const double* r) {
  EPos p;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    p.d[c] = r[c];
    split_ff_bits(r[c], p.h[c], p.l[c]);
  }
  return p;
}

// Shell s at displacement (x, y, z) = r - R_center. LEVEL 0: value. LEVEL 1: gradient (3)
// and Laplacian. LEVEL 2: value, gradient (3), Laplacian, Hessian (xx yy zz xy xz yz),
// gradient of the Laplacian (3). LEVEL kAoLevelP: the one row lap psi + 2 j . grad psi for the
// vector j (jv), the AO coefficients of a row of P = lap(phi) + 2 grad J . grad(phi), which is
// linear in C. out[c * stride + ao] for component c.
// With e_k = c_k exp(-a_k r^2), R0 = sum e_k, R1 = sum -2a_k e_k, R2 = sum 4a_k^2 e_k:
//   d_i F = x_i R1, d_i d_j F = x_i x_j R2 + delta_ij R1; for a harmonic homogeneous P of
//   degree l: lap(P F) = P sum_k -2a_k e_k ((2l+3) - 2 a_k r^2) and
//   d_k lap(P F) = P_k lap F + P x_k sum_k 4a_k^2 e_k ((2l+5) - 2 a_k r^2).
// Each primitive's factor (2l+3) - 2 a r^2 is where the Laplacian cancels; for primitives
// marked sharp (mixed mode only) a r^2 and the factors are formed in double from r2d.
constexpr int kAoLevelP = 3;

template <typename T, int LEVEL>
__device__ __forceinline__ void shell_eval(const DevSys& S, int s, T x, T y, T z, int smask, R2FF r2ff, T* out,
                                           int stride, const T* jv = nullptr) {
  const int4 sh = __ldg(S.shell + s);
  const int l = sh.y, np = sh.z, ao0 = sh.w;
  const T r2 = x * x + y * y + z * z;
  T R0 = 0, R1 = 0, R2 = 0, LF = 0, T3 = 0;
  for (int k = 0; k < np; ++k) {
    const T a = prim_alpha<T>(S, s, k);
    T e, f3, f5;
    if (sizeof(T) == 4 && ((smask >> k) & 1)) {
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
    R0 += e;
    if (LEVEL >= 1) {
      const T m2ae = T(-2) * a * e;
      R1 += m2ae;
      LF += m2ae * f3;
      if (LEVEL == 2) {
        const T a4e = T(4) * a * a * e;
        R2 += a4e;
        T3 += a4e * f5;
      }
    }
  }
  const int nc = 2 * l + 1;
  const T xs[3] = {x, y, z};
  for (int m = 0; m < nc; ++m) {
    T P, g[3], h[6];
    angular<T>(l, m, x, y, z, P, g, h);
    const int ao = ao0 + m;
    if (LEVEL == 0) {
      out[ao] = P * R0;
    } else {
      T grad[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) grad[i] = g[i] * R0 + P * xs[i] * R1;
      if (LEVEL == kAoLevelP) {
        out[ao] = P * LF + T(2) * (jv[0] * grad[0] + jv[1] * grad[1] + jv[2] * grad[2]);
      } else if (LEVEL == 1) {
        out[0 * stride + ao] = grad[0];
        out[1 * stride + ao] = grad[1];
        out[2 * stride + ao] = grad[2];
        out[3 * stride + ao] = P * LF;
      } else {
        out[0 * stride + ao] = P * R0;
        out[1 * stride + ao] = grad[0];
        out[2 * stride + ao] = grad[1];
        out[3 * stride + ao] = grad[2];
        out[4 * stride + ao] = P * LF;
        const int hi[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          const int i = hi[k][0], j = hi[k][1];
          out[(5 + k) * stride + ao] = h[k] * R0 + (g[i] * xs[j] + g[j] * xs[i]) * R1 +
                                       P * (xs[i] * xs[j] * R2 + (i == j ? R1 : T(0)));
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) out[(11 + k) * stride + ao] = g[k] * LF + P * xs[k] * T3;
      }
    }
  }
}

// Displacement of an electron from nucleus c: double in FP64 mode; in mixed mode the
// float-float difference, accurate to a float ulp of the displacement itself.
template <typename T>
__device__ __forceinline__ void disp_nuc(const DevSys& S, const EPos& p, int c, T d[3]);
template <>
__device__ __forceinline__ void disp_nuc<double>(const DevSys& S, const EPos& p, int c, double d[3]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) d[k] = p.d[k] - __ldg(S.R + 3 * c + k);
}
template <>
__device__ __forceinline__ void disp_nuc<float>(const DevSys& S, const EPos& p, int c, float d[3]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) d[k] = (p.h[k] - __ldg(S.Rh + 3 * c + k)) + (p.l[k] - __ldg(S.Rl + 3 * c + k));
}

// AO components of shell s at one point. SHARP: in mixed mode, form a r^2 of sharp
// primitives in float-float arithmetic.
template <typename T, int LEVEL, bool SHARP>
__device__ __forceinline__ void shell_point(const DevSys& S, const EPos& p, int s, T* out, int stride,
                                            const T* jv = nullptr) {
  {
    const int c = __ldg(S.shell + s).x;
    T d[3];
    R2FF r2ff{0.f, 0.f};
    int smask = 0;
    if (SHARP && sizeof(T) == 4 && (smask = __ldg(S.sharp + s))) {
      float hsum = 0.f, lsum = 0.f;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        float dh, dl, sdiff, eh;
        two_sum(p.h[k], -__ldg(S.Rh + 3 * c + k), sdiff, eh);
        fast_two_sum(sdiff, (p.l[k] - __ldg(S.Rl + 3 * c + k)) + eh, dh, dl);
        d[k] = (T)dh;
        const float pp = dh * dh, pe = fmaf(dh, dh, -pp);
        float tt;
        two_sum(hsum, pp, hsum, tt);
        lsum += tt + pe + 2.0f * dh * dl;
      }
      fast_two_sum(hsum, lsum, r2ff.h, r2ff.l);
    } else {
      disp_nuc<T>(S, p, c, d);
    }
    shell_eval<T, LEVEL>(S, s, d[0], d[1], d[2], smask, r2ff, out, stride, jv);
  }
}

template <typename T, int GS, int LEVEL, bool SHARP>
__device__ __forceinline__ void ao_point(const DevSys& S, const EPos& p, T* out, int stride) {
  const int t = threadIdx.x % GS;
  for (int s = t; s < S.nshell; s += GS) shell_point<T, LEVEL, SHARP>(S, p, s, out, stride);
}

// Electron-electron displacement from the shared-memory position arrays.
template <typename T>
__device__ __forceinline__ T edisp(const double* pos, const float* ph, const float* pl, int i, int j, int c);
template <>
__device__ __forceinline__ double edisp<double>(const double* pos, const float*, const float*, int i, int j, int c) {
  return pos[3 * i + c] - pos[3 * j + c];
}
template <>
__device__ __forceinline__ float edisp<float>(const double*, const float* ph, const float* pl, int i, int j, int c) {
  return (ph[3 * i + c] - ph[3 * j + c]) + (pl[3 * i + c] - pl[3 * j + c]);
}

// ---------------------------------------------------------------- Jastrow radial functions
// Pade a r / (1 + F r) and its first three derivatives.
template <typename T>
struct Rad3 { T h, h1, h2, h3; };
template <typename T>
__device__ __forceinline__ Rad3<T> pade(T a, T F, T r) {
  const T q = T(1) / (T(1) + F * r);
  const T q2 = q * q;
  return {a * r * q, a * q2, T(-2) * a * F * q2 * q, T(6) * a * F * F * q2 * q2};
}
template <typename T>
__device__ __forceinline__ T pade_value(T a, T F, T r) {
  return a * r / (T(1) + F * r);
}
// The same in mixed mode with the approximate reciprocal (a few float ulp; these terms are summed
// in float with many others) and, for a pair at squared distance r2, 1/r and r from the approximate
// reciprocal square root; in FP64 mode the exact operations.
template <typename T>
__device__ __forceinline__ Rad3<T> pade_fast(T a, T F, T r) {
  if constexpr (sizeof(T) == 8) {
    return pade<T>(a, F, r);
  } else {
    const float q = __fdividef(1.0f, 1.0f + F * r);
    const float q2 = q * q;
    return {a * r * q, a * q2, -2.0f * a * F * q2 * q, 6.0f * a * F * F * q2 * q2};
  }
}
template <typename T>
__device__ __forceinline__ T fast_rcp(T x) {
  if constexpr (sizeof(T) == 8) return 1.0 / x;
  else return __fdividef(1.0f, x);
}
template <typename T>
__device__ __forceinline__ void dist_inv(T r2, T& r, T& ri) {
  if constexpr (sizeof(T) == 8) {
    r = sqrt(r2);
    ri = 1.0 / r;
  } else {
    ri = rsqrtf(r2);
    r = r2 * ri;
  }
}

// Exponential form (a / F)(1 - exp(-F r)) (Eq. twobody_v_exp, cusp a) and its derivatives.
template <typename T> __device__ __forceinline__ T dexpm1(T x);
template <> __device__ __forceinline__ double dexpm1<double>(double x) { return expm1(x); }
template <> __device__ __forceinline__ float dexpm1<float>(float x) { return expm1f(x); }
template <typename T>
__device__ __forceinline__ Rad3<T> expo(T a, T F, T r) {
  const T q = dexp<T>(-F * r);
  return {-(a / F) * dexpm1<T>(-F * r), a * q, -a * F * q, a * F * F * q};
}
template <typename T>
__device__ __forceinline__ T expo_value(T a, T F, T r) {
  return -(a / F) * dexpm1<T>(-F * r);
}

// The two-body term of a pair of electrons with parallel (par) or antiparallel spins.
template <typename T>
__device__ __forceinline__ Rad3<T> pair_rad(const DevSys& S, bool par, T r) {
  const T a = jas_a<T>(S, par), F = jas_F<T>(S, par);
  return S.j2exp ? expo<T>(a, F, r) : pade<T>(a, F, r);
}
template <typename T>
__device__ __forceinline__ Rad3<T> pair_rad_fast(const DevSys& S, bool par, T r) {
  const T a = jas_a<T>(S, par), F = jas_F<T>(S, par);
  return S.j2exp ? expo<T>(a, F, r) : pade_fast<T>(a, F, r);
}
template <typename T>
__device__ __forceinline__ T pair_value(const DevSys& S, bool par, T r) {
  const T a = jas_a<T>(S, par), F = jas_F<T>(S, par);
  return S.j2exp ? expo_value<T>(a, F, r) : pade_value<T>(a, F, r);
}

// ---------------------------------------------------------------- FP64 Gauss-Jordan inverse
// In-place inversion of the n x n row-major matrix A (shared memory, double) with partial
// row pivoting. piv: int[n]; f: double[3 n + 1] scratch (column k, the pivot's reciprocal,
// the scaled pivot row and the row it replaces); flag: int (set to 1 if a pivot is zero or
// not finite). logabs/sign are accumulated when want_logdet. Every thread of the group must
// call it. Per pivot: the first warp finds the pivot; the group copies the pivot row (scaled),
// the row it displaces and column k; then every element is updated once, the row swap folded
// into the update, so each pivot costs three group barriers.
template <int GS>
__device__ void gj_inverse(double* A, int n, int* piv, double* f, int* flag, double* logabs, double* sgn,
                           bool want_logdet) {
  const int t = threadIdx.x % GS;
  double* rs = f + n + 1;      // scaled pivot row: the new row k
  double* rk = f + 2 * n + 1;  // old row k: the new row p
  // this thread's elements in row-major order: (i0, j0), then steps of GS elements
  const int i0 = t / n, j0 = t - i0 * n;
  const int di = GS / n, dj = GS - di * n;
  for (int k = 0; k < n; ++k) {
    // pivot search by the first warp of the group; |x| of doubles compared through their bit
    // patterns (monotone for non-negative values), so the search needs no FP64 instruction
    if (t < 32) {
      long long best = -1;
      int bi = k;
      for (int i = k + t; i < n; i += 32) {
        const long long v = __double_as_longlong(A[i * n + k]) & 0x7fffffffffffffffLL;
        if (v > best) { best = v; bi = i; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const long long ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (t == 0) {
        piv[k] = bi;
        const double p = A[bi * n + k];
        if (!(p != 0.0) || !isfinite(p)) *flag = 1;
        f[n] = 1.0 / p;  // the pivot's reciprocal, computed once
        if (want_logdet) {
          *logabs += log(fabs(p));
          if (p < 0) *sgn = -*sgn;
          if (bi != k) *sgn = -*sgn;
        }
      }
    }
    gsync<GS>();
    const int p = piv[k];
    const double pinv = f[n];
    for (int j = t; j < n; j += GS) {
      rs[j] = (j == k ? 1.0 : A[p * n + j]) * pinv;
      rk[j] = A[k * n + j];
    }
    for (int i = t; i < n; i += GS) f[i] = A[i * n + k];  // column k before the swap
    gsync<GS>();
    // after the swap, row p holds the old row k, whose column-k entry is f[k]
    const double fp = f[k];
    for (int i = i0, j = j0; i < n;) {
      double v;
      if (i == k) {
        v = rs[j];
      } else {
        const double fi = i == p ? fp : f[i];
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
    gsync<GS>();
  }
  // undo the row permutation as column swaps, last pivot first; a thread owns whole rows
  for (int i = t; i < n; i += GS)
    for (int k = n - 1; k >= 0; --k) {
      const int p = piv[k];
      if (p != k) {
        const double a = A[i * n + k];
        A[i * n + k] = A[i * n + p];
        A[i * n + p] = a;
      }
    }
  gsync<GS>();
}

// ---------------------------------------------------------------- orbital rows
// out[r][col] = sum_mu rows[r][mu] C[mu][col] for the R rows row0, row0 + ng, ... of a chunk of
// nrows rows (row stride M): independent accumulators that share each coefficient load. Rows
// past nrows are computed from a valid row and not stored.
template <typename T, int R, typename OutT>
__device__ __forceinline__ void orbital_rows(const T* rows, const T* C, int M, int n, int col, int row0, int ng,
                                             int nrows, OutT* out, int out_stride) {
  T v[R];
  const T* a[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    v[r] = T(0);
    const int row = row0 + r * ng;
    a[r] = rows + (row < nrows ? row : nrows - 1) * M;
  }
  for (int mu = 0; mu < M; ++mu) {
    const T c = __ldg(C + mu * n + col);
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] += a[r][mu] * c;
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int row = row0 + r * ng;
    if (row < nrows) out[row * out_stride + col] = (OutT)v[r];
  }
}

// The same rows of a float contraction with compensated accumulation, for the Slater matrix of a
// measurement in mixed mode: each product's rounding error (from an FMA) and each addition's (a
// two-sum) are carried in a second float and the result is assembled in double. Plain float
// accumulation over a few hundred AOs, with the cancellation between terms of both signs, leaves
// errors several times the rounding of the inputs, and the inverse of an ill-conditioned Slater
// matrix amplifies them by its condition number.
template <int R>
__device__ __forceinline__ void orbital_rows_comp(const float* rows, const float* C, int M, int n, int col, int row0,
                                                  int ng, int nrows, double* out, int out_stride) {
  float v[R], cmp[R];
  const float* a[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    v[r] = 0.f;
    cmp[r] = 0.f;
    const int row = row0 + r * ng;
    a[r] = rows + (row < nrows ? row : nrows - 1) * M;
  }
  for (int mu = 0; mu < M; ++mu) {
    const float c = __ldg(C + mu * n + col);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float x = a[r][mu], p = x * c, pe = fmaf(x, c, -p);
      float sv, se;
      two_sum(v[r], p, sv, se);
      v[r] = sv;
      cmp[r] += se + pe;
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int row = row0 + r * ng;
    if (row < nrows) out[row * out_stride + col] = f2d_bits(v[r]) + f2d_bits(cmp[r]);
  }
}

template <int GS>
__device__ __forceinline__ void orbital_block_comp(const float* rows, int nrows, const float* C, int M, int n,
                                                   double* out, int out_stride) {
  const int t = threadIdx.x % GS;
  const bool wide = GS >= n;
  const int ng = wide ? GS / n : 1;
  const int col0 = wide ? t % n : t, rg = wide ? t / n : 0, dcol = wide ? n : GS;
  for (int col = col0; col < n && rg < ng && rg < nrows; col += dcol) {
    switch ((nrows - rg + ng - 1) / ng) {  // rows of this thread
      case 1: orbital_rows_comp<1>(rows, C, M, n, col, rg, ng, nrows, out, out_stride); break;
      case 2: orbital_rows_comp<2>(rows, C, M, n, col, rg, ng, nrows, out, out_stride); break;
      case 3: orbital_rows_comp<3>(rows, C, M, n, col, rg, ng, nrows, out, out_stride); break;
      case 4: orbital_rows_comp<4>(rows, C, M, n, col, rg, ng, nrows, out, out_stride); break;
      case 5: orbital_rows_comp<5>(rows, C, M, n, col, rg, ng, nrows, out, out_stride); break;
      case 6: orbital_rows_comp<6>(rows, C, M, n, col, rg, ng, nrows, out, out_stride); break;
      case 7: orbital_rows_comp<7>(rows, C, M, n, col, rg, ng, nrows, out, out_stride); break;
      default: orbital_rows_comp<8>(rows, C, M, n, col, rg, ng, nrows, out, out_stride); break;
    }
  }
}

// All columns of nrows (<= 8 ng) rows of AO values times C^s (n columns), over the group:
// with GS >= n thread t owns column t % n and rows t / n + k ng (ng = GS / n); with GS < n it
// owns columns t, t + GS, ... and every row.
template <typename T, int GS, typename OutT>
__device__ __forceinline__ void orbital_block(const T* rows, int nrows, const T* C, int M, int n, OutT* out,
                                              int out_stride) {
  const int t = threadIdx.x % GS;
  const bool wide = GS >= n;
  const int ng = wide ? GS / n : 1;
  const int col0 = wide ? t % n : t, rg = wide ? t / n : 0, dcol = wide ? n : GS;
  for (int col = col0; col < n && rg < ng && rg < nrows; col += dcol) {
    switch ((nrows - rg + ng - 1) / ng) {  // rows of this thread
      case 1: orbital_rows<T, 1>(rows, C, M, n, col, rg, ng, nrows, out, out_stride); break;
      case 2: orbital_rows<T, 2>(rows, C, M, n, col, rg, ng, nrows, out, out_stride); break;
      case 3: orbital_rows<T, 3>(rows, C, M, n, col, rg, ng, nrows, out, out_stride); break;
      case 4: orbital_rows<T, 4>(rows, C, M, n, col, rg, ng, nrows, out, out_stride); break;
      case 5: orbital_rows<T, 5>(rows, C, M, n, col, rg, ng, nrows, out, out_stride); break;
      case 6: orbital_rows<T, 6>(rows, C, M, n, col, rg, ng, nrows, out, out_stride); break;
      case 7: orbital_rows<T, 7>(rows, C, M, n, col, rg, ng, nrows, out, out_stride); break;
      default: orbital_rows<T, 8>(rows, C, M, n, col, rg, ng, nrows, out, out_stride); break;
    }
  }
}

// ---------------------------------------------------------------- Slater matrix build
// A^s_{el, i} = phi_i(r_e) = sum_mu psi_mu(r_e) C^s_{mu i} (Eq. restricted-C), computed
// in T and stored in double for the inversion. aobuf: T[chunk * M] scratch; chunk electrons
// at a time: their AO values over (electron, shell) pairs, then their rows of A.
// COMP: in mixed mode, accumulate the contraction with compensation (orbital_rows_comp).
template <typename T, int GS, bool COMP = false>
__device__ void build_slater(const DevSys& S, const double* pos, int sg, double* A, T* aobuf, int chunk) {
  const int t = threadIdx.x % GS;
  const int n = sg == 0 ? S.nup : S.ndn, e0 = sg == 0 ? 0 : S.nup, M = S.M, ns = S.nshell;
  const T* C = coefC<T>(S, sg);
  const int ng = GS >= n ? GS / n : 1;
  chunk = chunk < 1 ? 1 : (chunk > 8 * ng ? 8 * ng : chunk);
  for (int c0 = 0; c0 < n; c0 += chunk) {
    const int nc = n - c0 < chunk ? n - c0 : chunk;
    for (int q = t; q < nc * ns; q += GS) {
      const int r = q / ns, sh = q - r * ns;
      shell_point<T, 0, true>(S, make_epos(pos + 3 * (e0 + c0 + r)), sh, aobuf + r * M, 0);
    }
    gsync<GS>();
    if constexpr (COMP && sizeof(T) == 4) orbital_block_comp<GS>(aobuf, nc, C, M, n, A + c0 * n, n);
    else orbital_block<T, GS>(aobuf, nc, C, M, n, A + c0 * n, n);
    gsync<GS>();
  }
}

}  // namespace vmcf
