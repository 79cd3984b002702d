// Host side of the C ABI declared in include/vmcf.h: input validation, basis
// normalisation, device tables, launch planning, the sampling loop and the estimator finish.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "../../include/vmcf.h"
#include "../../include/vmcf_diag.h"
#include "vmcf_host.h"

using namespace vmcf;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
  return VMCF_ECUDA;
}

#define VMCF_CUDA(call)                                  \
  do {                                                   \
    cudaError_t _e = (call);                             \
    if (_e != cudaSuccess) return cuda_fail(_e, #call);  \
  } while (0)

int align16(int x) { return (x + 15) & ~15; }

constexpr int kSmemCap = 227 * 1024;
constexpr double kSharpAlpha = 48.0;

}  // namespace

namespace {
// Event pair around one launch when profiling is on.
struct Timed {
  vmcf_walkers_s* wk;
  int kind;
  cudaStream_t st;
  cudaEvent_t a = nullptr, b = nullptr;
  Timed(vmcf_walkers_s* w, int k, cudaStream_t s) : wk(w), kind(k), st(s) {
    if (wk->profiling) {
      cudaEventCreate(&a);
      cudaEventCreate(&b);
      cudaEventRecord(a, st);
    }
  }
  ~Timed() {
    if (wk->profiling) {
      cudaEventRecord(b, st);
      wk->events.push_back({kind, {a, b}});
    }
  }
};
}  // namespace

namespace {

// ---------------------------------------------------------------- normalisation
// Radial normalisation of r^l exp(-a r^2) times a unit-sphere harmonic:
// N^2 = 2 (2a)^{l+3/2} / Gamma(l + 3/2).
double radial_norm(double a, int l) { return std::sqrt(2.0 * std::pow(2.0 * a, l + 1.5) / std::tgamma(l + 1.5)); }
// Overlap of two normalised primitives with the same centre, l and m:
// N_a N_b Gamma(l + 3/2) / (2 (a + b)^{l+3/2}).
double same_centre_overlap(double a, double b, int l) {
  return radial_norm(a, l) * radial_norm(b, l) * std::tgamma(l + 1.5) / (2.0 * std::pow(a + b, l + 1.5));
}

// Device tables of a basis (determinant or Jastrow): per shell (centre, l, nprim, first function),
// exponents and normalised contraction coefficients ([nshell][kMaxPrim]), the sharp-primitive
// masks, and the centre of every function. False (with the reason) on a bad shell.
bool shell_tables(const vmcf_basis& bas, int K, std::vector<int4>& shells, std::vector<int>& sharp,
                  std::vector<double>& alpha, std::vector<double>& coef, std::vector<int>& center, int* nfun,
                  std::string* why) {
  shells.assign(bas.nshell, make_int4(0, 0, 0, 0));
  sharp.assign(bas.nshell, 0);
  alpha.assign((size_t)bas.nshell * kMaxPrim, 0.0);
  coef.assign((size_t)bas.nshell * kMaxPrim, 0.0);
  center.clear();
  int M = 0;
  for (int sh = 0; sh < bas.nshell; ++sh) {
    const int c = bas.center[sh], l = bas.l[sh], np = bas.nprim[sh];
    if (c < 0 || c >= K || l < 0 || l > 2 || np < 1 || np > bas.maxprim) {
      *why = "bad shell (centre, l in 0..2, nprim)";
      return false;
    }
    double d[kMaxPrim], a[kMaxPrim];
    for (int k = 0; k < np; ++k) {
      a[k] = bas.exps[sh * bas.maxprim + k];
      d[k] = bas.coefs[sh * bas.maxprim + k];
      if (!(a[k] > 0.0) || !std::isfinite(a[k]) || !std::isfinite(d[k])) {
        *why = "exponents must be positive and finite";
        return false;
      }
    }
    double norm2 = 0.0;
    for (int p = 0; p < np; ++p)
      for (int q = 0; q < np; ++q) norm2 += d[p] * d[q] * same_centre_overlap(a[p], a[q], l);
    if (!(norm2 > 0.0)) {
      *why = "contraction has zero norm";
      return false;
    }
    for (int k = 0; k < np; ++k) {
      // In mixed mode a primitive this sharp has a r^2 and its Laplacian factors formed in
      // double: the float rounding of a r^2 times a would dominate the local energy error.
      if (a[k] > kSharpAlpha) sharp[sh] |= 1 << k;
      alpha[sh * kMaxPrim + k] = a[k];
      coef[sh * kMaxPrim + k] = d[k] * radial_norm(a[k], l) / std::sqrt(norm2);
    }
    shells[sh] = make_int4(c, l, np, M);
    for (int m = 0; m < 2 * l + 1; ++m) center.push_back(c);
    M += 2 * l + 1;
  }
  *nfun = M;
  return true;
}

// Whether the n columns of C [M][n] (row-major) are linearly independent: Gram-Schmidt, twice per
// column, against the columns before it; a column whose remainder is below 1e-10 of its own norm
// lies in their span.
bool independent_columns(const std::vector<double>& C, int M, int n) {
  std::vector<double> Q((size_t)M * n);
  for (int j = 0; j < n; ++j) {
    double n0 = 0.0;
    for (int mu = 0; mu < M; ++mu) {
      Q[(size_t)j * M + mu] = C[(size_t)mu * n + j];
      n0 += C[(size_t)mu * n + j] * C[(size_t)mu * n + j];
    }
    double* q = &Q[(size_t)j * M];
    for (int pass = 0; pass < 2; ++pass)
      for (int k = 0; k < j; ++k) {
        const double* qk = &Q[(size_t)k * M];
        double d = 0.0;
        for (int mu = 0; mu < M; ++mu) d += qk[mu] * q[mu];
        for (int mu = 0; mu < M; ++mu) q[mu] -= d * qk[mu];
      }
    double nr = 0.0;
    for (int mu = 0; mu < M; ++mu) nr += q[mu] * q[mu];
    if (!(nr > 1e-20 * n0) || !(n0 > 0.0)) return false;
    const double inv = 1.0 / std::sqrt(nr);
    for (int mu = 0; mu < M; ++mu) q[mu] *= inv;
  }
  return true;
}

template <typename T>
size_t tsize() { return sizeof(T); }

// Shared-memory plan of one walker group for the refresh and move kernels.
GroupLayout layout_refresh_move(const vmcf_system_s& s, size_t tsz, int GS) {
  GroupLayout L{};
  int o = 0;
  auto take = [&](int bytes) { int at = o; o = align16(o + bytes); return at; };
  L.pos = take(8 * 3 * s.Ne);
  L.ph = take(4 * 3 * s.Ne);
  L.pl = take(4 * 3 * s.Ne);
  L.Bd = take(8 * s.nmax * s.nmax);
  L.Bt = take((int)tsz * s.nB);
  L.ao_rows = 4;
  L.ao = take((int)tsz * s.M * L.ao_rows);
  L.row = take((int)tsz * s.nmax);
  L.wv = take((int)tsz * s.nmax);
  L.col = take((int)tsz * s.nmax);
  L.piv = take(4 * s.nmax);
  L.f = take(8 * (3 * s.nmax + 1));
  L.red = take(8 * 4 * std::max(1, GS / 32));
  L.scal = take(32);
  // AO-expanded Jastrow terms: t0 = xi + Xi s, the proposed and current Jastrow-basis values and
  // Xi (psi^J(r') - psi^J(r_e)) (the sum s while t0 is rebuilt)
  L.jw = s.MJ > 0 ? take((int)tsz * 4 * s.MJ) : 0;
  L.bytes = align16(o);
  return L;
}

// Shared-memory plan of one walker group for the measure kernel.
GroupLayout layout_measure_chunks(const vmcf_system_s& s, size_t tsz, int GS, bool withD, int tc_rows, int p2,
                              int p3) {
  GroupLayout L{};
  int o = 0;
  auto take = [&](int bytes) { int at = o; o = align16(o + bytes); return at; };
  L.pos = take(8 * 3 * s.Ne);
  L.ph = take(4 * 3 * s.Ne);
  L.pl = take(4 * 3 * s.Ne);
  // FP64: Bd holds both inverses and is Bt. Mixed: Bd holds one block during the inversion;
  // P (written after the last inversion) reuses its bytes (4 nB <= 8 nmax^2).
  L.Bd = take(8 * (tsz == 8 ? s.nB : s.nmax * s.nmax));
  L.Bt = (tsz == 8) ? L.Bd : take((int)tsz * s.nB);
  L.P = (tsz == 8) ? take((int)tsz * s.nB) : L.Bd;
  L.Q = take((int)tsz * s.nmax * s.nmax);
  L.Jg = take((int)tsz * 3 * s.Ne);
  L.Jl = take((int)tsz * s.Ne);
  L.gd = take((int)tsz * 3 * s.Ne);
  L.ao_rows = 8;
  L.p2_chunk = p2;  // 4 p2 electrons per chunk of the P-row pass: one AO row each
  L.p3_chunk = p3;  // electrons per step of the adjoint/force pass: 14 AO rows each
  L.ao = take((int)tsz * std::max(14 * L.p3_chunk, 4 * L.p2_chunk) * s.M);
  L.frc = take((int)tsz * 6 * s.K);
  L.fa = take((int)tsz * 6 * s.M);
  // space warp: dE_L/dr_e [3 Ne] (the kappa sums go to the AO buffer, free by then); in mixed mode
  // it shares the Gauss-Jordan scratch f, which is only used before (3 Ne floats <= 3 nmax + 1 doubles)
  // O per walker, or (tensor-core sums) a [tc_rows][8] bf16 staging tile of AO values
  L.Ow = tc_rows > 0 ? take(16 * tc_rows) : take((int)tsz * s.M * s.nmax);
  L.D = withD ? take((int)tsz * s.M * s.nmax) : L.Ow;
  L.piv = take(4 * s.nmax);
  L.f = take(8 * (3 * s.nmax + 1));
  L.ew = tsz == 4 ? L.f : take((int)tsz * 3 * s.Ne);
  L.red = take(8 * (32 + 4 * L.p2_chunk));  // group-sum scratch (<= 32 doubles), then per-electron sums
  L.scal = take(32);
  // AO-expanded Jastrow terms: t0, s (then sum_e w_e), P = Xi sum_e w_e, the per-function shares of
  // the nuclear derivatives [6][MJ], and the products with Xi of jch electrons at a time: inputs
  // [2 jch][MJ] and outputs [2 jch][MJ]. The work runs before the first and after the last use of
  // the per-walker O buffer, so it shares that buffer when it fits there.
  L.jch = tsz == 8 ? 2 : 4;
  // whole-warp subgroups, each covering every Jastrow-basis shell, for different electrons
  const int wpg = std::max(1, (s.nJs + 31) / 32), nw = std::max(1, GS / 32);
  L.jng = 1;
  while (L.jng < 4 && 2 * L.jng * wpg <= nw) L.jng *= 2;
  const int MJp = (s.MJ + 3) / 4 * 4;
  // inputs [2 jch][MJp] first (rows start on 16 bytes), outputs [2 jch][MJ], t0, s, P, shares [jng][6][MJ]
  const int jneed = (int)tsz * (2 * L.jch * MJp + 2 * L.jch * s.MJ + 3 * s.MJ + 6 * L.jng * s.MJ);
  L.jw = s.MJ == 0 ? 0 : (tc_rows == 0 && jneed <= (int)tsz * s.M * s.nmax ? L.Ow : take(jneed));
  L.bytes = align16(o);
  return L;
}

// Larger electron chunks where the layout fits and keeps as many walker groups per SM as the smallest
// (twelve electrons per P-row chunk, one per adjoint/force step): 24 per P-row chunk (half the chunks,
// each coefficient load shared by twice the rows) and two per adjoint/force step (half the steps and
// barriers, each coefficient load shared by both electrons), in that order of preference.
GroupLayout layout_measure(const vmcf_system_s& s, size_t tsz, int GS, bool withD, int tc_rows = 0) {
  const GroupLayout L0 = layout_measure_chunks(s, tsz, GS, withD, tc_rows, 3, 1);
  const int per_sm = 228 * 1024;
  const int want = per_sm / (L0.bytes + 1024);
  const int cand[3][2] = {{6, 2}, {6, 1}, {3, 2}};
  for (const auto& c : cand) {
    const GroupLayout L = layout_measure_chunks(s, tsz, GS, withD, tc_rows, c[0], c[1]);
    if (L.bytes <= kSmemCap && per_sm / (L.bytes + 1024) >= want) return L;
  }
  return L0;
}

// Measurement-kernel plan for group size s.GSm: layouts, groups per CTA, accumulator placement.
int plan_measure(vmcf_system_s& s) {
  const size_t tsz = s.precision == VMCF_FP64 ? 8 : 4;
  s.Lmeas = layout_measure(s, tsz, s.GSm, false);
  s.LmeasD = layout_measure(s, tsz, s.GSm, true);
  // mixed precision: the walker sums of O on the tensor cores (tiles of 128 AOs x 32 columns,
  // chunks of 16 electrons); the measurement then stages AO values instead of holding O
  s.LmeasTC = s.Lmeas;
  if (s.precision == VMCF_MIXED) {
    s.tcg_Mf = (s.M + 7) / 8 * 8;
    s.tcg_Nf = (2 * s.nmax + 15) / 16 * 16;
    s.tcg_nch = (s.nmax + 15) / 16;
    s.LmeasTC = layout_measure(s, tsz, s.GSm, false, s.tcg_Mf);
  }
  const int maxg = s.GSm == 32 ? 4 : 1;
  if (s.Lmeas.bytes > kSmemCap) return fail(VMCF_ENOTSUP, "system too large for the shared-memory plan (measure)");
  s.gpb_measD = s.LmeasD.bytes > kSmemCap ? 0 : std::max(1, std::min(maxg, kSmemCap / s.LmeasD.bytes));
  s.accL = 3 + 9 * s.K + 2 * s.M * (s.nup + s.ndn) + (s.swct ? 9 * s.K : 0);
  const int accBytes = align16((int)tsz * s.accL);
  int g = maxg;
  while (g > 1 && g * s.Lmeas.bytes + accBytes > kSmemCap) --g;
  if (g * s.Lmeas.bytes + accBytes <= kSmemCap) {
    s.acc_smem = true;
    s.gpb_meas = g;
    s.acc_off = g * s.Lmeas.bytes;
  } else {
    s.acc_smem = false;  // one group per CTA, sums go straight to the CTA's FP64 slot
    s.gpb_meas = 1;
    s.acc_off = -1;
  }
  return VMCF_OK;
}

int plan(vmcf_system_s& s) {
  const size_t tsz = s.precision == VMCF_FP64 ? 8 : 4;
  s.GS = (s.nmax <= 24) ? 32 : 128;
  s.GSm = (s.nmax <= 24) ? 32 : 256;
  s.Lrm = layout_refresh_move(s, tsz, s.GS);
  const int maxg = s.GS == 32 ? 4 : 1;
  s.gpb_rm = std::max(1, std::min(maxg, kSmemCap / std::max(1, s.Lrm.bytes)));
  if (s.Lrm.bytes > kSmemCap) return fail(VMCF_ENOTSUP, "system too large for the shared-memory plan (sampling)");
  return plan_measure(s);
}

// Small-system path: one lane per electron in the measurement, one lane per walker in the
// moves. Eligible when the electrons fit one warp, the orbitals per spin fit a 16-wide
// register row, and the shared-memory plan fits.
void plan_small(vmcf_system_s& s) {
  s.small = false;
  if (s.Ne > 32 || s.nmax > 16) return;
  const int tsz = s.precision == VMCF_FP64 ? 8 : 4;
  s.small_nm = s.nmax <= 8 ? 8 : (s.nmax <= 14 ? 14 : 16);  // register-row width; staged rows padded to 4
  SmallLayout L{};
  L.chunk = 21;  // odd row stride: lanes writing phi[e][c] fall in distinct banks
  int o = 0;
  auto take = [&](int bytes) { int at = o; o = align16(o + bytes); return at; };
  L.pd = take(8 * 3 * s.Ne);
  L.ph = take(4 * 3 * s.Ne);
  L.pl = take(4 * 3 * s.Ne);
  L.frc = take(tsz * 6 * s.K);
  L.red = take(16);
  L.scal = take(32);
  // from here to phi's end: work space that is dead before pass 1 and after pass 3
  const int dead0 = o;
  L.Ad = take(8 * s.nB);
  L.Bf = (tsz == 8) ? L.Ad : take(tsz * s.nB);
  L.Pm = take(tsz * s.nB);
  L.Q = take(tsz * s.nmax * s.nmax);
  L.piv = take(4 * 2 * s.nmax);           // both spin blocks are inverted at once
  L.f = take(8 * 2 * (3 * s.nmax + 1));
  L.phi = take(tsz * s.Ne * L.chunk);
  const int dead1 = o;
  if (s.MJ > 0) {  // AO-expanded Jastrow terms: [Ne][JS] rows (in the dead block when they fit), [3][MJp] vectors
    const int MJp = (s.MJ + 3) / 4 * 4;
    int JS = MJp;
    while ((JS * tsz / 16) % 2 == 0) JS += 16 / tsz;  // 16-byte row loads of a warp's lanes in distinct banks
    L.JS = JS;
    L.jv = take(tsz * 3 * MJp);
    const int need = tsz * s.Ne * JS;
    L.jA = need <= dead1 - dead0 ? dead0 : take(need);
  }
  L.bytes = align16(o);
  L.cta_C = 0;
  L.cta_acc = align16(tsz * 2 * s.M * ((s.small_nm + 3) / 4 * 4));
  L.cta_bytes = L.cta_acc + align16(tsz * s.accL);
  // with the tensor-core walker sums the accumulator leaves out the O range (2 M Ne entries)
  L.cta_bytes_tc = L.cta_acc + align16(tsz * (s.accL - 2 * s.M * s.Ne));
  int warps = 8;
  while (warps > 2 && L.cta_bytes + warps * L.bytes > kSmemCap) warps /= 2;
  if (L.cta_bytes + warps * L.bytes > kSmemCap) return;
  s.SL = L;
  s.small_warps = warps;
  // proposal kernel: staged C, and with the Jastrow-basis terms Xi and per warp the rows dphi_e and vectors s, t0
  const size_t cbytes = vmcf::propose_c_bytes(s.M, (s.small_nm + 3) / 4 * 4, tsz);
  const size_t pw = vmcf::propose_jb_bytes(s.Ne, s.MJ, L.JS, tsz);
  int pwarps = vmcf::kProposeWarps;
  const size_t xbytes = vmcf::propose_xi_bytes(s.MJ, tsz);
  while (pwarps > 1 && cbytes + xbytes + pwarps * pw > (size_t)kSmemCap) pwarps /= 2;
  if (cbytes + xbytes + pwarps * pw > (size_t)kSmemCap) return;
  s.propose_warps = pwarps;
  s.small_move_smem = cbytes + vmcf::propose_xi_bytes(s.MJ, tsz) + pwarps * pw;
  s.small = true;
  s.tc_Mp = (s.M + 7) / 8 * 8;
  s.tc_Np = (2 * s.nmax + 15) / 16 * 16;
  s.tc_nch = 1;
  s.tc_sums = s.precision == VMCF_MIXED;
}

Launch launch_rm(const vmcf_system_s& s, int W) {
  Launch lc{};
  lc.GS = s.GS;
  lc.groups = s.gpb_rm;
  lc.grid = (W + lc.groups - 1) / lc.groups;
  lc.L = s.Lrm;
  lc.smem = (size_t)lc.groups * s.Lrm.bytes;
  lc.acc_off = -1;
  return lc;
}

}  // namespace

GroupLayout vmcf::group_layout_rm(const vmcf_system_s& s, int GS) {
  return layout_refresh_move(s, s.precision == VMCF_FP64 ? 8 : 4, GS);
}

GroupLayout vmcf::group_layout_meas(const vmcf_system_s& s, int GS) {
  return layout_measure(s, s.precision == VMCF_FP64 ? 8 : 4, GS, false);
}

GroupLayout vmcf::group_layout_meas_tc(const vmcf_system_s& s, int GS) {
  return layout_measure(s, s.precision == VMCF_FP64 ? 8 : 4, GS, false, s.tcg_Mf);
}

Launch vmcf::launch_meas(const vmcf_system_s& s, int grid, bool accum, bool withD) {
  Launch lc{};
  lc.GS = s.GSm;
  if (withD) {
    lc.groups = s.gpb_measD;
    lc.L = s.LmeasD;
    lc.smem = (size_t)lc.groups * s.LmeasD.bytes;
    lc.acc_off = -1;
  } else if (accum && s.acc_smem) {
    lc.groups = s.gpb_meas;
    lc.L = s.Lmeas;
    lc.acc_off = s.acc_off;
    const size_t tsz = s.precision == VMCF_FP64 ? 8 : 4;
    lc.smem = (size_t)s.acc_off + align16((int)tsz * s.accL);
  } else if (accum) {
    lc.groups = 1;
    lc.L = s.Lmeas;
    lc.smem = s.Lmeas.bytes;
    lc.acc_off = -1;
  } else {
    lc.groups = s.gpb_meas;
    lc.L = s.Lmeas;
    lc.smem = (size_t)lc.groups * s.Lmeas.bytes;
    lc.acc_off = -1;
  }
  lc.grid = grid;
  return lc;
}

int vmcf::set_last_error(int code, const std::string& msg) { return fail(code, msg); }

namespace {

bool finite_all(const double* p, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}

// Small path: measurement kernel settings for `W` walkers (grid for evaluate/refresh).
SmallMeasParams small_params(const vmcf_system_s& s, int W) {
  SmallMeasParams P{};
  P.W = W;
  P.accL = s.accL;
  return P;
}

int launch_small_measure(vmcf_system_s* s, int grid, const SmallMeasParams& P, cudaStream_t st) {
  cudaError_t e = s->precision == VMCF_FP64
                      ? launch_measure_small<double>(s->dev, s->small_nm, s->SL, grid, s->small_warps, P, st)
                      : launch_measure_small<float>(s->dev, s->small_nm, s->SL, grid, s->small_warps, P, st);
  if (e != cudaSuccess) return cuda_fail(e, "small measurement kernel launch");
  return VMCF_OK;
}

// Walkers per CTA of the move kernel: one CTA per SM when the walkers, their inverses and
// positions fit shared memory, else as many as fit.
int move_walkers_per_cta(const vmcf_system_s& s, int W, int lpw) {
  const size_t tsz = s.precision == VMCF_FP64 ? 8 : 4;
  const size_t per = tsz * s.nB + 8 * 3 * (size_t)s.Ne;
  const size_t room = (size_t)kSmemCap - 8;  // inverses and positions only (8 bytes of alignment padding)
  int cap = (int)std::min<size_t>(room / per, (size_t)(256 / lpw));  // 256 threads per CTA at most
  int want = (W + s.small_sms - 1) / s.small_sms;
  return std::max(1, std::min(cap, want));
}

int eval_grid(const vmcf_system_s& s, int W) { return std::max(1, (W + 2 * s.small_warps - 1) / (2 * s.small_warps)); }

// Fresh inverses from the current positions.
int do_refresh(vmcf_system_s* s, vmcf_walkers_s* wk, cudaStream_t st) {
  if (s->small) {
    Timed tm(wk, 2, st);
    SmallMeasParams P = small_params(*s, wk->W);
    P.pos = wk->pos;
    P.pos_sk = wk->W;
    P.pos_sw = 1;
    P.mode = 0;
    P.Bout = wk->B;
    P.counters = wk->counters;
    // one wave of resident CTAs, each taking a contiguous range of walkers (no partial last wave)
    int rc = launch_small_measure(s, std::max(1, std::min(eval_grid(*s, wk->W), s->small_res)), P, st);
    if (rc != VMCF_OK) return rc;
    wk->counter = 0;
    return VMCF_OK;
  }
  const Launch lc = launch_rm(*s, wk->W);
  Timed tm(wk, 2, st);
  cudaError_t e = s->precision == VMCF_FP64
                      ? launch_refresh<double>(s->dev, lc, wk->pos, wk->B, wk->W, wk->counters, st)
                      : launch_refresh<float>(s->dev, lc, wk->pos, wk->B, wk->W, wk->counters, st);
  if (e != cudaSuccess) return cuda_fail(e, "refresh kernel launch");
  wk->counter = 0;
  return VMCF_OK;
}

// Bring positions in the ABI layout [W][Ne][3] (device or host) into the walker state.
int load_positions_state(vmcf_system_s* s, vmcf_walkers_s* wk, const double* pos, int is_host, cudaStream_t st) {
  const size_t bytes = 8 * (size_t)wk->W * 3 * s->Ne;
  const cudaMemcpyKind kind = is_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  if (!s->small) {
    VMCF_CUDA(cudaMemcpyAsync(wk->pos, pos, bytes, kind, st));
    return VMCF_OK;
  }
  VMCF_CUDA(cudaMemcpyAsync(wk->stage, pos, bytes, kind, st));
  VMCF_CUDA(launch_to_interleaved(wk->stage, wk->pos, wk->posf, wk->W, 3 * s->Ne, st));
  return VMCF_OK;
}

// FP64 slots of the tensor-core sums: [2 spins][tiles][nblocks * tc_cpb][128][32].
size_t tc_slot_doubles(const vmcf_system_s& s, const vmcf_walkers_s& wk) {
  const int Mf = s.small ? s.tc_Mp : s.tcg_Mf, Nf = s.small ? s.tc_Np : s.tcg_Nf;
  const size_t tiles = (size_t)((Mf + 127) / 128) * ((Nf + 31) / 32);
  return 2 * tiles * (size_t)wk.nblocks * wk.tc_cpb * 128 * 32;
}

// Tensor-core walker sums: bf16 tiles (zero-filled: electron slots beyond n, AO rows beyond M and
// Y columns beyond 2n are never written and must stay zero), FP64 slots and an error flag.
cudaError_t alloc_tc(vmcf_system_s* s, vmcf_walkers_s* wk) {
  const size_t W = wk->W;
  const size_t Mf = s->small ? s->tc_Mp : s->tcg_Mf, Nf = s->small ? s->tc_Np : s->tcg_Nf;
  const size_t nch = s->small ? s->tc_nch : s->tcg_nch;
  // CTAs per jackknife block of the walker-sum GEMM: as many as fit one wave of resident CTAs (a second,
  // partial wave would double the kernel's time), at most one per 16 walkers
  {
    int per_sm = 1, dev = 0, sms = 1;
    cudaError_t e0 = tc_sumprod_ctas_per_sm((int)Mf, (int)Nf, &per_sm);
    if (e0 == cudaSuccess) e0 = cudaGetDevice(&dev);
    if (e0 == cudaSuccess) e0 = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e0 != cudaSuccess) return e0;
    const size_t tiles = ((Mf + 127) / 128) * ((Nf + 31) / 32);
    const size_t wave = (size_t)std::max(1, per_sm) * sms / (2 * tiles * wk->nblocks);
    wk->tc_cpb = (int)std::max<size_t>(1, std::min<size_t>(wave, W / ((size_t)wk->nblocks * 16)));
  }
  cudaError_t e;
  for (int k = 0; k < 2; ++k) {
    if ((e = cudaMalloc(&wk->phiT[k], 2 * W * nch * Mf * 16))) return e;
    if ((e = cudaMalloc(&wk->yT[k], 2 * W * nch * Nf * 16))) return e;
    if ((e = cudaMemset(wk->phiT[k], 0, 2 * W * nch * Mf * 16))) return e;
    if ((e = cudaMemset(wk->yT[k], 0, 2 * W * nch * Nf * 16))) return e;
  }
  wk->tc_slot_doubles = tc_slot_doubles(*s, *wk);
  if ((e = cudaMalloc(&wk->tc_slots, 8 * wk->tc_slot_doubles))) return e;
  if ((e = cudaMemset(wk->tc_slots, 0, 8 * wk->tc_slot_doubles))) return e;
  if ((e = cudaMalloc(&wk->tc_flag, sizeof(int)))) return e;
  if ((e = cudaMemset(wk->tc_flag, 0, sizeof(int)))) return e;
  wk->tc = true;
  return cudaSuccess;
}

// One measurement of the walker state: the small-path kernel, and in tensor-core mode the
// walker-sum GEMM over the tiles it wrote.
int measure_state_small(vmcf_system_s* s, vmcf_walkers_s* wk, cudaStream_t st) {
  SmallMeasParams M = small_params(*s, wk->W);
  M.pos = wk->pos;
  M.pos_sk = wk->W;
  M.pos_sw = 1;
  M.mode = 2;
  M.Bout = wk->B;
  M.acc = wk->acc;
  M.swct_off = swct_offset(*s);
  M.eps = wk->eps;
  M.e_ref = wk->e_ref;
  M.counters = wk->counters;
  const bool tc = wk->tc && s->tc_sums;
  if (tc) {
    for (int k = 0; k < 2; ++k) {
      M.phiT[k] = wk->phiT[k];
      M.yT[k] = wk->yT[k];
    }
    M.Mp = s->tc_Mp;
    M.Np = s->tc_Np;
  }
  {
    Timed tm(wk, 1, st);
    int rc = launch_small_measure(s, wk->grid_meas, M, st);
    if (rc != VMCF_OK) return rc;
  }
  if (tc) {
    Timed tm(wk, 3, st);
    cudaError_t e = launch_tc_sumprod(wk->phiT[0], wk->phiT[1], wk->yT[0], wk->yT[1], wk->W, 1, s->tc_Mp, s->tc_Np,
                                      s->nup, s->ndn, wk->nblocks * wk->tc_cpb, wk->tc_slots, wk->tc_flag, st);
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core walker-sum kernel launch");
  }
  return VMCF_OK;
}

// One accumulate-mode measurement on the walker-group kernels; with tensor-core sums the kernel
// stages AO values and B rows as bf16 tiles and the GEMM kernel adds the O sums to its slots.
int measure_state_group(vmcf_system_s* s, vmcf_walkers_s* wk, cudaStream_t st) {
  MeasParams M{};
  M.pos = wk->pos;
  M.Bout = wk->B;
  M.acc = wk->acc;
  M.swct_off = swct_offset(*s);
  M.eps = wk->eps;
  M.accL = s->accL;
  M.acc_in_smem = s->acc_smem ? 1 : 0;
  M.e_ref = wk->e_ref;
  M.counters = wk->counters;
  M.W = wk->W;
  const bool tc = wk->tc && s->tcg_sums;
  Launch lme = launch_meas(*s, wk->grid_meas, true, false);
  if (tc) {
    for (int k = 0; k < 2; ++k) {
      M.phiT[k] = wk->phiT[k];
      M.yT[k] = wk->yT[k];
    }
    M.nch = s->tcg_nch;
    M.Mf = s->tcg_Mf;
    M.Nf = s->tcg_Nf;
    // one walker group per CTA, its non-O sums straight to the CTA's FP64 slot
    lme.L = s->LmeasTC;
    lme.groups = 1;
    lme.acc_off = -1;
    lme.smem = s->LmeasTC.bytes;
    M.acc_in_smem = 0;
  }
  {
    Timed tm(wk, 1, st);
    cudaError_t e = s->precision == VMCF_FP64 ? launch_measure<double>(s->dev, lme, M, st)
                                              : launch_measure<float>(s->dev, lme, M, st);
    if (e != cudaSuccess) return cuda_fail(e, "measure kernel launch");
  }
  if (tc) {
    Timed tm(wk, 3, st);
    cudaError_t e = launch_tc_sumprod(wk->phiT[0], wk->phiT[1], wk->yT[0], wk->yT[1], wk->W, s->tcg_nch, s->tcg_Mf,
                                      s->tcg_Nf, s->nup, s->ndn, wk->nblocks * wk->tc_cpb, wk->tc_slots, wk->tc_flag,
                                      st);
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core walker-sum kernel launch");
  }
  return VMCF_OK;
}
}  // namespace

// Re-inversion of a walker set from its positions (chain clock reset), for the batch entry points.
int vmcf::refresh_walker_set(vmcf_system_s* s, vmcf_walkers_s* wk, cudaStream_t st) { return do_refresh(s, wk, st); }

cudaError_t vmcf::small_sweep_launches(vmcf_system_s* s, vmcf_walkers_s* wk, const BatchClock* clk, int mode, int kref,
                                       double sigma, cudaStream_t st) {
  const bool fp64 = s->precision == VMCF_FP64;
  SmallProposeParams Q{};
  Q.pos = wk->pos;
  Q.posf = wk->posf;
  Q.pr = wk->pr;
  Q.W = wk->W;
  Q.wid0 = wk->wid0;
  Q.k0 = wk->k0;
  Q.k1 = wk->k1;
  Q.sigma = sigma;
  Q.sigma_f = (float)sigma;
  Q.jJS = s->SL.JS;
  Q.clk = clk;
  const int qgrid = std::max(1, std::min((wk->W + s->propose_warps - 1) / s->propose_warps, 8 * s->small_sms));
  cudaError_t e = fp64 ? launch_propose_small<double>(s->dev, s->small_nm, qgrid, s->propose_warps, s->small_move_smem, Q, st)
                       : launch_propose_small<float>(s->dev, s->small_nm, qgrid, s->propose_warps, s->small_move_smem, Q, st);
  SmallMoveParams P{};
  P.pos = wk->pos;
  P.posf = wk->posf;
  P.B = wk->B;
  P.pr = wk->pr;
  P.nacc = wk->nacc;
  P.nrej = wk->nrej;
  P.W = wk->W;
  P.wid0 = wk->wid0;
  P.k0 = wk->k0;
  P.k1 = wk->k1;
  P.sigma = sigma;
  P.eps = wk->eps;
  P.clk = clk;
  P.kref = kref;
  P.measure = mode != 0;
  const int lpw = wk->eps > 0.0 ? 2 : s->move_lpw;
  P.wpc = move_walkers_per_cta(*s, wk->W, lpw);
  SmallMeasParams R = small_params(*s, wk->W);
  R.pos = wk->pos;
  R.pos_sk = wk->W;
  R.pos_sw = 1;
  R.mode = 0;
  R.Bout = wk->B;
  R.counters = wk->counters;
  R.clk = clk;
  R.kref = kref;
  R.measure = mode != 0;
  // at most ceil(Ne / k) + 1 runs of moves per sweep (the first run is shorter when the sweep starts
  // part-way to a re-inversion); launches past the sweep's schedule do nothing
  const int nseg = (s->Ne + kref - 1) / kref + 1;
  for (int seg = 0; seg < nseg && e == cudaSuccess; ++seg) {
    P.seg = seg;
    R.seg = seg;
    e = fp64 ? launch_move_small<double>(s->dev, s->small_nm, lpw, wk->W, 0, P, st)
             : launch_move_small<float>(s->dev, s->small_nm, lpw, wk->W, 0, P, st);
    if (e == cudaSuccess)
      e = fp64 ? launch_measure_small<double>(s->dev, s->small_nm, s->SL, eval_grid(*s, wk->W), s->small_warps, R, st)
               : launch_measure_small<float>(s->dev, s->small_nm, s->SL, eval_grid(*s, wk->W), s->small_warps, R, st);
  }
  if (e != cudaSuccess || mode != 1) return e;
  SmallMeasParams M = small_params(*s, wk->W);
  M.pos = wk->pos;
  M.pos_sk = wk->W;
  M.pos_sw = 1;
  M.mode = 2;
  M.Bout = wk->B;
  M.acc = wk->acc;
  M.swct_off = swct_offset(*s);
  M.eps = wk->eps;
  M.e_ref = wk->e_ref;
  M.counters = wk->counters;
  const bool tc = wk->tc && s->tc_sums;
  if (tc) {
    for (int k = 0; k < 2; ++k) {
      M.phiT[k] = wk->phiT[k];
      M.yT[k] = wk->yT[k];
    }
    M.Mp = s->tc_Mp;
    M.Np = s->tc_Np;
  }
  e = fp64 ? launch_measure_small<double>(s->dev, s->small_nm, s->SL, wk->grid_meas, s->small_warps, M, st)
           : launch_measure_small<float>(s->dev, s->small_nm, s->SL, wk->grid_meas, s->small_warps, M, st);
  if (e == cudaSuccess && tc)
    e = launch_tc_sumprod(wk->phiT[0], wk->phiT[1], wk->yT[0], wk->yT[1], wk->W, 1, s->tc_Mp, s->tc_Np, s->nup, s->ndn,
                          wk->nblocks * wk->tc_cpb, wk->tc_slots, wk->tc_flag, st);
  return e;
}

extern "C" {

const char* vmcf_strerror(int status) {
  switch (status) {
    case VMCF_OK: return "ok";
    case VMCF_EINVAL: return "invalid argument";
    case VMCF_ENOMEM: return "out of memory";
    case VMCF_ECUDA: return "CUDA error";
    case VMCF_ESINGULAR: return "singular Slater matrix";
    case VMCF_ETIMEOUT: return "device wait timed out";
    case VMCF_ENOTSUP: return "not supported";
    default: return "unknown status";
  }
}

const char* vmcf_last_error(void) { return g_last_error.c_str(); }

int vmcf_init_system(const vmcf_nuclei* nuc, const vmcf_basis* bas, const double* C_up, const double* C_dn,
                     int n_up, int n_dn, const vmcf_jastrow* jas, const double* S, int precision,
                     vmcf_system_t* out) {
  if (!out) return fail(VMCF_EINVAL, "out is NULL");
  *out = nullptr;
  if (!nuc || !bas || !jas || !C_up) return fail(VMCF_EINVAL, "NULL input");
  const bool force_group = (precision & VMCF_FORCE_GROUP_PATH) != 0;
  const bool swct = (precision & VMCF_SPACE_WARP) != 0;
  precision &= ~(VMCF_FORCE_GROUP_PATH | VMCF_SPACE_WARP);
  if (precision != VMCF_FP64 && precision != VMCF_MIXED) return fail(VMCF_EINVAL, "bad precision");
  if (jas->two_body_exp && jas->enable_J2 && !(jas->F_anti > 0.0 && jas->F_par > 0.0))
    return fail(VMCF_EINVAL, "the exponential two-body form needs F_anti, F_par > 0");
  if (nuc->K < 1 || !nuc->Z || !nuc->R) return fail(VMCF_EINVAL, "need at least one nucleus");
  if (!finite_all(nuc->R, 3 * (size_t)nuc->K)) return fail(VMCF_EINVAL, "nuclear positions not finite");
  for (int I = 0; I < nuc->K; ++I)
    if (nuc->Z[I] < 1) return fail(VMCF_EINVAL, "nuclear charge < 1");
  if (bas->nshell < 1 || bas->maxprim < 1 || bas->maxprim > kMaxPrim || !bas->center || !bas->l || !bas->nprim ||
      !bas->exps || !bas->coefs)
    return fail(VMCF_EINVAL, "bad basis description");
  if (n_up < 1 || n_dn < 0 || n_dn > n_up || n_up > 64) return fail(VMCF_EINVAL, "need 1 <= n_dn <= n_up <= 64");
  if (n_dn > 0 && !C_dn) return fail(VMCF_EINVAL, "C_dn is NULL");

  auto* s = new vmcf_system_s();
  s->precision = precision;
  s->swct = swct;
  s->K = nuc->K;
  s->nshell = bas->nshell;
  s->nup = n_up;
  s->ndn = n_dn;
  s->Ne = n_up + n_dn;
  s->nB = n_up * n_up + n_dn * n_dn;
  s->nmax = std::max(n_up, n_dn);
  s->R.assign(nuc->R, nuc->R + 3 * s->K);
  s->Z.resize(s->K);
  for (int I = 0; I < s->K; ++I) s->Z[I] = nuc->Z[I];

  std::vector<int4> shells;
  std::vector<int> sharp;
  std::vector<double> alpha, coef;
  int M = 0;
  std::string why;
  if (!shell_tables(*bas, s->K, shells, sharp, alpha, coef, s->ao_center, &M, &why)) {
    delete s;
    return fail(VMCF_EINVAL, why);
  }
  s->M = M;
  if (M > 1024) {
    delete s;
    return fail(VMCF_ENOTSUP, "more than 1024 AOs");
  }
  // AO-expanded Jastrow terms: the Jastrow basis and its coefficients
  std::vector<int4> jshells;
  std::vector<int> jsharp, jcenter;
  std::vector<double> jalpha, jcoef, jxi, jXi;
  if (jas->basis) {
    const vmcf_basis* jb = jas->basis;
    if (jb->nshell < 1 || jb->maxprim < 1 || jb->maxprim > kMaxPrim || !jb->center || !jb->l || !jb->nprim ||
        !jb->exps || !jb->coefs) {
      delete s;
      return fail(VMCF_EINVAL, "bad Jastrow basis description");
    }
    int MJ = 0;
    if (!shell_tables(*jb, s->K, jshells, jsharp, jalpha, jcoef, jcenter, &MJ, &why)) {
      delete s;
      return fail(VMCF_EINVAL, "Jastrow basis: " + why);
    }
    if (MJ > 1024) {
      delete s;
      return fail(VMCF_ENOTSUP, "more than 1024 Jastrow basis functions");
    }
    jxi.assign(MJ, 0.0);
    jXi.assign((size_t)MJ * MJ, 0.0);
    if (jas->xi) jxi.assign(jas->xi, jas->xi + MJ);
    if (jas->Xi) jXi.assign(jas->Xi, jas->Xi + (size_t)MJ * MJ);
    jXi.resize((size_t)((MJ + 3) / 4 * 4) * MJ, 0.0);  // zero rows up to a multiple of 4
    if (!finite_all(jxi.data(), jxi.size()) || !finite_all(jXi.data(), jXi.size())) {
      delete s;
      return fail(VMCF_EINVAL, "Jastrow coefficients not finite");
    }
    double big = 0.0;
    for (double v : jXi) big = std::max(big, std::fabs(v));
    for (int a = 0; a < MJ; ++a)
      for (int b = a + 1; b < MJ; ++b)
        if (std::fabs(jXi[(size_t)a * MJ + b] - jXi[(size_t)b * MJ + a]) > 1e-12 * std::max(1.0, big)) {
          delete s;
          return fail(VMCF_EINVAL, "Xi must be symmetric");
        }
    s->MJ = MJ;
    s->nJs = jb->nshell;
  }
  s->C[0].assign(C_up, C_up + (size_t)M * n_up);
  if (n_dn > 0) s->C[1].assign(C_dn, C_dn + (size_t)M * n_dn);
  if (!finite_all(s->C[0].data(), s->C[0].size()) || !finite_all(s->C[1].data(), s->C[1].size())) {
    delete s;
    return fail(VMCF_EINVAL, "C not finite");
  }
  for (int sg = 0; sg < 2; ++sg)
    if (!independent_columns(s->C[sg], M, sg == 0 ? n_up : n_dn)) {
      delete s;
      return fail(VMCF_EINVAL, std::string("the columns of C_") + (sg == 0 ? "up" : "dn") +
                                   " are linearly dependent (every Slater matrix would be singular)");
    }
  if (S) {
    s->S.assign(S, S + (size_t)M * M);
    s->has_S = true;
  }
  // nuclear repulsion and its derivative
  double Vnn = 0.0;
  std::vector<double> dVnn(3 * s->K, 0.0);
  for (int I = 0; I < s->K; ++I)
    for (int J = 0; J < s->K; ++J) {
      if (I == J) continue;
      double d[3], r2 = 0.0;
      for (int k = 0; k < 3; ++k) {
        d[k] = s->R[3 * I + k] - s->R[3 * J + k];
        r2 += d[k] * d[k];
      }
      if (!(r2 > 1e-12)) {
        delete s;
        return fail(VMCF_EINVAL, "two nuclei at the same position");
      }
      const double r = std::sqrt(r2);
      if (J > I) Vnn += s->Z[I] * s->Z[J] / r;
      for (int k = 0; k < 3; ++k) dVnn[3 * I + k] -= s->Z[I] * s->Z[J] * d[k] / (r2 * r);
    }

  int rc = plan(*s);
  if (rc != VMCF_OK) {
    delete s;
    return rc;
  }
  if (!force_group) plan_small(*s);
  s->tcg_sums = !s->small && s->precision == VMCF_MIXED;

  // one device allocation for all tables
  std::vector<float> alpha_f(alpha.begin(), alpha.end()), coef_f(coef.begin(), coef.end());
  std::vector<float> alpha_lo(alpha.size());
  for (size_t i = 0; i < alpha.size(); ++i) alpha_lo[i] = (float)(alpha[i] - (double)alpha_f[i]);
  std::vector<float> Rh(3 * s->K), Rl(3 * s->K);
  for (int i = 0; i < 3 * s->K; ++i) {
    Rh[i] = (float)s->R[i];
    Rl[i] = (float)(s->R[i] - (double)Rh[i]);
  }
  std::vector<float> Cf0(s->C[0].begin(), s->C[0].end()), Cf1(s->C[1].begin(), s->C[1].end());
  // C^s transposed, [n_s][M]: read along mu by consecutive threads
  std::vector<double> CT[2];
  std::vector<float> CfT[2];
  for (int sg = 0; sg < 2; ++sg) {
    const int n = sg == 0 ? n_up : n_dn;
    CT[sg].assign((size_t)std::max(1, n * M), 0.0);
    CfT[sg].assign((size_t)std::max(1, n * M), 0.f);
    for (int mu = 0; mu < M; ++mu)
      for (int i = 0; i < n; ++i) {
        CT[sg][(size_t)i * M + mu] = s->C[sg][(size_t)mu * n + i];
        CfT[sg][(size_t)i * M + mu] = (float)s->C[sg][(size_t)mu * n + i];
      }
  }
  // shell groups: maximal runs of consecutive shells with one centre and one angular momentum,
  // (first shell, count, l + 256 if a shell of the run has sharp primitives, centre)
  std::vector<int4> groups;
  for (int sh = 0; sh < (int)shells.size(); ++sh) {
    const int sflag = sharp[sh] ? 256 : 0;
    if (!groups.empty() && groups.back().w == shells[sh].x && (groups.back().z & 255) == shells[sh].y &&
        groups.back().x + groups.back().y == sh) {
      ++groups.back().y;
      groups.back().z |= sflag;
    } else {
      groups.push_back(make_int4(sh, 1, shells[sh].y | sflag, shells[sh].x));
    }
  }
  size_t off = 0;
  auto slot = [&](size_t bytes) { size_t at = off; off = (off + bytes + 255) & ~size_t(255); return at; };
  const size_t oGrp = slot(sizeof(int4) * groups.size());
  std::vector<float> Zf(s->Z.begin(), s->Z.end());
  const size_t oZf = slot(4 * Zf.size());
  const size_t oR = slot(8 * s->R.size()), oZ = slot(8 * s->Z.size()), oSh = slot(sizeof(int4) * shells.size()),
               oA = slot(8 * alpha.size()), oC = slot(8 * coef.size()), oAf = slot(4 * alpha.size()),
               oCf = slot(4 * coef.size()), oAoc = slot(4 * (size_t)M), oC0 = slot(8 * s->C[0].size()),
               oC1 = slot(8 * std::max<size_t>(1, s->C[1].size())), oCf0 = slot(4 * Cf0.size()),
               oCf1 = slot(4 * std::max<size_t>(1, Cf1.size())), oDv = slot(8 * dVnn.size()), oCnt = slot(16),
               oRh = slot(4 * Rh.size()), oRl = slot(4 * Rl.size()), oSharp = slot(4 * sharp.size()),
               oAlo = slot(4 * alpha_lo.size()), oCT0 = slot(8 * CT[0].size()), oCT1 = slot(8 * CT[1].size()),
               oCfT0 = slot(4 * CfT[0].size()), oCfT1 = slot(4 * CfT[1].size());
  // Jastrow basis tables (AO-expanded Jastrow terms), double and float copies
  std::vector<float> jalpha_f(jalpha.begin(), jalpha.end()), jcoef_f(jcoef.begin(), jcoef.end());
  std::vector<float> jxi_f(jxi.begin(), jxi.end()), jXi_f(jXi.begin(), jXi.end());
  const int MJp = (s->MJ + 3) / 4 * 4;
  std::vector<double> jXr((size_t)s->MJ * MJp, 0.0);  // rows of Xi padded to MJp
  for (int a = 0; a < s->MJ; ++a)
    for (int c = 0; c < s->MJ; ++c) jXr[(size_t)a * MJp + c] = jXi[(size_t)a * s->MJ + c];
  std::vector<float> jXr_f(jXr.begin(), jXr.end());
  const size_t oJs = slot(sizeof(int4) * jshells.size()), oJa = slot(8 * jalpha.size()), oJc = slot(8 * jcoef.size()),
               oJaf = slot(4 * jalpha.size()), oJcf = slot(4 * jcoef.size()), oJcen = slot(4 * jcenter.size()),
               oJxi = slot(8 * jxi.size()), oJxif = slot(4 * jxi.size()), oJXi = slot(8 * jXi.size()),
               oJXif = slot(4 * jXi.size()), oJXr = slot(8 * jXr.size()), oJXrf = slot(4 * jXr.size());
  cudaError_t e = cudaMalloc(&s->dmem, off);
  if (e != cudaSuccess) {
    delete s;
    return cuda_fail(e, "cudaMalloc(system tables)");
  }
  if ((e = cudaGetDevice(&s->device)) != cudaSuccess) {
    cudaFree(s->dmem);
    delete s;
    return cuda_fail(e, "cudaGetDevice");
  }
  char* b = static_cast<char*>(s->dmem);
  auto up = [&](size_t at, const void* src, size_t bytes) {
    return bytes ? cudaMemcpy(b + at, src, bytes, cudaMemcpyHostToDevice) : cudaSuccess;
  };
  cudaError_t ce = cudaSuccess;
  ce = ce ? ce : up(oR, s->R.data(), 8 * s->R.size());
  ce = ce ? ce : up(oZ, s->Z.data(), 8 * s->Z.size());
  ce = ce ? ce : up(oSh, shells.data(), sizeof(int4) * shells.size());
  ce = ce ? ce : up(oGrp, groups.data(), sizeof(int4) * groups.size());
  ce = ce ? ce : up(oZf, Zf.data(), 4 * Zf.size());
  ce = ce ? ce : up(oA, alpha.data(), 8 * alpha.size());
  ce = ce ? ce : up(oC, coef.data(), 8 * coef.size());
  ce = ce ? ce : up(oAf, alpha_f.data(), 4 * alpha_f.size());
  ce = ce ? ce : up(oCf, coef_f.data(), 4 * coef_f.size());
  ce = ce ? ce : up(oAoc, s->ao_center.data(), 4 * (size_t)M);
  ce = ce ? ce : up(oC0, s->C[0].data(), 8 * s->C[0].size());
  ce = ce ? ce : up(oC1, s->C[1].data(), 8 * s->C[1].size());
  ce = ce ? ce : up(oCf0, Cf0.data(), 4 * Cf0.size());
  ce = ce ? ce : up(oCf1, Cf1.data(), 4 * Cf1.size());
  ce = ce ? ce : up(oDv, dVnn.data(), 8 * dVnn.size());
  ce = ce ? ce : cudaMemset(b + oCnt, 0, 16);
  ce = ce ? ce : up(oRh, Rh.data(), 4 * Rh.size());
  ce = ce ? ce : up(oRl, Rl.data(), 4 * Rl.size());
  ce = ce ? ce : up(oSharp, sharp.data(), 4 * sharp.size());
  ce = ce ? ce : up(oAlo, alpha_lo.data(), 4 * alpha_lo.size());
  ce = ce ? ce : up(oCT0, CT[0].data(), 8 * CT[0].size());
  ce = ce ? ce : up(oCT1, CT[1].data(), 8 * CT[1].size());
  ce = ce ? ce : up(oCfT0, CfT[0].data(), 4 * CfT[0].size());
  ce = ce ? ce : up(oCfT1, CfT[1].data(), 4 * CfT[1].size());
  ce = ce ? ce : up(oJs, jshells.data(), sizeof(int4) * jshells.size());
  ce = ce ? ce : up(oJa, jalpha.data(), 8 * jalpha.size());
  ce = ce ? ce : up(oJc, jcoef.data(), 8 * jcoef.size());
  ce = ce ? ce : up(oJaf, jalpha_f.data(), 4 * jalpha_f.size());
  ce = ce ? ce : up(oJcf, jcoef_f.data(), 4 * jcoef_f.size());
  ce = ce ? ce : up(oJcen, jcenter.data(), 4 * jcenter.size());
  ce = ce ? ce : up(oJxi, jxi.data(), 8 * jxi.size());
  ce = ce ? ce : up(oJxif, jxi_f.data(), 4 * jxi_f.size());
  ce = ce ? ce : up(oJXi, jXi.data(), 8 * jXi.size());
  ce = ce ? ce : up(oJXif, jXi_f.data(), 4 * jXi_f.size());
  ce = ce ? ce : up(oJXr, jXr.data(), 8 * jXr.size());
  ce = ce ? ce : up(oJXrf, jXr_f.data(), 4 * jXr_f.size());
  if (ce == cudaSuccess) ce = s->precision == VMCF_FP64 ? set_smem_limits<double>(s->GS) : set_smem_limits<float>(s->GS);
  if (ce == cudaSuccess && s->small)
    ce = s->precision == VMCF_FP64 ? set_smem_limits_small<double>() : set_smem_limits_small<float>();
  if (ce == cudaSuccess && s->precision == VMCF_MIXED) ce = set_smem_limits_tc();
  if (ce == cudaSuccess && s->small) {
    int dev = 0, sms = 0;
    ce = cudaGetDevice(&dev);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t cta = (size_t)(s->tc_sums ? s->SL.cta_bytes_tc : s->SL.cta_bytes) + (size_t)s->small_warps * s->SL.bytes;
    const int by_smem = (int)((228 * 1024) / (cta + 1024));
    const int by_regs = 65536 / (32 * s->small_warps * 128);
    s->small_res = std::max(1, sms * std::max(1, std::min(by_smem, by_regs)));
    s->small_sms = std::max(1, sms);
  }
  if (ce != cudaSuccess) {
    cudaFree(s->dmem);
    delete s;
    return cuda_fail(ce, "uploading system tables");
  }
  DevSys& D = s->dev;
  D.K = s->K; D.M = M; D.nup = n_up; D.ndn = n_dn; D.Ne = s->Ne; D.nshell = s->nshell; D.nB = s->nB; D.nmax = s->nmax;
  D.R = reinterpret_cast<const double*>(b + oR);
  D.Z = reinterpret_cast<const double*>(b + oZ);
  D.shell = reinterpret_cast<const int4*>(b + oSh);
  D.shgrp = reinterpret_cast<const int4*>(b + oGrp);
  D.ngrp = (int)groups.size();
  D.alpha = reinterpret_cast<const double*>(b + oA);
  D.coef = reinterpret_cast<const double*>(b + oC);
  D.alpha_f = reinterpret_cast<const float*>(b + oAf);
  D.coef_f = reinterpret_cast<const float*>(b + oCf);
  D.ao_center = reinterpret_cast<const int*>(b + oAoc);
  D.Rh = reinterpret_cast<const float*>(b + oRh);
  D.Rl = reinterpret_cast<const float*>(b + oRl);
  D.sharp = reinterpret_cast<const int*>(b + oSharp);
  D.alpha_lo = reinterpret_cast<const float*>(b + oAlo);
  D.C[0] = reinterpret_cast<const double*>(b + oC0);
  D.C[1] = reinterpret_cast<const double*>(b + oC1);
  D.Cf[0] = reinterpret_cast<const float*>(b + oCf0);
  D.Cf[1] = reinterpret_cast<const float*>(b + oCf1);
  D.CT[0] = reinterpret_cast<const double*>(b + oCT0);
  D.CT[1] = reinterpret_cast<const double*>(b + oCT1);
  D.CfT[0] = reinterpret_cast<const float*>(b + oCfT0);
  D.CfT[1] = reinterpret_cast<const float*>(b + oCfT1);
  D.Fa = jas->F_anti; D.Fp = jas->F_par; D.aa = jas->a_anti; D.ap = jas->a_par; D.ben = jas->b_en;
  D.Fa_f = (float)D.Fa; D.Fp_f = (float)D.Fp; D.aa_f = (float)D.aa; D.ap_f = (float)D.ap; D.ben_f = (float)D.ben;
  D.Zf = reinterpret_cast<const float*>(b + oZf);
  D.J1 = jas->enable_J1 ? 1 : 0;
  D.J2 = jas->enable_J2 ? 1 : 0;
  D.swct = s->swct ? 1 : 0;
  D.j2exp = jas->two_body_exp ? 1 : 0;
  D.Vnn = Vnn;
  D.dVnn = reinterpret_cast<const double*>(b + oDv);
  D.nJs = s->nJs;
  D.MJ = s->MJ;
  D.MJp = (s->MJ + 3) / 4 * 4;
  if (s->MJ > 0) {
    D.jshell = reinterpret_cast<const int4*>(b + oJs);
    D.jalpha = reinterpret_cast<const double*>(b + oJa);
    D.jcoef = reinterpret_cast<const double*>(b + oJc);
    D.jalpha_f = reinterpret_cast<const float*>(b + oJaf);
    D.jcoef_f = reinterpret_cast<const float*>(b + oJcf);
    D.jcenter = reinterpret_cast<const int*>(b + oJcen);
    D.jxi = reinterpret_cast<const double*>(b + oJxi);
    D.jxi_f = reinterpret_cast<const float*>(b + oJxif);
    D.jXi = reinterpret_cast<const double*>(b + oJXi);
    D.jXi_f = reinterpret_cast<const float*>(b + oJXif);
    D.jXr = reinterpret_cast<const double*>(b + oJXr);
    D.jXr_f = reinterpret_cast<const float*>(b + oJXrf);
  }
  s->scratch_counters = reinterpret_cast<double*>(b + oCnt);
  const int trc = tc_rows_setup(s);
  if (trc != VMCF_OK) {
    cudaFree(s->tcr_mem);
    cudaFree(s->dmem);
    delete s;
    return trc;
  }
  *out = s;
  return VMCF_OK;
}

int vmcf_system_set_geometry(vmcf_system_t s, const double* R, const double* C_up, const double* C_dn,
                              const double* S) {
  if (!s || !R || !C_up) return fail(VMCF_EINVAL, "NULL input");
  if (s->ndn > 0 && !C_dn) return fail(VMCF_EINVAL, "C_dn is NULL");
  const int K = s->K, M = s->M, n_up = s->nup, n_dn = s->ndn;
  if (!finite_all(R, 3 * (size_t)K)) return fail(VMCF_EINVAL, "nuclear positions not finite");
  std::vector<double> C[2];
  C[0].assign(C_up, C_up + (size_t)M * n_up);
  if (n_dn > 0) C[1].assign(C_dn, C_dn + (size_t)M * n_dn);
  if (!finite_all(C[0].data(), C[0].size()) || !finite_all(C[1].data(), C[1].size()))
    return fail(VMCF_EINVAL, "C not finite");
  for (int sg = 0; sg < 2; ++sg)
    if (!independent_columns(C[sg], M, sg == 0 ? n_up : n_dn))
      return fail(VMCF_EINVAL, std::string("the columns of C_") + (sg == 0 ? "up" : "dn") +
                                   " are linearly dependent (every Slater matrix would be singular)");
  // nuclear repulsion and its derivative, as at creation
  double Vnn = 0.0;
  std::vector<double> dVnn(3 * K, 0.0);
  for (int I = 0; I < K; ++I)
    for (int J = 0; J < K; ++J) {
      if (I == J) continue;
      double d[3], r2 = 0.0;
      for (int k = 0; k < 3; ++k) {
        d[k] = R[3 * I + k] - R[3 * J + k];
        r2 += d[k] * d[k];
      }
      if (!(r2 > 1e-12)) return fail(VMCF_EINVAL, "two nuclei at the same position");
      const double r = std::sqrt(r2);
      if (J > I) Vnn += s->Z[I] * s->Z[J] / r;
      for (int k = 0; k < 3; ++k) dVnn[3 * I + k] -= s->Z[I] * s->Z[J] * d[k] / (r2 * r);
    }
  std::vector<float> Rh(3 * K), Rl(3 * K);
  for (int i = 0; i < 3 * K; ++i) {
    Rh[i] = (float)R[i];
    Rl[i] = (float)(R[i] - (double)Rh[i]);
  }
  DevSys& D = s->dev;
  cudaError_t e = cudaSetDevice(s->device);
  auto up = [&](const void* dst, const void* src, size_t bytes) {
    if (e == cudaSuccess && bytes) e = cudaMemcpy(const_cast<void*>(dst), src, bytes, cudaMemcpyHostToDevice);
  };
  up(D.R, R, 8 * 3 * (size_t)K);
  up(D.Rh, Rh.data(), 4 * Rh.size());
  up(D.Rl, Rl.data(), 4 * Rl.size());
  up(D.dVnn, dVnn.data(), 8 * dVnn.size());
  for (int sg = 0; sg < 2; ++sg) {
    const int n = sg == 0 ? n_up : n_dn;
    if (n == 0) continue;
    std::vector<float> Cf(C[sg].begin(), C[sg].end());
    std::vector<double> CT((size_t)n * M);
    std::vector<float> CfT((size_t)n * M);
    for (int mu = 0; mu < M; ++mu)
      for (int i = 0; i < n; ++i) {
        CT[(size_t)i * M + mu] = C[sg][(size_t)mu * n + i];
        CfT[(size_t)i * M + mu] = (float)C[sg][(size_t)mu * n + i];
      }
    up(D.C[sg], C[sg].data(), 8 * C[sg].size());
    up(D.Cf[sg], Cf.data(), 4 * Cf.size());
    up(D.CT[sg], CT.data(), 8 * CT.size());
    up(D.CfT[sg], CfT.data(), 4 * CfT.size());
  }
  if (e != cudaSuccess) return cuda_fail(e, "uploading the new geometry");
  s->R.assign(R, R + 3 * (size_t)K);
  s->C[0].swap(C[0]);
  s->C[1].swap(C[1]);
  D.Vnn = Vnn;
  const int trc = tc_rows_upload(s);  // the tensor-core proposal pass's split coefficients
  if (trc != VMCF_OK) return trc;
  ++s->geometry_version;
  s->has_S = S != nullptr;
  if (S) s->S.assign(S, S + (size_t)M * M);
  else s->S.clear();
  return VMCF_OK;
}

int vmcf_system_destroy(vmcf_system_t s) {
  if (!s) return VMCF_OK;
  if (s->dmem) cudaFree(s->dmem);
  if (s->tcr_mem) cudaFree(s->tcr_mem);
  delete s;
  return VMCF_OK;
}

int vmcf_system_info(vmcf_system_t s, int* K, int* M, int* n_up, int* n_dn) {
  if (!s) return fail(VMCF_EINVAL, "NULL system");
  if (K) *K = s->K;
  if (M) *M = s->M;
  if (n_up) *n_up = s->nup;
  if (n_dn) *n_dn = s->ndn;
  return VMCF_OK;
}

int vmcf_accumulator_length(vmcf_system_t s) { return s ? s->accL : VMCF_EINVAL; }

// One sweep's proposals of every walker (small-system path): orbital rows, proposed positions,
// acceptance uniforms and electron-nucleus Jastrow changes, in one allocation.
// Proposals of one walker-group sweep: r' [W][Ne][3], the orbital rows [W][Ne][nmax], the uniforms and the
// electron-nucleus Jastrow changes [W][Ne].
static cudaError_t alloc_group_proposals(const vmcf_system_s* s, vmcf_walkers_s* wk) {
  const size_t tsz = s->precision == VMCF_FP64 ? 8 : 4, n = (size_t)wk->W * s->Ne;
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t o_rn = 0, o_row = o_rn + al(24 * n), o_u = o_row + al(tsz * n * s->nmax), o_dchi = o_u + al(8 * n),
               bytes = o_dchi + al(tsz * n);
  cudaError_t e = cudaMalloc(&wk->gprop, bytes);
  if (e != cudaSuccess) return e;
  char* b = static_cast<char*>(wk->gprop);
  wk->g_rn = reinterpret_cast<double*>(b + o_rn);
  wk->g_row = b + o_row;
  wk->g_u = reinterpret_cast<double*>(b + o_u);
  wk->g_dchi = b + o_dchi;
  return cudaSuccess;
}

static cudaError_t alloc_proposals(const vmcf_system_s* s, vmcf_walkers_s* wk) {
  const size_t tsz = s->precision == VMCF_FP64 ? 8 : 4, n = (size_t)wk->W * s->Ne;
  const int nms = (s->small_nm + 3) / 4 * 4;
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t npair = s->MJ > 0 ? (size_t)s->Ne * (s->Ne - 1) / 2 : 0;
  const size_t o_rows = 0, o_rnew = o_rows + al(tsz * n * nms), o_u = o_rnew + al(24 * n), o_dchi = o_u + al(8 * n),
               o_dpair = o_dchi + al(tsz * n), o_amask = o_dpair + al(tsz * npair * wk->W),
               bytes = o_amask + al(4 * (size_t)wk->W);
  cudaError_t e = cudaMalloc(&wk->prop, bytes);
  if (e != cudaSuccess) return e;
  char* b = static_cast<char*>(wk->prop);
  wk->pr.rows = b + o_rows;
  wk->pr.rnew = reinterpret_cast<double*>(b + o_rnew);
  wk->pr.u = reinterpret_cast<double*>(b + o_u);
  wk->pr.dchi = b + o_dchi;
  wk->pr.dpair = npair ? b + o_dpair : nullptr;
  wk->pr.amask = reinterpret_cast<uint32_t*>(b + o_amask);
  wk->pr.npair = (int)npair;
  wk->pr.nms = nms;
  return cudaSuccess;
}

int vmcf_walkers_create(vmcf_system_t s, int W, const double* pos, int is_host, uint64_t key0, uint64_t key1,
                        uint64_t wid0, int nblocks, void* stream, vmcf_walkers_t* out) {
  if (!out) return fail(VMCF_EINVAL, "out is NULL");
  *out = nullptr;
  if (!s || !pos) return fail(VMCF_EINVAL, "NULL system or positions");
  if (W < 1 || nblocks < 2 || nblocks > W) return fail(VMCF_EINVAL, "need W >= 1 and 2 <= nblocks <= W");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  auto* wk = new vmcf_walkers_s();
  wk->sys = s;
  wk->W = W;
  wk->nblocks = nblocks;
  wk->k0 = key0;
  wk->k1 = key1;
  wk->wid0 = wid0;
  const int per_cta = std::max(1, 4 * (s->acc_smem ? s->gpb_meas : 1));
  wk->cpb = std::max(1, (int)std::lround((double)W / ((double)nblocks * per_cta)));
  wk->grid_meas = nblocks * wk->cpb;
  const size_t tsz = s->precision == VMCF_FP64 ? 8 : 4;
  const size_t npos = (size_t)W * 3 * s->Ne;
  if (s->small) {
    // G = nblocks x cpb CTAs; pick cpb for the fewest walkers per warp times waves
    double best = 1e300;
    for (int cpb = 1; cpb <= 1024; ++cpb) {
      const long long G = (long long)nblocks * cpb;
      if (G > W) break;
      const long long per_cta = (W + G - 1) / G, per_warp = (per_cta + s->small_warps - 1) / s->small_warps;
      const long long waves = (G + s->small_res - 1) / s->small_res;
      const double est = (double)waves * per_warp + 1e-3 * cpb;
      if (est < best) {
        best = est;
        wk->cpb = cpb;
      }
    }
    wk->grid_meas = nblocks * wk->cpb;
  }
  cudaError_t e;
  if ((e = cudaMalloc(&wk->pos, 8 * npos)) || (e = cudaMalloc(&wk->B, tsz * (size_t)W * s->nB)) ||
      (e = cudaMalloc(&wk->nacc, 4 * (size_t)W)) || (e = cudaMalloc(&wk->nrej, 4 * (size_t)W)) ||
      (e = cudaMalloc(&wk->counters, 16)) ||
      (e = cudaMalloc(&wk->acc, 8 * (size_t)wk->grid_meas * s->accL)) ||
      (e = cudaMalloc(&wk->blocks, 8 * (size_t)nblocks * s->accL)) ||
      (e = cudaMallocHost(&wk->h_blocks, 8 * (size_t)nblocks * s->accL)) ||
      (e = cudaMalloc(&wk->d_fin, 8 * fin_doubles(*s) + 16)) || (e = cudaMallocHost(&wk->h_fin, 8 * fin_doubles(*s) + 16)) ||
      (s->small && (e = cudaMalloc(&wk->stage, 8 * npos))) ||
      (s->small && s->precision == VMCF_MIXED && (e = cudaMalloc(&wk->posf, sizeof(float2) * npos))) ||
      (s->small && (e = alloc_proposals(s, wk))) ||
      (!s->small && (e = alloc_group_proposals(s, wk))) ||
      (((s->small && s->tc_sums) || (!s->small && s->tcg_sums)) && (e = alloc_tc(s, wk)))) {
    vmcf_walkers_destroy(wk);
    return fail(VMCF_ENOMEM, std::string("walker state allocation: ") + cudaGetErrorString(e));
  }
  if ((e = cudaMemsetAsync(wk->nacc, 0, 4 * (size_t)W, st)) || (e = cudaMemsetAsync(wk->nrej, 0, 4 * (size_t)W, st)) ||
      (e = cudaMemsetAsync(wk->counters, 0, 16, st)) ||
      (e = cudaMemsetAsync(wk->acc, 0, 8 * (size_t)wk->grid_meas * s->accL, st))) {
    vmcf_walkers_destroy(wk);
    return cuda_fail(e, "walker state initialisation");
  }
  int rc = load_positions_state(s, wk, pos, is_host, st);
  if (rc == VMCF_OK) rc = do_refresh(s, wk, st);
  if (rc == VMCF_OK) {
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_fail(e, "initial refresh");
  }
  if (rc != VMCF_OK) {
    vmcf_walkers_destroy(wk);
    return rc;
  }
  *out = wk;
  return VMCF_OK;
}

int vmcf_walkers_destroy(vmcf_walkers_t wk) {
  if (!wk) return VMCF_OK;
  for (auto& ev : wk->events) {
    cudaEventDestroy(ev.second.first);
    cudaEventDestroy(ev.second.second);
  }
  cudaFree(wk->pos);
  cudaFree(wk->B);
  cudaFree(wk->nacc);
  cudaFree(wk->nrej);
  cudaFree(wk->counters);
  cudaFree(wk->acc);
  cudaFree(wk->blocks);
  cudaFreeHost(wk->h_blocks);
  cudaFree(wk->d_fin);
  cudaFreeHost(wk->h_fin);
  cudaFree(wk->stage);
  cudaFree(wk->posf);
  cudaFree(wk->prop);
  cudaFree(wk->gprop);
  for (int k = 0; k < 2; ++k) {
    cudaFree(wk->phiT[k]);
    cudaFree(wk->yT[k]);
  }
  cudaFree(wk->tc_slots);
  cudaFree(wk->tc_flag);
  delete wk;
  return VMCF_OK;
}

int vmcf_walkers_set_positions(vmcf_system_t s, vmcf_walkers_t wk, const double* pos, int is_host, void* stream) {
  if (!s || !wk || !pos || wk->sys != s) return fail(VMCF_EINVAL, "bad arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc = load_positions_state(s, wk, pos, is_host, st);
  if (rc != VMCF_OK) return rc;
  return do_refresh(s, wk, st);
}

int vmcf_walkers_get_positions(vmcf_walkers_t wk, double* pos, int is_host, void* stream) {
  if (!wk || !pos) return fail(VMCF_EINVAL, "bad arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const vmcf_system_s* s = wk->sys;
  const size_t bytes = 8 * (size_t)wk->W * 3 * s->Ne;
  const double* src = wk->pos;
  if (s->small) {
    VMCF_CUDA(launch_from_interleaved(wk->pos, wk->stage, wk->W, 3 * s->Ne, st));
    src = wk->stage;
  }
  VMCF_CUDA(cudaMemcpyAsync(pos, src, bytes, is_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
  if (is_host) VMCF_CUDA(cudaStreamSynchronize(st));
  return VMCF_OK;
}

int vmcf_set_guiding(vmcf_walkers_t wk, double eps) {
  if (!wk || !(eps >= 0.0) || !std::isfinite(eps)) return fail(VMCF_EINVAL, "need eps >= 0");
  wk->eps = eps;
  return VMCF_OK;
}

int vmcf_reset_accumulators(vmcf_walkers_t wk, double e_ref, void* stream) {
  if (!wk || !std::isfinite(e_ref)) return fail(VMCF_EINVAL, "bad arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  VMCF_CUDA(cudaMemsetAsync(wk->acc, 0, 8 * (size_t)wk->grid_meas * wk->sys->accL, st));
  if (wk->tc)
    VMCF_CUDA(cudaMemsetAsync(wk->tc_slots, 0, 8 * wk->tc_slot_doubles, st));
  wk->e_ref = e_ref;
  wk->measured = 0;
  return VMCF_OK;
}

int vmcf_sample(vmcf_system_t s, vmcf_walkers_t wk, int n_sweeps, double step_sigma, int refresh_k, int measure,
                void* stream) {
  if (!s || !wk || wk->sys != s) return fail(VMCF_EINVAL, "bad handles");
  if (n_sweeps < 0 || !(step_sigma > 0.0) || !std::isfinite(step_sigma) || refresh_k < 1)
    return fail(VMCF_EINVAL, "need n_sweeps >= 0, step_sigma > 0, refresh_k >= 1");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (n_sweeps > 0 && wk->counter >= refresh_k) {
    // k lowered since the last call: the moves since the last re-inversion already reach it
    int rc = do_refresh(s, wk, st);
    if (rc != VMCF_OK) return rc;
  }
  if (s->small) {
    const bool fp64 = s->precision == VMCF_FP64;
    SmallMoveParams P{};
    P.pos = wk->pos;
    P.posf = wk->posf;
    P.B = wk->B;
    P.nacc = wk->nacc;
    P.nrej = wk->nrej;
    P.W = wk->W;
    P.wid0 = wk->wid0;
    P.k0 = wk->k0;
    P.k1 = wk->k1;
    P.sigma = step_sigma;
    P.eps = wk->eps;
    const int lpw = wk->eps > 0.0 ? 2 : s->move_lpw;  // guided moves use two lanes per walker
    P.wpc = move_walkers_per_cta(*s, wk->W, lpw);
    SmallMeasParams M = small_params(*s, wk->W);
    M.pos = wk->pos;
    M.pos_sk = wk->W;
    M.pos_sw = 1;
    M.mode = 2;
    M.Bout = wk->B;
    M.acc = wk->acc;
    M.swct_off = swct_offset(*s);
    M.eps = wk->eps;
    M.e_ref = wk->e_ref;
    M.counters = wk->counters;
    P.pr = wk->pr;
    SmallProposeParams Q{};
    Q.pos = wk->pos;
    Q.posf = wk->posf;
    Q.pr = wk->pr;
    Q.W = wk->W;
    Q.wid0 = wk->wid0;
    Q.k0 = wk->k0;
    Q.k1 = wk->k1;
    Q.sigma = step_sigma;
    Q.sigma_f = (float)step_sigma;
    Q.jJS = s->SL.JS;
    const int qgrid = std::max(1, std::min((wk->W + s->propose_warps - 1) / s->propose_warps, 8 * s->small_sms));
    for (int sw = 0; sw < n_sweeps; ++sw) {
      {  // the sweep's proposals, from the positions at its start
        Timed tm(wk, 4, st);
        Q.sweep = wk->sweep;
        cudaError_t e = fp64 ? launch_propose_small<double>(s->dev, s->small_nm, qgrid, s->propose_warps, s->small_move_smem, Q, st)
                             : launch_propose_small<float>(s->dev, s->small_nm, qgrid, s->propose_warps, s->small_move_smem, Q, st);
        if (e != cudaSuccess) return cuda_fail(e, "small proposal kernel launch");
      }
      int done = 0;
      while (done < s->Ne) {
        const int chunk = std::min(s->Ne - done, refresh_k - wk->counter);
        P.move0 = wk->sweep * (uint64_t)s->Ne + (uint64_t)done;
        P.nmoves = chunk;
        {
          Timed tm(wk, 0, st);
          cudaError_t e =
              fp64 ? launch_move_small<double>(s->dev, s->small_nm, lpw, wk->W, 0, P, st)
                   : launch_move_small<float>(s->dev, s->small_nm, lpw, wk->W, 0, P, st);
          if (e != cudaSuccess) return cuda_fail(e, "small move kernel launch");
        }
        done += chunk;
        wk->counter += chunk;
        if (wk->counter == refresh_k) {
          const bool end_of_sweep = done == s->Ne;
          if (!(measure && end_of_sweep)) {
            int rc = do_refresh(s, wk, st);
            if (rc != VMCF_OK) return rc;
          }
          wk->counter = 0;
        }
      }
      wk->sweep += 1;
      if (measure) {
        int rc = measure_state_small(s, wk, st);
        if (rc != VMCF_OK) return rc;
        wk->counter = 0;
        wk->measured += 1;
      }
    }
    return VMCF_OK;
  }
  MoveParams P{};
  P.pos = wk->pos;
  P.B = wk->B;
  P.nacc = wk->nacc;
  P.nrej = wk->nrej;
  P.counters = wk->counters;
  P.W = wk->W;
  P.wid0 = wk->wid0;
  P.k0 = wk->k0;
  P.k1 = wk->k1;
  P.kref = refresh_k;
  P.sigma = step_sigma;
  P.eps = wk->eps;
  const Launch lm = launch_rm(*s, wk->W);
  const bool fp64 = s->precision == VMCF_FP64;
  auto move = [&](int nsw, int skip) -> int {
    if (!s->group_prepass || !wk->gprop) {  // every sweep's proposals drawn inside the move kernel
      P.sweep0 = wk->sweep;
      P.nsweeps = nsw;
      P.c0 = wk->counter;
      P.skip_final_refresh = skip;
      Timed tm(wk, 0, st);
      cudaError_t e = fp64 ? launch_move<double>(s->dev, lm, P, st) : launch_move<float>(s->dev, lm, P, st);
      if (e != cudaSuccess) return cuda_fail(e, "move kernel launch");
      wk->sweep += nsw;
      wk->counter = (int)((wk->counter + (long long)nsw * s->Ne) % refresh_k);
      return VMCF_OK;
    }
    // one sweep per launch, its proposals formed ahead for every (walker, electron) by propose_group
    GroupProposeParams Q{};
    Q.pos = wk->pos;
    Q.prn = wk->g_rn;
    Q.prow = wk->g_row;
    Q.pu = wk->g_u;
    Q.pdchi = wk->g_dchi;
    Q.W = wk->W;
    Q.wid0 = wk->wid0;
    Q.k0 = wk->k0;
    Q.k1 = wk->k1;
    Q.sigma = step_sigma;
    MoveParams Pp = P;
    Pp.prn = wk->g_rn;
    Pp.prow = wk->g_row;
    Pp.pu = wk->g_u;
    Pp.pdchi = wk->g_dchi;
    for (int k = 0; k < nsw; ++k) {
      Q.sweep = wk->sweep;
      Pp.sweep0 = wk->sweep;
      Pp.nsweeps = 1;
      Pp.c0 = wk->counter;
      Pp.skip_final_refresh = k == nsw - 1 ? skip : 0;
      {
        Timed tm(wk, 4, st);
        cudaError_t e = launch_propose_rows(*s, Q, st);
        if (e != cudaSuccess) return cuda_fail(e, "proposal kernel launch");
      }
      Timed tm(wk, 0, st);
      cudaError_t e = fp64 ? launch_move<double>(s->dev, lm, Pp, st) : launch_move<float>(s->dev, lm, Pp, st);
      if (e != cudaSuccess) return cuda_fail(e, "move kernel launch");
      wk->sweep += 1;
      wk->counter = (int)((wk->counter + (long long)s->Ne) % refresh_k);
    }
    return VMCF_OK;
  };
  if (!measure) {
    if (n_sweeps > 0) return move(n_sweeps, 0);
    return VMCF_OK;
  }
  for (int k = 0; k < n_sweeps; ++k) {
    int rc = move(1, 1);
    if (rc != VMCF_OK) return rc;
    rc = measure_state_group(s, wk, st);
    if (rc != VMCF_OK) return rc;
    wk->counter = 0;  // the measurement rebuilt the inverses
    wk->measured += 1;
  }
  return VMCF_OK;
}


int vmcf_measure(vmcf_system_t s, vmcf_walkers_t wk, void* stream) {
  if (!s || !wk || wk->sys != s) return fail(VMCF_EINVAL, "bad handles");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (s->small) {
    int rc = measure_state_small(s, wk, st);
    if (rc != VMCF_OK) return rc;
  } else {
    int rc = measure_state_group(s, wk, st);
    if (rc != VMCF_OK) return rc;
  }
  wk->counter = 0;
  wk->measured += 1;
  return VMCF_OK;
}

int vmcf_evaluate(vmcf_system_t s, const double* pos, int W, double* EL, double* logpsi, double* dlnpsi_dR,
                  double* dEL_dR, double* O, double* dEL_dC, void* stream) {
  if (!s || W < 0) return fail(VMCF_EINVAL, "bad arguments");
  if (W == 0) return VMCF_OK;  // nothing to read or write (pos may be NULL)
  if (!pos) return fail(VMCF_EINVAL, "NULL positions");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool withD = dEL_dC != nullptr;
  if (s->small && !withD) {
    SmallMeasParams P = small_params(*s, W);
    P.pos = pos;
    P.pos_sk = 1;
    P.pos_sw = 3 * s->Ne;
    P.mode = 1;
    P.EL = EL;
    P.logpsi = logpsi;
    P.dlnpsi = dlnpsi_dR;
    P.dEL = dEL_dR;
    P.O = O;
    P.counters = reinterpret_cast<unsigned long long*>(s->scratch_counters);
    return launch_small_measure(s, eval_grid(*s, W), P, st);
  }
  if (withD && s->gpb_measD == 0) return fail(VMCF_ENOTSUP, "dEL_dC output does not fit shared memory for this system");
  MeasParams M{};
  M.pos = pos;
  M.EL = EL;
  M.logpsi = logpsi;
  M.dlnpsi = dlnpsi_dR;
  M.dEL = dEL_dR;
  M.O = O;
  M.dELdC = dEL_dC;
  M.counters = reinterpret_cast<unsigned long long*>(s->scratch_counters);
  M.W = W;
  const int groups = withD ? s->gpb_measD : s->gpb_meas;
  const int grid = (W + 2 * groups - 1) / (2 * groups);
  const Launch lc = launch_meas(*s, grid, false, withD);
  cudaError_t e = s->precision == VMCF_FP64 ? launch_measure<double>(s->dev, lc, M, st)
                                            : launch_measure<float>(s->dev, lc, M, st);
  if (e != cudaSuccess) return cuda_fail(e, "measure kernel launch (evaluate)");
  return VMCF_OK;
}

namespace {
// Per-block sums of a walker set's CTA slots on the device, with the tensor-core slots folded in.
int reduce_blocks_on_device(vmcf_system_s* s, vmcf_walkers_s* wk, cudaStream_t st) {
  cudaError_t e = launch_block_reduce(wk->acc, wk->grid_meas, wk->cpb, s->accL, wk->blocks, wk->nblocks, st);
  if (e != cudaSuccess) return cuda_fail(e, "block reduce launch");
  if (wk->tc) {
    const int nO = s->M * (s->nup + s->ndn);
    e = launch_tc_fold(wk->tc_slots, wk->nblocks, wk->tc_cpb, s->small ? s->tc_Mp : s->tcg_Mf,
                       s->small ? s->tc_Np : s->tcg_Nf, s->M, s->nup, s->ndn, 3 + 9 * s->K, nO, s->accL, wk->blocks, st);
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core fold launch");
  }
  return VMCF_OK;
}
}  // namespace

int vmcf_block_sums(vmcf_system_t s, vmcf_walkers_t wk, double* out, void* stream) {
  if (!s || !wk || !out || wk->sys != s) return fail(VMCF_EINVAL, "bad arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int rc = reduce_blocks_on_device(s, wk, st);
  if (rc != VMCF_OK) return rc;
  if (wk->tc) {
    int flag = 0;
    VMCF_CUDA(cudaMemcpyAsync(&flag, wk->tc_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    VMCF_CUDA(cudaStreamSynchronize(st));
    if (flag) return fail(VMCF_ETIMEOUT, "tensor-core walker-sum kernel: a bounded wait timed out");
  }
  if (s->tcr_flag) {
    int flag = 0;
    VMCF_CUDA(cudaMemcpyAsync(&flag, s->tcr_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    VMCF_CUDA(cudaStreamSynchronize(st));
    if (flag) return fail(VMCF_ETIMEOUT, "tensor-core proposal kernel: a bounded wait timed out");
  }
  VMCF_CUDA(cudaMemcpyAsync(out, wk->blocks, 8 * (size_t)wk->nblocks * s->accL, cudaMemcpyDeviceToHost, st));
  VMCF_CUDA(cudaStreamSynchronize(st));
  return VMCF_OK;
}

namespace {
// Delete-one-block jackknife of the estimators from block sums: the full-sample estimates
// (E, F, B) and the nb leave-one-out estimates (Ej [nb], Fj [nb][3K], Bj [nb][nO]).
int jackknife_estimates(const double* blk, int nb, int K, int M, int n_up, int n_dn, double er, double* Ev,
                        std::vector<double>& Fv, std::vector<double>& Bv, std::vector<double>& Ej,
                        std::vector<double>& Fj, std::vector<double>& Bj) {
  if (!blk || nb < 2 || K < 1 || M < 0 || n_up < 0 || n_dn < 0) return fail(VMCF_EINVAL, "bad arguments");
  const int K3 = 3 * K, nO = M * (n_up + n_dn), L = 3 + 9 * K + 2 * nO;
  std::vector<double> tot(L, 0.0);
  for (int b = 0; b < nb; ++b)
    for (int i = 0; i < L; ++i) tot[i] += blk[(size_t)b * L + i];
  if (!(tot[0] > 0.0)) return fail(VMCF_EINVAL, "no measured samples");
  for (int b = 0; b < nb; ++b)
    if (!(tot[0] - blk[(size_t)b * L] > 0.0)) return fail(VMCF_EINVAL, "a jackknife block holds every sample");
  const int o_dEL = 3, o_d = 3 + K3, o_Ed = 3 + 2 * K3, o_O = 3 + 3 * K3, o_EO = 3 + 3 * K3 + nO;
  // estimates from a sum vector v (all blocks, or all but one); E_ref cancels algebraically
  // (the means of the force and orbital fields as products with 1/n: one division per vector, not two per entry)
  auto est = [&](const double* v, double* Eo, double* Fo, double* Bo) {
    const double n = v[0], Em = v[1] / n, in = 1.0 / n, c = Em - er;
    *Eo = Em;
    for (int i = 0; i < K3; ++i) Fo[i] = -(v[o_dEL + i] * in + 2.0 * (v[o_Ed + i] * in - c * (v[o_d + i] * in)));
    for (int i = 0; i < nO; ++i) Bo[i] = 2.0 * (v[o_EO + i] * in - c * (v[o_O + i] * in));
  };
  Fv.assign(K3, 0.0);
  Bv.assign(nO, 0.0);
  est(tot.data(), Ev, Fv.data(), Bv.data());
  Ej.resize(nb);  // every entry is written below
  Fj.resize((size_t)nb * K3);
  Bj.resize((size_t)nb * nO);
  std::vector<double> loo(L);
  for (int b = 0; b < nb; ++b) {
    for (int i = 0; i < L; ++i) loo[i] = tot[i] - blk[(size_t)b * L + i];
    est(loo.data(), &Ej[b], Fj.data() + (size_t)b * K3, Bj.data() + (size_t)b * nO);
  }
  return VMCF_OK;
}

// Mean over the nb leave-one-out estimates of component idx (stride = components per block).
double jk_mean(const std::vector<double>& th, int nb, int stride, int idx) {
  double m = 0.0;
  for (int b = 0; b < nb; ++b) m += th[(size_t)b * stride + idx];
  return m / nb;
}
}  // namespace

int vmcf_finish_estimators(const double* blk, int nb, int K, int M, int n_up, int n_dn, double er, double* E,
                           double* E_err, double* F, double* F_err, double* dEdC, double* dEdC_err) {
  if (M < 1) return fail(VMCF_EINVAL, "bad arguments");
  double Ev = 0.0;
  // per-thread work space, kept between calls (no fresh pages every call)
  thread_local std::vector<double> Fv, Bv, Ej, Fj, Bj, mean, var;
  int rc = jackknife_estimates(blk, nb, K, M, n_up, n_dn, er, &Ev, Fv, Bv, Ej, Fj, Bj);
  if (rc != VMCF_OK) return rc;
  const int K3 = 3 * K, nO = M * (n_up + n_dn);
  // jackknife errors of the components of th ([nb][n]): for each component the mean over the blocks, then the
  // sum of squared deviations, both summed over the blocks in order, a block's row at a time
  auto jk_all = [&](const std::vector<double>& th, int n, double* err) {
    mean.assign(n, 0.0);
    var.assign(n, 0.0);
    for (int b = 0; b < nb; ++b)
      for (int i = 0; i < n; ++i) mean[i] += th[(size_t)b * n + i];
    for (int i = 0; i < n; ++i) mean[i] /= nb;
    for (int b = 0; b < nb; ++b)
      for (int i = 0; i < n; ++i) {
        const double d = th[(size_t)b * n + i] - mean[i];
        var[i] += d * d;
      }
    for (int i = 0; i < n; ++i) err[i] = std::sqrt((nb - 1.0) / nb * var[i]);
  };
  if (E) *E = Ev;
  if (E_err) jk_all(Ej, 1, E_err);
  if (F) std::copy(Fv.begin(), Fv.end(), F);
  if (F_err) jk_all(Fj, K3, F_err);
  if (dEdC) std::copy(Bv.begin(), Bv.end(), dEdC);
  if (dEdC_err) jk_all(Bj, nO, dEdC_err);
  return VMCF_OK;
}

int vmcf_finish_covariance(const double* blk, int nb, int K, int M, int n_up, int n_dn, double er,
                           double* F_factor, double* B_factor) {
  if (M < 1) return fail(VMCF_EINVAL, "bad arguments");
  double Ev = 0.0;
  std::vector<double> Fv, Bv, Ej, Fj, Bj;
  int rc = jackknife_estimates(blk, nb, K, M, n_up, n_dn, er, &Ev, Fv, Bv, Ej, Fj, Bj);
  if (rc != VMCF_OK) return rc;
  const int K3 = 3 * K, nO = M * (n_up + n_dn);
  const double scale = std::sqrt((nb - 1.0) / nb);
  if (F_factor)
    for (int i = 0; i < K3; ++i) {
      const double m = jk_mean(Fj, nb, K3, i);
      for (int b = 0; b < nb; ++b) F_factor[(size_t)i * nb + b] = scale * (Fj[(size_t)b * K3 + i] - m);
    }
  if (B_factor)
    for (int i = 0; i < nO; ++i) {
      const double m = jk_mean(Bj, nb, nO, i);
      for (int b = 0; b < nb; ++b) B_factor[(size_t)i * nb + b] = scale * (Bj[(size_t)b * nO + i] - m);
    }
  return VMCF_OK;
}

int vmcf_finish_warp(const double* blk, int nb, int stride, int K, int M, int n_up, int n_dn, double er, double* F,
                     double* F_err) {
  if (!blk || nb < 2 || K < 1 || M < 1 || n_up < 0 || n_dn < 0) return fail(VMCF_EINVAL, "bad arguments");
  const int nO = M * (n_up + n_dn), Lb = 3 + 9 * K + 2 * nO;
  if (stride != Lb + 9 * K) return fail(VMCF_EINVAL, "stride must be 3 + 18 K + 2 M (n_up + n_dn)");
  // the base layout with the warped sums in place of the force fields, and no O sums
  const int Lw = 3 + 9 * K;
  std::vector<double> v((size_t)nb * Lw);
  for (int b = 0; b < nb; ++b) {
    const double* src = blk + (size_t)b * stride;
    double* dst = v.data() + (size_t)b * Lw;
    std::copy(src, src + 3, dst);
    std::copy(src + Lb, src + Lb + 9 * K, dst + 3);
  }
  double Ev = 0.0;
  std::vector<double> Fv, Bv, Ej, Fj, Bj;
  int rc = jackknife_estimates(v.data(), nb, K, 0, 0, 0, er, &Ev, Fv, Bv, Ej, Fj, Bj);
  if (rc != VMCF_OK) return rc;
  for (int i = 0; i < 3 * K; ++i) {
    if (F) F[i] = Fv[i];
    if (F_err) {
      const double m = jk_mean(Fj, nb, 3 * K, i);
      double s2 = 0.0;
      for (int b = 0; b < nb; ++b) s2 += (Fj[(size_t)b * 3 * K + i] - m) * (Fj[(size_t)b * 3 * K + i] - m);
      F_err[i] = std::sqrt((nb - 1.0) / nb * s2);
    }
  }
  return VMCF_OK;
}

int vmcf_reduce_warp(vmcf_system_t s, vmcf_walkers_t wk, double* F, double* F_err, void* stream) {
  if (!s || !wk || wk->sys != s) return fail(VMCF_EINVAL, "bad handles");
  if (!s->swct) return fail(VMCF_EINVAL, "the system was not created with VMCF_SPACE_WARP");
  int rc = vmcf_block_sums(s, wk, wk->h_blocks, stream);
  if (rc != VMCF_OK) return rc;
  return vmcf_finish_warp(wk->h_blocks, wk->nblocks, s->accL, s->K, s->M, s->nup, s->ndn, wk->e_ref, F, F_err);
}

int vmcf_evaluate_warp(vmcf_system_t s, const double* pos, int W, double* dEL_dr, double* dEL_sw, double* dlnpsi_sw,
                       void* stream) {
  if (!s || W < 0) return fail(VMCF_EINVAL, "bad arguments");
  if (W == 0) return VMCF_OK;  // nothing to read or write (pos may be NULL)
  if (!pos) return fail(VMCF_EINVAL, "NULL positions");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  MeasParams M{};
  M.pos = pos;
  M.dEL_dr = dEL_dr;
  M.dEL_sw = dEL_sw;
  M.dlnpsi_sw = dlnpsi_sw;
  M.counters = reinterpret_cast<unsigned long long*>(s->scratch_counters);
  M.W = W;
  const int grid = (W + 2 * s->gpb_meas - 1) / (2 * s->gpb_meas);
  const Launch lc = launch_meas(*s, grid, false, false);
  cudaError_t e = s->precision == VMCF_FP64 ? launch_measure<double>(s->dev, lc, M, st)
                                            : launch_measure<float>(s->dev, lc, M, st);
  if (e != cudaSuccess) return cuda_fail(e, "measure kernel launch (space warp)");
  return VMCF_OK;
}

namespace {
// -B Q^s per spin from B (host): Q^s = 1 - C^s C^s^T S (Eq. Q_projector); rhs_{nu i} = -sum_mu B_{mu i} Q_{mu nu}
int rhs_from_B(const vmcf_system_s* s, const std::vector<double>& Bv, double* rhs_BQ) {
  const int M = s->M;
  int ooff = 0;
  for (int sg = 0; sg < 2; ++sg) {
    const int n = sg == 0 ? s->nup : s->ndn;
    const std::vector<double>& C = s->C[sg];
    std::vector<double> CtB((size_t)n * n, 0.0);  // (C^T B)_{k i}
    for (int k = 0; k < n; ++k)
      for (int i = 0; i < n; ++i) {
        double v = 0.0;
        for (int mu = 0; mu < M; ++mu) v += C[(size_t)mu * n + k] * Bv[ooff + (size_t)mu * n + i];
        CtB[(size_t)k * n + i] = v;
      }
    std::vector<double> SC((size_t)M * n, 0.0);  // (S C)_{nu k}
    for (int nu = 0; nu < M; ++nu)
      for (int k = 0; k < n; ++k) {
        double v = 0.0;
        for (int la = 0; la < M; ++la) v += s->S[(size_t)nu * M + la] * C[(size_t)la * n + k];
        SC[(size_t)nu * n + k] = v;
      }
    for (int nu = 0; nu < M; ++nu)
      for (int i = 0; i < n; ++i) {
        double v = Bv[ooff + (size_t)nu * n + i];
        for (int k = 0; k < n; ++k) v -= SC[(size_t)nu * n + k] * CtB[(size_t)k * n + i];
        rhs_BQ[ooff + (size_t)nu * n + i] = -v;
      }
    ooff += M * n;
  }
  return VMCF_OK;
}
}  // namespace

int vmcf_reduce_estimators(vmcf_system_t s, vmcf_walkers_t wk, double* E, double* E_err, double* F, double* F_err,
                           double* dEdC, double* dEdC_err, double* rhs_BQ, void* stream) {
  if (!s || !wk || wk->sys != s) return fail(VMCF_EINVAL, "bad handles");
  if (rhs_BQ && !s->has_S) return fail(VMCF_EINVAL, "rhs_BQ needs the AO overlap S at init");
  const int L = s->accL, nb = wk->nblocks, nO = s->M * (s->nup + s->ndn);
  thread_local std::vector<double> Bv;
  if (nb <= kFinishMaxBlocks && wk->d_fin) {
    // on the device: block sums, then the estimators and their jackknife errors (the host routine's arithmetic);
    // only the results and the status flags come back, after one synchronisation
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = reduce_blocks_on_device(s, wk, st);
    if (rc != VMCF_OK) return rc;
    const int K3 = 3 * s->K;
    const size_t fn = fin_doubles(*s);
    int* dstat = reinterpret_cast<int*>(wk->d_fin + fn);
    int* hflag = reinterpret_cast<int*>(wk->h_fin + fn);  // [0] finish status, [1] tensor-core sums, [2] rows
    VMCF_CUDA(cudaMemsetAsync(dstat, 0, sizeof(int), st));
    cudaError_t e = launch_finish(wk->blocks, nb, L, K3, nO, wk->e_ref, wk->d_fin, dstat, st);
    if (e != cudaSuccess) return cuda_fail(e, "estimator finish launch");
    hflag[1] = hflag[2] = 0;
    VMCF_CUDA(cudaMemcpyAsync(wk->h_fin, wk->d_fin, 8 * fn + sizeof(int), cudaMemcpyDeviceToHost, st));
    if (wk->tc) VMCF_CUDA(cudaMemcpyAsync(hflag + 1, wk->tc_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    if (s->tcr_flag) VMCF_CUDA(cudaMemcpyAsync(hflag + 2, s->tcr_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    VMCF_CUDA(cudaStreamSynchronize(st));
    if (hflag[1]) return fail(VMCF_ETIMEOUT, "tensor-core walker-sum kernel: a bounded wait timed out");
    if (hflag[2]) return fail(VMCF_ETIMEOUT, "tensor-core proposal kernel: a bounded wait timed out");
    if (hflag[0] & 1) return fail(VMCF_EINVAL, "no measured samples");
    if (hflag[0] & 2) return fail(VMCF_EINVAL, "a jackknife block holds every sample");
    const double* o = wk->h_fin;
    const double* Bo = o + 2 + 2 * K3;
    if (E) *E = o[0];
    if (E_err) *E_err = o[1];
    if (F) std::copy(o + 2, o + 2 + K3, F);
    if (F_err) std::copy(o + 2 + K3, o + 2 + 2 * K3, F_err);
    if (dEdC) std::copy(Bo, Bo + nO, dEdC);
    if (dEdC_err) std::copy(Bo + nO, Bo + 2 * nO, dEdC_err);
    if (!rhs_BQ) return VMCF_OK;
    Bv.assign(Bo, Bo + nO);
    return rhs_from_B(s, Bv, rhs_BQ);
  }
  // the block sums land in the walker set's pinned host buffer (a direct copy, no staging)
  int rc = vmcf_block_sums(s, wk, wk->h_blocks, stream);
  if (rc != VMCF_OK) return rc;
  const int Lb = 3 + 9 * s->K + 2 * nO;  // base fields; the space-warp sums (if any) follow
  const double* blk = wk->h_blocks;
  std::vector<double> base;
  if (L != Lb) {
    base.resize((size_t)nb * Lb);
    for (int b = 0; b < nb; ++b) std::copy(blk + (size_t)b * L, blk + (size_t)b * L + Lb, &base[(size_t)b * Lb]);
    blk = base.data();
  }
  Bv.resize(nO);
  rc = vmcf_finish_estimators(blk, nb, s->K, s->M, s->nup, s->ndn, wk->e_ref, E, E_err, F, F_err,
                              Bv.data(), dEdC_err);
  if (rc != VMCF_OK) return rc;
  if (dEdC) std::copy(Bv.begin(), Bv.end(), dEdC);
  return rhs_BQ ? rhs_from_B(s, Bv, rhs_BQ) : VMCF_OK;
}

int vmcf_set_tuning(vmcf_system_t s, const char* key, int value) {
  if (!s || !key) return fail(VMCF_EINVAL, "bad arguments");
  const std::string k(key);
  if (k == "group_proposal_pass") {  // walker-group sweeps: proposals formed ahead (1) or in the move kernel (0)
    s->group_prepass = value != 0;
    return VMCF_OK;
  }
  if (k == "tensor_core_rows") {  // walker-group proposal pass, mixed precision: orbital rows on the tensor cores
    if (value != 0 && !s->tcr_mem)
      return fail(VMCF_EINVAL, "tensor-core orbital rows need mixed precision on the walker-group kernels");
    s->tc_rows = value != 0;
    return VMCF_OK;
  }
  if (k == "move_lanes_per_walker") {
    if (value != 1 && value != 2 && value != 4 && value != 8) return fail(VMCF_EINVAL, "lanes per walker: 1, 2, 4 or 8");
    s->move_lpw = value;
    return VMCF_OK;
  }
  if (k == "tensor_core_sums") {
    const bool want = value != 0;
    if (want && s->precision != VMCF_MIXED) return fail(VMCF_EINVAL, "tensor-core walker sums need mixed precision");
    if (s->small) s->tc_sums = want;
    else s->tcg_sums = want;
    return VMCF_OK;
  }
  if (k == "measure_group_size") {
    if (s->small || (value != 32 && value != 128 && value != 256))
      return fail(VMCF_EINVAL, "measure group size (walker-group kernels): 32, 128 or 256");
    const int old = s->GSm;
    s->GSm = value;
    int rc = plan_measure(*s);
    if (rc != VMCF_OK) {
      s->GSm = old;
      plan_measure(*s);
    }
    return rc;
  }
  if (k == "measure_warps") {
    if (!s->small || (value != 2 && value != 4 && value != 8)) return fail(VMCF_EINVAL, "measure warps: 2, 4 or 8");
    if (s->SL.cta_bytes + value * s->SL.bytes > kSmemCap) return fail(VMCF_EINVAL, "does not fit shared memory");
    s->small_warps = value;
    return VMCF_OK;
  }
  return fail(VMCF_EINVAL, "unknown tuning key");
}

int vmcf_profile(vmcf_walkers_t wk, int enable) {
  if (!wk) return fail(VMCF_EINVAL, "NULL walkers");
  wk->profiling = enable != 0;
  return VMCF_OK;
}

int vmcf_kernel_times(vmcf_walkers_t wk, double* ms, long long* count, int reset) {
  if (!wk) return fail(VMCF_EINVAL, "NULL walkers");
  for (auto& ev : wk->events) {
    VMCF_CUDA(cudaEventSynchronize(ev.second.second));
    float t = 0.f;
    VMCF_CUDA(cudaEventElapsedTime(&t, ev.second.first, ev.second.second));
    wk->kernel_ms[ev.first] += t;
    wk->kernel_n[ev.first] += 1;
    cudaEventDestroy(ev.second.first);
    cudaEventDestroy(ev.second.second);
  }
  wk->events.clear();
  for (int k = 0; k < 5; ++k) {
    if (ms) ms[k] = wk->kernel_ms[k];
    if (count) count[k] = wk->kernel_n[k];
    if (reset) {
      wk->kernel_ms[k] = 0.0;
      wk->kernel_n[k] = 0;
    }
  }
  return VMCF_OK;
}

int vmcf_diag_group_proposals(vmcf_walkers_t wk, double step_sigma, double* rnew, double* rows, double* u,
                              double* dchi, void* stream) {
  if (!wk || !rnew || !rows || !u || !dchi || !(step_sigma > 0.0)) return fail(VMCF_EINVAL, "bad arguments");
  vmcf_system_s* s = wk->sys;
  if (s->small || !wk->gprop) return fail(VMCF_EINVAL, "the proposal pass of the walker-group kernels only");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  GroupProposeParams Q{};
  Q.pos = wk->pos;
  Q.prn = wk->g_rn;
  Q.prow = wk->g_row;
  Q.pu = wk->g_u;
  Q.pdchi = wk->g_dchi;
  Q.W = wk->W;
  Q.wid0 = wk->wid0;
  Q.k0 = wk->k0;
  Q.k1 = wk->k1;
  Q.sweep = wk->sweep;
  Q.sigma = step_sigma;
  if (wk->W == 0) return VMCF_OK;
  cudaError_t e = launch_propose_rows(*s, Q, st);
  if (e != cudaSuccess) return cuda_fail(e, "proposal kernel launch");
  const size_t n = (size_t)wk->W * s->Ne, nr = n * s->nmax;
  const bool fp64 = s->precision == VMCF_FP64;
  std::vector<float> rf(fp64 ? 0 : nr), df(fp64 ? 0 : n);
  VMCF_CUDA(cudaMemcpyAsync(rnew, wk->g_rn, 24 * n, cudaMemcpyDeviceToHost, st));
  VMCF_CUDA(cudaMemcpyAsync(u, wk->g_u, 8 * n, cudaMemcpyDeviceToHost, st));
  if (fp64) {
    VMCF_CUDA(cudaMemcpyAsync(rows, wk->g_row, 8 * nr, cudaMemcpyDeviceToHost, st));
    VMCF_CUDA(cudaMemcpyAsync(dchi, wk->g_dchi, 8 * n, cudaMemcpyDeviceToHost, st));
  } else {
    VMCF_CUDA(cudaMemcpyAsync(rf.data(), wk->g_row, 4 * nr, cudaMemcpyDeviceToHost, st));
    VMCF_CUDA(cudaMemcpyAsync(df.data(), wk->g_dchi, 4 * n, cudaMemcpyDeviceToHost, st));
  }
  VMCF_CUDA(cudaStreamSynchronize(st));
  if (!fp64) {
    for (size_t i = 0; i < nr; ++i) rows[i] = rf[i];
    for (size_t i = 0; i < n; ++i) dchi[i] = df[i];
  }
  if (s->tcr_flag) {
    int flag = 0;
    VMCF_CUDA(cudaMemcpy(&flag, s->tcr_flag, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) return fail(VMCF_ETIMEOUT, "tensor-core proposal kernel: a bounded wait timed out");
  }
  return VMCF_OK;
}

int vmcf_probe_pipes(double* fp64_tflops, double* fp32_tflops, double* exp_gops, void* stream) {
  cudaError_t e = run_probes(fp64_tflops, fp32_tflops, exp_gops, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "pipe probes");
  return VMCF_OK;
}

int vmcf_refresh_residual(vmcf_walkers_t wk, double* max_rel, double* mean_rel, void* stream) {
  if (!wk) return fail(VMCF_EINVAL, "NULL walkers");
  vmcf_system_s* s = wk->sys;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (max_rel) *max_rel = 0.0;
  if (mean_rel) *mean_rel = 0.0;
  const int W = wk->W, nB = s->nB;
  if (W == 0) return VMCF_OK;
  const bool fp64 = s->precision == VMCF_FP64;
  const size_t tsz = fp64 ? 8 : 4, bytes = tsz * (size_t)W * nB;
  void* fresh = nullptr;
  VMCF_CUDA(cudaMalloc(&fresh, bytes));
  // fresh inverses of the current positions into the temporary buffer, with the walker set's own re-inversion
  // kernel; the evaluation's scratch counters take the kernel's counts
  cudaError_t e;
  if (s->small) {
    SmallMeasParams P = small_params(*s, W);
    P.pos = wk->pos;
    P.pos_sk = W;
    P.pos_sw = 1;
    P.mode = 0;
    P.Bout = fresh;
    P.counters = reinterpret_cast<unsigned long long*>(s->scratch_counters);
    e = fp64 ? launch_measure_small<double>(s->dev, s->small_nm, s->SL, eval_grid(*s, W), s->small_warps, P, st)
             : launch_measure_small<float>(s->dev, s->small_nm, s->SL, eval_grid(*s, W), s->small_warps, P, st);
  } else {
    const Launch lc = launch_rm(*s, W);
    e = fp64 ? launch_refresh<double>(s->dev, lc, wk->pos, fresh, W,
                                      reinterpret_cast<unsigned long long*>(s->scratch_counters), st)
             : launch_refresh<float>(s->dev, lc, wk->pos, fresh, W,
                                     reinterpret_cast<unsigned long long*>(s->scratch_counters), st);
  }
  std::vector<unsigned char> cur(bytes), frs(bytes);
  if (e == cudaSuccess) e = cudaMemcpyAsync(cur.data(), wk->B, bytes, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(frs.data(), fresh, bytes, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(fresh);
  if (e != cudaSuccess) return cuda_fail(e, "refresh residual");
  // entry k of walker w: [k][W] (one-warp kernels, walker-interleaved) or [W][nB] (walker groups)
  auto at = [&](const std::vector<unsigned char>& v, int w, int k) -> double {
    const size_t i = s->small ? (size_t)k * W + w : (size_t)w * nB + k;
    return fp64 ? reinterpret_cast<const double*>(v.data())[i] : (double)reinterpret_cast<const float*>(v.data())[i];
  };
  double mx = 0.0, sum = 0.0;
  for (int w = 0; w < W; ++w) {
    double dmax = 0.0, bmax = 0.0;
    for (int k = 0; k < nB; ++k) {
      const double b = at(frs, w, k);
      dmax = std::max(dmax, std::fabs(at(cur, w, k) - b));
      bmax = std::max(bmax, std::fabs(b));
    }
    const double r = bmax > 0.0 ? dmax / bmax : dmax;
    mx = std::max(mx, r);
    sum += r;
  }
  if (max_rel) *max_rel = mx;
  if (mean_rel) *mean_rel = sum / W;
  return VMCF_OK;
}

int vmcf_status_counters(vmcf_walkers_t wk, vmcf_counters* out, void* stream) {
  if (!wk || !out) return fail(VMCF_EINVAL, "bad arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::vector<uint32_t> a(wk->W), r(wk->W);
  unsigned long long c[2];
  VMCF_CUDA(cudaMemcpyAsync(a.data(), wk->nacc, 4 * (size_t)wk->W, cudaMemcpyDeviceToHost, st));
  VMCF_CUDA(cudaMemcpyAsync(r.data(), wk->nrej, 4 * (size_t)wk->W, cudaMemcpyDeviceToHost, st));
  VMCF_CUDA(cudaMemcpyAsync(c, wk->counters, 16, cudaMemcpyDeviceToHost, st));
  VMCF_CUDA(cudaStreamSynchronize(st));
  std::memset(out, 0, sizeof(*out));
  for (int w = 0; w < wk->W; ++w) {
    out->accepted += a[w];
    out->rejected_nonfinite += r[w];
  }
  out->sweeps = wk->sweep;
  out->moves = wk->sweep * (uint64_t)wk->W * (uint64_t)wk->sys->Ne;
  out->singular = c[0];
  out->refreshes = c[1];
  out->measured_sweeps = wk->measured;
  return VMCF_OK;
}

}  // extern "C"
