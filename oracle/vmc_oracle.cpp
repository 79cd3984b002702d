// Plain FP64 CPU oracle for the VMC hot path of "Fast Evaluation of Unbiased Atomic Forces
// in ab initio VMC via the Lagrangian Technique" (arXiv:2511.05222).
//
// TEST INFRASTRUCTURE ONLY. It is called by the tests, by the smoke check and by the
// benchmark's CPU baseline; the product path never links or calls it. It shares no code,
// header, table or constant generator with the CUDA library.
//
// Style: plain loops in double precision, no BLAS, no blocking, no fusion; OpenMP only over
// independent walkers. Build with -O2 -ffp-contract=off so that x86 and Arm give the same
// bits. Every function names the passage of the paper (or of the workload definition) it
// follows.
//
// Wavefunction (App. A, "Wavefunction Ansatz"): Psi = exp(J) * det A_up * det A_dn, the
// Jastrow-Slater determinant that the JAGP reduces to when the geminal is expanded over the
// occupied orbitals only. A^s_{e i} = phi^s_i(r_e) with phi^s_i = sum_mu C^s_{mu i} psi_mu
// (Eq. restricted-C). Electrons 0..n_up-1 are spin up, n_up..Ne-1 spin down.
// Jastrow: J = sum_{i<j} u_{s_i s_j}(r_ij) + sum_{e,I} chi_I(|r_e - R_I|), with the Pade
// form a r / (1 + F r) of Eq. twobody_v made spin dependent (a = 1/2 antiparallel, 1/4
// parallel) and the e-n cusp term chi_I(r) = -Z_I r / (1 + b r). Optionally, the AO-expanded
// terms over a separate Jastrow basis psi^J (App., Eqs. onebody_J_inhom and threebody_jas):
// sum_e sum_mu xi_mu psi^J_mu(r_e) + sum_{i<j} sum_{mu,nu} Xi_{mu nu} psi^J_mu(r_i) psi^J_nu(r_j),
// read as further terms of the exponent J, with Xi symmetric.
// Local energy (App. A, E_L = H Psi / Psi): E_L = -1/2 sum_e lap_e Psi / Psi + V_ee + V_en + V_nn.
// Forces (Eqs. hf, pulay): total partial derivatives of E_L and ln|Psi| with respect to the
// nuclear positions at fixed electron positions and fixed C.
// O = d ln Psi / d C (App. A, Eq. fc-vmc-eval).

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#include <algorithm>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

const double kPi = 3.14159265358979323846;

struct Mono { double c; int e[3]; };

struct Shell {
  int center, l, nprim;
  double alpha[8];
  double coef[8];   // normalised contraction coefficients
};

struct AO { int shell; std::vector<Mono> poly; };

struct OSys {
  int K = 0;
  std::vector<int> Z;
  std::vector<double> R;  // [K][3]
  std::vector<Shell> shells;
  std::vector<AO> aos;
  int M = 0;
  int nup = 0, ndn = 0;
  std::vector<double> C[2];  // [M][n_s]
  double Fa = 0.8, Fp = 0.8, aa = 0.5, ap = 0.25, ben = 1.5;
  int J1 = 1, J2 = 1;
  int j2exp = 0;  // two-body form: 0 Pade (Eq. twobody_v), 1 exponential (Eq. twobody_v_exp)
  // Jastrow basis of the AO-expanded terms (MJ = 0: none), its one-body coefficients xi [MJ] and
  // its symmetric pair coefficients Xi [MJ][MJ]
  std::vector<Shell> jshells;
  std::vector<AO> jaos;
  int MJ = 0;
  std::vector<double> xi, Xi;
};

// ---------------------------------------------------------------- basis (convention P1)
// Real solid harmonics r^l Y_lm, unit-sphere normalised; p = (x, y, z);
// d = (xy, yz, 3z^2 - r^2, xz, x^2 - y^2).
std::vector<std::vector<Mono>> solid_harmonics(int l) {
  std::vector<std::vector<Mono>> out;
  if (l == 0) {
    out.push_back({{std::sqrt(1.0 / (4 * kPi)), {0, 0, 0}}});
  } else if (l == 1) {
    double c = std::sqrt(3.0 / (4 * kPi));
    out.push_back({{c, {1, 0, 0}}});
    out.push_back({{c, {0, 1, 0}}});
    out.push_back({{c, {0, 0, 1}}});
  } else {
    double c1 = std::sqrt(15.0 / (4 * kPi));
    double c0 = std::sqrt(5.0 / (16 * kPi));
    double c2 = std::sqrt(15.0 / (16 * kPi));
    out.push_back({{c1, {1, 1, 0}}});
    out.push_back({{c1, {0, 1, 1}}});
    out.push_back({{2 * c0, {0, 0, 2}}, {-c0, {2, 0, 0}}, {-c0, {0, 2, 0}}});
    out.push_back({{c1, {1, 0, 1}}});
    out.push_back({{c2, {2, 0, 0}}, {-c2, {0, 2, 0}}});
  }
  return out;
}

double dfact(int n) {  // n!!, with (-1)!! = 1
  double r = 1.0;
  for (int k = n; k > 1; k -= 2) r *= k;
  return r;
}

// Primitive normalisation: integral of r^{2l+2} exp(-2 a r^2) dr over [0, inf) equals
// (2l+1)!! / (2^{l+2} (2a)^{l+1}) sqrt(pi / (2a)); the angular factor integrates to one.
double prim_norm(double a, int l) {
  double radial = dfact(2 * l + 1) / (std::pow(2.0, l + 2) * std::pow(2 * a, l + 1)) * std::sqrt(kPi / (2 * a));
  return 1.0 / std::sqrt(radial);
}

// Overlap of two normalised same-centre primitives of equal l, m.
double prim_overlap(double a, double b, int l) {
  return std::pow(2.0 * std::sqrt(a * b) / (a + b), l + 1.5);
}

// ---------------------------------------------------------------- AO evaluation
// One factor x^a exp(-al x^2): its value and first three derivatives, by applying
// D = d/dx - 2 al x to the polynomial part (the Gaussian factor is multiplied in outside).
void poly1d_derivs(int a, double al, double x, double out[4]) {
  double p[8] = {0};  // polynomial coefficients in x
  p[a] = 1.0;
  for (int d = 0; d < 4; ++d) {
    double v = 0.0, xp = 1.0;
    for (int k = 0; k < 8; ++k) { v += p[k] * xp; xp *= x; }
    out[d] = v;
    double q[8] = {0};
    for (int k = 1; k < 8; ++k) q[k - 1] += k * p[k];
    for (int k = 0; k < 7; ++k) q[k + 1] += -2.0 * al * p[k];
    std::memcpy(p, q, sizeof p);
  }
}

// comps: 0 value, 1..3 gradient, 4 Laplacian, 5..10 Hessian (xx, yy, zz, xy, xz, yz),
// 11..13 gradient of the Laplacian.
const int NC = 14;

// Every function of a basis (shells, functions) at the point r.
void basis_eval_point(const std::vector<Shell>& shells, const std::vector<AO>& aos, const std::vector<double>& R,
                      const double r[3], double* out /*[n][NC]*/) {
  const int nf = (int)aos.size();
  std::fill(out, out + (size_t)nf * NC, 0.0);
  for (int mu = 0; mu < nf; ++mu) {
    const AO& ao = aos[mu];
    const Shell& sh = shells[ao.shell];
    double x[3];
    for (int d = 0; d < 3; ++d) x[d] = r[d] - R[3 * sh.center + d];
    double r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
    double* o = out + (size_t)mu * NC;
    for (int k = 0; k < sh.nprim; ++k) {
      double al = sh.alpha[k];
      double g = sh.coef[k] * std::exp(-al * r2);
      for (const Mono& m : ao.poly) {
        double f[3][4];
        for (int d = 0; d < 3; ++d) poly1d_derivs(m.e[d], al, x[d], f[d]);
        double w = g * m.c;
        o[0] += w * f[0][0] * f[1][0] * f[2][0];
        o[1] += w * f[0][1] * f[1][0] * f[2][0];
        o[2] += w * f[0][0] * f[1][1] * f[2][0];
        o[3] += w * f[0][0] * f[1][0] * f[2][1];
        double hxx = f[0][2] * f[1][0] * f[2][0];
        double hyy = f[0][0] * f[1][2] * f[2][0];
        double hzz = f[0][0] * f[1][0] * f[2][2];
        o[4] += w * (hxx + hyy + hzz);
        o[5] += w * hxx;
        o[6] += w * hyy;
        o[7] += w * hzz;
        o[8] += w * f[0][1] * f[1][1] * f[2][0];
        o[9] += w * f[0][1] * f[1][0] * f[2][1];
        o[10] += w * f[0][0] * f[1][1] * f[2][1];
        o[11] += w * (f[0][3] * f[1][0] * f[2][0] + f[0][1] * f[1][2] * f[2][0] + f[0][1] * f[1][0] * f[2][2]);
        o[12] += w * (f[0][2] * f[1][1] * f[2][0] + f[0][0] * f[1][3] * f[2][0] + f[0][0] * f[1][1] * f[2][2]);
        o[13] += w * (f[0][2] * f[1][0] * f[2][1] + f[0][0] * f[1][2] * f[2][1] + f[0][0] * f[1][0] * f[2][3]);
      }
    }
  }
}

void ao_eval_point(const OSys& s, const double r[3], double* out /*[M][NC]*/) {
  basis_eval_point(s.shells, s.aos, s.R, r, out);
}

// Index of the Hessian component (d, c) in the comps layout.
int hidx(int d, int c) {
  if (d == c) return 5 + d;
  int a = std::min(d, c), b = std::max(d, c);
  if (a == 0 && b == 1) return 8;
  if (a == 0 && b == 2) return 9;
  return 10;
}

// ---------------------------------------------------------------- linear algebra
// LU with partial (row) pivoting, Doolittle; then the inverse column by column.
// Returns 0, or 1 when a zero pivot makes the matrix singular.
int lu_inverse(int n, const double* A, double* inv, double* logabs, double* sgn) {
  std::vector<double> LU(A, A + (size_t)n * n);
  std::vector<int> perm(n);
  for (int i = 0; i < n; ++i) perm[i] = i;
  double s = 1.0, la = 0.0;
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(LU[(size_t)i * n + k]) > std::fabs(LU[(size_t)p * n + k])) p = i;
    if (LU[(size_t)p * n + k] == 0.0) { *logabs = -INFINITY; *sgn = 0.0; return 1; }
    if (p != k) {
      for (int j = 0; j < n; ++j) std::swap(LU[(size_t)k * n + j], LU[(size_t)p * n + j]);
      std::swap(perm[k], perm[p]);
      s = -s;
    }
    double piv = LU[(size_t)k * n + k];
    la += std::log(std::fabs(piv));
    if (piv < 0) s = -s;
    for (int i = k + 1; i < n; ++i) {
      double f = LU[(size_t)i * n + k] / piv;
      LU[(size_t)i * n + k] = f;
      for (int j = k + 1; j < n; ++j) LU[(size_t)i * n + j] -= f * LU[(size_t)k * n + j];
    }
  }
  // Solve A x = e_c for each column c: P A = L U.
  std::vector<double> y(n);
  for (int c = 0; c < n; ++c) {
    for (int i = 0; i < n; ++i) {
      double v = (perm[i] == c) ? 1.0 : 0.0;
      for (int j = 0; j < i; ++j) v -= LU[(size_t)i * n + j] * y[j];
      y[i] = v;
    }
    for (int i = n - 1; i >= 0; --i) {
      double v = y[i];
      for (int j = i + 1; j < n; ++j) v -= LU[(size_t)i * n + j] * y[j];
      y[i] = v / LU[(size_t)i * n + i];
    }
    for (int i = 0; i < n; ++i) inv[(size_t)i * n + c] = y[i];
  }
  *logabs = la;
  *sgn = s;
  return 0;
}

// ---------------------------------------------------------------- Jastrow pieces
// Radial function h(r) and its first three derivatives.
struct Rad { double h, h1, h2, h3; };

Rad pade(double a, double F, double r) {  // a r / (1 + F r)
  double q = 1.0 / (1.0 + F * r);
  return {a * r * q, a * q * q, -2.0 * a * F * q * q * q, 6.0 * a * F * F * q * q * q * q};
}

// Exponential form (a / F) (1 - exp(-F r)) of Eq. twobody_v_exp, with the cusp a in place of 1/2.
Rad expo(double a, double F, double r) {
  double q = std::exp(-F * r);
  return {-(a / F) * std::expm1(-F * r), a * q, -a * F * q, a * F * F * q};
}

Rad chi(double Z, double b, double r) {  // -Z r / (1 + b r)
  Rad p = pade(-Z, b, r);
  return p;
}

// The two-body term u_{s_i s_j}(r) of the pair: antiparallel or parallel cusp and F, in the
// chosen form.
Rad pair_u(const OSys& s, bool par, double r) {
  const double a = par ? s.ap : s.aa, F = par ? s.Fp : s.Fa;
  return s.j2exp ? expo(a, F, r) : pade(a, F, r);
}

// For a radial function h(|s|): gradient, Hessian, Laplacian and gradient of the Laplacian
// with respect to s.
struct RadDeriv { double g[3]; double H[3][3]; double lap; double glap[3]; };

RadDeriv radial_derivs(const Rad& f, const double s[3]) {
  RadDeriv o;
  double r = std::sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
  double n[3] = {s[0] / r, s[1] / r, s[2] / r};
  for (int d = 0; d < 3; ++d) {
    o.g[d] = f.h1 * n[d];
    for (int c = 0; c < 3; ++c)
      o.H[d][c] = f.h2 * n[d] * n[c] + f.h1 / r * ((d == c ? 1.0 : 0.0) - n[d] * n[c]);
  }
  o.lap = f.h2 + 2.0 * f.h1 / r;
  double dl = f.h3 + 2.0 * f.h2 / r - 2.0 * f.h1 / (r * r);  // d/dr of the Laplacian
  for (int d = 0; d < 3; ++d) o.glap[d] = dl * n[d];
  return o;
}

inline int spin_of(const OSys& s, int e) { return e < s.nup ? 0 : 1; }
inline int nspin(const OSys& s, int sg) { return sg == 0 ? s.nup : s.ndn; }
inline int first_e(const OSys& s, int sg) { return sg == 0 ? 0 : s.nup; }

struct WalkerOut {
  double EL, logpsi, sgn, J;
  std::vector<double> dlnpsi_dR, dEL_dR;     // [K][3]
  std::vector<double> O[2], dELdC[2];         // [M][n_s]
  std::vector<double> glnpsi, laplnpsi;       // [Ne][3], [Ne]
  std::vector<double> dEL_dr;                 // [Ne][3] (want_electron)
  std::vector<double> dEL_sw, dlnpsi_sw;      // [K][3] space-warp force vectors (want_electron)
  double Vee, Ven, Vnn, Ekin;
  int singular;
};

// ---------------------------------------------------------------- one walker, all outputs
void eval_walker(const OSys& s, const double* pos, bool want_dC, WalkerOut& w, bool want_electron = false) {
  const int Ne = s.nup + s.ndn, M = s.M, K = s.K;
  // AO table at every electron.
  std::vector<double> ao((size_t)Ne * M * NC);
  for (int e = 0; e < Ne; ++e) ao_eval_point(s, pos + 3 * e, ao.data() + (size_t)e * M * NC);
  auto AOv = [&](int e, int mu, int c) { return ao[((size_t)e * M + mu) * NC + c]; };

  // MO matrices per spin: A (value), G[3] (gradient), L (Laplacian).
  std::vector<double> A[2], G[2][3], L[2], B[2];
  w.logpsi = 0.0;
  w.sgn = 1.0;
  w.singular = 0;
  for (int sg = 0; sg < 2; ++sg) {
    int n = nspin(s, sg), e0 = first_e(s, sg);
    A[sg].assign((size_t)n * n, 0.0);
    L[sg].assign((size_t)n * n, 0.0);
    for (int c = 0; c < 3; ++c) G[sg][c].assign((size_t)n * n, 0.0);
    for (int el = 0; el < n; ++el)
      for (int i = 0; i < n; ++i) {
        double v = 0, gx = 0, gy = 0, gz = 0, lp = 0;
        for (int mu = 0; mu < M; ++mu) {
          double c = s.C[sg][(size_t)mu * n + i];
          v += AOv(e0 + el, mu, 0) * c;
          gx += AOv(e0 + el, mu, 1) * c;
          gy += AOv(e0 + el, mu, 2) * c;
          gz += AOv(e0 + el, mu, 3) * c;
          lp += AOv(e0 + el, mu, 4) * c;
        }
        A[sg][(size_t)el * n + i] = v;
        G[sg][0][(size_t)el * n + i] = gx;
        G[sg][1][(size_t)el * n + i] = gy;
        G[sg][2][(size_t)el * n + i] = gz;
        L[sg][(size_t)el * n + i] = lp;
      }
    B[sg].assign((size_t)n * n, 0.0);
    if (n > 0) {
      double la, sgn;
      if (lu_inverse(n, A[sg].data(), B[sg].data(), &la, &sgn)) w.singular = 1;
      w.logpsi += la;
      w.sgn *= sgn;
    }
  }

  // Determinant drift and Laplacian ratio per electron: g_e = sum_i G_ei B_ie,
  // l_e = sum_i L_ei B_ie (B = A^{-1}, indexed [i][e]).
  std::vector<double> gdet((size_t)Ne * 3, 0.0), ldet(Ne, 0.0);
  for (int e = 0; e < Ne; ++e) {
    int sg = spin_of(s, e), n = nspin(s, sg), el = e - first_e(s, sg);
    for (int i = 0; i < n; ++i) {
      double b = B[sg][(size_t)i * n + el];
      for (int c = 0; c < 3; ++c) gdet[3 * e + c] += G[sg][c][(size_t)el * n + i] * b;
      ldet[e] += L[sg][(size_t)el * n + i] * b;
    }
  }

  // Jastrow value, gradient and Laplacian per electron; potentials.
  std::vector<double> Jg((size_t)Ne * 3, 0.0), Jl(Ne, 0.0);
  double J = 0.0, Vee = 0.0, Ven = 0.0, Vnn = 0.0;
  for (int i = 0; i < Ne; ++i)
    for (int j = i + 1; j < Ne; ++j) {
      double d[3];
      for (int c = 0; c < 3; ++c) d[c] = pos[3 * i + c] - pos[3 * j + c];
      double r = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      Vee += 1.0 / r;
      if (s.J2) {
        bool par = spin_of(s, i) == spin_of(s, j);
        Rad u = pair_u(s, par, r);
        J += u.h;
        RadDeriv du = radial_derivs(u, d);  // derivatives with respect to r_i
        for (int c = 0; c < 3; ++c) {
          Jg[3 * i + c] += du.g[c];
          Jg[3 * j + c] -= du.g[c];
        }
        Jl[i] += du.lap;
        Jl[j] += du.lap;
      }
    }
  for (int e = 0; e < Ne; ++e)
    for (int I = 0; I < K; ++I) {
      double d[3];
      for (int c = 0; c < 3; ++c) d[c] = pos[3 * e + c] - s.R[3 * I + c];
      double r = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      Ven -= s.Z[I] / r;
      if (s.J1) {
        Rad f = chi(s.Z[I], s.ben, r);
        J += f.h;
        RadDeriv df = radial_derivs(f, d);
        for (int c = 0; c < 3; ++c) Jg[3 * e + c] += df.g[c];
        Jl[e] += df.lap;
      }
    }
  // AO-expanded Jastrow terms (Eqs. onebody_J_inhom, threebody_jas) by their definition:
  // U = sum_e sum_mu xi_mu psi^J_mu(r_e) + sum_{i<j} sum_{mu,nu} Xi_{mu nu} psi^J_mu(r_i) psi^J_nu(r_j).
  // U is linear in the functions of any one electron; with Xi symmetric its derivative with respect
  // to psi^J_mu(r_e) is t_{e mu} = xi_mu + sum_{j != e} sum_nu Xi_{mu nu} psi^J_nu(r_j), so that
  // grad_e U = sum_mu t_{e mu} grad psi^J_mu(r_e) and lap_e U = sum_mu t_{e mu} lap psi^J_mu(r_e).
  const int MJ = s.MJ;
  std::vector<double> jv, tJ;
  auto JV = [&](int e, int mu, int c) { return jv[((size_t)e * MJ + mu) * NC + c]; };
  auto XI = [&](int mu, int nu) { return s.Xi[(size_t)mu * MJ + nu]; };
  if (MJ > 0) {
    jv.resize((size_t)Ne * MJ * NC);
    for (int e = 0; e < Ne; ++e) basis_eval_point(s.jshells, s.jaos, s.R, pos + 3 * e, jv.data() + (size_t)e * MJ * NC);
    for (int e = 0; e < Ne; ++e)
      for (int mu = 0; mu < MJ; ++mu) J += s.xi[mu] * JV(e, mu, 0);
    for (int i = 0; i < Ne; ++i)
      for (int j = i + 1; j < Ne; ++j)
        for (int mu = 0; mu < MJ; ++mu)
          for (int nu = 0; nu < MJ; ++nu) J += JV(i, mu, 0) * XI(mu, nu) * JV(j, nu, 0);
    tJ.assign((size_t)Ne * MJ, 0.0);
    for (int e = 0; e < Ne; ++e)
      for (int mu = 0; mu < MJ; ++mu) {
        double t = s.xi[mu];
        for (int j = 0; j < Ne; ++j) {
          if (j == e) continue;
          for (int nu = 0; nu < MJ; ++nu) t += XI(mu, nu) * JV(j, nu, 0);
        }
        tJ[(size_t)e * MJ + mu] = t;
        for (int c = 0; c < 3; ++c) Jg[3 * e + c] += t * JV(e, mu, 1 + c);
        Jl[e] += t * JV(e, mu, 4);
      }
  }
  for (int I = 0; I < K; ++I)
    for (int Jn = I + 1; Jn < K; ++Jn) {
      double d[3];
      for (int c = 0; c < 3; ++c) d[c] = s.R[3 * I + c] - s.R[3 * Jn + c];
      Vnn += s.Z[I] * s.Z[Jn] / std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    }
  w.logpsi += J;
  w.J = J;

  // Local energy: lap Psi / Psi = l_e + lap J + |grad J|^2 + 2 grad J . g_e per electron.
  double Ekin = 0.0;
  w.glnpsi.assign((size_t)Ne * 3, 0.0);
  w.laplnpsi.assign(Ne, 0.0);
  for (int e = 0; e < Ne; ++e) {
    double jj = 0, jg = 0, gg = 0;
    for (int c = 0; c < 3; ++c) {
      jj += Jg[3 * e + c] * Jg[3 * e + c];
      jg += Jg[3 * e + c] * gdet[3 * e + c];
      gg += gdet[3 * e + c] * gdet[3 * e + c];
      w.glnpsi[3 * e + c] = gdet[3 * e + c] + Jg[3 * e + c];
    }
    Ekin += -0.5 * (ldet[e] + Jl[e] + jj + 2.0 * jg);
    // lap ln Psi = lap Psi / Psi - |grad ln Psi|^2
    w.laplnpsi[e] = (ldet[e] - gg) + Jl[e];
  }
  w.Vee = Vee; w.Ven = Ven; w.Vnn = Vnn; w.Ekin = Ekin;
  w.EL = Ekin + Vee + Ven + Vnn;

  // ------------------------------------------------ nuclear derivatives, forward mode
  // For each nuclear coordinate lambda = R_{I,d}: the AOs centred on I move with it, so
  // d psi/d lambda = -d_d psi, d grad psi / d lambda = -d_d grad psi, d lap psi / d lambda =
  // -d_d lap psi. dB = -B dA B. chi_I moves with R_I; V_en and V_nn are differentiated
  // directly.
  w.dlnpsi_dR.assign((size_t)K * 3, 0.0);
  w.dEL_dR.assign((size_t)K * 3, 0.0);
  for (int I = 0; I < K; ++I)
    for (int d = 0; d < 3; ++d) {
      double dlnpsi = 0.0, dEL = 0.0;
      std::vector<double> dg((size_t)Ne * 3, 0.0), dl(Ne, 0.0);
      for (int sg = 0; sg < 2; ++sg) {
        int n = nspin(s, sg), e0 = first_e(s, sg);
        if (n == 0) continue;
        std::vector<double> dA((size_t)n * n, 0.0), dL((size_t)n * n, 0.0), dG[3];
        for (int c = 0; c < 3; ++c) dG[c].assign((size_t)n * n, 0.0);
        for (int el = 0; el < n; ++el)
          for (int i = 0; i < n; ++i)
            for (int mu = 0; mu < M; ++mu) {
              if (s.shells[s.aos[mu].shell].center != I) continue;
              double c = s.C[sg][(size_t)mu * n + i];
              int e = e0 + el;
              dA[(size_t)el * n + i] -= AOv(e, mu, 1 + d) * c;
              for (int cc = 0; cc < 3; ++cc) dG[cc][(size_t)el * n + i] -= AOv(e, mu, hidx(d, cc)) * c;
              dL[(size_t)el * n + i] -= AOv(e, mu, 11 + d) * c;
            }
        // d ln det = tr(B dA)
        for (int el = 0; el < n; ++el)
          for (int i = 0; i < n; ++i) dlnpsi += B[sg][(size_t)i * n + el] * dA[(size_t)el * n + i];
        // dB = -B dA B
        std::vector<double> tmp((size_t)n * n, 0.0), dB((size_t)n * n, 0.0);
        for (int i = 0; i < n; ++i)
          for (int e = 0; e < n; ++e) {
            double v = 0;
            for (int k = 0; k < n; ++k) v += B[sg][(size_t)i * n + k] * dA[(size_t)k * n + e];
            tmp[(size_t)i * n + e] = v;
          }
        for (int i = 0; i < n; ++i)
          for (int e = 0; e < n; ++e) {
            double v = 0;
            for (int k = 0; k < n; ++k) v += tmp[(size_t)i * n + k] * B[sg][(size_t)k * n + e];
            dB[(size_t)i * n + e] = -v;
          }
        for (int el = 0; el < n; ++el) {
          int e = e0 + el;
          for (int i = 0; i < n; ++i) {
            double b = B[sg][(size_t)i * n + el], db = dB[(size_t)i * n + el];
            for (int c = 0; c < 3; ++c)
              dg[3 * e + c] += dG[c][(size_t)el * n + i] * b + G[sg][c][(size_t)el * n + i] * db;
            dl[e] += dL[(size_t)el * n + i] * b + L[sg][(size_t)el * n + i] * db;
          }
        }
      }
      // Jastrow: only chi_I depends on R_I; d/dR_I = -d/ds.
      std::vector<double> dJg((size_t)Ne * 3, 0.0), dJl(Ne, 0.0);
      if (s.J1)
        for (int e = 0; e < Ne; ++e) {
          double sv[3];
          for (int c = 0; c < 3; ++c) sv[c] = pos[3 * e + c] - s.R[3 * I + c];
          double r = std::sqrt(sv[0] * sv[0] + sv[1] * sv[1] + sv[2] * sv[2]);
          RadDeriv df = radial_derivs(chi(s.Z[I], s.ben, r), sv);
          dlnpsi -= df.g[d];
          for (int c = 0; c < 3; ++c) dJg[3 * e + c] += -df.H[d][c];
          dJl[e] += -df.glap[d];
        }
      // AO-expanded terms: the Jastrow functions centred on I move with it, d psi^J_nu(r_j) =
      // -d_d psi^J_nu(r_j) (and one order up for their gradients and Laplacians); d U =
      // sum_{e,mu} t_{e mu} d psi^J_mu(r_e), and t_{e mu} changes by sum_{j != e} sum_nu Xi_{mu nu} d psi^J_nu(r_j).
      if (MJ > 0) {
        std::vector<double> dphi((size_t)Ne * MJ, 0.0);
        std::vector<char> onI(MJ, 0);
        for (int mu = 0; mu < MJ; ++mu) onI[mu] = s.jshells[s.jaos[mu].shell].center == I;
        for (int e = 0; e < Ne; ++e)
          for (int nu = 0; nu < MJ; ++nu)
            if (onI[nu]) dphi[(size_t)e * MJ + nu] = -JV(e, nu, 1 + d);
        for (int e = 0; e < Ne; ++e)
          for (int mu = 0; mu < MJ; ++mu) {
            double dt = 0.0;
            for (int j = 0; j < Ne; ++j) {
              if (j == e) continue;
              for (int nu = 0; nu < MJ; ++nu)
                if (onI[nu]) dt += XI(mu, nu) * dphi[(size_t)j * MJ + nu];
            }
            const double t = tJ[(size_t)e * MJ + mu];
            dlnpsi += t * dphi[(size_t)e * MJ + mu];
            for (int c = 0; c < 3; ++c)
              dJg[3 * e + c] += (onI[mu] ? -JV(e, mu, hidx(d, c)) : 0.0) * t + JV(e, mu, 1 + c) * dt;
            dJl[e] += (onI[mu] ? -JV(e, mu, 11 + d) : 0.0) * t + JV(e, mu, 4) * dt;
          }
      }
      for (int e = 0; e < Ne; ++e) {
        double t = dl[e] + dJl[e];
        for (int c = 0; c < 3; ++c)
          t += 2.0 * Jg[3 * e + c] * dJg[3 * e + c] + 2.0 * dJg[3 * e + c] * gdet[3 * e + c] +
               2.0 * Jg[3 * e + c] * dg[3 * e + c];
        dEL += -0.5 * t;
      }
      // V_en: d/dR_I of -Z_I / |r_e - R_I| is -Z_I (r_e - R_I)_d / |r_e - R_I|^3.
      for (int e = 0; e < Ne; ++e) {
        double sv[3];
        for (int c = 0; c < 3; ++c) sv[c] = pos[3 * e + c] - s.R[3 * I + c];
        double r = std::sqrt(sv[0] * sv[0] + sv[1] * sv[1] + sv[2] * sv[2]);
        dEL += -s.Z[I] * sv[d] / (r * r * r);
      }
      // V_nn
      for (int Jn = 0; Jn < K; ++Jn) {
        if (Jn == I) continue;
        double sv[3];
        for (int c = 0; c < 3; ++c) sv[c] = s.R[3 * I + c] - s.R[3 * Jn + c];
        double r = std::sqrt(sv[0] * sv[0] + sv[1] * sv[1] + sv[2] * sv[2]);
        dEL += -s.Z[I] * s.Z[Jn] * sv[d] / (r * r * r);
      }
      w.dlnpsi_dR[3 * I + d] = dlnpsi;
      w.dEL_dR[3 * I + d] = dEL;
    }

  // ------------------------------------------------ electron derivatives, forward mode
  // For each electron coordinate lambda = r_{q,d}: row q of A, G and L moves (d psi / d lambda
  // = d_d psi at r_q, and likewise one order up); dB = -B dA B. In the Jastrow, every pair
  // term u(r_q - r_j) and every chi_I(r_q - R_I) depends on r_q; V_ee and V_en directly.
  if (want_electron) {
    w.dEL_dr.assign((size_t)Ne * 3, 0.0);
    for (int q = 0; q < Ne; ++q)
      for (int d = 0; d < 3; ++d) {
        const int sq = spin_of(s, q), n = nspin(s, sq), e0 = first_e(s, sq), elq = q - e0;
        std::vector<double> dg((size_t)Ne * 3, 0.0), dl(Ne, 0.0);
        // the moved rows: dA_{elq, i}, dG_{elq, i}, dL_{elq, i}
        std::vector<double> dArow(n, 0.0), dLrow(n, 0.0), dGrow[3];
        for (int c = 0; c < 3; ++c) dGrow[c].assign(n, 0.0);
        for (int i = 0; i < n; ++i)
          for (int mu = 0; mu < M; ++mu) {
            double c = s.C[sq][(size_t)mu * n + i];
            dArow[i] += AOv(q, mu, 1 + d) * c;
            for (int cc = 0; cc < 3; ++cc) dGrow[cc][i] += AOv(q, mu, hidx(d, cc)) * c;
            dLrow[i] += AOv(q, mu, 11 + d) * c;
          }
        // dB = -B dA B with dA nonzero in row elq only: dB_{i e} = -B_{i, elq} v_e,
        // v_e = sum_k dA_{elq, k} B_{k e}
        std::vector<double> v(n, 0.0);
        for (int e = 0; e < n; ++e)
          for (int k = 0; k < n; ++k) v[e] += dArow[k] * B[sq][(size_t)k * n + e];
        for (int el = 0; el < n; ++el) {
          int e = e0 + el;
          for (int i = 0; i < n; ++i) {
            double b = B[sq][(size_t)i * n + el], db = -B[sq][(size_t)i * n + elq] * v[el];
            for (int c = 0; c < 3; ++c)
              dg[3 * e + c] += (el == elq ? dGrow[c][i] : 0.0) * b + G[sq][c][(size_t)el * n + i] * db;
            dl[e] += (el == elq ? dLrow[i] : 0.0) * b + L[sq][(size_t)el * n + i] * db;
          }
        }
        double dEL = 0.0;
        std::vector<double> dJg((size_t)Ne * 3, 0.0), dJl(Ne, 0.0);
        for (int j = 0; j < Ne; ++j) {
          if (j == q) continue;
          double sv[3];
          for (int c = 0; c < 3; ++c) sv[c] = pos[3 * q + c] - pos[3 * j + c];
          double r = std::sqrt(sv[0] * sv[0] + sv[1] * sv[1] + sv[2] * sv[2]);
          dEL += -sv[d] / (r * r * r);  // V_ee
          if (s.J2) {
            bool par = spin_of(s, q) == spin_of(s, j);
            RadDeriv du = radial_derivs(pair_u(s, par, r), sv);
            for (int c = 0; c < 3; ++c) {
              dJg[3 * q + c] += du.H[d][c];  // grad_q u(r_q - r_j) moves with r_q
              dJg[3 * j + c] -= du.H[d][c];  // grad_j u = -grad_q u
            }
            dJl[q] += du.glap[d];  // both Laplacians of the pair term equal lap u(r_q - r_j)
            dJl[j] += du.glap[d];
          }
        }
        for (int I = 0; I < K; ++I) {
          double sv[3];
          for (int c = 0; c < 3; ++c) sv[c] = pos[3 * q + c] - s.R[3 * I + c];
          double r = std::sqrt(sv[0] * sv[0] + sv[1] * sv[1] + sv[2] * sv[2]);
          dEL += s.Z[I] * sv[d] / (r * r * r);  // V_en
          if (s.J1) {
            RadDeriv df = radial_derivs(chi(s.Z[I], s.ben, r), sv);
            for (int c = 0; c < 3; ++c) dJg[3 * q + c] += df.H[d][c];
            dJl[q] += df.glap[d];
          }
        }
        // AO-expanded terms: only the functions at r_q move; t_q does not depend on r_q, and for
        // e != q, t_{e mu} changes by sum_nu Xi_{mu nu} d_d psi^J_nu(r_q).
        if (MJ > 0)
          for (int e = 0; e < Ne; ++e)
            for (int mu = 0; mu < MJ; ++mu) {
              if (e == q) {
                const double t = tJ[(size_t)q * MJ + mu];
                for (int c = 0; c < 3; ++c) dJg[3 * q + c] += JV(q, mu, hidx(d, c)) * t;
                dJl[q] += JV(q, mu, 11 + d) * t;
              } else {
                double dt = 0.0;
                for (int nu = 0; nu < MJ; ++nu) dt += XI(mu, nu) * JV(q, nu, 1 + d);
                for (int c = 0; c < 3; ++c) dJg[3 * e + c] += JV(e, mu, 1 + c) * dt;
                dJl[e] += JV(e, mu, 4) * dt;
              }
            }
        for (int e = 0; e < Ne; ++e) {
          double t = dl[e] + dJl[e];
          for (int c = 0; c < 3; ++c)
            t += 2.0 * Jg[3 * e + c] * dJg[3 * e + c] + 2.0 * dJg[3 * e + c] * gdet[3 * e + c] +
                 2.0 * Jg[3 * e + c] * dg[3 * e + c];
          dEL += -0.5 * t;
        }
        w.dEL_dr[3 * q + d] = dEL;
      }
    // Space-warp coordinate transformation (force expression with omega, Sec. Methods /
    // App.): electrons near nucleus a move with it, with weight
    // omega_a(r) = kappa(|r - R_a|) / sum_b kappa(|r - R_b|), kappa(r) = 1 / r^4;
    // dE_L^sw/dR_a = dE_L/dR_a + sum_e omega_a(r_e) dE_L/dr_e,
    // d ln Psi^sw/dR_a = d ln Psi/dR_a + sum_e [omega_a(r_e) d ln Psi/dr_e + 1/2 grad omega_a(r_e)].
    w.dEL_sw = w.dEL_dR;
    w.dlnpsi_sw = w.dlnpsi_dR;
    std::vector<double> kap(K), gk((size_t)K * 3);
    for (int e = 0; e < Ne; ++e) {
      double ks = 0.0, gks[3] = {0, 0, 0};
      for (int b = 0; b < K; ++b) {
        double sv[3];
        for (int c = 0; c < 3; ++c) sv[c] = pos[3 * e + c] - s.R[3 * b + c];
        double r2 = sv[0] * sv[0] + sv[1] * sv[1] + sv[2] * sv[2];
        kap[b] = 1.0 / (r2 * r2);
        for (int c = 0; c < 3; ++c) gk[3 * b + c] = -4.0 * sv[c] / (r2 * r2 * r2);  // grad of r^-4
        ks += kap[b];
        for (int c = 0; c < 3; ++c) gks[c] += gk[3 * b + c];
      }
      for (int a = 0; a < K; ++a) {
        double om = kap[a] / ks;
        for (int c = 0; c < 3; ++c) {
          double gom = (gk[3 * a + c] * ks - kap[a] * gks[c]) / (ks * ks);
          w.dEL_sw[3 * a + c] += om * w.dEL_dr[3 * e + c];
          w.dlnpsi_sw[3 * a + c] += om * w.glnpsi[3 * e + c] + 0.5 * gom;
        }
      }
    }
  }

  // ------------------------------------------------ orbital-coefficient derivatives
  // O^s_{mu i} = d ln Psi / d C^s_{mu i} = sum_{e in s} psi_mu(r_e) B_{i e}.
  for (int sg = 0; sg < 2; ++sg) {
    int n = nspin(s, sg), e0 = first_e(s, sg);
    w.O[sg].assign((size_t)M * n, 0.0);
    for (int mu = 0; mu < M; ++mu)
      for (int i = 0; i < n; ++i) {
        double v = 0;
        for (int el = 0; el < n; ++el) v += AOv(e0 + el, mu, 0) * B[sg][(size_t)i * n + el];
        w.O[sg][(size_t)mu * n + i] = v;
      }
    w.dELdC[sg].assign((size_t)M * n, 0.0);
    if (!want_dC || n == 0) continue;
    // Forward mode in C^s_{mu i}: dA_{e k} = psi_mu(r_e) delta_{k i}, and likewise for the
    // gradient and Laplacian rows; dB = -B dA B has elements dB_{j e} = -O_{mu j} B_{i e}.
    for (int mu = 0; mu < M; ++mu)
      for (int i = 0; i < n; ++i) {
        double dEL = 0.0;
        for (int el = 0; el < n; ++el) {
          int e = e0 + el;
          double dge[3] = {0, 0, 0}, dle = 0.0;
          // terms with dG, dL (column i only)
          double b = B[sg][(size_t)i * n + el];
          for (int c = 0; c < 3; ++c) dge[c] += AOv(e, mu, 1 + c) * b;
          dle += AOv(e, mu, 4) * b;
          // terms with dB
          for (int j = 0; j < n; ++j) {
            double dbje = -w.O[sg][(size_t)mu * n + j] * b;
            for (int c = 0; c < 3; ++c) dge[c] += G[sg][c][(size_t)el * n + j] * dbje;
            dle += L[sg][(size_t)el * n + j] * dbje;
          }
          double t = dle;
          for (int c = 0; c < 3; ++c) t += 2.0 * Jg[3 * e + c] * dge[c];
          dEL += -0.5 * t;
        }
        w.dELdC[sg][(size_t)mu * n + i] = dEL;
      }
  }
}

// ---------------------------------------------------------------- Philox4x64-10
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11).
void philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
  uint64_t x[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
  uint64_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += W0; k1 += W1; }
    unsigned __int128 p0 = (unsigned __int128)M0 * x[0];
    unsigned __int128 p1 = (unsigned __int128)M1 * x[2];
    uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
    uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
    uint64_t y0 = hi1 ^ x[1] ^ k0, y1 = lo1, y2 = hi0 ^ x[3] ^ k1, y3 = lo0;
    x[0] = y0; x[1] = y1; x[2] = y2; x[3] = y3;
  }
  for (int i = 0; i < 4; ++i) out[i] = x[i];
}

inline double u01(uint64_t x) { return (double)(x >> 11) * (1.0 / 9007199254740992.0); }

// ---------------------------------------------------------------- sampling (App. A, MCMC)
// The Metropolis proposal, the refresh cadence and the generator are not specified by the
// paper; this follows the workload definition: Gaussian single-electron moves of width
// sigma, Philox counter (walker, sweep, electron, j), Sherman-Morrison updates of the
// inverse and a full re-inversion every k attempted moves.
void refresh(const OSys& s, const double* pos, double* Bst, int* singular) {
  const int M = s.M;
  std::vector<double> aov(M * NC);
  int off = 0;
  for (int sg = 0; sg < 2; ++sg) {
    int n = nspin(s, sg), e0 = first_e(s, sg);
    if (n == 0) continue;
    std::vector<double> A((size_t)n * n);
    for (int el = 0; el < n; ++el) {
      ao_eval_point(s, pos + 3 * (e0 + el), aov.data());
      for (int i = 0; i < n; ++i) {
        double v = 0;
        for (int mu = 0; mu < M; ++mu) v += aov[(size_t)mu * NC] * s.C[sg][(size_t)mu * n + i];
        A[(size_t)el * n + i] = v;
      }
    }
    double la, sgn;
    if (lu_inverse(n, A.data(), Bst + off, &la, &sgn)) *singular = 1;
    off += n * n;
  }
}

double u_pair(const OSys& s, int i, int j, double r) {
  bool par = spin_of(s, i) == spin_of(s, j);
  return pair_u(s, par, r).h;
}

// Guiding function for reweighted sampling (App., reweighting: sample |Psi_G|^2 and weight each
// sample by |Psi / Psi_G|^2). Reading of the Attaccalite-Sorella regularisation: Psi_G = Psi g with
// g(x) = max(1, eps sqrt(S(x))), S = sum over both spin blocks of the squared entries of the inverse
// Slater matrices; 1 / sqrt(S) vanishes linearly on the nodal surface of the determinants, so
// Psi_G stays finite there. eps = 0 gives g = 1 (plain sampling).
double frob2(const OSys& s, const double* Bst) {
  const size_t nb = (size_t)s.nup * s.nup + (size_t)s.ndn * s.ndn;
  double v = 0.0;
  for (size_t k = 0; k < nb; ++k) v += Bst[k] * Bst[k];
  return v;
}
double guide_g(double eps, double S) { return std::max(1.0, eps * std::sqrt(S)); }

// Change of the Jastrow exponent J when electron e moves from pos[e] to rn: the two-body terms
// of its pairs, its e-n terms and the AO-expanded terms that hold it.
double move_jastrow_diff(const OSys& s, const double* pos, int e, const double rn[3]) {
  const int Ne = s.nup + s.ndn;
  double dJ = 0.0;
  if (s.J2)
    for (int j = 0; j < Ne; ++j) {
      if (j == e) continue;
      double dn[3], d0[3];
      for (int d = 0; d < 3; ++d) { dn[d] = rn[d] - pos[3 * j + d]; d0[d] = pos[3 * e + d] - pos[3 * j + d]; }
      dJ += u_pair(s, e, j, std::sqrt(dn[0] * dn[0] + dn[1] * dn[1] + dn[2] * dn[2])) -
            u_pair(s, e, j, std::sqrt(d0[0] * d0[0] + d0[1] * d0[1] + d0[2] * d0[2]));
    }
  if (s.J1)
    for (int I = 0; I < s.K; ++I) {
      double dn[3], d0[3];
      for (int d = 0; d < 3; ++d) { dn[d] = rn[d] - s.R[3 * I + d]; d0[d] = pos[3 * e + d] - s.R[3 * I + d]; }
      dJ += chi(s.Z[I], s.ben, std::sqrt(dn[0] * dn[0] + dn[1] * dn[1] + dn[2] * dn[2])).h -
            chi(s.Z[I], s.ben, std::sqrt(d0[0] * d0[0] + d0[1] * d0[1] + d0[2] * d0[2])).h;
    }
  if (s.MJ > 0) {
    // AO-expanded terms (Eqs. onebody_J_inhom, threebody_jas): the terms that hold electron e,
    // sum_mu xi_mu dphi_mu + sum_{j != e} sum_{mu,nu} dphi_mu Xi_{mu nu} psi^J_nu(r_j), with
    // dphi = psi^J(r') - psi^J(r_e)
    const int MJ = s.MJ;
    std::vector<double> jn((size_t)MJ * NC), jo((size_t)MJ * NC), jj((size_t)MJ * NC), dphi(MJ);
    basis_eval_point(s.jshells, s.jaos, s.R, rn, jn.data());
    basis_eval_point(s.jshells, s.jaos, s.R, pos + 3 * e, jo.data());
    for (int mu = 0; mu < MJ; ++mu) {
      dphi[mu] = jn[(size_t)mu * NC] - jo[(size_t)mu * NC];
      dJ += s.xi[mu] * dphi[mu];
    }
    for (int j = 0; j < Ne; ++j) {
      if (j == e) continue;
      basis_eval_point(s.jshells, s.jaos, s.R, pos + 3 * j, jj.data());
      for (int mu = 0; mu < MJ; ++mu)
        for (int nu = 0; nu < MJ; ++nu) dJ += dphi[mu] * s.Xi[(size_t)mu * MJ + nu] * jj[(size_t)nu * NC];
    }
  }
  return dJ;
}

void sample_walker(const OSys& s, int wid, double* pos, double* Bst, uint64_t k0, uint64_t k1,
                   uint64_t sweep0, int nsweeps, double sigma, int kref, int* counter,
                   uint32_t* nacc, uint32_t* nsing, double* margin, double eps = 0.0) {
  const int Ne = s.nup + s.ndn, M = s.M;
  std::vector<double> aov(M * NC), row(std::max(s.nup, s.ndn) + 1), w(std::max(s.nup, s.ndn) + 1);
  const uint64_t key[2] = {k0, k1};
  int c = *counter;
  for (int sw = 0; sw < nsweeps; ++sw) {
    uint64_t sweep = sweep0 + sw;
    for (int e = 0; e < Ne; ++e) {
      int sg = spin_of(s, e), n = nspin(s, sg), el = e - first_e(s, sg);
      double* B = Bst + (sg == 0 ? 0 : s.nup * s.nup);
      uint64_t ctr[4] = {(uint64_t)wid, sweep, (uint64_t)e, 0}, rnd[4];
      philox4x64_10(ctr, key, rnd);
      double u1 = u01(rnd[0]), u2 = u01(rnd[1]), u3 = u01(rnd[2]), u4 = u01(rnd[3]);
      double rad1 = std::sqrt(-2.0 * std::log(1.0 - u1));
      double rad2 = std::sqrt(-2.0 * std::log(1.0 - u3));
      const double twopi = 6.283185307179586;
      double xi[3] = {rad1 * std::cos(twopi * u2), rad1 * std::sin(twopi * u2), rad2 * std::cos(twopi * u4)};
      double rn[3];
      for (int d = 0; d < 3; ++d) rn[d] = pos[3 * e + d] + sigma * xi[d];
      // determinant ratio from the new orbital row
      ao_eval_point(s, rn, aov.data());
      double R = 0.0;
      for (int i = 0; i < n; ++i) {
        double v = 0;
        for (int mu = 0; mu < M; ++mu) v += aov[(size_t)mu * NC] * s.C[sg][(size_t)mu * n + i];
        row[i] = v;
        R += v * B[(size_t)i * n + el];
      }
      // Jastrow ratio
      const double dJ = move_jastrow_diff(s, pos, e, rn);
      double p = R * R * std::exp(2.0 * dJ);
      if (eps > 0.0 && R != 0.0) {
        // the guiding factor at the proposed configuration, from the updated inverse formed explicitly
        const size_t nbst = (size_t)s.nup * s.nup + (size_t)s.ndn * s.ndn;
        std::vector<double> Bn(Bst, Bst + nbst);
        double* Bp = Bn.data() + (sg == 0 ? 0 : s.nup * s.nup);
        std::vector<double> wt(n);
        for (int j = 0; j < n; ++j) {
          double v = 0;
          for (int i = 0; i < n; ++i) v += row[i] * B[(size_t)i * n + j];
          wt[j] = v - (j == el ? 1.0 : 0.0);
        }
        for (int k = 0; k < n; ++k)
          for (int j = 0; j < n; ++j) Bp[(size_t)k * n + j] -= B[(size_t)k * n + el] * wt[j] / R;
        const double g0 = guide_g(eps, frob2(s, Bst)), g1 = guide_g(eps, frob2(s, Bn.data()));
        p *= (g1 / g0) * (g1 / g0);
      }
      uint64_t ctr2[4] = {(uint64_t)wid, sweep, (uint64_t)e, 1};
      philox4x64_10(ctr2, key, rnd);
      double u = u01(rnd[0]);
      bool ok = std::isfinite(p) && R != 0.0;
      if (!ok) ++*nsing;
      if (ok && p > 0) *margin = std::min(*margin, std::fabs(u - p) / p);
      if (ok && u < p) {
        // Sherman-Morrison: row el of A replaced by the new row.
        for (int j = 0; j < n; ++j) {
          double v = 0;
          for (int i = 0; i < n; ++i) v += row[i] * B[(size_t)i * n + j];
          w[j] = v - (j == el ? 1.0 : 0.0);
        }
        std::vector<double> col(n);
        for (int k = 0; k < n; ++k) col[k] = B[(size_t)k * n + el];
        for (int k = 0; k < n; ++k)
          for (int j = 0; j < n; ++j) B[(size_t)k * n + j] -= col[k] * w[j] / R;
        for (int d = 0; d < 3; ++d) pos[3 * e + d] = rn[d];
        ++*nacc;
      }
      if (++c == kref) {
        int sing = 0;
        refresh(s, pos, Bst, &sing);
        c = 0;
      }
    }
  }
  *counter = c;
}

}  // namespace

// Shells of a basis: each primitive normalised, then the contraction renormalised (convention
// P1); returns the number of functions added.
static int add_shells(std::vector<Shell>& shells, std::vector<AO>& aos, int nshell, const int* center, const int* l,
               const int* nprim, const double* exps, const double* coefs, int maxprim) {
  int nf = 0;
  for (int sh = 0; sh < nshell; ++sh) {
    Shell x;
    x.center = center[sh];
    x.l = l[sh];
    x.nprim = nprim[sh];
    double d[8], S = 0.0;
    for (int k = 0; k < x.nprim; ++k) {
      x.alpha[k] = exps[sh * maxprim + k];
      d[k] = coefs[sh * maxprim + k];
    }
    for (int a = 0; a < x.nprim; ++a)
      for (int b = 0; b < x.nprim; ++b) S += d[a] * d[b] * prim_overlap(x.alpha[a], x.alpha[b], x.l);
    for (int k = 0; k < x.nprim; ++k) x.coef[k] = d[k] * prim_norm(x.alpha[k], x.l) / std::sqrt(S);
    const int first = (int)shells.size();
    shells.push_back(x);
    for (auto& poly : solid_harmonics(x.l)) {
      aos.push_back({first, poly});
      ++nf;
    }
  }
  return nf;
}

// ==================================================================== C interface
extern "C" {

void* osys_create(int K, const int* Z, const double* R, int nshell, const int* center, const int* l,
                  const int* nprim, const double* exps, const double* coefs, int maxprim, int n_up,
                  int n_dn, const double* C_up, const double* C_dn, const double* jas, int enable_J1,
                  int enable_J2, int j2exp) {
  OSys* s = new OSys();
  s->K = K;
  s->Z.assign(Z, Z + K);
  s->R.assign(R, R + 3 * K);
  s->M = add_shells(s->shells, s->aos, nshell, center, l, nprim, exps, coefs, maxprim);
  s->nup = n_up;
  s->ndn = n_dn;
  s->C[0].assign(C_up, C_up + (size_t)s->M * n_up);
  s->C[1].assign(C_dn, C_dn + (size_t)s->M * n_dn);
  s->Fa = jas[0]; s->Fp = jas[1]; s->aa = jas[2]; s->ap = jas[3]; s->ben = jas[4];
  s->J1 = enable_J1;
  s->J2 = enable_J2;
  s->j2exp = j2exp;
  return s;
}

// Jastrow basis of the AO-expanded terms (same conventions as the determinant basis, centred on
// the same nuclei), one-body coefficients xi [MJ] and symmetric pair coefficients Xi [MJ][MJ]
// (either may be NULL: zero). Returns MJ.
int osys_set_jastrow_basis(void* p, int nshell, const int* center, const int* l, const int* nprim,
                           const double* exps, const double* coefs, int maxprim, const double* xi,
                           const double* Xi) {
  OSys* s = static_cast<OSys*>(p);
  s->jshells.clear();
  s->jaos.clear();
  s->MJ = add_shells(s->jshells, s->jaos, nshell, center, l, nprim, exps, coefs, maxprim);
  const size_t MJ = (size_t)s->MJ;
  s->xi.assign(MJ, 0.0);
  s->Xi.assign(MJ * MJ, 0.0);
  if (xi) s->xi.assign(xi, xi + MJ);
  if (Xi) s->Xi.assign(Xi, Xi + MJ * MJ);
  return s->MJ;
}

// Change of the Jastrow exponent that the sampler uses when electron e of the walker at pos
// [Ne][3] moves to rn [3].
double osys_move_jastrow_diff(void* p, const double* pos, int e, const double* rn) {
  return move_jastrow_diff(*static_cast<OSys*>(p), pos, e, rn);
}

void osys_destroy(void* p) { delete static_cast<OSys*>(p); }
int osys_nao(void* p) { return static_cast<OSys*>(p)->M; }

void osys_norm_coefs(void* p, double* out, int maxprim) {
  OSys* s = static_cast<OSys*>(p);
  for (size_t sh = 0; sh < s->shells.size(); ++sh)
    for (int k = 0; k < s->shells[sh].nprim; ++k) out[sh * maxprim + k] = s->shells[sh].coef[k];
}

// out: [npts][M][14] (value, grad 3, Laplacian, Hessian xx yy zz xy xz yz, grad-Laplacian 3)
void osys_ao_eval(void* p, int npts, const double* pts, double* out) {
  OSys* s = static_cast<OSys*>(p);
  for (int i = 0; i < npts; ++i) ao_eval_point(*s, pts + 3 * i, out + (size_t)i * s->M * NC);
}

int oracle_lu_inverse(int n, const double* A, double* inv, double* logabs, double* sgn) {
  return lu_inverse(n, A, inv, logabs, sgn);
}

void oracle_philox4x64_10(const uint64_t* ctr, const uint64_t* key, uint64_t* out) { philox4x64_10(ctr, key, out); }

// Per-walker evaluation. Any output pointer may be NULL.
// EL, logpsi, sgn: [W]; dlnpsi_dR, dEL_dR: [W][K][3]; O, dELdC: [W][M*n_up + M*n_dn];
// glnpsi: [W][Ne][3]; laplnpsi: [W][Ne]; parts: [W][5] = (Ekin, Vee, Ven, Vnn, J).
int osys_eval(void* p, int W, const double* pos, int nthreads, double* EL, double* logpsi, double* sgn,
              double* dlnpsi_dR, double* dEL_dR, double* O, double* dELdC, double* glnpsi,
              double* laplnpsi, double* parts) {
  OSys* s = static_cast<OSys*>(p);
  const int Ne = s->nup + s->ndn, K = s->K, M = s->M;
  const size_t nO = (size_t)M * (s->nup + s->ndn);
  int nsing = 0;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : nsing)
#endif
  for (int w = 0; w < W; ++w) {
    WalkerOut o;
    eval_walker(*s, pos + (size_t)w * Ne * 3, dELdC != nullptr, o);
    nsing += o.singular;
    if (EL) EL[w] = o.EL;
    if (logpsi) logpsi[w] = o.logpsi;
    if (sgn) sgn[w] = o.sgn;
    if (dlnpsi_dR) std::copy(o.dlnpsi_dR.begin(), o.dlnpsi_dR.end(), dlnpsi_dR + (size_t)w * K * 3);
    if (dEL_dR) std::copy(o.dEL_dR.begin(), o.dEL_dR.end(), dEL_dR + (size_t)w * K * 3);
    if (O) {
      std::copy(o.O[0].begin(), o.O[0].end(), O + w * nO);
      std::copy(o.O[1].begin(), o.O[1].end(), O + w * nO + o.O[0].size());
    }
    if (dELdC) {
      std::copy(o.dELdC[0].begin(), o.dELdC[0].end(), dELdC + w * nO);
      std::copy(o.dELdC[1].begin(), o.dELdC[1].end(), dELdC + w * nO + o.dELdC[0].size());
    }
    if (glnpsi) std::copy(o.glnpsi.begin(), o.glnpsi.end(), glnpsi + (size_t)w * Ne * 3);
    if (laplnpsi) std::copy(o.laplnpsi.begin(), o.laplnpsi.end(), laplnpsi + (size_t)w * Ne);
    if (parts) {
      double* q = parts + (size_t)w * 5;
      q[0] = o.Ekin; q[1] = o.Vee; q[2] = o.Ven; q[3] = o.Vnn; q[4] = o.J;
    }
  }
  return nsing;
}

// Electron derivatives and space-warp force vectors per walker (any output may be NULL):
// dEL_dr [W][Ne][3], dEL_sw and dlnpsi_sw [W][K][3].
int osys_eval_warp(void* p, int W, const double* pos, int nthreads, double* dEL_dr, double* dEL_sw,
                   double* dlnpsi_sw) {
  OSys* s = static_cast<OSys*>(p);
  const int Ne = s->nup + s->ndn, K = s->K;
  int nsing = 0;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 2) reduction(+ : nsing)
#endif
  for (int w = 0; w < W; ++w) {
    WalkerOut o;
    eval_walker(*s, pos + (size_t)w * Ne * 3, false, o, true);
    nsing += o.singular;
    if (dEL_dr) std::copy(o.dEL_dr.begin(), o.dEL_dr.end(), dEL_dr + (size_t)w * Ne * 3);
    if (dEL_sw) std::copy(o.dEL_sw.begin(), o.dEL_sw.end(), dEL_sw + (size_t)w * K * 3);
    if (dlnpsi_sw) std::copy(o.dlnpsi_sw.begin(), o.dlnpsi_sw.end(), dlnpsi_sw + (size_t)w * K * 3);
  }
  return nsing;
}

// Reweighting factor |Psi / Psi_G|^2 = 1 / g^2 of every walker from fresh inverses.
int osys_guide_weight(void* p, int W, const double* pos, double eps, double* wt, int nthreads) {
  OSys* s = static_cast<OSys*>(p);
  const int Ne = s->nup + s->ndn;
  const size_t nb = (size_t)s->nup * s->nup + (size_t)s->ndn * s->ndn;
  int nsing = 0;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : nsing)
#endif
  for (int w = 0; w < W; ++w) {
    std::vector<double> B(std::max<size_t>(nb, 1));
    int sing = 0;
    refresh(*s, pos + (size_t)w * Ne * 3, B.data(), &sing);
    nsing += sing;
    const double g = guide_g(eps, frob2(*s, B.data()));
    wt[w] = 1.0 / (g * g);
  }
  return nsing;
}

// Fresh inverses for every walker: Bst [W][n_up^2 + n_dn^2].
int osys_refresh(void* p, int W, const double* pos, double* Bst, int nthreads) {
  OSys* s = static_cast<OSys*>(p);
  const int Ne = s->nup + s->ndn;
  const size_t nb = (size_t)s->nup * s->nup + (size_t)s->ndn * s->ndn;
  int nsing = 0;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : nsing)
#endif
  for (int w = 0; w < W; ++w) {
    int sing = 0;
    refresh(*s, pos + (size_t)w * Ne * 3, Bst + w * nb, &sing);
    nsing += sing;
  }
  return nsing;
}

// Metropolis sweeps. pos [W][Ne][3] and Bst are updated in place. wid0 is the global id
// of walker 0 (Philox counter word 0). counter: attempted moves since the last refresh,
// the same for every walker (in/out). nacc, nsing: per-walker counts (added to).
// margin: per-walker minimum of |u - p| / p over all decisions (in/out).
void osys_sample(void* p, int W, double* pos, double* Bst, uint64_t wid0, uint64_t k0, uint64_t k1,
                 uint64_t sweep0, int nsweeps, double sigma, int kref, int* counter, uint32_t* nacc,
                 uint32_t* nsing, double* margin, int nthreads, double eps) {
  OSys* s = static_cast<OSys*>(p);
  const int Ne = s->nup + s->ndn;
  const size_t nb = (size_t)s->nup * s->nup + (size_t)s->ndn * s->ndn;
  int c0 = *counter;
  if (nsweeps > 0 && c0 >= kref) {
    // k lowered since the last call: the attempted moves since the last re-inversion already
    // reach it, so the inverses are rebuilt before the first move
    osys_refresh(p, W, pos, Bst, nthreads);
    c0 = 0;
  }
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
#endif
  for (int w = 0; w < W; ++w) {
    const uint64_t wid = wid0 + (uint64_t)w;
    int c = c0;
    sample_walker(*s, (int)wid, pos + (size_t)w * Ne * 3, Bst + w * nb, k0, k1, sweep0, nsweeps, sigma, kref,
                  &c, nacc + w, nsing + w, margin + w, eps);
  }
  *counter = (int)((c0 + (long long)nsweeps * Ne) % kref);  // the common counter
}

}  // extern "C"
