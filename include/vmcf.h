/*
 * vmcf — GB300-native VMC evaluation of a Jastrow x spin-block Slater wavefunction with
 * frozen orbitals: local energy, Hellmann-Feynman + Pulay atomic forces and the
 * orbital-coefficient gradient dE/dC, over many independent walkers.
 *
 * Method: arXiv:2511.05222, "Fast Evaluation of Unbiased Atomic Forces in ab initio
 * Variational Monte Carlo via the Lagrangian Technique".
 *   - wavefunction: App. A ("Wavefunction Ansatz"): Psi = exp(J) det A_up det A_dn, the
 *     Jastrow-Slater determinant that the JAGP becomes when the geminal is expanded over
 *     the occupied orbitals; MOs phi_i = sum_mu C_{mu i} psi_mu (Eq. restricted-C);
 *     Pade two-body Jastrow (Eq. twobody_v) made spin dependent, plus the one-body
 *     e-n cusp term chi_I(r) = -Z_I r / (1 + b r);
 *   - local energy E_L = H Psi / Psi and the MCMC averages (App. A, Eq. eval-observable);
 *   - forces F = -<dE_L/dR> - 2 <(E_L - E) d ln Psi / dR> (Eqs. hf, pulay); the
 *     non-variational term (Eq. add) needs the CPKS response and is not computed here;
 *   - dE/dC = 2 (<E_L O> - E <O>), O = d ln Psi / dC (App. A, Eq. fc-vmc-eval, whose
 *     printed sign is the generalised-force convention -dE/dC);
 *   - optional right-hand side -B Q of the Z-vector equations (Eqs. Q_projector,
 *     AZ_eq_B_elements) when the AO overlap S is supplied;
 *   - jackknife error bars over walker blocks (Sec. II, last paragraph).
 *
 * Conventions shared by every entry point:
 *   - atomic units (bohr, hartree); row-major arrays; double precision at the boundary;
 *   - every call returns a vmcf_status code; no exception crosses the boundary; the text
 *     of the last error of the calling thread is returned by vmcf_last_error();
 *   - "device" pointers are CUDA device (or managed) memory owned by the caller;
 *     "host" pointers are host memory owned by the caller; the library copies what it
 *     keeps and never frees a caller's pointer;
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream);
 *     calls are asynchronous on that stream unless stated otherwise;
 *   - electrons are ordered spin up first: 0..n_up-1 up, n_up..n_up+n_dn-1 down.
 *     Positions are [W][Ne][3]; O and dE/dC are [2 spin blocks] = [M][n_up] followed by
 *     [M][n_dn] (compound index (mu i sigma) of the paper's App. B);
 *   - AOs: real solid harmonics r^l Y_lm (unit-sphere normalised), p = (x, y, z),
 *     d = (xy, yz, 3z^2 - r^2, xz, x^2 - y^2); each primitive normalised, then the
 *     contraction renormalised; AOs are numbered shell by shell in input order.
 */
#ifndef VMCF_H
#define VMCF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  VMCF_OK = 0,
  VMCF_EINVAL = -1,     /* bad argument (sizes, pointers, basis, NaN input) */
  VMCF_ENOMEM = -2,     /* device or host allocation failed */
  VMCF_ECUDA = -3,      /* a CUDA runtime call or kernel launch failed */
  VMCF_ESINGULAR = -4,  /* a Slater matrix had a zero pivot (walker on a node) */
  VMCF_ETIMEOUT = -5,   /* a bounded device-side wait gave up */
  VMCF_ENOTSUP = -6     /* configuration not supported by this build */
} vmcf_status;

typedef enum {
  VMCF_FP64 = 0,  /* every step in double precision */
  VMCF_MIXED = 1  /* FP32 AOs, MOs, Jastrow, adjoint and O; FP64 LU/inverse, ratio,
                     refresh and walker sums */
} vmcf_precision;

/* OR-ed into `precision` at vmcf_init_system: run a system that fits the small-system
 * kernels (at most 32 electrons and 16 orbitals per spin) on the general walker-group kernels
 * instead. Both give the same results within rounding; this exists to test one against the
 * other. */
#define VMCF_FORCE_GROUP_PATH 0x100

/* OR-ed into `precision` at vmcf_init_system: also accumulate the space-warp (SWCT) force
 * estimator (the force expression with the warp weights omega, Methods/appendix: electrons
 * near nucleus a move with it with weight omega_a(r) = kappa(|r - R_a|) / sum_b kappa(|r - R_b|),
 * kappa(r) = r^-4). Its walker sums are appended to each block (see vmcf_block_sums); read the
 * estimate with vmcf_reduce_warp. Same expectation as the plain forces, smaller variance. */
#define VMCF_SPACE_WARP 0x200

typedef struct vmcf_system_s* vmcf_system_t;   /* opaque, library-owned */
typedef struct vmcf_walkers_s* vmcf_walkers_t; /* opaque, library-owned device state */

typedef struct {
  int K;            /* number of nuclei, >= 1 */
  const int* Z;     /* host [K], nuclear charges >= 1 */
  const double* R;  /* host [K][3], positions */
} vmcf_nuclei;

typedef struct {
  int nshell;           /* >= 1 */
  int maxprim;          /* row stride of exps/coefs, 1..8 */
  const int* center;    /* host [nshell], 0..K-1 */
  const int* l;         /* host [nshell], 0..2 */
  const int* nprim;     /* host [nshell], 1..maxprim */
  const double* exps;   /* host [nshell][maxprim], > 0 */
  const double* coefs;  /* host [nshell][maxprim], coefficients of normalised primitives */
} vmcf_basis;

typedef struct {
  double F_anti, F_par; /* Pade denominators F (Eq. twobody_v); default 0.8, 0.8 */
  double a_anti, a_par; /* Pade numerators; Kato cusps: 0.5 antiparallel, 0.25 parallel */
  double b_en;          /* one-body chi_I(r) = -Z_I r / (1 + b_en r); default 1.5 */
  int enable_J1;        /* one-body term on/off */
  int enable_J2;        /* two-body term on/off */
  int two_body_exp;     /* two-body form: 0 Pade a r / (1 + F r) (Eq. twobody_v), 1 exponential
                           (a / F)(1 - exp(-F r)) (Eq. twobody_v_exp); a is the cusp in both */
  /* AO-expanded Jastrow terms over a separate Jastrow basis psi^J (App., Eqs. onebody_J_inhom and
   * threebody_jas), read as further terms of the Jastrow exponent:
   *   sum_e sum_mu xi_mu psi^J_mu(r_e) + sum_{i<j} sum_{mu,nu} Xi_{mu nu} psi^J_mu(r_i) psi^J_nu(r_j)
   * (the inhomogeneous one-body term and the three-body term; entries of Xi between functions of
   * different nuclei are the four-body terms). NULL basis: none. The basis follows the conventions
   * of the determinant basis, on the same nuclei, with at most 1024 functions (MJ); xi: host [MJ]
   * or NULL (zero); Xi: host [MJ][MJ] or NULL (zero), symmetric to 1e-12 relative (else
   * VMCF_EINVAL). Systems with these terms run on the walker-group kernels. */
  const vmcf_basis* basis;
  const double* xi;
  const double* Xi;
} vmcf_jastrow;

typedef struct {
  uint64_t moves;            /* attempted single-electron moves since creation */
  uint64_t accepted;         /* accepted moves */
  uint64_t rejected_nonfinite; /* moves rejected because the ratio was 0 or not finite */
  uint64_t singular;         /* Slater inversions that met a zero pivot */
  uint64_t refreshes;        /* full re-inversions performed (per walker, summed) */
  uint64_t sweeps;           /* sweeps performed */
  uint64_t measured_sweeps;  /* sweeps accumulated into the estimators */
} vmcf_counters;

/* Build a system: validates the input, normalises the basis, uploads tables and C.
 * Defines the wavefunction of App. A ("Wavefunction Ansatz"): the JAGP expanded over the n_up,
 * n_dn occupied orbitals, i.e. the Jastrow-Slater determinant Psi = exp(J) det A_up det A_dn with
 * A^s_{ei} = phi^s_i(r_e) and phi^s_i = sum_mu C^s_{mu i} psi_mu (Eqs. agp_expansion, restricted-C,
 * occ-expansion); psi_mu are the contracted GTOs of `basis` on `nuclei`; J is the one-body and
 * two-body Jastrow of `jastrow` (Eqs. twobody_v, twobody_v_exp, onebody_J_inhom, threebody_jas).
 * C is frozen (the paper's coefficients come from DFT and stay fixed in VMC); R and C are the two
 * parameter sets the forces and dE/dC differentiate.
 * C_up [M][n_up], C_dn [M][n_dn]: host, double, row-major [mu][i] (M = number of AOs).
 * S: host [M][M] AO overlap, or NULL (then rhs_BQ is unavailable).
 * n_up >= n_dn >= 0, n_up >= 1, n_up <= 64, M <= 1024.
 * Rejected with VMCF_EINVAL before any CUDA call: NULL inputs, non-finite nuclear positions or
 * coefficients, charges < 1, two nuclei at the same position, invalid shells (l > 2, exponents
 * <= 0, centres out of range, a contraction of zero norm), and a C_up or C_dn with linearly
 * dependent columns (every Slater matrix would be singular). Walker positions are not scanned:
 * a non-finite position makes that walker's moves rejected (counted in rejected_nonfinite).
 * The call synchronises the current device. */
int vmcf_init_system(const vmcf_nuclei* nuclei, const vmcf_basis* basis, const double* C_up,
                     const double* C_dn, int n_up, int n_dn, const vmcf_jastrow* jastrow,
                     const double* S, int precision, vmcf_system_t* out);
int vmcf_system_destroy(vmcf_system_t sys);
/* Sizes of a system: number of nuclei, AOs, up and down electrons (any pointer may be NULL). */
int vmcf_system_info(vmcf_system_t sys, int* K, int* M, int* n_up, int* n_dn);
/* Replaces the nuclear positions R [K][3] (bohr) and the frozen orbital coefficients C_up [M][n_up], C_dn [M][n_dn]
 * (row-major, host memory, copied) of an existing system, keeping its basis, charges, Jastrow factor, precision and
 * kernel plans: the wavefunction of App. "Wavefunction Ansatz" at another geometry, e.g. for the forces of Eqs. hf,
 * pulay along a trajectory or for derivatives with respect to R and C. S: the AO overlap at the new geometry
 * ([M][M], host) for vmcf_reduce_estimators' rhs_BQ, or NULL (rhs_BQ is then refused until S is given again).
 * Validated as at creation (VMCF_EINVAL before any CUDA call: non-finite values, two nuclei at one position,
 * linearly dependent columns of C); the system is unchanged on error. The call synchronises the system's device and
 * must not overlap kernels that use this system. Walker sets of the system keep their positions, but their inverses
 * and accumulated sums belong to the old wavefunction: re-invert them (vmcf_walkers_set_positions) and reset their
 * sums (vmcf_reset_accumulators) before sampling or reducing. Batches notice the change at their next
 * vmcf_batch_sample. */
int vmcf_system_set_geometry(vmcf_system_t sys, const double* R, const double* C_up, const double* C_dn,
                             const double* S);

/* Walker state for sampling: positions, Slater inverses, counters, accumulators. The walkers are
 * the set {x_i} of App. A ("Variational Monte Carlo Methods") that the Markov chain draws from
 * pi(x) = Psi^2 / int Psi^2; each walker is one independent chain, and the estimators are the
 * averages over walkers and measured sweeps (Eq. eq-eval-observable).
 * pos: [W][Ne][3] double, device (is_host = 0) or host (is_host = 1) memory.
 * key0, key1: Philox4x64-10 key; wid0: global id of walker 0 (Philox counter word 0), so
 * that shards of one walker set on several GPUs draw the same streams as one GPU would.
 * nblocks: jackknife blocks (contiguous walker groups), 2 <= nblocks <= W.
 * The initial inverses are built (a full FP64 inversion) before the call returns. */
int vmcf_walkers_create(vmcf_system_t sys, int W, const double* pos, int is_host, uint64_t key0,
                        uint64_t key1, uint64_t wid0, int nblocks, void* stream, vmcf_walkers_t* out);
int vmcf_walkers_destroy(vmcf_walkers_t wk);
/* Replace the positions (device or host memory) and rebuild the inverses. */
int vmcf_walkers_set_positions(vmcf_system_t sys, vmcf_walkers_t wk, const double* pos, int is_host,
                               void* stream);
/* Copy the current positions out ([W][Ne][3], device or host memory). */
int vmcf_walkers_get_positions(vmcf_walkers_t wk, double* pos, int is_host, void* stream);
/* Zero the estimator accumulators and set the reference energy subtracted from E_L
 * before it multiplies d ln Psi / dR or O (cancellation control; results do not depend
 * on it except by rounding). */
int vmcf_reset_accumulators(vmcf_walkers_t wk, double e_ref, void* stream);
/* Reweighted (guided) sampling (App., reweighting; the Attaccalite-Sorella scheme the paper uses to
 * keep the force and dE/dC estimators finite-variance near the nodal surface). With eps > 0 the
 * walker set samples |Psi_G|^2, Psi_G = Psi g, g = max(1, eps sqrt(S)), where S is the sum over
 * both spin blocks of the squared entries of the inverse Slater matrices (1/sqrt(S) vanishes
 * linearly on the nodal surface), and every measured sample enters the walker sums with weight
 * |Psi/Psi_G|^2 = 1/g^2 (the sample count becomes the sum of the weights), so that every estimator
 * is sum(W O) / sum(W). eps = 0 (the default) is plain |Psi|^2 sampling, bit for bit. The moves
 * track S through each Sherman-Morrison update and recompute it at every refresh. Takes effect at
 * the next vmcf_sample / vmcf_measure. */
int vmcf_set_guiding(vmcf_walkers_t wk, double eps);

/* Metropolis sweeps (App. A, MCMC). Each sweep moves every electron once, in order, with
 * a Gaussian proposal of width step_sigma; the Philox counter is (walker id, sweep index,
 * electron, 0) for the three normals (Box-Muller) and (..., 1) for the acceptance draw.
 * Accepted moves update the inverse by Sherman-Morrison; every refresh_k attempted moves
 * the inverses are rebuilt from scratch in FP64. measure != 0: after each sweep the
 * inverse is rebuilt (if not fresh) and E_L, d ln Psi/dR, dE_L/dR and O are accumulated
 * into the estimator sums. */
int vmcf_sample(vmcf_system_t sys, vmcf_walkers_t wk, int n_sweeps, double step_sigma, int refresh_k,
                int measure, void* stream);

/* One measurement of the walkers' current positions, without moving them: the inverses
 * are rebuilt in FP64 and E_L, d ln Psi/dR, dE_L/dR and O are added to the walker sums (as
 * one measured sweep of vmcf_sample does). Used for estimators on fixed configurations. */
int vmcf_measure(vmcf_system_t sys, vmcf_walkers_t wk, void* stream);

/* Fixed-walker evaluation (no sampling): the per-sample quantities whose averages make up the
 * estimators. E_L = H Psi / Psi (App. A, the local energy of Eq. eq-eval-observable); d ln Psi/dR and
 * dE_L/dR, the per-sample terms of the Pulay and Hellmann-Feynman forces (Eqs. pulay, hf), as total
 * derivatives at fixed electron positions (AOs and one-body terms move with their nucleus, C fixed);
 * O = d ln Psi / dC (App. A, "Computing derivatives", Eq. fc-vmc-eval).
 * pos: device [W][Ne][3], W >= 0 (W = 0: nothing is
 * read or written and pos may be NULL). Outputs are device buffers owned by the caller; any may
 * be NULL:
 *   EL [W], logpsi [W] (ln|Psi|), dlnpsi_dR [W][K][3], dEL_dR [W][K][3],
 *   O [W][M*(n_up+n_dn)], dEL_dC [W][M*(n_up+n_dn)] (the explicit dE_L/dC, for tests). */
int vmcf_evaluate(vmcf_system_t sys, const double* pos, int W, double* EL, double* logpsi,
                  double* dlnpsi_dR, double* dEL_dR, double* O, double* dEL_dC, void* stream);

/* Finish the estimators from the accumulated sums (synchronises the stream): E = <E_L>
 * (Eq. eq-eval-observable), F = -<dE_L/dR> - 2 (<E_L d ln Psi/dR> - E <d ln Psi/dR>) (Eqs. hf,
 * pulay, with E the same-sample mean), dEdC = 2 (<E_L O> - E <O>) (Eq. fc-vmc-eval, as dE/dC), and
 * rhs_BQ, the right-hand side of the Z-vector equations projected on the virtual space (Eqs.
 * Q_projector, AZ_eq_B_elements). Host outputs
 * (any may be NULL): E, E_err (scalars), F, F_err [K][3], dEdC, dEdC_err [M*(n_up+n_dn)],
 * rhs_BQ [M*(n_up+n_dn)] = -sum_mu B_{mu i} Q_{mu nu} (needs S at init, else VMCF_EINVAL).
 * Error bars: delete-one-block jackknife over the walker blocks. With at most 4096 blocks the block
 * sums, the estimators and their errors are formed on the device (the arithmetic of
 * vmcf_finish_estimators, every sum over the blocks in block order) and only the results come back;
 * beyond that the block sums are copied back and finished on the host. */
int vmcf_reduce_estimators(vmcf_system_t sys, vmcf_walkers_t wk, double* E, double* E_err, double* F,
                           double* F_err, double* dEdC, double* dEdC_err, double* rhs_BQ, void* stream);
/* Raw block sums (synchronises): host [nblocks][vmcf_accumulator_length()] doubles, layout
 * n, sum E_L, sum E_L^2, sum dE_L/dR [3K], sum dlnPsi/dR [3K], sum (E_L-E_ref) dlnPsi/dR [3K],
 * sum O [nO], sum (E_L-E_ref) O [nO], with nO = M (n_up + n_dn); with VMCF_SPACE_WARP followed by
 * sum dE_L^sw/dR [3K], sum dlnPsi^sw/dR [3K], sum (E_L-E_ref) dlnPsi^sw/dR [3K]. */
int vmcf_block_sums(vmcf_system_t sys, vmcf_walkers_t wk, double* out, void* stream);
int vmcf_accumulator_length(vmcf_system_t sys);

/* Host-only estimator finish (no GPU needed): Eqs. hf/pulay and fc-vmc-eval from block sums
 * `blocks` [nblocks][3 + 9K + 2 M (n_up + n_dn)] in the vmcf_block_sums layout, with e_ref the
 * reference energy the sums were taken with. This is what several ranks call after gathering
 * their block sums (the blocks of all ranks side by side); vmcf_reduce_estimators follows the same
 * arithmetic on the device.
 * Host outputs as in vmcf_reduce_estimators (any may be NULL). */
int vmcf_finish_estimators(const double* blocks, int nblocks, int K, int M, int n_up, int n_dn, double e_ref,
                           double* E, double* E_err, double* F, double* F_err, double* dEdC, double* dEdC_err);

/* Space-warp forces (VMCF_SPACE_WARP):
 * F^sw_a = -<dE_L^sw/dR_a> - 2 <(E_L - E) dlnPsi^sw/dR_a>, with
 *   dE_L^sw/dR_a = dE_L/dR_a + sum_e omega_a(r_e) dE_L/dr_e,
 *   dlnPsi^sw/dR_a = dlnPsi/dR_a + sum_e [omega_a(r_e) dlnPsi/dr_e + 1/2 grad_{r_e} omega_a(r_e)]
 * (the component of the gradient of omega along the force component), jackknife error bars.
 * vmcf_finish_warp: host only, from block sums with row length `stride` = 3 + 18K + 2 M (n_up +
 *   n_dn) (the layout above with the warped sums); F, F_err host [K][3] or NULL.
 * vmcf_reduce_warp: the same from a walker set's own sums (synchronises).
 * vmcf_evaluate_warp: per-walker values at device positions pos [W][Ne][3] (any output may be
 *   NULL; device, caller-owned): dE_L/dr_e [W][Ne][3], dE_L^sw/dR [W][K][3], dlnPsi^sw/dR
 *   [W][K][3]. Works with or without VMCF_SPACE_WARP. W = 0: nothing is read or written. */
int vmcf_finish_warp(const double* blocks, int nblocks, int stride, int K, int M, int n_up, int n_dn, double e_ref,
                     double* F, double* F_err);
int vmcf_reduce_warp(vmcf_system_t sys, vmcf_walkers_t wk, double* F, double* F_err, void* stream);
int vmcf_evaluate_warp(vmcf_system_t sys, const double* pos, int W, double* dEL_dr, double* dEL_sw,
                       double* dlnpsi_sw, void* stream);

/* Host-only covariance of the estimators, as the low-rank factor that the error propagation
 * through the Z-vector equations needs (App. "Error propagation": Var(F^c) = R^T G Cov(B) G^T R,
 * with Cov(B) = b b^T for a factor b with few columns). From block sums in the vmcf_block_sums
 * layout, with theta_k the estimate that leaves block k out (k < nblocks) and theta-bar their
 * mean, the delete-one-block jackknife covariance is
 *   Cov = (nb - 1)/nb sum_k (theta_k - theta-bar)(theta_k - theta-bar)^T = b b^T,
 *   b[i][k] = sqrt((nb - 1)/nb) (theta_k[i] - theta-bar[i]),
 * so diag(b b^T) is the square of the error bars of vmcf_finish_estimators. Outputs (any may be
 * NULL): F_factor host [3K][nblocks] for the forces, B_factor host [nO][nblocks] for dE/dC, with
 * nO = M (n_up + n_dn) in the dEdC order. Blocks of several ranks placed side by side give the
 * factor of the combined estimate. */
int vmcf_finish_covariance(const double* blocks, int nblocks, int K, int M, int n_up, int n_dn, double e_ref,
                           double* F_factor, double* B_factor);

/* Counters of the Markov chain of App. A ("Variational Monte Carlo Methods"): attempted and
 * accepted Metropolis moves, moves rejected on a zero or non-finite ratio, Slater inversions that
 * met a zero pivot, FP64 re-inversions, sweeps (synchronises the stream). Not part of the paper's
 * estimators; they show whether the chain is healthy (acceptance rate, walkers on a node). */
int vmcf_status_counters(vmcf_walkers_t wk, vmcf_counters* out, void* stream);

/* Refresh residual: how far the walker set's current inverses (Sherman-Morrison-updated since the
 * last FP64 re-inversion, the S6/S7 steps of the sampler in App. A) are from a fresh FP64
 * re-inversion of its current positions. Per walker the normwise deviation
 * max_k |B_k - B^fresh_k| / max_k |B^fresh_k| over both spin blocks' entries; outputs (either may be
 * NULL): max_rel the largest over the walkers, mean_rel their mean. The walker state is not changed
 * (the fresh inverses go to a temporary device buffer, allocated and freed inside the call; the
 * counters are not touched). Synchronises the stream. 0 right after a re-inversion (the same kernel
 * forms both), of order the working precision times the moves since then otherwise. W = 0: both 0. */
int vmcf_refresh_residual(vmcf_walkers_t wk, double* max_rel, double* mean_rel, void* stream);

/* Checkpoint and resume of a walker set, between library calls. A checkpoint holds everything
 * the chains and the accumulated sums depend on: positions, the current inverses (as the
 * Sherman-Morrison updates left them, so a chain resumes anywhere, not only after a
 * re-inversion), accepted and rejected move counts, the status counters, the per-CTA walker sums
 * (and the tensor-core sum slots of the mixed path), the chain clock, E_ref, the guiding
 * threshold and the Philox key and walker-id base. The Philox counter of a move is (walker id,
 * sweep, electron, draw), so a walker set that loads a checkpoint draws exactly the numbers the
 * saved one would have drawn: its chains continue bit for bit; its sums continue to within the
 * ordering of the in-CTA accumulation.
 * Layout of the host buffer: one vmcf_walkers_state header, then its segments back to back in
 * the order of `bytes` (raw device contents, in layouts private to the library; 0 bytes: segment
 * absent). The header is public so that callers can read the chain clock and E_ref.
 * vmcf_walkers_state_bytes: the buffer size for this walker set.
 * vmcf_walkers_save: writes the checkpoint into host buf [bytes] (synchronises the stream).
 * vmcf_walkers_load: restores it into a walker set created for the same system with the same W
 *   and nblocks (VMCF_EINVAL if the header or any segment size differs; nothing is changed
 *   then); synchronises the stream. */
typedef struct {
  char magic[8];        /* "vmcfwk1" (NUL-terminated) */
  int32_t W, nblocks;   /* walkers, jackknife blocks */
  int32_t Ne, n_up, n_dn, M, K, precision; /* the system (precision without flags) */
  int32_t counter;      /* attempted moves since the last re-inversion */
  int32_t reserved;
  uint64_t sweep;       /* sweeps done (the Philox counter's sweep word) */
  uint64_t measured;    /* sweeps accumulated into the sums */
  uint64_t key0, key1, wid0;
  double e_ref, eps;
  uint64_t bytes[8];    /* positions, inverses, accepted, rejected, status counters, per-CTA sums,
                           float-float positions, tensor-core sum slots */
} vmcf_walkers_state;
int vmcf_walkers_state_bytes(vmcf_walkers_t wk, uint64_t* bytes);
int vmcf_walkers_save(vmcf_walkers_t wk, void* buf, uint64_t bytes, void* stream);
int vmcf_walkers_load(vmcf_walkers_t wk, const void* buf, uint64_t bytes, void* stream);

/* Fixed-walker evaluation reduced to walker sums, allocating nothing (the paper has no
 * counterpart; this is a deployment variant of vmcf_evaluate plus vmcf_block_sums).
 * It is for callers that must not allocate GPU memory while they run, for example code
 * embedded in a host application that hands the library only buffers it already owns, or
 * a loop that cannot afford the device-wide synchronisation a cudaMalloc or cudaFree can
 * cause. The system must already exist (vmcf_init_system allocates once, at set-up), and its
 * device (the device current at vmcf_init_system) must be the current device (else VMCF_EINVAL).
 *   pos: device [W][Ne][3]; e_ref: reference energy, as in vmcf_reset_accumulators;
 *   sums: device [vmcf_accumulator_length()] doubles, written (not added to) with the sums
 *   over all W walkers in the vmcf_block_sums layout for one block.
 *   W = 0: only the once-per-device set-up below (pos and sums may be NULL, nothing launches).
 * Scratch: a fixed array of 2^21 doubles (16 MiB) in this library's device memory holds the
 * per-CTA partial sums; every GPU that loads the library keeps it until the process exits.
 * A system whose sum vector is longer than 2^21 doubles is rejected with VMCF_EINVAL. Every
 * walker sum is accumulated in FP64 (in mixed precision each walker's terms go straight to its
 * CTA's FP64 partial sum).
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress). With
 * CUDA's lazy module loading that lookup may load the library's device code and commit the
 * 16 MiB array at that moment, so the first call can synchronise or fail for lack of memory:
 * make it at set-up (a call with W = 0 does only this), and before any stream capture.
 * All calls share the array: each call clears the part it uses, and calls whose kernels
 * overlap on the GPU race with each other (serialise them, e.g. on one stream). The call
 * calls no cudaMalloc, cudaFree or other allocating routine. */
int vmcf_evaluate_sums_noalloc(vmcf_system_t sys, const double* pos, int W, double e_ref, double* sums,
                               void* stream);

/* Launch-shape and kernel-choice knobs of a system (not part of the paper's method). The launch
 * shapes leave every result unchanged; the two tensor-core switches change mixed-precision results
 * by rounding only:
 *   "move_lanes_per_walker": 1, 2, 4 or 8 lanes share one walker in the Metropolis kernel of
 *                            the small-system path (default 2);
 *   "measure_warps":         2, 4 or 8 walkers (one warp each) per CTA of the small-system
 *                            measurement kernel (default: the most that fit shared memory, up to 8);
 *   "measure_group_size":    32, 128 or 256 threads per walker in the walker-group measurement
 *                            kernel (default from the orbital count);
 *   "group_proposal_pass":   1: walker-group sweeps take their proposals from a pass over every
 *                            (walker, electron) ahead of the sweep (default); 0: drawn inside the
 *                            sweep kernel, with the same arithmetic as the SIMT pass;
 *   "tensor_core_sums":      1: in mixed precision, the walker sums of O and (E_L - E_ref) O are
 *                            one bf16 GEMM on the tensor cores (tcgen05, FP32 accumulation in
 *                            tensor memory, FP64 across CTAs); 0: FP32 SIMT sums (default 1);
 *   "tensor_core_rows":      1: in mixed precision on the walker-group kernels, the orbital rows
 *                            of that proposal pass are a split-bf16 GEMM on the tensor cores
 *                            (default where the tile fits shared memory); 0: FP32 SIMT rows;
 *                            VMCF_EINVAL where the system has no tensor-core form of them.
 * Takes effect for walker sets created afterwards (measure_warps) or at the next call. */
int vmcf_set_tuning(vmcf_system_t sys, const char* key, int value);


/* ---- Ragged batches of geometries.
 * Many independent geometries (different nuclei, electron and AO counts, walker counts) are
 * sampled together: each VMC sweep of the whole batch is one replay of a captured CUDA graph
 * with two phases, the Metropolis sweep of every walker and (when measuring) the evaluation
 * of every walker (E_L, forces, O, walker sums). Each phase is one persistent kernel per
 * launch shape, run side by side; geometries that fit the small-system kernels (at most 32
 * electrons and 16 orbitals per spin, created without VMCF_FORCE_GROUP_PATH) run in branches of
 * their own beside them (proposals, runs of moves with the re-inversions, the evaluation), their
 * launches reading the sweep's schedule from the geometry's chain clock on the device; a
 * one-thread-block kernel then advances the chain clocks.
 * Walker groups in the persistent kernels pull work items (one geometry, one range of its
 * walkers) from a device queue, longest first, so that small and large geometries share the
 * SMs. The method per walker is exactly that of vmcf_sample (App. A, the MCMC sampling and
 * the estimators of Eqs. hf, pulay and fc-vmc-eval); batching changes neither a walker's chain
 * nor its contributions, only where and when they are computed. The paper batches nothing
 * across geometries: this is the deployment form for many molecules (or many displaced
 * geometries) at once.
 *
 * vmcf_batch_create: systems[g], walkers[g] for g < G: each walker set belongs to its system;
 *   every system has the same precision (else VMCF_EINVAL). The batch keeps the handles (the caller keeps ownership and must keep them
 *   alive until vmcf_batch_destroy) and allocates its own device tables. Geometries on the
 *   walker-group kernels are put in buckets by (ceil(Ne / 16), ceil(M / 64)); every bucket starts, per phase, with the default
 *   launch shape (32 threads per walker while n_up, n_dn <= 24, with as many walker groups per
 *   CTA, up to 4, as fit shared memory; else 128 threads per walker for the sweep and 256 for
 *   the evaluation). Synchronises `stream`.
 * vmcf_batch_autotune: for every bucket and phase, time one sweep (phase 0) or one evaluation
 *   (phase 1) of the bucket's walkers with each feasible launch shape (threads per walker x
 *   walker groups per CTA: 32 x 1, 2, 4, 8; 128 x 1, 2; 256 x 1) and keep the fastest; also
 *   records each geometry's measured cost for the longest-first order. The timed sweeps are
 *   real sweeps of the chains (as vmcf_sample with measure = 0) and the timed evaluations
 *   rebuild the inverses and discard their sums: call it during equilibration. Synchronises
 *   `stream`.
 * vmcf_batch_set_shape: force the launch shape of `phase` (0 sweep, 1 evaluation) for the
 *   bucket that holds geometry g; VMCF_EINVAL if unsupported, too large for shared memory, or g
 *   runs on the small-system kernels.
 * vmcf_batch_sample: n_sweeps sweeps of every geometry, as vmcf_sample on each walker set
 *   (same arguments and meaning; measure != 0 adds each sweep's evaluation to each walker
 *   set's sums, read with vmcf_reduce_estimators / vmcf_block_sums on that walker set).
 *   The first call with a given (measure, refresh_k, step_sigma) captures the graph; later
 *   calls replay it. Asynchronous on `stream`.
 * vmcf_batch_info: number of buckets and of persistent kernels per measured sweep; for
 *   geometry g (if 0 <= g < G) its bucket and shapes[4] = {sweep GS, sweep groups per CTA,
 *   evaluation GS, evaluation groups per CTA}; a geometry on the small-system kernels has bucket
 *   -1 and shapes {lanes per walker of its moves, 0, 32 (one warp per walker), walkers per
 *   evaluation CTA}; any output may be NULL.
 * A small-system geometry's launches are captured with its walker set's E_ref and guiding
 * threshold; vmcf_batch_sample captures the graph again when either has changed. */
typedef struct vmcf_batch_s* vmcf_batch_t; /* opaque, library-owned */
int vmcf_batch_create(const vmcf_system_t* systems, const vmcf_walkers_t* walkers, int G, void* stream,
                      vmcf_batch_t* out);
int vmcf_batch_destroy(vmcf_batch_t batch);
int vmcf_batch_autotune(vmcf_batch_t batch, double step_sigma, int refresh_k, void* stream);
int vmcf_batch_set_shape(vmcf_batch_t batch, int g, int phase, int GS, int groups);
int vmcf_batch_sample(vmcf_batch_t batch, int n_sweeps, double step_sigma, int refresh_k, int measure,
                      void* stream);
int vmcf_batch_info(vmcf_batch_t batch, int* n_buckets, int* n_launches, int g, int* bucket, int* shapes);

const char* vmcf_strerror(int status);
const char* vmcf_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* VMCF_H */
