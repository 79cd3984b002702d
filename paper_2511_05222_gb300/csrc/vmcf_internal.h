// Internal interfaces between the host API (vmcf_api.cu) and the kernel translation units.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "vmcf_device.cuh"

namespace vmcf {

struct BatchClock;  // per-geometry chain clock of a ragged batch (below)

// Byte offsets of one walker group's shared-memory region; computed on the host.
struct GroupLayout {
  int pos, ph, pl, Bd, Bt, P, Q, Jg, Jl, gd, ao, frc, fa, ew, Ow, D, piv, f, red, scal, row, wv, col;
  int ao_rows;   // AO rows of M values the ao buffer holds (electrons per Slater-build chunk)
  int p2_chunk;  // the P-row pass takes 4 p2_chunk electrons per chunk (one AO row each)
  int p3_chunk;  // electrons per step of the adjoint/force pass (14 AO rows each): 1 or 2
  int jw;        // AO-expanded Jastrow work space (systems with a Jastrow basis, else 0)
  int jch;       // electrons per chunk of the Jastrow-basis products (measurement)
  int jng;       // subgroups of whole warps that take different electrons in the Jastrow-basis loops
  int bytes;    // size of one group's region (16-byte multiple)
};

struct Launch {
  int GS;          // threads per walker group: 32 or 128
  int groups;      // groups per CTA
  int grid;        // CTAs
  size_t smem;     // dynamic shared memory per CTA
  GroupLayout L;
  int acc_off;     // CTA accumulator region offset (measure kernel), -1 if none
};

struct MoveParams {
  double* pos;      // [W][Ne][3]
  void* B;          // T [W][nB]
  uint32_t* nacc;   // [W]
  uint32_t* nrej;   // [W]
  unsigned long long* counters;  // [0] singular inversions, [1] refreshes
  int W;
  uint64_t wid0, k0, k1, sweep0;
  int nsweeps, kref, c0, skip_final_refresh;
  double sigma;
  double eps;       // guiding function max(1, eps sqrt(S)) of reweighted sampling; 0: plain |Psi|^2
  // the proposals of this launch's sweep (nsweeps = 1) from propose_group, or NULL: computed in the kernel,
  // with the same arithmetic. Electron e of walker w at index w Ne + e.
  const double* prn;  // [W][Ne][3] r'_e
  const void* prow;   // T [W][Ne][nmax]: orbital row of the electron's spin at r'_e
  const double* pu;   // [W][Ne] acceptance uniform
  const void* pdchi;  // T [W][Ne] change of the electron-nucleus Jastrow terms
};

// The proposals of one sweep for every (walker, electron), computed ahead of the walker-group moves.
struct GroupProposeParams {
  const double* pos;  // [W][Ne][3] positions at the start of the sweep
  double* prn;
  void* prow;
  double* pu;
  void* pdchi;
  int W;
  uint64_t wid0, k0, k1, sweep;
  double sigma;
  const BatchClock* clk;  // in a batch graph: the sweep index comes from the geometry's device clock
};

struct MeasParams {
  const double* pos;  // [W][Ne][3]
  void* Bout;         // T [W][nB] or NULL
  double *EL, *logpsi, *dlnpsi, *dEL, *O, *dELdC;  // outputs or NULL
  double *dEL_dr, *dEL_sw, *dlnpsi_sw;               // space-warp outputs ([W][Ne][3], [W][K][3]) or NULL
  void* phiT[2];      // mixed accumulate: tensor-core tiles of the O sums ([W][nch][Mf][16] bf16 per spin), or NULL
  void* yT[2];        // [W][nch][Nf][16] bf16 per spin
  int nch, Mf, Nf;
  double* acc;        // [grid][accL] FP64 slots, or NULL
  int accL, acc_in_smem;
  int swct_off;       // offset (> 0) of the space-warp sums in a slot, 0 if none
  double eps;         // guided chain: weight the sums by |Psi / Psi_G|^2; 0: unweighted
  double e_ref;
  unsigned long long* counters;
  int W;
};


// Launchers (one instantiation per precision and group size, see k_fp64.cu / k_fp32.cu).
template <typename T>
cudaError_t launch_refresh(const DevSys& S, const Launch& lc, const double* pos, void* B, int W,
                           unsigned long long* counters, cudaStream_t st);
template <typename T>
cudaError_t launch_move(const DevSys& S, const Launch& lc, const MoveParams& P, cudaStream_t st);
template <typename T>
cudaError_t launch_measure(const DevSys& S, const Launch& lc, const MeasParams& P, cudaStream_t st);
template <typename T>
cudaError_t set_smem_limits(int GS);
template <typename T>
cudaError_t launch_propose_group(const DevSys& S, const GroupProposeParams& P, cudaStream_t st);

// ---- small-system path (kernels_small.cuh)

// The proposals of one sweep for every walker and electron (filled by propose_small before the
// sweep's moves): electron e of walker w at index w * Ne + e.
struct SmallProposals {
  void* rows;    // T [W][Ne][nms]: orbital row phi(r'_e) of the electron's spin (zero beyond n_s)
  double* rnew;  // [W][Ne][3]: proposed position r'_e (FP64 mode); mixed mode: the same bytes hold
                 // float2 [W][Ne][3], r'_e as float-float pairs (high, low)
  double* u;     // [W][Ne]: acceptance uniform
  void* dchi;    // T [W][Ne]: change of the electron-nucleus Jastrow terms, chi(r'_e) - chi(r_e), plus (with
                 // AO-expanded Jastrow terms) the part of their change that does not depend on earlier moves
  // AO-expanded Jastrow pair terms of a sweep: the move of e changes U by dphi_e . (t0 - Xi psi_e) plus, for every
  // accepted j < e, dphi_e . Xi dphi_j (dphi: psi^J(r') - psi^J(r) of the electron's own proposal; t0, psi: at the
  // start of the sweep)
  void* dpair;       // T [W][npair]: dphi_e . Xi dphi_j at pair index e (e - 1) / 2 + j, j < e (NULL without the terms)
  uint32_t* amask;   // [W]: bit j set when electron j's move of the current sweep was accepted
  int npair;         // Ne (Ne - 1) / 2 with the terms, else 0
  int nms;       // row stride (c_stride of the register-row width)
};

// Shared memory of the proposal kernel: the staged coefficient rows C^up, C^dn ([2][M][nms] of the
// working type).
__host__ __device__ inline size_t propose_c_bytes(int M, int nms, size_t tsz) {
  return (tsz * 2 * (size_t)M * nms + 15) / 16 * 16;
}
// With AO-expanded Jastrow terms: per CTA, Xi's rows padded to MJp ([MJ][MJp]); per warp, the rows dphi_e of every
// electron ([Ne][JS]) and the vectors s and t0 ([2][MJp]). Nothing without them.
__host__ __device__ inline size_t propose_xi_bytes(int MJ, size_t tsz) {
  return MJ > 0 ? (tsz * (size_t)MJ * ((MJ + 3) / 4 * 4) + 15) / 16 * 16 : 0;
}
__host__ __device__ inline size_t propose_jb_bytes(int Ne, int MJ, int JS, size_t tsz) {
  return MJ > 0 ? (tsz * ((size_t)Ne * JS + 2 * (size_t)((MJ + 3) / 4 * 4)) + 15) / 16 * 16 : 0;
}
constexpr int kProposeWarps = 8;  // most warps per CTA of the proposal kernel

struct SmallProposeParams {
  const double* pos;   // [3 Ne][W], positions at the start of the sweep (FP64 mode)
  const float2* posf;  // [3 Ne][W], the same as float-float pairs (mixed mode)
  SmallProposals pr;
  int W;
  uint64_t wid0, k0, k1, sweep;
  double sigma;
  float sigma_f;
  const BatchClock* clk;  // in a batch graph: the sweep index comes from the geometry's device clock
  int jJS;                // row stride of the Jastrow-basis rows (SmallLayout::JS)
};

struct SmallMoveParams {
  double* pos;   // [3 Ne][W]
  float2* posf;  // [3 Ne][W] float-float (mixed mode) or NULL
  void* B;       // T [nB][W]
  SmallProposals pr;  // this sweep's proposals
  uint32_t* nacc;
  uint32_t* nrej;
  int W;
  uint64_t wid0, k0, k1;
  uint64_t move0;  // global index of the first move: sweep = move0 / Ne, electron = move0 % Ne
  int nmoves;
  // in a batch graph: move0 and nmoves come from segment seg of the sweep's schedule, replayed from
  // the geometry's device clock with re-inversions every kref moves (measure: the sweep is measured)
  const BatchClock* clk;
  int seg, kref, measure;
  int wpc;         // walkers per CTA
  double sigma;
  double eps;      // guiding function max(1, eps sqrt(S)); 0: plain |Psi|^2
};

struct SmallLayout {
  int pd, ph, pl, Ad, Bf, Pm, Q, piv, f, frc, phi, red, scal;
  int jA, jv, JS;  // AO-expanded Jastrow terms: [Ne][JS] rows (may share Ad..phi), vectors [3][MJp]; JS row stride
  int bytes;  // per warp
  int cta_C, cta_acc, cta_bytes;
  int cta_bytes_tc;  // the CTA region with the tensor-core walker sums (no O range in the accumulator)
  int chunk;  // AOs per O chunk (Phi buffer width)
};

struct SmallMeasParams {
  const double* pos;  // positions, element (w, k) at pos[k * pos_sk + w * pos_sw], k = 3 e + xyz
  long long pos_sk, pos_sw;
  int mode;             // 0 refresh only, 1 evaluate, 2 accumulate
  void* Bout;           // T [nB][W] (refresh and accumulate modes) or NULL
  float2* posf_out;     // float-float positions [3 Ne][W] to refresh (mixed, refresh mode) or NULL
  double *EL, *logpsi, *dlnpsi, *dEL, *O;  // evaluate-mode outputs (any may be NULL)
  double* acc;          // [grid][accL] FP64 slots (accumulate mode)
  void* phiT[2];        // tensor-core walker sums (mixed accumulate mode): [W][Mp][16] bf16 per spin, or NULL
  void* yT[2];          // [W][Np][16] bf16 per spin
  int Mp, Np;
  int accL;
  double e_ref;
  unsigned long long* counters;
  int W;
  int swct_off;  // offset (> 0) of the space-warp sums in a slot (accumulate mode), 0 if none
  double eps;    // guided chain: weight the sums by |Psi / Psi_G|^2; 0: unweighted
  // refresh mode in a batch graph: the re-inversion after segment seg of the sweep's schedule (replayed
  // from the geometry's device clock, as for the moves); the launch does nothing when there is none
  const BatchClock* clk;
  int seg, kref, measure;
};

template <typename T>
cudaError_t launch_move_small(const DevSys& S, int nm, int lpw, int W, size_t smem, const SmallMoveParams& P,
                              cudaStream_t st);
template <typename T>
cudaError_t launch_propose_small(const DevSys& S, int nm, int grid, int warps, size_t smem, const SmallProposeParams& P,
                                 cudaStream_t st);
// the instances for systems with AO-expanded Jastrow terms (k_small_fp32_jb.cu, k_small_fp64_jb.cu)
template <typename T>
cudaError_t launch_propose_small_jb(const DevSys& S, int nm, int grid, int warps, size_t smem,
                                    const SmallProposeParams& P, cudaStream_t st);
template <typename T>
cudaError_t launch_measure_small_jb(const DevSys& S, int nm, const SmallLayout& L, int grid, int warps,
                                    const SmallMeasParams& P, cudaStream_t st);
template <typename T>
cudaError_t set_smem_limits_small_jb();
template <typename T>
cudaError_t launch_measure_small(const DevSys& S, int nm, const SmallLayout& L, int grid, int warps,
                                 const SmallMeasParams& P, cudaStream_t st);
template <typename T>
cudaError_t set_smem_limits_small();
cudaError_t launch_to_interleaved(const double* src, double* dst, float2* dstf, int W, int n3, cudaStream_t st);
cudaError_t launch_from_interleaved(const double* src, double* dst, int W, int n3, cudaStream_t st);

// Tensor-core walker sums of O: PhiT[s] [W][nch] chunks of Mf x 16 and YT[s] [W][nch] chunks of Nf x 16
// bf16 per spin, element (row r, electron slot k) of a chunk at tc_tile_index(r, k);
// slots [2][tiles][grid_x][128][32] FP64 with tiles = ceil(Mf / 128) ceil(Nf / 32).
cudaError_t launch_tc_sumprod(const void* phiT_up, const void* phiT_dn, const void* yT_up, const void* yT_dn, int W,
                              int nch, int Mf, int Nf, int n_up, int n_dn, int grid_x, double* slots, int* flag,
                              cudaStream_t st);
cudaError_t set_smem_limits_tc();
cudaError_t tc_sumprod_ctas_per_sm(int Mf, int Nf, int* n);
cudaError_t launch_tc_fold(const double* slots, int nblocks, int cpb, int Mf, int Nf, int M, int n_up, int n_dn,
                           int oo, int nO, int accL, double* blocks, cudaStream_t st);

// ---- ragged batch of geometries (k_batch.cu): one persistent kernel per launch shape
// Everything a walker group needs to work on one geometry; copied into the group's shared
// memory when it switches geometry.
struct BatchGeom {
  DevSys S;
  GroupLayout Lrm, Lmeas;
  MoveParams P;   // walker state; sweep0, c0, nsweeps, kref, skip_final_refresh and sigma set per launch
  MeasParams Mp;  // accumulator slots [grid_meas][accL]; acc_in_smem = 0
  int grid_meas;  // slot c holds walkers [W c / grid_meas, W (c + 1) / grid_meas)
  int pad_;
};

// Per-geometry chain clock: global sweep index and moves since the last refresh.
struct BatchClock {
  unsigned long long sweep;
  int c;
  int Ne;
};

struct BatchArgs {
  const BatchGeom* geo;
  const BatchClock* clk;
  const int2* items;  // (geometry, slot) in processing order
  int n_items;
  int* queue;         // next item index (reset to 0 after each sweep)
  int mode;           // 0 moves only, 1 moves + measurement into the slots, 2 moves + measurement without sums
  int kref;
  double sigma;
  int region;         // bytes of shared memory per walker group (header + working set)
  int hdr;            // header bytes (geometry copy and the group's scalars) at the start of a region
};

// phase 0: Metropolis sweep of each walker; phase 1: evaluation (and walker sums when mode 1)
template <typename T>
cudaError_t launch_batch(int phase, int GS, int groups, int grid, size_t smem, const BatchArgs& A, bool jb,
                         cudaStream_t st);
template <typename T>
cudaError_t batch_occupancy(int phase, int GS, int groups, size_t smem, bool jb, int* ctas_per_sm);
cudaError_t launch_batch_advance(BatchClock* clk, int G, int mode, int kref, int* queues, int nq, cudaStream_t st);

cudaError_t run_probes(double* fp64_tflops, double* fp32_tflops, double* exp_gops, cudaStream_t st);

// Estimators and jackknife errors of a walker set's block sums on the device (k_reduce.cu); blocks up to
// kFinishMaxBlocks (shared memory of the per-block scalars).
constexpr int kFinishMaxBlocks = 4096;
cudaError_t launch_finish(const double* blk, int nb, int L, int K3, int nO, double er, double* out, int* status,
                          cudaStream_t st);
cudaError_t launch_block_reduce(const double* acc, int grid, int cpb, int accL, double* out, int nblocks,
                                cudaStream_t st);

}  // namespace vmcf
