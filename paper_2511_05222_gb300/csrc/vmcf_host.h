// Host-side state of the C ABI handles, shared by the translation units that implement
// entry points (vmcf_api.cu, noalloc.cu).
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <utility>
#include <vector>

#include "vmcf_internal.h"

struct vmcf_system_s {
  int precision = 0;
  int device = -1;
  int geometry_version = 0;  // incremented by vmcf_system_set_geometry      // the CUDA device the system's tables live on (current at vmcf_init_system)
  int K = 0, M = 0, nup = 0, ndn = 0, Ne = 0, nshell = 0, nB = 0, nmax = 0;
  int MJ = 0, nJs = 0;  // functions and shells of the Jastrow basis (AO-expanded Jastrow terms)
  std::vector<double> R, Z, S, C[2];
  std::vector<int> ao_center;
  bool has_S = false;
  bool swct = false;  // accumulate the space-warp force sums (VMCF_SPACE_WARP)
  vmcf::DevSys dev{};
  void* dmem = nullptr;
  // launch planning
  int GS = 32;   // threads per walker group: sweep and refresh kernels
  int GSm = 32;  // threads per walker group: measurement kernel
  vmcf::GroupLayout Lrm{}, Lmeas{}, LmeasD{};
  int gpb_rm = 1, gpb_meas = 1, gpb_measD = 1;
  int accL = 0;
  bool acc_smem = false;
  int acc_off = -1;
  double* scratch_counters = nullptr;  // device [2] for evaluate
  // small-system path (at most 32 electrons and 16 orbitals per spin)
  bool small = false;
  int small_nm = 16;          // register row width: 8, 14 or 16 (staged coefficient rows padded to 4)
  int small_warps = 8;        // warps per CTA of the measurement kernel
  int small_res = 1;          // resident measurement CTAs on the device
  int small_sms = 1;          // SMs on the device
  vmcf::SmallLayout SL{};
  size_t small_move_smem = 0;  // shared memory of the proposal kernel (C staging, Jastrow-basis rows)
  int propose_warps = 8;       // warps per CTA of the proposal kernel
  int move_lpw = 2;            // lanes per walker in the move kernel (1, 2, 4 or 8)
  bool group_prepass = true;   // walker-group sweeps take their proposals from propose_group
  bool tc_sums = false;        // mixed small path: walker sums of O on the tensor cores
  int tc_Mp = 0, tc_Np = 0;    // padded AO rows and Y columns of those tiles
  int tc_nch = 1;              // chunks of 16 electron slots per walker
  // walker-group path, mixed precision: the same sums on the tensor cores (tiles and chunks)
  bool tcg_sums = false;
  int tcg_Mf = 0, tcg_Nf = 0, tcg_nch = 1;
  vmcf::GroupLayout LmeasTC{};  // measurement layout that stages AO values instead of holding O
  // walker-group path, mixed precision: orbital rows of the proposal pass on the tensor cores (k_tc_rows.cu)
  bool tc_rows = false;
  int tcr_Kp = 0, tcr_Np = 0;   // AO columns and orbital rows of the operands, padded to 16
  size_t tcr_smem = 0;
  int tcr_grid = 1;             // CTAs per spin
  void* tcr_mem = nullptr;      // [spin][part][Np][Kp] bf16 split coefficients (part 0 hi, 1 lo), then the flag
  int* tcr_flag = nullptr;      // set by a timed-out wait of the kernel
  alignas(64) unsigned char tcr_map[128] = {};  // tensor map (CUtensorMap) over the split coefficients
};

struct vmcf_walkers_s {
  vmcf_system_s* sys = nullptr;
  int W = 0, nblocks = 0, cpb = 1, grid_meas = 1;
  uint64_t k0 = 0, k1 = 0, wid0 = 0;
  double* pos = nullptr;
  void* B = nullptr;
  uint32_t* nacc = nullptr;
  uint32_t* nrej = nullptr;
  unsigned long long* counters = nullptr;  // [0] singular, [1] refreshes
  double* acc = nullptr;                   // [grid_meas][accL]
  double* blocks = nullptr;                // [nblocks][accL]
  double* h_blocks = nullptr;              // pinned host copy of the block sums [nblocks][accL] (reductions)
  // estimators finished on the device: [E, E_err, F [3K], F_err [3K], B [nO], B_err [nO]] then int flags
  // (device: the finish status; pinned host copy: status, tensor-core sum flag, tensor-core row flag)
  double* d_fin = nullptr;
  double* h_fin = nullptr;
  uint64_t sweep = 0, measured = 0;
  int counter = 0;
  double e_ref = 0.0;
  double eps = 0.0;  // guided sampling: Psi_G = Psi max(1, eps sqrt(S)); 0: plain |Psi|^2
  // small-system path state: positions and inverses walker-interleaved
  float2* posf = nullptr;   // float-float positions (mixed mode)
  void* phiT[2] = {nullptr, nullptr};  // tensor-core walker sums: [W][Mp][16] bf16 per spin
  void* yT[2] = {nullptr, nullptr};    // [W][Np][16] bf16 per spin
  double* tc_slots = nullptr;          // [2][nblocks * tc_cpb][Mp][Np]
  int* tc_flag = nullptr;
  int tc_cpb = 1;
  size_t tc_slot_doubles = 0;
  bool tc = false;
  double* stage = nullptr;  // [W][Ne][3] staging for layout conversion
  void* prop = nullptr;     // small-system path: one sweep's proposals (see pr)
  vmcf::SmallProposals pr{};
  // walker-group path: one sweep's proposals from propose_group ([W][Ne][3] r', [W][Ne][nmax] rows, [W][Ne] u, dchi)
  void* gprop = nullptr;
  double* g_rn = nullptr;
  void* g_row = nullptr;
  double* g_u = nullptr;
  void* g_dchi = nullptr;
  // per-kernel timing (kind 0 move, 1 measure, 2 refresh, 3 tensor-core sums, 4 proposals): event pairs
  bool profiling = false;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> events;
  double kernel_ms[5] = {0, 0, 0, 0, 0};  // move, measure, refresh, tensor-core walker sums, proposal pass
  long long kernel_n[5] = {0, 0, 0, 0, 0};
};


namespace vmcf {
// Launch planning shared by the entry points (defined in vmcf_api.cu).
Launch launch_meas(const vmcf_system_s& s, int grid, bool accum, bool withD);
// Offset of the space-warp sums in an accumulator slot (after the base fields), 0 if off.
inline int swct_offset(const vmcf_system_s& s) { return s.swct ? 3 + 9 * s.K + 2 * s.M * (s.nup + s.ndn) : 0; }
// Doubles of the estimators finished on the device: E, E_err, F and F_err (3K each), B and B_err (nO each).
inline size_t fin_doubles(const vmcf_system_s& s) { return 2 + 6 * (size_t)s.K + 2 * (size_t)s.M * (s.nup + s.ndn); }
// Walker-group shared-memory plans of the sweep and measurement kernels for group size GS.
GroupLayout group_layout_rm(const vmcf_system_s& s, int GS);
GroupLayout group_layout_meas(const vmcf_system_s& s, int GS);
// the measurement plan that stages AO values for the tensor-core sums (mixed, walker-group path)
GroupLayout group_layout_meas_tc(const vmcf_system_s& s, int GS);
constexpr int kSmemCapBytes = 227 * 1024;
int set_last_error(int code, const std::string& msg);
// Rebuild a walker set's inverses from its positions and reset its re-inversion count (vmcf_api.cu).
int refresh_walker_set(vmcf_system_s* s, vmcf_walkers_s* wk, cudaStream_t st);
// The launches of one sweep of a small-system walker set (proposals, runs of moves with the
// re-inversions between them, and for mode 1 the measurement and its tensor-core sums) onto st, with
// the sweep's schedule read from the geometry's device clock clk, for capture into a batch graph.
cudaError_t small_sweep_launches(vmcf_system_s* s, vmcf_walkers_s* wk, const BatchClock* clk, int mode, int kref,
                                 double sigma, cudaStream_t st);
// Tensor-core orbital rows of the walker-group proposal pass (k_tc_rows.cu): plan, buffer and tensor map at system
// set-up; the split coefficients again after a geometry change; the proposal-pass launch of either precision.
int tc_rows_setup(vmcf_system_s* s);
int tc_rows_upload(vmcf_system_s* s);
cudaError_t launch_propose_rows(const vmcf_system_s& s, const GroupProposeParams& P, cudaStream_t st);
}  // namespace vmcf
