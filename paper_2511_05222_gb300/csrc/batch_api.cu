// Host side of the ragged-batch entry points (vmcf_batch_*): buckets, launch shapes per
// phase (Metropolis sweep, evaluation), the autotuner, the longest-first work order and the
// captured sweep graph.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/vmcf.h"
#include "vmcf_host.h"

using namespace vmcf;

namespace {

int fail(int code, const std::string& msg) { return vmcf::set_last_error(code, msg); }

int cuda_fail(cudaError_t e, const std::string& where) {
  return vmcf::set_last_error(VMCF_ECUDA, where + ": " + cudaGetErrorString(e));
}

#define BATCH_CUDA(call)                                 \
  do {                                                   \
    cudaError_t _e = (call);                             \
    if (_e != cudaSuccess) return cuda_fail(_e, #call);  \
  } while (0)

int align16(int x) { return (x + 15) & ~15; }

// Header of a walker group's shared-memory region: the geometry copy and two ints.
constexpr int kHdr = (int)((sizeof(BatchGeom) + 16 + 15) / 16 * 16);

struct Shape {
  int GS = 32, groups = 1;
  bool operator<(const Shape& o) const { return std::tie(GS, groups) < std::tie(o.GS, o.groups); }
};

struct LaunchPlan {
  int phase = 0;  // 0 Metropolis sweep, 1 evaluation
  Shape shape;
  int grid = 1;
  size_t smem = 0;
  int region = 0;
  int item0 = 0, n_items = 0;
};

}  // namespace

struct vmcf_batch_s {
  int G = 0, precision = 0, sms = 1;
  bool jb = false;  // some geometry has AO-expanded Jastrow terms: the kernels that hold their code
  std::vector<vmcf_system_s*> sys;
  std::vector<vmcf_walkers_s*> wk;
  std::vector<int> bucket;              // per geometry
  std::vector<Shape> bucket_shape[2];   // per phase, per bucket
  std::vector<double> cost[2];          // per phase, per geometry: relative cost of one walker
  std::vector<LaunchPlan> launches;     // phase-0 launches first
  int n_launch[2] = {0, 0};
  std::vector<BatchGeom> h_geo;
  std::vector<BatchClock> h_clk;
  BatchGeom* d_geo = nullptr;
  BatchClock* d_clk = nullptr;
  int2* d_items = nullptr;
  size_t items_cap = 0;
  int* d_queue = nullptr;  // one counter per launch
  int queue_cap = 0;
  // captured sweep graph and the (mode, kref, sigma) it was captured for
  cudaGraphExec_t exec = nullptr;
  int g_mode = -1, g_kref = -1;
  double g_sigma = 0.0;
  cudaStream_t cap = nullptr;
  std::vector<cudaStream_t> forks;
  std::vector<cudaEvent_t> joins;
  cudaEvent_t fork_ev = nullptr;
  // geometries on the small-system kernels: their own branch of the graph each, with the E_ref and
  // guiding threshold their launches were captured with
  std::vector<int> small_g;
  std::vector<cudaStream_t> sforks;
  std::vector<cudaEvent_t> sjoins;
  std::vector<double> s_eref, s_eps;
  std::vector<int> geo_version;  // each system's geometry version when its descriptors were last filled
};

namespace {

// Geometry g forms its O sums on the tensor cores (its walker set holds the bf16 tiles).
bool uses_tc(const vmcf_batch_s& b, int g) { return b.wk[g]->tc && b.sys[g]->tcg_sums; }

GroupLayout meas_layout(const vmcf_batch_s& b, int g, int GS) {
  return uses_tc(b, g) ? group_layout_meas_tc(*b.sys[g], GS) : group_layout_meas(*b.sys[g], GS);
}

// Bytes of one walker group's region for geometry g in `phase` at group size GS.
int region_bytes(const vmcf_batch_s& b, int phase, int g, int GS) {
  const GroupLayout L = phase == 0 ? group_layout_rm(*b.sys[g], GS) : meas_layout(b, g, GS);
  return kHdr + align16(L.bytes);
}

int bucket_region(const vmcf_batch_s& b, int phase, int bk, int GS) {
  int r = 0;
  for (int g = 0; g < b.G; ++g)
    if (b.bucket[g] == bk) r = std::max(r, region_bytes(b, phase, g, GS));
  return r;
}

int occupancy(const vmcf_batch_s& b, int phase, const Shape& sh, size_t smem, int* ctas) {
  cudaError_t e = b.precision == VMCF_FP64 ? batch_occupancy<double>(phase, sh.GS, sh.groups, smem, b.jb, ctas)
                                           : batch_occupancy<float>(phase, sh.GS, sh.groups, smem, b.jb, ctas);
  if (e != cudaSuccess) return cuda_fail(e, "occupancy query of the batch kernel");
  return VMCF_OK;
}

// Shapes the batch kernels support: 32 threads x 1, 2, 4 or 8 groups, 128 x 1 or 2, 256 x 1.
bool shape_supported(const Shape& sh) {
  return (sh.GS == 32 && (sh.groups == 1 || sh.groups == 2 || sh.groups == 4 || sh.groups == 8)) ||
         (sh.GS == 128 && (sh.groups == 1 || sh.groups == 2)) || (sh.GS == 256 && sh.groups == 1);
}

bool shape_fits(const vmcf_batch_s& b, int phase, int bk, const Shape& sh) {
  if (!shape_supported(sh)) return false;
  return (size_t)sh.groups * bucket_region(b, phase, bk, sh.GS) <= (size_t)kSmemCapBytes;
}

const Shape kCandidates[] = {{32, 1}, {32, 2}, {32, 4}, {32, 8}, {128, 1}, {128, 2}, {256, 1}};

// Default shape: the single-geometry plan's group size (32 threads while n_up, n_dn <= 24;
// else 128 for sweeps and 256 for evaluations), as many groups per CTA as fit (up to 4).
Shape default_shape(const vmcf_batch_s& b, int phase, int bk) {
  int nmax = 0;
  for (int g = 0; g < b.G; ++g)
    if (b.bucket[g] == bk) nmax = std::max(nmax, b.sys[g]->nmax);
  Shape sh{nmax <= 24 ? 32 : (phase == 0 ? 128 : 256), 1};
  if (sh.GS == 32)
    for (int gr : {4, 2}) {
      const Shape t{32, gr};
      if (shape_fits(b, phase, bk, t)) {
        sh = t;
        break;
      }
    }
  if (!shape_fits(b, phase, bk, sh)) sh = Shape{128, 1};
  return sh;
}

// Relative cost of one walker-sweep (phase 0) or evaluation (phase 1), from the operation
// counts of the method: AO/MO rows per move and per evaluation, inversions, Jastrow pairs, and
// the products with Xi of the AO-expanded Jastrow terms (one per move; three row blocks per
// electron in an evaluation).
double heuristic_cost(const vmcf_system_s& s, int phase) {
  const double Ne = s.Ne, M = s.M, n = s.nmax, K = s.K, MJ = s.MJ;
  if (phase == 0)
    return Ne * (2.0 * M * n + 4.0 * n * n + 30.0 * (Ne + K) + 2.0 * MJ * MJ + 6.0 * MJ) +
           (Ne / 26.0) * (Ne * M * n + 4.0 * n * n * n + Ne * MJ + 2.0 * MJ * MJ);
  return Ne * (12.0 * M * n + 40.0 * M + 6.0 * MJ * MJ + 60.0 * MJ) + 4.0 * n * n * n + 60.0 * Ne * (Ne + K);
}

void fill_geo(vmcf_batch_s& b, int g) {
  const vmcf_system_s& s = *b.sys[g];
  const vmcf_walkers_s& w = *b.wk[g];
  BatchGeom G{};
  G.S = s.dev;
  // (a geometry on the small-system kernels keeps a table the persistent kernels never read)
  G.Lrm = group_layout_rm(s, b.bucket[g] >= 0 ? b.bucket_shape[0][b.bucket[g]].GS : 32);
  G.Lmeas = meas_layout(b, g, b.bucket[g] >= 0 ? b.bucket_shape[1][b.bucket[g]].GS : 32);
  G.P.pos = w.pos;
  G.P.B = w.B;
  G.P.nacc = w.nacc;
  G.P.nrej = w.nrej;
  G.P.counters = w.counters;
  G.P.W = w.W;
  G.P.wid0 = w.wid0;
  G.P.k0 = w.k0;
  G.P.k1 = w.k1;
  G.Mp.pos = w.pos;
  G.Mp.Bout = w.B;
  G.Mp.acc = w.acc;
  G.Mp.swct_off = swct_offset(s);
  if (uses_tc(b, g)) {
    for (int k = 0; k < 2; ++k) {
      G.Mp.phiT[k] = w.phiT[k];
      G.Mp.yT[k] = w.yT[k];
    }
    G.Mp.nch = s.tcg_nch;
    G.Mp.Mf = s.tcg_Mf;
    G.Mp.Nf = s.tcg_Nf;
  }
  G.Mp.eps = w.eps;
  G.P.eps = w.eps;
  if (b.bucket[g] >= 0 && s.group_prepass && w.gprop) {  // the sweep's proposals come from propose_group
    G.P.prn = w.g_rn;
    G.P.prow = w.g_row;
    G.P.pu = w.g_u;
    G.P.pdchi = w.g_dchi;
  }
  G.Mp.accL = s.accL;
  G.Mp.acc_in_smem = 0;
  G.Mp.e_ref = w.e_ref;
  G.Mp.counters = w.counters;
  G.Mp.W = w.W;
  G.grid_meas = w.grid_meas;
  b.h_geo[g] = G;
}

void invalidate_graph(vmcf_batch_s& b) {
  if (b.exec) cudaGraphExecDestroy(b.exec);
  b.exec = nullptr;
  b.g_mode = -1;
}

// Launch list and work order for the current bucket shapes, for the phases in `phases`
// (bit 0: sweep, bit 1: evaluation) and the geometries with take[g] (all when take is
// empty). Items of one launch are ordered by the cost of the walkers they hold, largest first.
int build_plan(vmcf_batch_s& b, const std::vector<char>& take, int phases, cudaStream_t st) {
  std::vector<int2> items;
  b.launches.clear();
  b.n_launch[0] = b.n_launch[1] = 0;
  for (int g = 0; g < b.G; ++g) fill_geo(b, g);
  for (int phase = 0; phase < 2; ++phase) {
    if (!(phases & (1 << phase))) continue;
    std::map<Shape, std::vector<int>> by_shape;
    for (int g = 0; g < b.G; ++g)
      if (b.bucket[g] >= 0 && (take.empty() || take[g])) by_shape[b.bucket_shape[phase][b.bucket[g]]].push_back(g);
    for (auto& kv : by_shape) {
      LaunchPlan lp;
      lp.phase = phase;
      lp.shape = kv.first;
      int region = 0;
      for (int g : kv.second) region = std::max(region, region_bytes(b, phase, g, lp.shape.GS));
      lp.region = region;
      lp.smem = (size_t)lp.shape.groups * region;
      if (lp.smem > (size_t)kSmemCapBytes) return fail(VMCF_ENOTSUP, "batch launch shape does not fit shared memory");
      std::vector<std::pair<double, int2>> its;
      for (int g : kv.second) {
        const vmcf_walkers_s& w = *b.wk[g];
        for (int c = 0; c < w.grid_meas; ++c) {
          const long long n = (long long)w.W * (c + 1) / w.grid_meas - (long long)w.W * c / w.grid_meas;
          its.push_back({b.cost[phase][g] * (double)n, make_int2(g, c)});
        }
      }
      std::stable_sort(its.begin(), its.end(), [](const auto& x, const auto& y) { return x.first > y.first; });
      lp.item0 = (int)items.size();
      lp.n_items = (int)its.size();
      for (auto& it : its) items.push_back(it.second);
      int ctas = 0;
      int rc = occupancy(b, phase, lp.shape, lp.smem, &ctas);
      if (rc != VMCF_OK) return rc;
      if (ctas < 1) return fail(VMCF_ENOTSUP, "batch kernel cannot be resident with this launch shape");
      const long long grid_full = (long long)ctas * b.sms;
      lp.grid = (int)std::max(1LL, std::min(grid_full, ((long long)lp.n_items + lp.shape.groups - 1) / lp.shape.groups));
      b.launches.push_back(lp);
      b.n_launch[phase] += 1;
    }
  }
  if (items.size() > b.items_cap) {
    cudaFree(b.d_items);
    b.d_items = nullptr;
    BATCH_CUDA(cudaMalloc(&b.d_items, sizeof(int2) * items.size()));
    b.items_cap = items.size();
  }
  if ((int)b.launches.size() > b.queue_cap) {
    cudaFree(b.d_queue);
    b.d_queue = nullptr;
    BATCH_CUDA(cudaMalloc(&b.d_queue, sizeof(int) * b.launches.size()));
    b.queue_cap = (int)b.launches.size();
  }
  if (!items.empty())
    BATCH_CUDA(cudaMemcpyAsync(b.d_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice, st));
  BATCH_CUDA(cudaStreamSynchronize(st));
  while (b.forks.size() < b.launches.size()) {
    cudaStream_t s2;
    cudaEvent_t ev;
    BATCH_CUDA(cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking));
    BATCH_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    b.forks.push_back(s2);
    b.joins.push_back(ev);
  }
  invalidate_graph(b);
  return VMCF_OK;
}

// Geometry tables (with the current E_ref of each walker set), chain clocks and queues.
int upload_state(vmcf_batch_s& b, cudaStream_t st) {
  for (int g = 0; g < b.G; ++g) {
    b.h_geo[g].Mp.e_ref = b.wk[g]->e_ref;
    b.h_clk[g].sweep = b.wk[g]->sweep;
    b.h_clk[g].c = b.wk[g]->counter;
    b.h_clk[g].Ne = b.sys[g]->Ne;
  }
  BATCH_CUDA(cudaMemcpyAsync(b.d_geo, b.h_geo.data(), sizeof(BatchGeom) * b.G, cudaMemcpyHostToDevice, st));
  BATCH_CUDA(cudaMemcpyAsync(b.d_clk, b.h_clk.data(), sizeof(BatchClock) * b.G, cudaMemcpyHostToDevice, st));
  if (!b.launches.empty()) BATCH_CUDA(cudaMemsetAsync(b.d_queue, 0, sizeof(int) * b.launches.size(), st));
  return VMCF_OK;
}

BatchArgs args_for(const vmcf_batch_s& b, int k, int mode, int kref, double sigma) {
  const LaunchPlan& lp = b.launches[k];
  BatchArgs A{};
  A.geo = b.d_geo;
  A.clk = b.d_clk;
  A.items = b.d_items + lp.item0;
  A.n_items = lp.n_items;
  A.queue = b.d_queue + k;
  A.mode = mode;
  A.kref = kref;
  A.sigma = sigma;
  A.region = lp.region;
  A.hdr = kHdr;
  return A;
}

cudaError_t launch_k(const vmcf_batch_s& b, int k, int mode, int kref, double sigma, cudaStream_t st) {
  const LaunchPlan& lp = b.launches[k];
  const BatchArgs A = args_for(b, k, mode, kref, sigma);
  return b.precision == VMCF_FP64
             ? launch_batch<double>(lp.phase, lp.shape.GS, lp.shape.groups, lp.grid, lp.smem, A, b.jb, st)
             : launch_batch<float>(lp.phase, lp.shape.GS, lp.shape.groups, lp.grid, lp.smem, A, b.jb, st);
}

// One sweep of the batch as a graph: per phase (the evaluation only when measuring), fork
// one branch per persistent kernel and join; then advance the clocks and rewind the queues.
// The proposals of the coming sweep for every walker-group geometry with take[g] (all when take is empty) whose
// descriptor reads them, each geometry's sweep index from its device clock.
cudaError_t launch_batch_proposals(const vmcf_batch_s& b, const std::vector<char>& take, double sigma, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  for (int g = 0; g < b.G && e == cudaSuccess; ++g) {
    if (b.bucket[g] < 0 || !b.h_geo[g].P.prn || !(take.empty() || take[g])) continue;
    const vmcf_system_s& s = *b.sys[g];
    const vmcf_walkers_s& w = *b.wk[g];
    GroupProposeParams Q{};
    Q.pos = w.pos;
    Q.prn = w.g_rn;
    Q.prow = w.g_row;
    Q.pu = w.g_u;
    Q.pdchi = w.g_dchi;
    Q.W = w.W;
    Q.wid0 = w.wid0;
    Q.k0 = w.k0;
    Q.k1 = w.k1;
    Q.sigma = sigma;
    Q.clk = b.d_clk + g;
    e = launch_propose_rows(s, Q, st);
  }
  return e;
}

int capture(vmcf_batch_s& b, int mode, int kref, double sigma) {
  invalidate_graph(b);
  BATCH_CUDA(cudaStreamBeginCapture(b.cap, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  // small-system geometries: each a branch of its own for the whole sweep (proposals, runs of moves and
  // re-inversions, the measurement), beside the persistent kernels of both phases
  if (!b.small_g.empty()) e = cudaEventRecord(b.fork_ev, b.cap);
  for (size_t i = 0; e == cudaSuccess && i < b.small_g.size(); ++i) {
    const int g = b.small_g[i];
    e = cudaStreamWaitEvent(b.sforks[i], b.fork_ev, 0);
    if (e == cudaSuccess) e = small_sweep_launches(b.sys[g], b.wk[g], b.d_clk + g, mode, kref, sigma, b.sforks[i]);
    if (e == cudaSuccess) e = cudaEventRecord(b.sjoins[i], b.sforks[i]);
    b.s_eref[i] = b.wk[g]->e_ref;
    b.s_eps[i] = b.wk[g]->eps;
  }
  // the walker-group geometries' proposals, ahead of the sweep phase
  if (e == cudaSuccess) e = launch_batch_proposals(b, {}, sigma, b.cap);
  for (int phase = 0; phase < 2 && e == cudaSuccess; ++phase) {
    if (phase == 1 && mode == 0) break;
    e = cudaEventRecord(b.fork_ev, b.cap);
    for (size_t k = 0; e == cudaSuccess && k < b.launches.size(); ++k) {
      if (b.launches[k].phase != phase) continue;
      cudaStream_t sk = b.forks[k];
      e = cudaStreamWaitEvent(sk, b.fork_ev, 0);
      if (e == cudaSuccess) e = launch_k(b, (int)k, mode, kref, sigma, sk);
      if (e == cudaSuccess) e = cudaEventRecord(b.joins[k], sk);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(b.cap, b.joins[k], 0);
    }
  }
  for (size_t i = 0; e == cudaSuccess && i < b.small_g.size(); ++i) e = cudaStreamWaitEvent(b.cap, b.sjoins[i], 0);
  // measured sweeps: the tensor-core GEMM of each geometry's O sums over the tiles just written
  for (int g = 0; e == cudaSuccess && mode == 1 && g < b.G; ++g) {
    if (!uses_tc(b, g)) continue;
    const vmcf_system_s& s = *b.sys[g];
    const vmcf_walkers_s& w = *b.wk[g];
    e = launch_tc_sumprod(w.phiT[0], w.phiT[1], w.yT[0], w.yT[1], w.W, s.tcg_nch, s.tcg_Mf, s.tcg_Nf, s.nup, s.ndn,
                          w.nblocks * w.tc_cpb, w.tc_slots, w.tc_flag, b.cap);
  }
  if (e == cudaSuccess) e = launch_batch_advance(b.d_clk, b.G, mode, kref, b.d_queue, (int)b.launches.size(), b.cap);
  cudaGraph_t graph = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(b.cap, &graph);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b.exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    b.exec = nullptr;
    return cuda_fail(e, "capturing the batch sweep graph");
  }
  b.g_mode = mode;
  b.g_kref = kref;
  b.g_sigma = sigma;
  return VMCF_OK;
}

void advance_host(vmcf_batch_s& b, const std::vector<char>& take, int n, int mode, int kref) {
  for (int g = 0; g < b.G; ++g) {
    if (!take.empty() && !take[g]) continue;
    vmcf_walkers_s& w = *b.wk[g];
    w.sweep += (uint64_t)n;
    if (mode != 0) {
      w.counter = 0;
      if (mode == 1) w.measured += (uint64_t)n;
    } else {
      w.counter = (int)((w.counter + (long long)n * b.sys[g]->Ne) % kref);
    }
  }
}

}  // namespace

extern "C" {

int vmcf_batch_destroy(vmcf_batch_t b) {
  if (!b) return VMCF_OK;
  invalidate_graph(*b);
  for (auto s : b->forks) cudaStreamDestroy(s);
  for (auto e : b->joins) cudaEventDestroy(e);
  for (auto s : b->sforks) cudaStreamDestroy(s);
  for (auto e : b->sjoins) cudaEventDestroy(e);
  if (b->fork_ev) cudaEventDestroy(b->fork_ev);
  if (b->cap) cudaStreamDestroy(b->cap);
  cudaFree(b->d_geo);
  cudaFree(b->d_clk);
  cudaFree(b->d_items);
  cudaFree(b->d_queue);
  delete b;
  return VMCF_OK;
}

int vmcf_batch_create(const vmcf_system_t* systems, const vmcf_walkers_t* walkers, int G, void* stream,
                      vmcf_batch_t* out) {
  if (!out) return fail(VMCF_EINVAL, "out is NULL");
  *out = nullptr;
  if (!systems || !walkers || G < 1) return fail(VMCF_EINVAL, "need G >= 1 systems and walker sets");
  for (int g = 0; g < G; ++g) {
    if (!systems[g] || !walkers[g] || walkers[g]->sys != systems[g])
      return fail(VMCF_EINVAL, "geometry " + std::to_string(g) + ": walker set does not belong to its system");
    if (systems[g]->precision != systems[0]->precision)
      return fail(VMCF_EINVAL, "all systems of a batch must have the same precision");
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  auto* b = new vmcf_batch_s();
  b->G = G;
  b->precision = systems[0]->precision;
  b->sys.assign(systems, systems + G);
  b->wk.assign(walkers, walkers + G);
  for (int g = 0; g < G; ++g) b->jb = b->jb || systems[g]->MJ > 0;
  b->h_geo.resize(G);
  b->h_clk.resize(G);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_geo, sizeof(BatchGeom) * G);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_clk, sizeof(BatchClock) * G);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    vmcf_batch_destroy(b);
    return cuda_fail(e, "batch set-up");
  }
  // buckets by (ceil(Ne / 16), ceil(M / 64)) for the walker-group kernels; geometries on the
  // small-system kernels get a graph branch each instead (bucket -1)
  std::map<std::pair<int, int>, int> keys;
  b->bucket.resize(G);
  for (int g = 0; g < G; ++g) {
    b->cost[0].push_back(0.0);
    b->cost[1].push_back(0.0);
    if (systems[g]->small) {
      b->bucket[g] = -1;
      b->small_g.push_back(g);
      cudaStream_t s2 = nullptr;
      cudaEvent_t ev = nullptr;
      cudaError_t e2 = cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking);
      if (e2 == cudaSuccess) e2 = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      if (s2) b->sforks.push_back(s2);
      if (ev) b->sjoins.push_back(ev);
      if (e2 != cudaSuccess) {
        vmcf_batch_destroy(b);
        return cuda_fail(e2, "batch set-up");
      }
      continue;
    }
    const std::pair<int, int> k{(systems[g]->Ne + 15) / 16, (systems[g]->M + 63) / 64};
    auto it = keys.find(k);
    if (it == keys.end()) it = keys.emplace(k, (int)keys.size()).first;
    b->bucket[g] = it->second;
    for (int ph = 0; ph < 2; ++ph) b->cost[ph][g] = heuristic_cost(*systems[g], ph);
  }
  b->s_eref.assign(b->small_g.size(), 0.0);
  b->geo_version.resize(G);
  for (int g = 0; g < G; ++g) b->geo_version[g] = systems[g]->geometry_version;
  b->s_eps.assign(b->small_g.size(), 0.0);
  for (int ph = 0; ph < 2; ++ph) {
    b->bucket_shape[ph].resize(keys.size());
    for (int bk = 0; bk < (int)keys.size(); ++bk) b->bucket_shape[ph][bk] = default_shape(*b, ph, bk);
  }
  int rc = build_plan(*b, {}, 3, st);
  if (rc != VMCF_OK) {
    vmcf_batch_destroy(b);
    return rc;
  }
  *out = b;
  return VMCF_OK;
}

int vmcf_batch_set_shape(vmcf_batch_t b, int g, int phase, int GS, int groups) {
  if (!b || g < 0 || g >= b->G || phase < 0 || phase > 1) return fail(VMCF_EINVAL, "bad batch, geometry or phase");
  const int bk = b->bucket[g];
  if (bk < 0) return fail(VMCF_EINVAL, "geometry runs on the small-system kernels (no launch shape to set)");
  const Shape sh{GS, groups};
  if (!shape_fits(*b, phase, bk, sh))
    return fail(VMCF_EINVAL, "launch shape not supported or does not fit shared memory");
  b->bucket_shape[phase][bk] = sh;
  return build_plan(*b, {}, 3, nullptr);
}

int vmcf_batch_info(vmcf_batch_t b, int* n_buckets, int* n_launches, int g, int* bucket, int* shapes) {
  if (!b) return fail(VMCF_EINVAL, "NULL batch");
  if (n_buckets) *n_buckets = (int)b->bucket_shape[0].size();
  if (n_launches) *n_launches = (int)b->launches.size();
  if (g >= 0 && g < b->G) {
    if (bucket) *bucket = b->bucket[g];
    if (shapes) {
      if (b->bucket[g] < 0) {  // small-system kernels: lanes per walker of the moves, warps per evaluation CTA
        const vmcf_system_s& s = *b->sys[g];
        shapes[0] = s.move_lpw;
        shapes[1] = 0;
        shapes[2] = 32;
        shapes[3] = s.small_warps;
      } else {
        for (int ph = 0; ph < 2; ++ph) {
          shapes[2 * ph] = b->bucket_shape[ph][b->bucket[g]].GS;
          shapes[2 * ph + 1] = b->bucket_shape[ph][b->bucket[g]].groups;
        }
      }
    }
  }
  return VMCF_OK;
}

int vmcf_batch_sample(vmcf_batch_t b, int n_sweeps, double step_sigma, int refresh_k, int measure, void* stream) {
  if (!b) return fail(VMCF_EINVAL, "NULL batch");
  if (n_sweeps < 0 || !(step_sigma > 0.0) || !std::isfinite(step_sigma) || refresh_k < 1)
    return fail(VMCF_EINVAL, "need n_sweeps >= 0, step_sigma > 0, refresh_k >= 1");
  if (n_sweeps == 0) return VMCF_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (int g = 0; g < b->G; ++g)
    if (b->wk[g]->counter >= refresh_k) {  // k lowered since the last call: re-invert before the first move
      int rc = vmcf::refresh_walker_set(b->sys[g], b->wk[g], st);
      if (rc != VMCF_OK) return rc;
    }
  const int mode = measure ? 1 : 0;
  bool stale = false;  // a small-system geometry's launches were captured with another E_ref or threshold
  for (int g = 0; g < b->G; ++g)
    if (b->geo_version[g] != b->sys[g]->geometry_version) {  // vmcf_system_set_geometry since: new descriptors
      fill_geo(*b, g);
      b->geo_version[g] = b->sys[g]->geometry_version;
      stale = true;
    }
  for (size_t i = 0; i < b->small_g.size(); ++i)
    stale = stale || b->s_eref[i] != b->wk[b->small_g[i]]->e_ref || b->s_eps[i] != b->wk[b->small_g[i]]->eps;
  if (!b->exec || stale || b->g_mode != mode || b->g_kref != refresh_k || b->g_sigma != step_sigma) {
    int rc = capture(*b, mode, refresh_k, step_sigma);
    if (rc != VMCF_OK) return rc;
  }
  int rc = upload_state(*b, st);
  if (rc != VMCF_OK) return rc;
  for (int i = 0; i < n_sweeps; ++i) BATCH_CUDA(cudaGraphLaunch(b->exec, st));
  advance_host(*b, {}, n_sweeps, mode, refresh_k);
  return VMCF_OK;
}

int vmcf_batch_autotune(vmcf_batch_t b, double step_sigma, int refresh_k, void* stream) {
  if (!b) return fail(VMCF_EINVAL, "NULL batch");
  if (!(step_sigma > 0.0) || !std::isfinite(step_sigma) || refresh_k < 1)
    return fail(VMCF_EINVAL, "need step_sigma > 0, refresh_k >= 1");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEvent_t t0, t1;
  BATCH_CUDA(cudaEventCreate(&t0));
  if (cudaError_t e = cudaEventCreate(&t1); e != cudaSuccess) {
    cudaEventDestroy(t0);
    return cuda_fail(e, "cudaEventCreate(&t1)");
  }
  const int nb = (int)b->bucket_shape[0].size();
  int rc = VMCF_OK;
  // per bucket and phase: one sweep (phase 0) or one evaluation without sums (phase 1) of
  // the bucket's walkers per feasible shape
  for (int phase = 0; phase < 2 && rc == VMCF_OK; ++phase)
    for (int bk = 0; bk < nb && rc == VMCF_OK; ++bk) {
      std::vector<char> take(b->G, 0);
      for (int g = 0; g < b->G; ++g) take[g] = b->bucket[g] == bk;
      Shape best = b->bucket_shape[phase][bk];
      float best_ms = 1e30f;
      for (const Shape& cand : kCandidates) {
        if (!shape_fits(*b, phase, bk, cand)) continue;
        b->bucket_shape[phase][bk] = cand;
        rc = build_plan(*b, take, 1 << phase, st);
        if (rc != VMCF_OK) break;
        rc = upload_state(*b, st);
        if (rc != VMCF_OK) break;
        const int mode = phase == 0 ? 0 : 2;
        cudaError_t e = phase == 0 ? launch_batch_proposals(*b, take, step_sigma, st) : cudaSuccess;
        if (e == cudaSuccess) e = cudaEventRecord(t0, st);
        if (e == cudaSuccess) e = launch_k(*b, 0, mode, refresh_k, step_sigma, st);
        if (e == cudaSuccess) e = cudaEventRecord(t1, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
        if (e != cudaSuccess) {
          rc = cuda_fail(e, "autotuning launch");
          break;
        }
        if (phase == 0) {
          advance_host(*b, take, 1, 0, refresh_k);
        } else {
          for (int g = 0; g < b->G; ++g)
            if (take[g]) b->wk[g]->counter = 0;  // the evaluation rebuilt the inverses
        }
        if (ms < best_ms) {
          best_ms = ms;
          best = cand;
        }
      }
      b->bucket_shape[phase][bk] = best;
      // measured cost per walker of this bucket, shared by its geometries in proportion to
      // their operation counts
      if (rc == VMCF_OK && best_ms < 1e29f) {
        double hsum = 0.0;
        for (int g = 0; g < b->G; ++g)
          if (take[g]) hsum += heuristic_cost(*b->sys[g], phase) * b->wk[g]->W;
        for (int g = 0; g < b->G; ++g)
          if (take[g] && hsum > 0.0) b->cost[phase][g] = (double)best_ms * heuristic_cost(*b->sys[g], phase) / hsum;
      }
    }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  if (rc != VMCF_OK) return rc;
  return build_plan(*b, {}, 3, st);
}

}  // extern "C"
