// vmcf_evaluate_sums_noalloc: fixed-walker evaluation reduced to walker sums, for callers
// that must not allocate GPU memory while they run (see include/vmcf.h).
//
// The measurement kernel normally writes its per-CTA FP64 partial sums into a buffer that
// the walker object allocated. Here the same kernel writes them into g_noalloc_scratch, a
// file-scope device array of fixed size, and the block-reduction kernel folds them into
// the caller's output. Nothing is allocated: the array exists on every GPU that loads this
// library, from load until process exit.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/vmcf.h"
#include "vmcf_host.h"

namespace {

// 2^21 doubles = 16 MiB of per-CTA partial sums.
constexpr size_t kScratchDoubles = size_t(1) << 21;
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

// Device address of g_noalloc_scratch, looked up once per device with that device current.
// In host code the symbol's name is only a host-side stand-in, never a device address.
constexpr int kMaxDevices = 64;
double* g_scratch_dev[kMaxDevices] = {};
std::mutex g_scratch_mu;

// The scratch of device `dev`, which must be the current device (the system's own device).
int scratch_for_device(int dev, double** out) {
  if (dev < 0 || dev >= kMaxDevices) return vmcf::set_last_error(VMCF_ENOTSUP, "device index beyond 63");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return vmcf::set_last_error(VMCF_ECUDA, std::string("cudaGetSymbolAddress(g_noalloc_scratch): ") +
                                                  cudaGetErrorString(e));
    g_scratch_dev[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_dev[dev];
  return VMCF_OK;
}

}  // namespace

extern "C" int vmcf_evaluate_sums_noalloc(vmcf_system_t s, const double* pos, int W, double e_ref, double* sums,
                                          void* stream) {
  if (!s || W < 0 || (W > 0 && (!pos || !sums)))
    return vmcf::set_last_error(VMCF_EINVAL, "need a system, W >= 0, and positions and an output when W > 0");
  const int accL = s->accL;
  const size_t fit = kScratchDoubles / (size_t)accL;  // CTAs whose partial sums fit the scratch
  if (fit < 1)
    return vmcf::set_last_error(VMCF_EINVAL, "the system's walker-sum vector exceeds the no-alloc scratch of 2^21 doubles");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return vmcf::set_last_error(VMCF_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev != s->device)
    return vmcf::set_last_error(VMCF_EINVAL, "the system's device must be the current device");
  double* scratch = nullptr;
  int rc = scratch_for_device(dev, &scratch);
  if (rc != VMCF_OK || W == 0) return rc;  // W = 0: the once-per-device set-up only
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  vmcf::MeasParams M{};
  vmcf::Launch lc = vmcf::launch_meas(*s, 1, true, false);
  M.acc_in_smem = s->acc_smem ? 1 : 0;
  if (s->precision != VMCF_FP64 && s->acc_smem) {
    // Mixed precision: the shared-memory accumulator is FP32 and is meant for the few walkers of
    // one CTA; with the grid capped by the scratch a CTA may take many, so every walker goes
    // straight to its CTA's FP64 slot instead (one walker group per CTA).
    lc.groups = 1;
    lc.L = s->Lmeas;
    lc.smem = s->Lmeas.bytes;
    lc.acc_off = -1;
    M.acc_in_smem = 0;
  }
  const int per_cta = 4 * (M.acc_in_smem ? s->gpb_meas : 1);
  long long grid = (W + per_cta - 1) / per_cta;
  if (grid > (long long)fit) grid = (long long)fit;
  if (grid > W) grid = W;
  lc.grid = (int)grid;
  // every call reuses the scratch: clear the slots this call accumulates into
  e = cudaMemsetAsync(scratch, 0, sizeof(double) * (size_t)grid * accL, st);
  if (e != cudaSuccess) return vmcf::set_last_error(VMCF_ECUDA, std::string("clearing scratch: ") + cudaGetErrorString(e));
  M.pos = pos;
  M.acc = scratch;
  M.swct_off = vmcf::swct_offset(*s);
  M.accL = accL;
  M.e_ref = e_ref;
  M.counters = reinterpret_cast<unsigned long long*>(s->scratch_counters);
  M.W = W;
  e = s->precision == VMCF_FP64 ? vmcf::launch_measure<double>(s->dev, lc, M, st)
                                : vmcf::launch_measure<float>(s->dev, lc, M, st);
  if (e != cudaSuccess) return vmcf::set_last_error(VMCF_ECUDA, std::string("measure kernel launch: ") + cudaGetErrorString(e));
  e = vmcf::launch_block_reduce(scratch, (int)grid, (int)grid, accL, sums, 1, st);
  if (e != cudaSuccess) return vmcf::set_last_error(VMCF_ECUDA, std::string("reduce kernel launch: ") + cudaGetErrorString(e));
  return VMCF_OK;
}
