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

int scratch_for_current_device(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return vmcf::set_last_error(VMCF_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return vmcf::set_last_error(VMCF_ENOTSUP, "device index beyond 63");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
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
  if (!s || !pos || !sums || W < 1) return vmcf::set_last_error(VMCF_EINVAL, "need a system, positions, W >= 1 and an output");
  const int accL = s->accL;
  const size_t fit = kScratchDoubles / (size_t)accL;  // CTAs whose partial sums fit the scratch
  if (fit < 1)
    return vmcf::set_last_error(VMCF_EINVAL, "the system's walker-sum vector exceeds the no-alloc scratch of 2^21 doubles");
  double* scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc != VMCF_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int per_cta = 4 * (s->acc_smem ? s->gpb_meas : 1);
  long long grid = (W + per_cta - 1) / per_cta;
  if (grid > (long long)fit) grid = (long long)fit;
  if (grid > W) grid = W;
  // every call reuses the scratch: clear the slots this call accumulates into
  cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(double) * (size_t)grid * accL, st);
  if (e != cudaSuccess) return vmcf::set_last_error(VMCF_ECUDA, std::string("clearing scratch: ") + cudaGetErrorString(e));
  vmcf::MeasParams M{};
  M.pos = pos;
  M.acc = scratch;
  M.swct_off = vmcf::swct_offset(*s);
  M.accL = accL;
  M.acc_in_smem = s->acc_smem ? 1 : 0;
  M.e_ref = e_ref;
  M.counters = reinterpret_cast<unsigned long long*>(s->scratch_counters);
  M.W = W;
  const vmcf::Launch lc = vmcf::launch_meas(*s, (int)grid, true, false);
  e = s->precision == VMCF_FP64 ? vmcf::launch_measure<double>(s->dev, lc, M, st)
                                : vmcf::launch_measure<float>(s->dev, lc, M, st);
  if (e != cudaSuccess) return vmcf::set_last_error(VMCF_ECUDA, std::string("measure kernel launch: ") + cudaGetErrorString(e));
  e = vmcf::launch_block_reduce(scratch, (int)grid, (int)grid, accL, sums, 1, st);
  if (e != cudaSuccess) return vmcf::set_last_error(VMCF_ECUDA, std::string("reduce kernel launch: ") + cudaGetErrorString(e));
  return VMCF_OK;
}
