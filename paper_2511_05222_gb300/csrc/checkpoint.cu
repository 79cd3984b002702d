// Checkpoint and resume of a walker set (see include/vmcf.h): the walker state's device buffers
// copied to and from one host buffer behind a vmcf_walkers_state header. Host code only.
#include <cuda_runtime.h>

#include <cstring>
#include <string>

#include "../../include/vmcf.h"
#include "vmcf_host.h"

namespace {

constexpr char kMagic[8] = "vmcfwk1";
constexpr int kSegments = 8;

int fail(int code, const std::string& msg) { return vmcf::set_last_error(code, msg); }

// The walker set's device segments in header order, with their sizes in bytes (nullptr / 0:
// absent for this system). The sizes are those the walker set was allocated with.
void segments(const vmcf_walkers_s& wk, void* ptr[kSegments], uint64_t bytes[kSegments]) {
  const vmcf_system_s& s = *wk.sys;
  const uint64_t W = (uint64_t)wk.W, npos = W * 3 * (uint64_t)s.Ne;
  const uint64_t tsz = s.precision == VMCF_FP64 ? 8 : 4;
  ptr[0] = wk.pos;
  bytes[0] = 8 * npos;
  ptr[1] = wk.B;
  bytes[1] = tsz * W * (uint64_t)s.nB;
  ptr[2] = wk.nacc;
  bytes[2] = 4 * W;
  ptr[3] = wk.nrej;
  bytes[3] = 4 * W;
  ptr[4] = wk.counters;
  bytes[4] = 16;
  ptr[5] = wk.acc;
  bytes[5] = 8 * (uint64_t)wk.grid_meas * (uint64_t)s.accL;
  ptr[6] = wk.posf;
  bytes[6] = wk.posf ? sizeof(float2) * npos : 0;
  ptr[7] = wk.tc ? wk.tc_slots : nullptr;
  bytes[7] = wk.tc ? 8 * (uint64_t)wk.tc_slot_doubles : 0;
}

vmcf_walkers_state header_of(const vmcf_walkers_s& wk) {
  vmcf_walkers_state h;
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, kMagic, sizeof(kMagic));
  const vmcf_system_s& s = *wk.sys;
  h.W = wk.W;
  h.nblocks = wk.nblocks;
  h.Ne = s.Ne;
  h.n_up = s.nup;
  h.n_dn = s.ndn;
  h.M = s.M;
  h.K = s.K;
  h.precision = s.precision;
  h.counter = wk.counter;
  h.sweep = wk.sweep;
  h.measured = wk.measured;
  h.key0 = wk.k0;
  h.key1 = wk.k1;
  h.wid0 = wk.wid0;
  h.e_ref = wk.e_ref;
  h.eps = wk.eps;
  void* ptr[kSegments];
  segments(wk, ptr, h.bytes);
  return h;
}

uint64_t total_bytes(const vmcf_walkers_state& h) {
  uint64_t n = sizeof(vmcf_walkers_state);
  for (int i = 0; i < kSegments; ++i) n += h.bytes[i];
  return n;
}

}  // namespace

extern "C" {

int vmcf_walkers_state_bytes(vmcf_walkers_t wk, uint64_t* bytes) {
  if (!wk || !bytes) return fail(VMCF_EINVAL, "NULL walker set or output");
  *bytes = total_bytes(header_of(*wk));
  return VMCF_OK;
}

int vmcf_walkers_save(vmcf_walkers_t wk, void* buf, uint64_t bytes, void* stream) {
  if (!wk || !buf) return fail(VMCF_EINVAL, "NULL walker set or buffer");
  const vmcf_walkers_state h = header_of(*wk);
  if (bytes < total_bytes(h)) return fail(VMCF_EINVAL, "checkpoint buffer too small (see vmcf_walkers_state_bytes)");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned char* out = static_cast<unsigned char*>(buf);
  std::memcpy(out, &h, sizeof(h));
  uint64_t off = sizeof(h);
  void* ptr[kSegments];
  uint64_t seg[kSegments];
  segments(*wk, ptr, seg);
  for (int i = 0; i < kSegments; ++i) {
    if (seg[i] == 0) continue;
    cudaError_t e = cudaMemcpyAsync(out + off, ptr[i], seg[i], cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return fail(VMCF_ECUDA, std::string("checkpoint copy: ") + cudaGetErrorString(e));
    off += seg[i];
  }
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(VMCF_ECUDA, std::string("checkpoint copy: ") + cudaGetErrorString(e));
  return VMCF_OK;
}

int vmcf_walkers_load(vmcf_walkers_t wk, const void* buf, uint64_t bytes, void* stream) {
  if (!wk || !buf) return fail(VMCF_EINVAL, "NULL walker set or buffer");
  if (bytes < sizeof(vmcf_walkers_state)) return fail(VMCF_EINVAL, "checkpoint buffer shorter than its header");
  vmcf_walkers_state h;
  std::memcpy(&h, buf, sizeof(h));
  const vmcf_walkers_state mine = header_of(*wk);
  if (std::memcmp(h.magic, kMagic, sizeof(kMagic)) != 0) return fail(VMCF_EINVAL, "not a walker-set checkpoint");
  if (h.W != mine.W || h.nblocks != mine.nblocks || h.Ne != mine.Ne || h.n_up != mine.n_up || h.n_dn != mine.n_dn ||
      h.M != mine.M || h.K != mine.K || h.precision != mine.precision)
    return fail(VMCF_EINVAL, "checkpoint of a different system, walker count, block count or precision");
  for (int i = 0; i < kSegments; ++i)
    if (h.bytes[i] != mine.bytes[i]) return fail(VMCF_EINVAL, "checkpoint segment sizes differ from this walker set's");
  if (bytes < total_bytes(h)) return fail(VMCF_EINVAL, "checkpoint buffer shorter than its segments");
  if (h.counter < 0 || !(h.eps >= 0.0)) return fail(VMCF_EINVAL, "checkpoint header holds an invalid chain clock");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const unsigned char* in = static_cast<const unsigned char*>(buf);
  uint64_t off = sizeof(h);
  void* ptr[kSegments];
  uint64_t seg[kSegments];
  segments(*wk, ptr, seg);
  for (int i = 0; i < kSegments; ++i) {
    if (seg[i] == 0) continue;
    cudaError_t e = cudaMemcpyAsync(ptr[i], in + off, seg[i], cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return fail(VMCF_ECUDA, std::string("checkpoint restore: ") + cudaGetErrorString(e));
    off += seg[i];
  }
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(VMCF_ECUDA, std::string("checkpoint restore: ") + cudaGetErrorString(e));
  wk->counter = h.counter;
  wk->sweep = h.sweep;
  wk->measured = h.measured;
  wk->k0 = h.key0;
  wk->k1 = h.key1;
  wk->wid0 = h.wid0;
  wk->e_ref = h.e_ref;
  wk->eps = h.eps;
  return VMCF_OK;
}

}  // extern "C"
