// Walker sums of O on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// For one spin block, the walker-weighted orbital-coefficient sums of App. A (Eq. fc-vmc-eval)
//   S[mu][j] = sum over walkers w of the block, electrons el of the spin:
//              psi_mu(r_{w,el}) * Y_{w,el,j},   Y = [B_{i,el} (j < n) | c_w B_{i,el} (n <= j < 2n)]
// are one GEMM with K = walkers x electron slots: D[mu][j] = sum_k PhiT[mu][k] Y[k][j]. The
// measurement kernels write, per walker and chunk of 16 electron slots, PhiT as [Mf][16] and YT as
// [Nf][16] bf16 (slots beyond n, rows beyond M and columns beyond 2n are zero). A CTA owns a range
// of walkers inside one jackknife block, one spin and one 128 x 32 tile of D, keeps the tile
// (FP32) in tensor memory across the whole range, and adds it to its FP64 slot at the end.
//
// Operands are K-major without swizzle: 8-row x 16-byte core matrices, the K-adjacent core at
// +128 bytes (leading byte offset), the M/N-adjacent core at +KC*128 bytes (stride byte offset),
// KC = 16-byte K chunks per stage. One thread issues the MMAs; completion is tracked with an
// mbarrier whose waits are bounded (a timeout sets the error flag and the CTA stops cleanly).
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>

#include "vmcf_internal.h"

namespace vmcf {

namespace {

constexpr int kTcThreads = 128;       // 4 warps: all stage copies; warps 0-3 read TMEM lanes 0-127
constexpr int kTcWalkersPerStage = 8; // K per stage = 8 walkers x 16 slots = 128
constexpr int kTcKC = 2 * kTcWalkersPerStage;  // 16-byte K chunks per stage (8 bf16 each)
constexpr long long kSpinLimit = 1LL << 26;    // bounded mbarrier wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// tcgen05 shared-memory matrix descriptor: start >> 4 (bits 0-13), leading byte offset >> 4
// (16-29), stride byte offset >> 4 (32-45), descriptor version 1 (46-47), no swizzle (61-63 = 0).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator (bits 4-5 = 1), A and B bf16 (bits 7-9 and
// 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__device__ __forceinline__ uint32_t instr_desc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Wait for the phase with the given parity to complete; false after kSpinLimit polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (long long it = 0; it < kSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

}  // namespace

// grid.x = nblocks * cpb CTAs (walker ranges), grid.y = 2 spins, grid.z = output tiles of 128 AO
// rows x 32 Y columns (z = mt * Nt + nt). Each walker holds nch chunks of 16 electron slots:
// PhiT[s]: [W][nch][Mf][16] bf16, YT[s]: [W][nch][Nf][16] bf16 (a chunk is one K step of 16).
// slots: [2][gridDim.z][gridDim.x][128][32] FP64, added to. flag: set to 1 on a timed-out wait.
__global__ void __launch_bounds__(kTcThreads, 1)
    tc_sumprod_kernel(const __nv_bfloat16* __restrict__ phiT_up, const __nv_bfloat16* __restrict__ phiT_dn,
                      const __nv_bfloat16* __restrict__ yT_up, const __nv_bfloat16* __restrict__ yT_dn, int W, int nch,
                      int Mf, int Nf, int n_up, int n_dn, double* __restrict__ slots, int* flag) {
  __shared__ __align__(128) unsigned char sA[128 * kTcKC * 16];  // 128 rows (mu) x K stage
  __shared__ __align__(128) unsigned char sB[32 * kTcKC * 16];   // up to 32 rows (j) x K stage
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int spin = blockIdx.y;
  if ((spin == 0 ? n_up : n_dn) == 0) return;
  const __nv_bfloat16* phiT = spin == 0 ? phiT_up : phiT_dn;
  const __nv_bfloat16* yT = spin == 0 ? yT_up : yT_dn;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int Nt = (Nf + 31) / 32, mt = blockIdx.z / Nt, nt = blockIdx.z - mt * Nt;
  const int m0 = 128 * mt, j0 = 32 * nt;
  const int Mp = Mf - m0 < 128 ? Mf - m0 : 128, Np = Nf - j0 < 32 ? Nf - j0 : 32;  // rows of this tile
  // the CTA's walkers (never split between CTAs, so a jackknife block keeps whole walkers),
  // as nch chunks each
  const long long w0 = (long long)nch * ((long long)W * blockIdx.x / gridDim.x);
  const long long w1 = (long long)nch * ((long long)W * (blockIdx.x + 1) / gridDim.x);

  // zero both tiles once: rows mu >= Mp and j >= Np stay zero for the whole kernel
  for (int i = tid; i < (int)(sizeof(sA) / 16); i += kTcThreads) reinterpret_cast<uint4*>(sA)[i] = make_uint4(0, 0, 0, 0);
  for (int i = tid; i < (int)(sizeof(sB) / 16); i += kTcThreads) reinterpret_cast<uint4*>(sB)[i] = make_uint4(0, 0, 0, 0);
  if (tid == 0) {
    mbar_init(&mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {  // tensor-memory accumulator: 32 columns x 128 lanes, FP32
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(smem_u32(&tmem_base))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = instr_desc_bf16(128, 32);
  const uint32_t aBase = smem_u32(sA), bBase = smem_u32(sB);
  const uint32_t sbo = kTcKC * 128;  // next 8-row core group
  uint32_t phase = 0;
  bool ok = true, first = true;

  for (long long ws = w0; ws < w1 && ok; ws += kTcWalkersPerStage) {
    // stage: core (row group g, K chunk kc) at (g * KC + kc) * 128 bytes; row r of it at +16 r
    const int nw = (int)((w1 - ws) < kTcWalkersPerStage ? (w1 - ws) : kTcWalkersPerStage);
    for (int idx = tid; idx < kTcWalkersPerStage * Mp * 2; idx += kTcThreads) {
      const int s = idx / (Mp * 2), rem = idx - s * Mp * 2, mu = rem >> 1, h = rem & 1;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (s < nw) v = *reinterpret_cast<const uint4*>(phiT + ((size_t)(ws + s) * Mf + m0 + mu) * 16 + 8 * h);
      const int kc = 2 * s + h;
      *reinterpret_cast<uint4*>(sA + ((mu >> 3) * kTcKC + kc) * 128 + (mu & 7) * 16) = v;
    }
    for (int idx = tid; idx < kTcWalkersPerStage * Np * 2; idx += kTcThreads) {
      const int s = idx / (Np * 2), rem = idx - s * Np * 2, j = rem >> 1, h = rem & 1;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (s < nw) v = *reinterpret_cast<const uint4*>(yT + ((size_t)(ws + s) * Nf + j0 + j) * 16 + 8 * h);
      const int kc = 2 * s + h;
      *reinterpret_cast<uint4*>(sB + ((j >> 3) * kTcKC + kc) * 128 + (j & 7) * 16) = v;
    }
    // the MMA reads shared memory through the async proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int t = 0; t < kTcWalkersPerStage; ++t) {  // K = 16 per MMA: two 16-byte chunks
        const uint64_t da = smem_desc(aBase + t * 256, 128, sbo);
        const uint64_t db = smem_desc(bBase + t * 256, 128, sbo);
        const uint32_t acc = first ? 0u : 1u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(da), "l"(db), "r"(idesc), "r"(acc)
            : "memory");
        first = false;
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(&mbar))
                   : "memory");
    }
    first = false;
    // everyone waits until the MMAs have read the tiles before they are overwritten; a
    // timed-out wait is made CTA-uniform so that every thread leaves the loop together
    const bool timed_out = !mbar_wait(&mbar, phase);
    phase ^= 1;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (__syncthreads_or(timed_out ? 1 : 0)) {
      ok = false;
      if (tid == 0) atomicExch(flag, 1);
    }
  }

  // accumulator -> FP64 slot (lane = row mu; 32 columns j); rows >= Mp and columns >= Np unused
  if (ok && w1 > w0) {  // ok is CTA-uniform
    const int row = warp * 32 + (tid & 31);
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(tmem + ((uint32_t)(warp * 32) << 16)));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    if (row < Mp) {
      double* slot = slots + ((((size_t)spin * gridDim.z + blockIdx.z) * gridDim.x + blockIdx.x) * 128 + row) * 32;
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (j < Np) slot[j] += (double)__uint_as_float(r[j]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem) : "memory");
}

cudaError_t launch_tc_sumprod(const void* phiT_up, const void* phiT_dn, const void* yT_up, const void* yT_dn, int W,
                              int nch, int Mf, int Nf, int n_up, int n_dn, int grid_x, double* slots, int* flag,
                              cudaStream_t st) {
  if (nch < 1 || Mf < 8 || Nf < 16 || (Nf % 16) != 0 || (Mf % 8) != 0) return cudaErrorInvalidValue;
  const int tiles = ((Mf + 127) / 128) * ((Nf + 31) / 32);
  tc_sumprod_kernel<<<dim3(grid_x, 2, tiles), kTcThreads, 0, st>>>(
      static_cast<const __nv_bfloat16*>(phiT_up), static_cast<const __nv_bfloat16*>(phiT_dn),
      static_cast<const __nv_bfloat16*>(yT_up), static_cast<const __nv_bfloat16*>(yT_dn), W, nch, Mf, Nf, n_up, n_dn,
      slots, flag);
  return cudaGetLastError();
}

}  // namespace vmcf
