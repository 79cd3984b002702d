// Walker sums of O on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// For one spin block, the walker-weighted orbital-coefficient sums of App. A (Eq. fc-vmc-eval)
//   S[mu][j] = sum over walkers w of the block, electrons el of the spin:
//              psi_mu(r_{w,el}) * Y_{w,el,j},   Y = [B_{i,el} (j < n) | c_w B_{i,el} (n <= j < 2n)]
// are one GEMM with K = walkers x electron slots: D[mu][j] = sum_k PhiT[mu][k] Y[k][j]. The
// measurement kernels write, per walker and chunk of 16 electron slots, PhiT as Mf rows and YT as
// Nf rows of 16 bf16 (slots beyond n, rows beyond M and columns beyond 2n are zero), each chunk
// already in the tensor cores' K-major layout without swizzle: 8-row x 16-byte core matrices, the
// core of electron slots 8..15 at +128 bytes from that of slots 0..7 (leading byte offset), the next
// 8 rows at +256 bytes (stride byte offset). Element (row r, slot k) of a chunk is at bf16 index
// tc_tile_index(r, k). A chunk's rows [r0, r0 + R) are then R x 32 contiguous bytes, so a chunk
// reaches shared memory in one bulk asynchronous copy (TMA engine) and is one MMA operand as is.
//
// A CTA owns a range of walkers inside one jackknife block, one spin and one 128 x 32 tile of D,
// keeps the tile (FP32) in tensor memory across the whole range, and adds it to its FP64 slot at the
// end. One thread runs a ring of kTcStages shared-memory stages: bulk copies of kTcCPS chunks per
// stage complete on the stage's "full" mbarrier; the stage's MMAs (K = 16 each) are committed to its
// "empty" mbarrier, which the thread waits on before refilling that stage, one stage behind the
// MMAs it has just issued, so copies of later stages overlap the MMAs. Every wait is bounded: a
// timeout sets the error flag, the thread waits (again bounded) for its copies and MMAs in flight,
// and the CTA skips the read-out, frees its tensor memory and returns.
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>

#include "vmcf_internal.h"

namespace vmcf {

namespace {

constexpr int kTcThreads = 128;  // 4 warps; warps 0-3 read TMEM lanes 0-127 at the end
constexpr int kTcCPS = 4;        // chunks (K = 16 each) per stage
constexpr int kTcStages = 4;     // stages in the ring
constexpr int kTcPad = 4096;     // an MMA reads 128 A rows (32 rows of B) from a chunk's start: the
                                 // rows past a chunk's own (past the tile's M or N) land in the next
                                 // chunk or in this pad, and only feed D rows/columns never read
constexpr long long kSpinLimit = 1LL << 26;  // bounded mbarrier wait

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

// Arrive once on the barrier and add `bytes` to the transaction count its phase waits for.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// Bulk asynchronous copy global -> shared (16-byte aligned addresses, size a multiple of 16),
// completing `bytes` transactions on the barrier.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

}  // namespace

// grid.x = nblocks * cpb CTAs (walker ranges), grid.y = 2 spins, grid.z = output tiles of 128 AO
// rows x 32 Y columns (z = mt * Nt + nt). Each walker holds nch chunks of 16 electron slots:
// PhiT[s]: [W][nch] chunks of Mf x 16 bf16, YT[s]: [W][nch] chunks of Nf x 16 bf16, both in the
// layout of tc_tile_index. slots: [2][gridDim.z][gridDim.x][128][32] FP64, added to. flag: set to 1
// on a timed-out wait. Dynamic shared memory: tc_sumprod_smem(Mp, Np) for the tile's row counts.
__global__ void __launch_bounds__(kTcThreads, 1)
    tc_sumprod_kernel(const __nv_bfloat16* __restrict__ phiT_up, const __nv_bfloat16* __restrict__ phiT_dn,
                      const __nv_bfloat16* __restrict__ yT_up, const __nv_bfloat16* __restrict__ yT_dn, int W, int nch,
                      int Mf, int Nf, int n_up, int n_dn, double* __restrict__ slots, int* flag) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  __shared__ __align__(8) uint64_t full[kTcStages], empty[kTcStages], done;
  __shared__ uint32_t tmem_base;
  const int spin = blockIdx.y;
  if ((spin == 0 ? n_up : n_dn) == 0) return;
  const unsigned char* phiT = reinterpret_cast<const unsigned char*>(spin == 0 ? phiT_up : phiT_dn);
  const unsigned char* yT = reinterpret_cast<const unsigned char*>(spin == 0 ? yT_up : yT_dn);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int Nt = (Nf + 31) / 32, mt = blockIdx.z / Nt, nt = blockIdx.z - mt * Nt;
  const int m0 = 128 * mt, j0 = 32 * nt;
  const int Mp = Mf - m0 < 128 ? Mf - m0 : 128, Np = Nf - j0 < 32 ? Nf - j0 : 32;  // rows of this tile
  // the CTA's walkers (never split between CTAs, so a jackknife block keeps whole walkers), as a
  // range of chunks
  const long long q0 = (long long)nch * ((long long)W * blockIdx.x / gridDim.x);
  const long long q1 = (long long)nch * ((long long)W * (blockIdx.x + 1) / gridDim.x);
  const int nst = (int)((q1 - q0 + kTcCPS - 1) / kTcCPS);
  // stage b, chunk c: A rows at sA + (b kTcCPS + c) aSlot, B rows at sB + (b kTcCPS + c) bSlot
  const uint32_t aSlot = 32u * Mp, bSlot = 32u * Np;
  unsigned char* sA = dsm;
  unsigned char* sB = dsm + (size_t)kTcStages * kTcCPS * aSlot;
  const unsigned char* gA = phiT + (size_t)m0 * 32;  // rows m0.. of chunk 0
  const unsigned char* gB = yT + (size_t)j0 * 32;
  const size_t aChunk = (size_t)Mf * 32, bChunk = (size_t)Nf * 32;

  if (tid == 0) {
    for (int b = 0; b < kTcStages; ++b) {
      mbar_init(&full[b], 1);
      mbar_init(&empty[b], 1);
    }
    mbar_init(&done, 1);
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

  int bad = 0;
  if (tid == 0) {
    const uint32_t idesc = instr_desc_bf16(128, 32);
    auto chunks_of = [&](int s) {
      const long long c0 = q0 + (long long)s * kTcCPS;
      return (int)(q1 - c0 < kTcCPS ? q1 - c0 : kTcCPS);
    };
    auto load = [&](int s) {  // stage s into ring slot s % kTcStages
      const int b = s % kTcStages, nc = chunks_of(s);
      const long long c0 = q0 + (long long)s * kTcCPS;
      mbar_arrive_expect_tx(&full[b], (uint32_t)nc * (aSlot + bSlot));
      for (int c = 0; c < nc; ++c) {
        bulk_g2s(sA + (size_t)(b * kTcCPS + c) * aSlot, gA + (size_t)(c0 + c) * aChunk, aSlot, &full[b]);
        bulk_g2s(sB + (size_t)(b * kTcCPS + c) * bSlot, gB + (size_t)(c0 + c) * bChunk, bSlot, &full[b]);
      }
    };
    int loaded = 0, consumed = 0;  // stages whose copies were issued / waited for
    for (; loaded < nst && loaded < kTcStages; ++loaded) load(loaded);
    for (int s = 0; s < nst; ++s) {
      const int b = s % kTcStages;
      if (!mbar_wait(&full[b], (uint32_t)(s / kTcStages) & 1u)) {
        bad = 1;
        break;
      }
      consumed = s + 1;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int nc = chunks_of(s);
      for (int c = 0; c < nc; ++c) {
        const uint64_t da = smem_desc(smem_u32(sA + (size_t)(b * kTcCPS + c) * aSlot), 128, 256);
        const uint64_t db = smem_desc(smem_u32(sB + (size_t)(b * kTcCPS + c) * bSlot), 128, 256);
        const uint32_t acc = (s | c) != 0 ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(da), "l"(db), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&empty[b]))
                   : "memory");
      // refill the previous stage's slot once its MMAs have read it (they were issued a stage ago)
      if (s >= 1 && loaded < nst) {
        const int pb = (s - 1) % kTcStages;
        if (!mbar_wait(&empty[pb], (uint32_t)((s - 1) / kTcStages) & 1u)) {
          bad = 1;
          break;
        }
        load(loaded++);
      }
    }
    // copies issued but not waited for (only after a timeout) must land before the CTA exits
    for (int s = consumed; s < loaded; ++s) mbar_wait(&full[s % kTcStages], (uint32_t)(s / kTcStages) & 1u);
    // every MMA issued by this thread has completed once `done` flips
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(&done))
                 : "memory");
    if (!mbar_wait(&done, 0)) bad = 1;
    if (bad) atomicExch(flag, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  const bool ok = __syncthreads_or(bad) == 0;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  // accumulator -> FP64 slot (lane = row mu; 32 columns j); rows >= Mp and columns >= Np unused
  if (ok && nst > 0) {  // CTA-uniform
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

// Dynamic shared memory of a CTA whose tile has Mp A rows and Np B rows (at most 128 and 32).
static size_t tc_sumprod_smem(int Mp, int Np) {
  return (size_t)kTcStages * kTcCPS * 32 * (Mp + Np) + kTcPad;
}

cudaError_t set_smem_limits_tc() {
  cudaError_t e = cudaFuncSetAttribute(tc_sumprod_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)tc_sumprod_smem(128, 32));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tc_sumprod_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  return e;
}

// CTAs of the walker-sum kernel resident per SM for a launch over tiles of at most Mf x Nf, from the kernel's
// registers and shared memory against the SM's (the kernel is always launched with the largest shared-memory
// carve-out, which set_smem_limits_tc requests).
cudaError_t tc_sumprod_ctas_per_sm(int Mf, int Nf, int* n) {
  const size_t smem = tc_sumprod_smem(Mf < 128 ? Mf : 128, Nf < 32 ? Nf : 32);
  cudaFuncAttributes fa{};
  int dev = 0, smem_sm = 0, reserved = 0, regs_sm = 0, thr_sm = 0;
  cudaError_t e = cudaFuncGetAttributes(&fa, tc_sumprod_kernel);
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
  if (e != cudaSuccess) return e;
  const size_t per_cta = smem + fa.sharedSizeBytes + (size_t)reserved;
  const int by_smem = (int)((size_t)smem_sm / per_cta);
  const int by_regs = fa.numRegs > 0 ? regs_sm / (fa.numRegs * kTcThreads) : by_smem;
  const int by_thr = thr_sm / kTcThreads;
  int v = by_smem < by_regs ? by_smem : by_regs;
  v = v < by_thr ? v : by_thr;
  *n = v > 0 ? v : 1;
  return cudaSuccess;
}

cudaError_t launch_tc_sumprod(const void* phiT_up, const void* phiT_dn, const void* yT_up, const void* yT_dn, int W,
                              int nch, int Mf, int Nf, int n_up, int n_dn, int grid_x, double* slots, int* flag,
                              cudaStream_t st) {
  if (nch < 1 || Mf < 8 || Nf < 16 || (Nf % 16) != 0 || (Mf % 8) != 0) return cudaErrorInvalidValue;
  const int tiles = ((Mf + 127) / 128) * ((Nf + 31) / 32);
  // every tile's ring fits the largest (128 x 32) tile's size
  const size_t smem = tc_sumprod_smem(Mf < 128 ? Mf : 128, Nf < 32 ? Nf : 32);
  tc_sumprod_kernel<<<dim3(grid_x, 2, tiles), kTcThreads, smem, st>>>(
      static_cast<const __nv_bfloat16*>(phiT_up), static_cast<const __nv_bfloat16*>(phiT_dn),
      static_cast<const __nv_bfloat16*>(yT_up), static_cast<const __nv_bfloat16*>(yT_dn), W, nch, Mf, Nf, n_up, n_dn,
      slots, flag);
  return cudaGetLastError();
}

}  // namespace vmcf
