// Orbital rows of the walker-group proposal pass on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// Every electron of a walker-group sweep moves once, from its position at the start of the sweep, so the proposal
// pass forms ahead, for every (walker, electron), the row of orbital values of the electron's spin at its proposed
// position, phi_i(r'_e) = sum_mu psi_mu(r'_e) C_{mu i} (App. A, "Computing derivatives": the orbitals are the AOs
// contracted with C). Over the (walker, electron) pairs of one spin these rows are one GEMM,
// [pairs x M] . [M x n_s]. This kernel forms it in tiles of 128 pairs of one spin:
//  - the CTA's warps evaluate the AO values of the tile's pairs (one warp per pair, with the arithmetic of the
//    SIMT pass, so the values are the same) and store them in shared memory as split bf16 pairs
//    hi = bf16(x), lo = bf16(x - hi), already in the MMA operand layout (K-major, no swizzle): the 8 x 16-byte
//    core matrix of rows 8a..8a+7 and AO columns 8g..8g+7 at g (128 x 16) + a 128 bytes;
//  - C^s, split the same way and transposed at system set-up into [part][n_p][K_p] bf16 (part 0 hi, 1 lo, rows
//    beyond n_s and columns beyond M zero), reaches shared memory once per CTA through tensor-map copies
//    (cp.async.bulk.tensor, the TMA engine), one box of 8 AO columns x n_p rows per copy, so that box g lands at
//    g (n_p x 16) bytes: the same core-matrix layout with n_p rows;
//  - one thread issues, per 16 AO columns, tcgen05.mma kind::f16 (M = 128, N = n_p) for hi.hi, hi.lo and lo.hi
//    with the FP32 accumulator in tensor memory and commits them to an mbarrier; the first four warps then read
//    the accumulator (tcgen05.ld, lane = pair) into the proposal buffer.
// Without the lo.lo term and with the lo parts rounded, each product carries a relative error of at most 3 2^-18
// (about 1e-5). The rows feed the Metropolis ratio and the Sherman-Morrison update between FP64 re-inversions;
// the measurement rebuilds the Slater matrix from the positions and never reads them.
//
// Every wait is bounded: a timeout sets the error flag, the waiting thread waits once more (bounded) for the
// copies or MMAs in flight, and the CTA frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "kernels.cuh"
#include "vmcf.h"
#include "vmcf_host.h"

namespace vmcf {

namespace {

constexpr int kRowTile = 128;   // (walker, electron) pairs per tile: the MMA's M
constexpr int kRowWarps = 16;   // warps per CTA; warps 0-3 read the accumulator's 128 lanes
constexpr int kRowThreads = 32 * kRowWarps;
constexpr int kRowsPerWarp = kRowTile / kRowWarps;  // a warp's rows of a tile: warp, warp + kRowWarps, ...

// A pair's proposal and start position, formed once by one lane and read by the warp.
struct PairProp {
  EPos pn, po;
};
constexpr long long kRowSpin = 1LL << 26;  // bounded mbarrier wait (polls)

__device__ __forceinline__ uint32_t s_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// tcgen05 shared-memory matrix descriptor, K-major without swizzle: start >> 4 (bits 0-13), byte offset between
// core matrices adjacent in K >> 4 (16-29), byte offset between core matrices adjacent in M or N >> 4 (32-45),
// descriptor version 1 (46-47).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t k_off, uint32_t mn_off) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((k_off >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((mn_off >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator, A and B bf16, both K-major, N >> 3 at bits 17-22,
// M >> 4 at bits 24-28.
__device__ __forceinline__ uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = s_u32(bar);
  for (long long it = 0; it < kRowSpin; ++it) {
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

__device__ __forceinline__ uint32_t pack_bf16(float a, float b, bool lo_part) {
  __nv_bfloat16 x = __float2bfloat16_rn(a), y = __float2bfloat16_rn(b);
  if (lo_part) {
    x = __float2bfloat16_rn(a - __bfloat162float(x));
    y = __float2bfloat16_rn(b - __bfloat162float(y));
  }
  return (uint32_t)__bfloat16_as_ushort(x) | ((uint32_t)__bfloat16_as_ushort(y) << 16);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

}  // namespace

// grid.x: CTAs per spin (each takes tiles blockIdx.x, blockIdx.x + gridDim.x, ...), grid.y = 2 spins. Pair q of
// spin s is electron e0_s + q mod n_s of walker q / n_s. Dynamic shared memory: A hi and lo (128 x Kp bf16 each),
// C^s hi and lo (Np x Kp bf16 each), one AO row of Kp floats per warp, the proposals of a warp's rows.
__global__ void __launch_bounds__(kRowThreads, 1)
    propose_group_tc(DevSys S, GroupProposeParams P, const __grid_constant__ CUtensorMap mapC, int Kp, int Np,
                     int* flag) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  __shared__ __align__(8) uint64_t bar_c, bar_mma;
  __shared__ uint32_t tmem_base;
  const int spin = blockIdx.y;
  const int n = spin == 0 ? S.nup : S.ndn, e0 = spin == 0 ? 0 : S.nup, Ne = S.Ne;
  const long long items = (long long)P.W * n;
  const long long tiles = (items + kRowTile - 1) / kRowTile;
  if (n == 0 || (long long)blockIdx.x >= tiles) return;  // CTA-uniform, before any tensor memory is held
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const size_t aPart = (size_t)kRowTile * Kp * 2, bPart = (size_t)Np * Kp * 2;
  unsigned char* sAh = dsm;
  unsigned char* sAl = dsm + aPart;
  unsigned char* sBh = dsm + 2 * aPart;
  unsigned char* sBl = sBh + bPart;
  float* aob = reinterpret_cast<float*>(sBh + 2 * bPart) + (size_t)warp * Kp;
  PairProp* pp = reinterpret_cast<PairProp*>(sBh + 2 * bPart + (size_t)kRowWarps * Kp * 4) + warp * kRowsPerWarp;
  const int ncols = Np <= 32 ? 32 : Np <= 64 ? 64 : Np <= 128 ? 128 : 256;
  const int KG = Kp / 8;

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_u32(&bar_c)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_u32(&bar_mma)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_u32(&tmem_base)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  if (tid == 0) {  // C^s, hi and lo parts: one tensor-map copy per 8 AO columns and part
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(
                     s_u32(&bar_c)),
                 "r"((uint32_t)(2 * bPart))
                 : "memory");
    for (int part = 0; part < 2; ++part)
      for (int g = 0; g < KG; ++g)
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
            "[%4];" ::"r"(s_u32((part ? sBl : sBh) + (size_t)g * Np * 16)),
            "l"(reinterpret_cast<uint64_t>(&mapC)), "r"(8 * g), "r"((2 * spin + part) * Np), "r"(s_u32(&bar_c))
            : "memory");
  }

  const uint32_t idesc = idesc_bf16(kRowTile, Np);
  const uint64_t sweep = P.clk ? P.clk->sweep : P.sweep;
  float* prow_base = reinterpret_cast<float*>(P.prow);
  float* dchi = reinterpret_cast<float*>(P.pdchi);
  int bad = 0, c_wait_failed = 0, mma_wait_failed = 0;
  uint32_t phase = 0;
  for (long long t = blockIdx.x; t < tiles; t += gridDim.x) {
    // the proposals of the warp's rows, one lane per pair (the FP64 arithmetic of a proposal runs once per pair,
    // not once per lane: an FP64 instruction takes the pipe for a whole warp whatever its active lanes), with the
    // arithmetic of the SIMT pass
    if (lane < kRowsPerWarp) {
      const long long q = t * kRowTile + warp + lane * kRowWarps;
      if (q < items) {
        const int w = (int)(q / n), e = e0 + (int)(q - (long long)w * n);
        const long long it = (long long)w * Ne + e;
        const uint64_t wid = P.wid0 + (uint64_t)w;
        uint64_t rr[4] = {wid, sweep, (uint64_t)e, 0};
        philox4x64_10(rr, P.k0, P.k1);
        double xi[3];
        normals3(rr, xi, 0.0f);
        double po3[3], rn[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          po3[k] = P.pos[(size_t)it * 3 + k];
          rn[k] = po3[k] + P.sigma * xi[k];
          P.prn[(size_t)it * 3 + k] = rn[k];
        }
        pp[lane].pn = make_epos(rn);
        pp[lane].po = make_epos(po3);
        uint64_t r2[4] = {wid, sweep, (uint64_t)e, 1};
        philox4x64_10(r2, P.k0, P.k1);
        P.pu[it] = u01(r2[0]);
      }
    }
    __syncwarp();
    // the tile's AO rows, split into the A operand, and the electron-nucleus Jastrow changes
    for (int j = 0; j < kRowsPerWarp; ++j) {
      const int r = warp + j * kRowWarps;
      const long long q = t * kRowTile + r;
      if (q < items) {  // warp-uniform
        const int w = (int)(q / n), e = e0 + (int)(q - (long long)w * n);
        const long long it = (long long)w * Ne + e;
        const EPos pn = pp[j].pn;
        const EPos po = pp[j].po;
        ao_point<float, 32, 0, false>(S, pn, aob, 0);
        __syncwarp();
        for (int g = lane; g < KG; g += 32) {
          float x[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) x[i] = 8 * g + i < S.M ? aob[8 * g + i] : 0.0f;
          const size_t off = (size_t)g * (kRowTile * 16) + (size_t)r * 16;
          *reinterpret_cast<uint4*>(sAh + off) = make_uint4(pack_bf16(x[0], x[1], false), pack_bf16(x[2], x[3], false),
                                                            pack_bf16(x[4], x[5], false), pack_bf16(x[6], x[7], false));
          *reinterpret_cast<uint4*>(sAl + off) = make_uint4(pack_bf16(x[0], x[1], true), pack_bf16(x[2], x[3], true),
                                                            pack_bf16(x[4], x[5], true), pack_bf16(x[6], x[7], true));
        }
        const float en = en_change_warp<float>(S, pn, po, lane);
        if (lane == 0) dchi[it] = en;
        __syncwarp();  // the AO row buffer is reused for the warp's next pair
      } else {         // rows past the last pair: zero (their accumulator lanes are never read)
        for (int g = lane; g < KG; g += 32) {
          const size_t off = (size_t)g * (kRowTile * 16) + (size_t)r * 16;
          *reinterpret_cast<uint4*>(sAh + off) = make_uint4(0u, 0u, 0u, 0u);
          *reinterpret_cast<uint4*>(sAl + off) = make_uint4(0u, 0u, 0u, 0u);
        }
      }
    }
    // the generic-proxy stores above are read by the tensor cores (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) {
      if (t == (long long)blockIdx.x && !bar_wait(&bar_c, 0)) c_wait_failed = 1;
      if (!c_wait_failed) {
        for (int s = 0; s < Kp / 16; ++s) {
          const uint32_t ka = 2u * s * (kRowTile * 16), kb = 2u * s * (uint32_t)(Np * 16);
          const uint64_t ah = sdesc(s_u32(sAh) + ka, kRowTile * 16, 128);
          const uint64_t al = sdesc(s_u32(sAl) + ka, kRowTile * 16, 128);
          const uint64_t bh = sdesc(s_u32(sBh) + kb, Np * 16, 128);
          const uint64_t bl = sdesc(s_u32(sBl) + kb, Np * 16, 128);
          mma_bf16(tmem, ah, bh, idesc, s > 0 ? 1u : 0u);
          mma_bf16(tmem, ah, bl, idesc, 1u);
          mma_bf16(tmem, al, bh, idesc, 1u);
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         s_u32(&bar_mma))
                     : "memory");
      } else {  // no MMA issued: complete the phase so that no thread waits for it
        asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(s_u32(&bar_mma))
                     : "memory");
      }
    }
    // the MMAs have read the tile and written the accumulator once the phase completes
    const bool done = bar_wait(&bar_mma, phase);
    if (!done && tid == 0) mma_wait_failed = 1;
    phase ^= 1u;
    if (__syncthreads_or(!done || c_wait_failed)) {  // CTA-uniform
      bad = 1;
      break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp < 4) {  // accumulator lane = pair 32 warp + lane of the tile, column = orbital
      const int row = 32 * warp + lane;
      const long long q = t * kRowTile + row;
      const bool valid = q < items;
      float* prow = nullptr;
      if (valid) {
        const int w = (int)(q / n), e = e0 + (int)(q - (long long)w * n);
        prow = prow_base + ((long long)w * Ne + e) * S.nmax;
      }
      for (int c0 = 0; c0 < Np; c0 += 16) {
        uint32_t v[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
            "%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (valid) {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (c0 + j < n) prow[c0 + j] = __uint_as_float(v[j]);
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  if (tid == 0) {  // after a timeout, let the copies or MMAs in flight land before the memory is released
    if (c_wait_failed) bar_wait(&bar_c, 0);
    if (mma_wait_failed) bar_wait(&bar_mma, phase ^ 1u);
    if (bad) atomicExch(flag, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

namespace {

// bf16 of a finite float, rounded to nearest even, and back
uint16_t bf16_rn_host(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}
float bf16_to_float_host(uint16_t h) {
  const uint32_t u = (uint32_t)h << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

size_t tc_rows_smem(int Kp, int Np) {
  return 2 * (size_t)kRowTile * Kp * 2 + 2 * (size_t)Np * Kp * 2 + (size_t)kRowWarps * Kp * 4 +
         (size_t)kRowWarps * kRowsPerWarp * sizeof(PairProp);
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

}  // namespace

// The split, transposed coefficients [spin][part][Np][Kp] bf16 from the system's C (float values, as the SIMT
// pass uses), uploaded into the system's buffer.
int tc_rows_upload(vmcf_system_s* s) {
  if (!s->tcr_mem) return VMCF_OK;
  const int Kp = s->tcr_Kp, Np = s->tcr_Np, M = s->M;
  std::vector<uint16_t> ct((size_t)4 * Np * Kp, 0);
  for (int sg = 0; sg < 2; ++sg) {
    const int n = sg == 0 ? s->nup : s->ndn;
    for (int mu = 0; mu < M; ++mu)
      for (int i = 0; i < n; ++i) {
        const float c = (float)s->C[sg][(size_t)mu * n + i];
        const uint16_t h = bf16_rn_host(c);
        const uint16_t l = bf16_rn_host(c - bf16_to_float_host(h));
        ct[((size_t)(2 * sg) * Np + i) * Kp + mu] = h;
        ct[((size_t)(2 * sg + 1) * Np + i) * Kp + mu] = l;
      }
  }
  cudaError_t e = cudaMemcpy(s->tcr_mem, ct.data(), 2 * ct.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return set_last_error(VMCF_ECUDA, std::string("uploading split coefficients: ") + cudaGetErrorString(e));
  return VMCF_OK;
}

// Plan, buffer and tensor map of the tensor-core orbital rows (mixed precision, walker-group kernels), at system
// set-up. A system whose tile does not fit shared memory keeps the SIMT proposal pass.
int tc_rows_setup(vmcf_system_s* s) {
  s->tc_rows = false;
  if (s->precision != VMCF_MIXED || s->small) return VMCF_OK;
  const int Kp = (s->M + 15) / 16 * 16, Np = (s->nmax + 15) / 16 * 16;
  const size_t smem = tc_rows_smem(Kp, Np);
  // The kernel's dynamic shared-memory limit is one setting for the whole process, shared by every system (a
  // batch launches several systems' tiles): it is set to the device's largest, not to this system's size.
  int dev = 0, sms = 0, optin = 0;
  cudaFuncAttributes fa{};
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, propose_group_tc);
  if (e != cudaSuccess) return set_last_error(VMCF_ECUDA, std::string("device attributes: ") + cudaGetErrorString(e));
  const int lim = optin - (int)fa.sharedSizeBytes;
  if (Np > 256 || lim <= 0 || smem > (size_t)lim) return VMCF_OK;  // the tile does not fit: the SIMT pass
  if ((e = cudaFuncSetAttribute(propose_group_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)) != cudaSuccess)
    return set_last_error(VMCF_ECUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
  s->tcr_Kp = Kp;
  s->tcr_Np = Np;
  s->tcr_smem = smem;
  s->tcr_grid = std::max(1, sms / 2);  // one CTA per SM (shared memory) over both spins: one wave
  const size_t cbytes = (size_t)4 * Np * Kp * 2;
  if ((e = cudaMalloc(&s->tcr_mem, cbytes + 256)) != cudaSuccess)
    return set_last_error(VMCF_ECUDA, std::string("cudaMalloc(split coefficients): ") + cudaGetErrorString(e));
  s->tcr_flag = reinterpret_cast<int*>(static_cast<char*>(s->tcr_mem) + cbytes);
  if ((e = cudaMemset(s->tcr_flag, 0, sizeof(int))) != cudaSuccess)
    return set_last_error(VMCF_ECUDA, std::string("cudaMemset: ") + cudaGetErrorString(e));
  int rc = tc_rows_upload(s);
  if (rc != VMCF_OK) return rc;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q{};
  e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
  if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
    return set_last_error(VMCF_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
  CUtensorMap map;
  const cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)4 * Np};
  const cuuint64_t strides[1] = {(cuuint64_t)Kp * 2};
  const cuuint32_t box[2] = {8, (cuuint32_t)Np};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult cr = reinterpret_cast<EncodeTiled>(fn)(
      &map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, s->tcr_mem, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
      CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) return set_last_error(VMCF_ECUDA, "cuTensorMapEncodeTiled failed for the split coefficients");
  static_assert(sizeof(map) == sizeof(s->tcr_map), "tensor map size");
  std::memcpy(s->tcr_map, &map, sizeof(map));
  s->tc_rows = true;
  return VMCF_OK;
}

// The proposal pass of a walker-group sweep: FP64 SIMT in FP64 mode; in mixed mode the tensor-core rows when the
// system has them switched on, else the FP32 SIMT pass.
cudaError_t launch_propose_rows(const vmcf_system_s& s, const GroupProposeParams& P, cudaStream_t st) {
  if (s.precision == VMCF_FP64) return launch_propose_group<double>(s.dev, P, st);
  if (!s.tc_rows || !s.tcr_mem) return launch_propose_group<float>(s.dev, P, st);
  if (P.W == 0) return cudaSuccess;
  const long long items = (long long)P.W * std::max(s.nup, s.ndn);
  const long long tiles = (items + kRowTile - 1) / kRowTile;
  const int grid = (int)std::min<long long>(tiles, s.tcr_grid);
  CUtensorMap map;
  std::memcpy(&map, s.tcr_map, sizeof(map));
  propose_group_tc<<<dim3(grid, 2), kRowThreads, s.tcr_smem, st>>>(s.dev, P, map, s.tcr_Kp, s.tcr_Np, s.tcr_flag);
  return cudaGetLastError();
}

}  // namespace vmcf
