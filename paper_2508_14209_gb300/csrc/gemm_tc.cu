// gemm_tc.cu — the Gaussian stage Z = G Y on the 5th-generation tensor cores
// (tcgen05, kind::f16, FP32 accumulation in tensor memory), the only dense
// contraction of the multisketch (Section 1 "Count-Gauss"; the paper runs it
// as a cuBLAS GEMM, Section 6.1).
//
// Operands (both K-major, bf16 or fp16):
//   A = G, p x k row-major, generated directly in the 16-bit type;
//   B = Y^T split into PARTS 16-bit parts, Yt[t][n][k]:
//     PARTS = 1 for BF16 / F16 (Y rounded once);
//     PARTS = 3 for BF16X3: Y = Y1 + Y2 + Y3 exactly up to 2^-24 |Y|, each
//     Yt a bfloat16 rounding of what the previous parts left (Henry, Tang,
//     Heinecke, ARITH 2019); G is exactly bfloat16, so every product is exact
//     and the three MMAs accumulate into one FP32 accumulator.
// Tiling: a CTA owns a 128 x NT tile of Z and a slice of the K tiles (split-K:
// the output is tiny, K = k is long).  Warp 0 (one lane) streams 128x64 A tiles
// and NTx64 B tiles with TMA (128-byte swizzle) through a ring of shared-memory
// stages; warp 1 (one lane) issues tcgen05.mma (K = 16 per instruction, four
// per 64-wide K tile, times PARTS) into a TMEM accumulator and frees each stage
// with tcgen05.commit; all four warps then read the accumulator back with
// tcgen05.ld and write FP32 partial tiles, which a second kernel sums in FP64
// in a fixed order.  Every mbarrier wait is bounded (1 s): on expiry the kernel
// records a timeout flag, waits (bounded) for its own copies in flight, frees
// its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "msk_device.cuh"
#include "msk_internal.h"
#include "msk_tc.cuh"

namespace msk {

__device__ int g_tc_timeout = 0;  // set by a tensor-core kernel whose bounded wait expired

constexpr int kTcBM = 128;       // M per CTA (one UMMA M)
constexpr int kTcBK = 64;        // K per stage: 64 x 2 bytes = one 128-byte swizzle row
constexpr int kTcThreads = 128;  // 4 warps
// Instruction descriptor of kind::f16 with FP32 accumulation, K-major A and B:
// bits 4-5 D format (1 = F32), 7-9 A format, 10-12 B format (0 = F16,
// 1 = BF16), 17-22 N >> 3, 24-28 M >> 4.
static uint32_t make_idesc(int M, int N, bool bf16) {
  return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

template <int PARTS>
__global__ void __launch_bounds__(kTcThreads, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   int p, int ncol, int NT, int KT, int kt_per, int stages, uint32_t idesc,
                   float* __restrict__ part) {
  extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t a_bytes = kTcBM * kTcBK * 2;
  const uint32_t b_bytes = (uint32_t)NT * kTcBK * 2;
  const uint32_t stage_bytes = a_bytes + PARTS * b_bytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)stages * stage_bytes);
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bars + 2 * stages + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * kTcBM, n0 = blockIdx.y * NT;
  const int kt0 = blockIdx.z * kt_per;
  const int nk = min(KT, kt0 + kt_per) - kt0;
  const uint32_t tmem_cols = NT <= 32 ? 32u : NT <= 64 ? 64u : NT <= 128 ? 128u : 256u;

  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(smem_u32(&bars[s]), 1);
      mbar_init(smem_u32(&bars[stages + s]), 1);
    }
    mbar_init(smem_u32(&bars[2 * stages]), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_holder)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  if (warp == 0 && lane == 0) {
    // TMA producer
    int issued = 0;
    for (int it = 0; it < nk; ++it) {
      const int s = it % stages;
      if (it >= stages && !mbar_wait(smem_u32(&bars[stages + s]), ((it / stages) & 1) ^ 1, &g_tc_timeout)) {
        *abort_flag = 1;
        break;
      }
      if (*abort_flag) break;
      const uint32_t full = smem_u32(&bars[s]);
      mbar_expect_tx(full, stage_bytes);
      unsigned char* st = smem + (size_t)s * stage_bytes;
      const int kc = (kt0 + it) * kTcBK;
      tma_load_2d(smem_u32(st), &tmA, kc, m0, full);
#pragma unroll
      for (int t = 0; t < PARTS; ++t)
        tma_load_3d(smem_u32(st + a_bytes + t * b_bytes), &tmB, kc, n0, t, full);
      ++issued;
    }
    if (*abort_flag) {
      // let this CTA's copies in flight land before leaving (bounded waits)
      for (int it = (issued > stages ? issued - stages : 0); it < issued; ++it)
        mbar_wait(smem_u32(&bars[it % stages]), (it / stages) & 1, &g_tc_timeout);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    for (int it = 0; it < nk; ++it) {
      const int s = it % stages;
      if (!mbar_wait(smem_u32(&bars[s]), (it / stages) & 1, &g_tc_timeout)) {
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      const uint32_t a_base = smem_u32(smem + (size_t)s * stage_bytes);
#pragma unroll
      for (int kk = 0; kk < kTcBK / 16; ++kk) {
        const uint64_t ad = sw128_desc(a_base + kk * 32);
#pragma unroll
        for (int t = 0; t < PARTS; ++t) {
          const uint64_t bd = sw128_desc(a_base + a_bytes + t * b_bytes + kk * 32);
          umma_f16(tmem, ad, bd, idesc, (it > 0 || kk > 0 || t > 0) ? 1u : 0u);
        }
      }
      umma_commit(smem_u32(&bars[stages + s]));
    }
    umma_commit(smem_u32(&bars[2 * stages]));
  }
  __syncwarp();
  // epilogue: TMEM lane (warp*32 + lane) holds row m0 + warp*32 + lane
  const bool done = mbar_wait(smem_u32(&bars[2 * stages]), 0, &g_tc_timeout);
  tc_fence_after();
  // tcgen05.ld is warp-collective: take the decision per warp
  if (__all_sync(0xffffffffu, done && !*abort_flag && nk > 0)) {
    const int row = m0 + warp * 32 + lane;
    float* out = part + (int64_t)blockIdx.z * p * ncol;
    for (int c0 = 0; c0 < NT; c0 += 16) {
      uint32_t v[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int col = n0 + c0 + q;
        if (row < p && col < ncol) out[(int64_t)col * p + row] = __uint_as_float(v[q]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols)
                 : "memory");
}

// ---------------------------------------------------------------------------
// BF16X3 with per-K-tile draining.  A single FP32 accumulator over a CTA's
// whole K slice loses about sqrt(C/2) ulps over a chain of C products
// (C ~ 4e4 here), which made R too inexact to precondition kappa(A) ~ 1e8.
// So the MMA warp restarts the accumulator every 64-wide K tile (C = 192 exact
// products) in one of two TMEM buffers, and 16 drain warps read each finished
// buffer (tcgen05.ld) and add it into double-single registers (hi + lo binary32
// pairs, TwoSum), while the MMA warp fills the other buffer.  Drain warp w
// covers TMEM lanes 32 (w mod 4) .. +31 and a quarter of the NT columns.
// Per-CTA results are written as FP64 partials.
constexpr int kDsDrainWarps = 16;
constexpr int kDsThreads = (2 + kDsDrainWarps) * 32;
constexpr int kDsMaxCpw = 24;  // columns per drain warp (NT <= 96): keeps hi/lo in registers

// One CTA's tile (mt, nt) and K slice sidx of one problem.  tmA / tmB point
// at tensor maps in parameter or global memory.
__device__ __forceinline__ void tc_ds_body(const CUtensorMap* tmA, const CUtensorMap* tmB, int p,
                                           int ncol, int NT, int KT, int kt_per, int stages,
                                           uint32_t idesc, double* __restrict__ part, int mt,
                                           int nt, int sidx) {
  constexpr int PARTS = 3;
  extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t a_bytes = kTcBM * kTcBK * 2;
  const uint32_t b_bytes = (uint32_t)NT * kTcBK * 2;
  const uint32_t stage_bytes = a_bytes + PARTS * b_bytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)stages * stage_bytes);
  // bars: full[stages], empty[stages], accf[2], acce[2]
  uint64_t* accf = bars + 2 * stages;
  uint64_t* acce = accf + 2;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(acce + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = mt * kTcBM, n0 = nt * NT;
  const int kt0 = sidx * kt_per;
  const int nk = min(KT, kt0 + kt_per) - kt0;
  constexpr uint32_t kCols = 512;  // two accumulator buffers at columns 0 and 256

  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(smem_u32(&bars[s]), 1);
      mbar_init(smem_u32(&bars[stages + s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&accf[b]), 1);
      mbar_init(smem_u32(&acce[b]), kDsDrainWarps);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_holder)),
                 "r"(kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  if (warp == 0) {
    if (lane == 0) {
      int issued = 0;
      for (int it = 0; it < nk; ++it) {
        const int s = it % stages;
        if (it >= stages && !mbar_wait(smem_u32(&bars[stages + s]), ((it / stages) & 1) ^ 1, &g_tc_timeout)) {
          *abort_flag = 1;
          break;
        }
        if (*abort_flag) break;
        const uint32_t full = smem_u32(&bars[s]);
        mbar_expect_tx(full, stage_bytes);
        unsigned char* st = smem + (size_t)s * stage_bytes;
        const int kc = (kt0 + it) * kTcBK;
        tma_load_2d(smem_u32(st), tmA, kc, m0, full);
#pragma unroll
        for (int t = 0; t < PARTS; ++t)
          tma_load_3d(smem_u32(st + a_bytes + t * b_bytes), tmB, kc, n0, t, full);
        ++issued;
      }
      if (*abort_flag)
        for (int it = (issued > stages ? issued - stages : 0); it < issued; ++it)
          mbar_wait(smem_u32(&bars[it % stages]), (it / stages) & 1, &g_tc_timeout);
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      for (int it = 0; it < nk; ++it) {
        const int s = it % stages;
        const int b = it & 1, u = it >> 1;
        if (u >= 1 && !mbar_wait(smem_u32(&acce[b]), (u - 1) & 1, &g_tc_timeout)) {
          *abort_flag = 1;
          break;
        }
        if (!mbar_wait(smem_u32(&bars[s]), (it / stages) & 1, &g_tc_timeout)) {
          *abort_flag = 1;
          break;
        }
        tc_fence_after();
        const uint32_t a_base = smem_u32(smem + (size_t)s * stage_bytes);
        const uint32_t d = tmem + (uint32_t)b * 256u;
#pragma unroll
        for (int kk = 0; kk < kTcBK / 16; ++kk) {
          const uint64_t ad = sw128_desc(a_base + kk * 32);
#pragma unroll
          for (int t = 0; t < PARTS; ++t) {
            const uint64_t bd = sw128_desc(a_base + a_bytes + t * b_bytes + kk * 32);
            umma_f16(d, ad, bd, idesc, (kk > 0 || t > 0) ? 1u : 0u);
          }
        }
        umma_commit(smem_u32(&bars[stages + s]));
        umma_commit(smem_u32(&accf[b]));
      }
    }
    __syncwarp();
  } else {
    // drain warps
    const int dw = warp - 2;
    const int quad = warp & 3;
    const int cpw = NT / 4;
    const int c_begin = (dw >> 2) * cpw;
    float hi[kDsMaxCpw], lo[kDsMaxCpw];
#pragma unroll
    for (int c = 0; c < kDsMaxCpw; ++c) {
      hi[c] = 0.f;
      lo[c] = 0.f;
    }
    bool ok = true;
    for (int it = 0; it < nk; ++it) {
      const int b = it & 1, u = it >> 1;
      const bool got = mbar_wait(smem_u32(&accf[b]), u & 1, &g_tc_timeout);
      if (!__all_sync(0xffffffffu, got && !*abort_flag)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t base = tmem + (uint32_t)b * 256u + ((uint32_t)(quad * 32) << 16) + (uint32_t)c_begin;
#pragma unroll
      for (int c = 0; c < kDsMaxCpw; c += 4) {
        if (c < cpw) {
          uint32_t v[4];
          tmem_ld4(base + (uint32_t)c, v);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int q = 0; q < 4; ++q) ds_accum(hi[c + q], lo[c + q], __uint_as_float(v[q]));
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&acce[b]));
    }
    if (ok && nk > 0) {
      const int row = m0 + quad * 32 + lane;
      double* out = part + (int64_t)sidx * p * ncol;
#pragma unroll
      for (int c = 0; c < kDsMaxCpw; ++c) {
        const int col = n0 + c_begin + c;
        if (c < cpw && row < p && col < ncol)
          out[(int64_t)col * p + row] = (double)hi[c] + (double)lo[c];
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols)
                 : "memory");
}

__global__ void __launch_bounds__(kDsThreads, 1)
    tc_gemm_ds_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                      int p, int ncol, int NT, int KT, int kt_per, int stages, uint32_t idesc,
                      double* __restrict__ part) {
  tc_ds_body(&tmA, &tmB, p, ncol, NT, KT, kt_per, stages, idesc, part, blockIdx.x, blockIdx.y,
             blockIdx.z);
}

// Batched form: CTA b takes work item b; jobs[j] covers items
// [jobs[j].item_begin, jobs[j + 1].item_begin) in (s, nt, mt) order.  The
// tensor maps live in global memory (64-byte aligned inside TcJob); the
// producer thread acquires them for the tensor-map proxy before the first TMA.
__global__ void __launch_bounds__(kDsThreads, 1)
    tc_gemm_ds_batch_kernel(const TcJob* __restrict__ jobs, int njobs, int stages) {
  int lo = 0, hi = njobs - 1;
  const int b = blockIdx.x;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].item_begin <= b) lo = mid; else hi = mid - 1;
  }
  const TcJob& J = jobs[lo];
  MSK_CHECK_OR(J.item_begin <= b, kCheckBatch, return);
  const int local = b - J.item_begin;
  const int mt = local % J.Mt, nt = (local / J.Mt) % J.Nt, sidx = local / (J.Mt * J.Nt);
  if (threadIdx.x == 0) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&J.mapA) : "memory");
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&J.mapB) : "memory");
  }
  tc_ds_body(&J.mapA, &J.mapB, J.p, J.ncol, J.NT, J.KT, J.kt_per, stages, J.idesc, J.part, mt, nt,
             sidx);
}

// Yt[t][n][kk] (row pitch kpitch) from the FP32 row-major Y (k x ncol, ldy):
// PARTS = 1: round once (bf16 or fp16); PARTS = 3: bf16 split of the residues.
// Rows n >= ncol (up to npad) are zero.  32x32 tiles transposed in shared memory.
template <int PARTS, bool BF16>
__global__ void split_transpose_kernel(const float* __restrict__ Y, int64_t ldy, int64_t k, int ncol,
                                       int npad, int64_t kpitch, uint16_t* __restrict__ Yt) {
  __shared__ float tile[32][33];
  const int64_t k0 = (int64_t)blockIdx.x * 32;
  const int n0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
  for (int r = ty; r < 32; r += 8) {
    const int64_t kk = k0 + r;
    const int n = n0 + tx;
    tile[r][tx] = (kk < k && n < ncol) ? Y[kk * ldy + n] : 0.0f;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int n = n0 + r;
    const int64_t kk = k0 + tx;
    if (n >= npad || kk >= k) continue;
    float y = tile[tx][r];
#pragma unroll
    for (int t = 0; t < PARTS; ++t) {
      uint16_t bits;
      float back;
      if (BF16) {
        const __nv_bfloat16 h = __float2bfloat16_rn(y);
        bits = __bfloat16_as_ushort(h);
        back = __bfloat162float(h);
      } else {
        const __half h = __float2half_rn(y);
        bits = __half_as_ushort(h);
        back = __half2float(h);
      }
      Yt[((int64_t)t * npad + n) * kpitch + kk] = bits;
      y = y - back;  // exact in binary32 (the rounded part shares y's leading bits)
    }
  }
}

// Z[r + c*ldz] = sum_s part[s][c*p + r] in FP64, slices in order.
__global__ void tc_reduce_kernel(const float* __restrict__ part, int S, int64_t p, int64_t ncol,
                                 double* __restrict__ Z, int64_t ldz) {
  const int64_t total = p * ncol;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < S; ++q) s += (double)part[(int64_t)q * total + e];
    const int64_t c = e / p, r = e - c * p;
    Z[r + c * ldz] = s;
  }
}

// ---------------------------------------------------------------------------
struct TcPlan {
  int parts, npad, NT, Mt, Nt, KT, kt_per, S, stages;
  int64_t kpitch;
};

static int tc_parts(int prec) { return prec == MSK_GEMM_BF16X3 ? 3 : 1; }

static TcPlan tc_plan(int64_t p, int64_t k, int64_t ncol, int prec) {
  TcPlan t;
  t.parts = tc_parts(prec);
  t.npad = (int)((ncol + 15) / 16 * 16);
  const bool drain = t.parts == 3 && tune_get("tc.drain", 1) != 0;
  const int nt_max = drain ? 4 * kDsMaxCpw : (t.parts == 3 ? 144 : 256);
  const int ntiles = (t.npad + nt_max - 1) / nt_max;
  t.NT = (int)(((t.npad + ntiles - 1) / ntiles + 15) / 16 * 16);
  t.Nt = (t.npad + t.NT - 1) / t.NT;
  t.Mt = (int)((p + kTcBM - 1) / kTcBM);
  t.KT = (int)((k + kTcBK - 1) / kTcBK);
  t.kpitch = (k + 7) / 8 * 8;
  const int tiles = t.Mt * t.Nt;
  int s = std::max(1, num_sms() / std::max(1, tiles));
  s = std::min(s, t.KT);
  t.kt_per = (t.KT + s - 1) / s;
  t.S = (t.KT + t.kt_per - 1) / t.kt_per;
  const int stage_bytes = kTcBM * kTcBK * 2 + t.parts * t.NT * kTcBK * 2;
  t.stages = std::max(1, std::min(6, (kTcSmemBudget - 2048) / stage_bytes));
  return t;
}

size_t tc_gemm_workspace(int64_t p, int64_t k, int64_t ncol, int prec) {
  TcPlan t = tc_plan(p, k, ncol, prec);
  Need nd;
  nd.add((size_t)p * t.kpitch * 2);                        // G (16-bit)
  nd.add((size_t)t.parts * t.npad * t.kpitch * 2);         // Yt parts (16-bit)
  nd.add((size_t)t.S * p * ncol * sizeof(double));         // partials (FP32 or FP64)
  return nd.used;
}


int launch_tc_gemm(uint64_t gkey, int64_t p, int64_t k, int64_t ncol, const float* Y, int64_t ldy,
                   int prec, double* Z, int64_t ldz, void* ws, size_t ws_bytes, cudaStream_t st) {
  if (p < 1 || ncol < 1 || k < 1) return MSK_OK;
  if (ncol > 512) return MSK_ENOTSUP;
  TcPlan t = tc_plan(p, k, ncol, prec);
  const bool bf16 = prec != MSK_GEMM_F16;
  Carve cv(ws, ws_bytes);
  uint16_t* G = static_cast<uint16_t*>(cv.take((size_t)p * t.kpitch * 2));
  uint16_t* Yt = static_cast<uint16_t*>(cv.take((size_t)t.parts * t.npad * t.kpitch * 2));
  float* part = static_cast<float*>(cv.take((size_t)t.S * p * ncol * sizeof(double)));
  if (!G || !Yt || !part) return MSK_ENOMEM;
  int rc = launch_gaussian(gkey, p, k, bf16 ? MSK_GEMM_BF16 : MSK_GEMM_F16, G, t.kpitch, st);
  if (rc) return rc;
  {
    dim3 grid((unsigned)((k + 31) / 32), (unsigned)((t.npad + 31) / 32));
    if (t.parts == 3)
      split_transpose_kernel<3, true><<<grid, 256, 0, st>>>(Y, ldy, k, (int)ncol, t.npad, t.kpitch, Yt);
    else if (bf16)
      split_transpose_kernel<1, true><<<grid, 256, 0, st>>>(Y, ldy, k, (int)ncol, t.npad, t.kpitch, Yt);
    else
      split_transpose_kernel<1, false><<<grid, 256, 0, st>>>(Y, ldy, k, (int)ncol, t.npad, t.kpitch, Yt);
    MSK_CHECK_LAUNCH("split_transpose_kernel");
  }
  auto enc = tensor_map_encoder();
  if (!enc) {
    set_error_text("cuTensorMapEncodeTiled entry point not available");
    return MSK_ECUDA;
  }
  const CUtensorMapDataType dt = bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  CUtensorMap tmA, tmB;
  {
    cuuint64_t dims[2] = {(cuuint64_t)k, (cuuint64_t)p};
    cuuint64_t strides[1] = {(cuuint64_t)t.kpitch * 2};
    cuuint32_t box[2] = {(cuuint32_t)kTcBK, (cuuint32_t)kTcBM};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(&tmA, dt, 2, G, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
      set_error_text("cuTensorMapEncodeTiled failed for G");
      return MSK_ECUDA;
    }
  }
  {
    cuuint64_t dims[3] = {(cuuint64_t)k, (cuuint64_t)t.npad, (cuuint64_t)t.parts};
    cuuint64_t strides[2] = {(cuuint64_t)t.kpitch * 2, (cuuint64_t)t.npad * t.kpitch * 2};
    cuuint32_t box[3] = {(cuuint32_t)kTcBK, (cuuint32_t)t.NT, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(&tmB, dt, 3, Yt, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
      set_error_text("cuTensorMapEncodeTiled failed for Y");
      return MSK_ECUDA;
    }
  }
  const uint32_t idesc = make_idesc(kTcBM, t.NT, bf16);
  const int stage_bytes = kTcBM * kTcBK * 2 + t.parts * t.NT * kTcBK * 2;
  const size_t smem = (size_t)t.stages * stage_bytes + 1024 + 256;
  dim3 grid(t.Mt, t.Nt, t.S);
  const bool drain = t.parts == 3 && tune_get("tc.drain", 1) != 0;
  if (drain) {
    MSK_ALLOW_SMEM(tc_gemm_ds_kernel);
    tc_gemm_ds_kernel<<<grid, kDsThreads, smem, st>>>(tmA, tmB, (int)p, (int)ncol, t.NT, t.KT, t.kt_per,
                                                      t.stages, idesc, reinterpret_cast<double*>(part));
    MSK_CHECK_LAUNCH("tc_gemm_ds_kernel");
    const int64_t total = p * ncol;
    splitk_reduce_kernel<<<(unsigned)std::min<int64_t>((total + 255) / 256, num_sms() * 8), 256, 0, st>>>(
        reinterpret_cast<const double*>(part), t.S, p, ncol, Z, ldz);
    MSK_CHECK_LAUNCH("splitk_reduce_kernel");
    return MSK_OK;
  }
  if (t.parts == 3) {
    MSK_ALLOW_SMEM(tc_gemm_kernel<3>);
    tc_gemm_kernel<3><<<grid, kTcThreads, smem, st>>>(tmA, tmB, (int)p, (int)ncol, t.NT, t.KT, t.kt_per,
                                                      t.stages, idesc, part);
  } else {
    MSK_ALLOW_SMEM(tc_gemm_kernel<1>);
    tc_gemm_kernel<1><<<grid, kTcThreads, smem, st>>>(tmA, tmB, (int)p, (int)ncol, t.NT, t.KT, t.kt_per,
                                                      t.stages, idesc, part);
  }
  MSK_CHECK_LAUNCH("tc_gemm_kernel");
  const int64_t total = p * ncol;
  tc_reduce_kernel<<<(unsigned)std::min<int64_t>((total + 255) / 256, num_sms() * 8), 256, 0, st>>>(
      part, t.S, p, ncol, Z, ldz);
  MSK_CHECK_LAUNCH("tc_reduce_kernel");
  return MSK_OK;
}


// ---------------------------------------------------------------------------
// Batched draining BF16x3 stage (used by the batch engine).

// Shapes of one problem in the batched stage: N tiles of <= 96 columns,
// K slices of kt_per K tiles.
void tc_ds_shape(int64_t p, int64_t k, int64_t ncol, int kt_per, TcShape* s) {
  s->npad = (int)((ncol + 15) / 16 * 16);
  const int nt_max = 4 * kDsMaxCpw;
  const int ntiles = (s->npad + nt_max - 1) / nt_max;
  s->NT = (int)(((s->npad + ntiles - 1) / ntiles + 15) / 16 * 16);
  s->Nt = (s->npad + s->NT - 1) / s->NT;
  s->Mt = (int)((p + kTcBM - 1) / kTcBM);
  s->KT = (int)((k + kTcBK - 1) / kTcBK);
  s->kpitch = (k + 7) / 8 * 8;
  s->kt_per = std::max(1, std::min(kt_per, s->KT));
  s->S = (s->KT + s->kt_per - 1) / s->kt_per;
  s->items = s->Mt * s->Nt * s->S;
}

// Fill a TcJob: tensor maps over G (p x k bf16, pitch kpitch) and Yt (3 parts
// of npad x k bf16).
int tc_ds_make_job(int64_t p, int64_t k, int64_t ncol, const TcShape& s, const void* G,
                   const void* Yt, double* part, int item_begin, TcJob* job) {
  auto enc = tensor_map_encoder();
  if (!enc) {
    set_error_text("cuTensorMapEncodeTiled entry point not available");
    return MSK_ECUDA;
  }
  {
    cuuint64_t dims[2] = {(cuuint64_t)k, (cuuint64_t)p};
    cuuint64_t strides[1] = {(cuuint64_t)s.kpitch * 2};
    cuuint32_t box[2] = {(cuuint32_t)kTcBK, (cuuint32_t)kTcBM};
    cuuint32_t estr[2] = {1, 1};
    if (enc(&job->mapA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(G), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
      set_error_text("cuTensorMapEncodeTiled failed for a batched G");
      return MSK_ECUDA;
    }
  }
  {
    cuuint64_t dims[3] = {(cuuint64_t)k, (cuuint64_t)s.npad, 3};
    cuuint64_t strides[2] = {(cuuint64_t)s.kpitch * 2, (cuuint64_t)s.npad * s.kpitch * 2};
    cuuint32_t box[3] = {(cuuint32_t)kTcBK, (cuuint32_t)s.NT, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    if (enc(&job->mapB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(Yt), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
      set_error_text("cuTensorMapEncodeTiled failed for a batched Y");
      return MSK_ECUDA;
    }
  }
  job->part = part;
  job->p = (int)p;
  job->ncol = (int)ncol;
  job->NT = s.NT;
  job->KT = s.KT;
  job->kt_per = s.kt_per;
  job->Mt = s.Mt;
  job->Nt = s.Nt;
  job->S = s.S;
  job->idesc = make_idesc(kTcBM, s.NT, true);
  job->item_begin = item_begin;
  return MSK_OK;
}

int launch_tc_ds_batch(const TcJob* jobs, int njobs, int total_items, int max_nt, cudaStream_t st) {
  if (total_items <= 0) return MSK_OK;
  const int stage_bytes = kTcBM * kTcBK * 2 + 3 * max_nt * kTcBK * 2;
  const int stages = std::max(1, std::min(6, (kTcSmemBudget - 2048) / stage_bytes));
  const size_t smem = (size_t)stages * stage_bytes + 1024 + 256;
  MSK_ALLOW_SMEM(tc_gemm_ds_batch_kernel);
  tc_gemm_ds_batch_kernel<<<total_items, kDsThreads, smem, st>>>(jobs, njobs, stages);
  MSK_CHECK_LAUNCH("tc_gemm_ds_batch_kernel");
  return MSK_OK;
}

// Test hook: a wait on an mbarrier that nothing arrives on, through the same
// bounded wait as the pipelined kernels; it expires and sets g_tc_timeout.
__global__ void tc_wait_selftest_kernel() {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_wait(smem_u32(&bar), 0, &g_tc_timeout);
}

int launch_tc_wait_selftest(cudaStream_t st) {
  tc_wait_selftest_kernel<<<1, 32, 0, st>>>();
  MSK_CHECK_LAUNCH("tc_wait_selftest_kernel");
  return MSK_OK;
}

// Device address of the timeout flag, for kernels of other files (looked up
// once per device and context with that device current).
int tc_timeout_flag(int** out) {
  constexpr int kMaxDev = 64;
  static int* addr[kMaxDev] = {nullptr};
  int dev = 0;
  MSK_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDev) return MSK_ENOTSUP;
  if (!addr[dev]) {
    void* p = nullptr;
    MSK_CUDA(cudaGetSymbolAddress(&p, g_tc_timeout));
    addr[dev] = static_cast<int*>(p);
  }
  *out = addr[dev];
  return MSK_OK;
}

// Reads and clears the timeout flag of the tensor-core kernel (synchronises).
int tc_take_timeout(cudaStream_t st) {
  int h = 0, zero = 0;
  MSK_CUDA(cudaStreamSynchronize(st));
  MSK_CUDA(cudaMemcpyFromSymbol(&h, g_tc_timeout, sizeof(int)));
  if (h) MSK_CUDA(cudaMemcpyToSymbol(g_tc_timeout, &zero, sizeof(int)));
  return h ? MSK_ETIMEOUT : MSK_OK;
}

}  // namespace msk
