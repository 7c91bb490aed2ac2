// gemm_oz.cu — the FP64 Gaussian stage Z = G Y of the multisketch (Section 1
// "Count-Gauss", Section 6.2) on the tcgen05 tensor cores, by error-free
// slicing of both operands into 8-bit integers (the Ozaki scheme: Ozaki,
// Ogita, Oishi, Rump, "Error-free transformations of matrix multiplication by
// using fast routines of matrix multiplication and its applications",
// Numerical Algorithms 59, 2012).  GB300 runs FP64 at about 1 TFLOP/s and
// BF16 MMAs at about 2 PFLOP/s: 36 exact BF16 products cost far less than one
// FP64 product.
//
// Slices.  With a power-of-two scale per row of G (one bound for every row:
// the polar-method Gaussian is below 8.1/sqrt(p)) and per column of Y (its
// largest magnitude), each operand is written as eight 8-bit slices:
//   G[r][i] = 2^(eG - 7)   (g_0 + g_1 2^-8 + ... + g_7 2^-56) + rest_G,
//   Y[i][c] = 2^(eY_c - 7) (y_0 + y_1 2^-8 + ... + y_7 2^-56) + rest_Y,
// g_j, y_l integers in [-128, 128] (exact in bfloat16), |rest| at most half
// a unit of the last slice: each operand is rounded once to 64-bit fixed
// point, whose balanced base-256 digits are the slices (exact).
//
// Products.  g_j y_l is an integer of magnitude <= 2^14, exact in the tensor
// core's FP32 accumulator, and so is every partial sum of up to 1024 of them
// (<= 2^24).  The pairs with j + l <= 7 are kept (36 of them); a pair's level
// is j + l.  A CTA takes one group of G slices — {0, 7}, {1, 6}, {2, 5} or
// {3, 4}, nine pairs each — with all the Y slices they pair with, and one
// TMEM accumulator per level; a level receives at most two pairs over at most
// 512 K values, so at most 1024 products: every accumulator stays exact.  The
// epilogue reads the levels (tcgen05.ld) and combines them exactly into two
// 64-bit integers; one kernel sums the partials of all K slices and groups
// exactly in 64-bit integers (so the result is the same in any order) and
// rounds once to FP64.  Slicing, combining and summing use integer
// arithmetic only: GB300's FP64 pipe would otherwise bound the stage.
//
// Error.  Per term i the dropped pairs (levels 8..14) and the two rests
// contribute at most 9.1 * 2^(eG + eY_c - 64); with 2^eG < 2 * 8.1/sqrt(p)
// and 2^eY_c <= 2 max_i |Y[i][c]|,
//   |Z_computed - G Y| <= k * 9.1 * 2^(eG + eY_c - 64) + 3 u |Z|,
// i.e. about 0.15 k u max|Y[:,c]| / sqrt(p) (u = 2^-53), below the worst
// case of an FP64 dot product of the same length.  (Seven slices, 2^8 times
// less accurate, moved the sketch-and-solve residual at kappa(A) = 1e10 by
// 2e-8 relative.)  The stage is used from k >= 1024 (below, the FP64 SIMT
// kernel is cheap anyway).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "msk_device.cuh"
#include "msk_internal.h"
#include "msk_tc.cuh"

namespace msk {

constexpr int kOzSlices = 8;      // slices of each operand; levels 0..7 kept
constexpr int kOzGroups = 4;      // G-slice groups {0,7} {1,6} {2,5} {3,4}
constexpr int kOzBM = 128;        // M per CTA (one UMMA M)
constexpr int kOzBK = 64;         // K per stage (one 128-byte swizzle row of bf16)
constexpr int kOzMaxKtPer = 8;    // K tiles per CTA: 2 pairs x 512 products <= 1024
constexpr int kOzThreads = 128;
constexpr int kOzMaxNT = 64;      // 8 levels x NT TMEM columns <= 512
constexpr double kOzGaussBound = 8.1;  // |polar-method N(0,1) sample| < 8.1

// ---------------------------------------------------------------------------
// Fixed-point forms, in integer arithmetic only (GB300's FP64 pipe is slow).
// The integer nearest to m 2^sh (0 <= m < 2^53), ties upward, for shifts
// that keep it below 2^63.
__device__ __forceinline__ long long oz_shift_round(unsigned long long m, int sh) {
  if (sh >= 0) return (long long)(m << sh);
  const int s = -sh;
  if (s >= 64) return 0;
  return (long long)((m + (1ull << (s - 1))) >> s);
}
// X = round(y 2^(63 - e)) for a finite |y| < 2^e, so |X| < 2^63.
__device__ __forceinline__ long long oz_fixed_f64(double y, int e) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(y);
  const int E = (int)((bits >> 52) & 0x7FF);
  const unsigned long long frac = bits & ((1ull << 52) - 1);
  const unsigned long long m = E ? (frac | (1ull << 52)) : frac;
  const long long X = oz_shift_round(m, (E ? E : 1) - 1075 + 63 - e);  // y = m 2^(E - 1075)
  return (bits >> 63) ? -X : X;
}
__device__ __forceinline__ long long oz_fixed_f32(float g, int e) {
  const unsigned bits = __float_as_uint(g);
  const int E = (int)((bits >> 23) & 0xFF);
  const unsigned long long m = E ? ((bits & 0x7FFFFFu) | 0x800000u) : (bits & 0x7FFFFFu);
  const long long X = oz_shift_round(m, (E ? E : 1) - 150 + 63 - e);  // g = m 2^(E - 150)
  return (bits >> 31) ? -X : X;
}
// bfloat16 bits of the integer e - 128 (0 <= e <= 256): 2^23 + 2^22 + e - 128
// assembled as binary32 bits, less 1.5 2^23 (exact, FP32 add), whose top 16
// bits are the bfloat16 (the value has at most 8 significant bits).  One
// integer add, one FP32 add and one shift: no conversion instruction.
__device__ __forceinline__ uint16_t oz_bf16_of_biased(unsigned e) {
  return (uint16_t)(__float_as_uint(__uint_as_float(0x4B3FFF80u + e) - 12582912.0f) >> 16);
}
// The eight slices of X as bfloat16 bits: X = sum_l s_l 2^(56 - 8 l) exactly,
// with balanced base-256 digits.  Adding 128 to each of the low seven bytes
// (0x0080808080808080, carries included) turns them into the digits s_1..s_7
// plus 128, in [0, 255]; the carry out of byte 6 goes to s_0 = (X >> 56) +
// carry, in [-128, 128].
__device__ __forceinline__ void oz_slices(long long X, uint16_t (&s)[kOzSlices]) {
  const unsigned long long L = ((unsigned long long)X & 0x00FFFFFFFFFFFFFFull) + 0x0080808080808080ull;
  const unsigned lo = (unsigned)L, hi = (unsigned)(L >> 32);
  s[0] = oz_bf16_of_biased((unsigned)((int)(X >> 56) + (int)(hi >> 24) + 128));
  s[1] = oz_bf16_of_biased((hi >> 16) & 0xFFu);
  s[2] = oz_bf16_of_biased((hi >> 8) & 0xFFu);
  s[3] = oz_bf16_of_biased(hi & 0xFFu);
  s[4] = oz_bf16_of_biased(lo >> 24);
  s[5] = oz_bf16_of_biased((lo >> 16) & 0xFFu);
  s[6] = oz_bf16_of_biased((lo >> 8) & 0xFFu);
  s[7] = oz_bf16_of_biased(lo & 0xFFu);
}

// G slices: entry (r, i) is the same binary32 number the Gaussian kernel
// writes (standard normal number r*k + i of the stream, divided by sqrt(p)),
// in fixed point at 2^(eG - 63) and cut into eight slices Gs[j][r][i]
// (pitch kpitch).  Rows over gridDim.y, columns over gridDim.x.
__global__ void oz_split_g_kernel(uint64_t key, int64_t p, int64_t k, float sqrt_p, int eG,
                                  int64_t kpitch, __nv_bfloat16* __restrict__ Gs) {
  const int64_t plane = p * kpitch;
  for (int64_t r = blockIdx.y; r < p; r += gridDim.y)
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < k;
         c += (int64_t)gridDim.x * blockDim.x) {
      const float g = __fdiv_rn(gauss_std(key, (uint64_t)(r * k + c)), sqrt_p);
      MSK_CHECK_OR(fabsf(g) < ldexpf(1.0f, eG), kCheckSlice, continue);
      uint16_t sl[kOzSlices];
      oz_slices(oz_fixed_f32(g, eG), sl);
      uint16_t* out = reinterpret_cast<uint16_t*>(Gs) + r * kpitch + c;
#pragma unroll
      for (int j = 0; j < kOzSlices; ++j) out[j * plane] = sl[j];
    }
}

// Largest |Y[i][c]| of every column, as the bit pattern of a non-negative
// double (ordered like the value), combined with atomicMax.  mx is zeroed by
// the caller.  Block 32 x 8: 32 columns, 8 rows at a time.
__global__ void oz_colmax_kernel(const double* __restrict__ Y, int64_t ldy, int64_t k, int ncol,
                                 unsigned long long* __restrict__ mx) {
  __shared__ unsigned long long red[8][32];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int c = blockIdx.x * 32 + tx;
  unsigned long long m = 0;
  if (c < ncol)
    for (int64_t i = (int64_t)blockIdx.y * 8 + ty; i < k; i += (int64_t)gridDim.y * 8) {
      const unsigned long long b =
          (unsigned long long)__double_as_longlong(Y[i * ldy + c]) & 0x7FFFFFFFFFFFFFFFull;
      m = b > m ? b : m;
    }
  red[ty][tx] = m;
  __syncthreads();
  if (ty == 0 && c < ncol) {
#pragma unroll
    for (int q = 1; q < 8; ++q) m = red[q][tx] > m ? red[q][tx] : m;
    atomicMax(mx + c, m);
  }
}

// Exponent e with max < 2^e from the bit pattern of a non-negative max
// (-1022 for zero or subnormal maxima: every such value is below 2^-1022).
__device__ __forceinline__ int oz_exp_of(unsigned long long bits) {
  const int E = (int)((bits >> 52) & 0x7FF);
  return E == 0 ? -1022 : E - 1022;
}

// Y slices: Ys[l][c][i] (K-major, pitch kpitch, npad rows; rows >= ncol
// zero) from the row-major FP64 Y, in fixed point at 2^(eY_c - 63); 32x32
// tiles transposed in shared memory; eY[c] the column exponents (0 for the
// padding columns).
__global__ void oz_split_y_kernel(const double* __restrict__ Y, int64_t ldy, int64_t k, int ncol,
                                  int npad, int64_t kpitch, const unsigned long long* __restrict__ mx,
                                  int* __restrict__ eY, __nv_bfloat16* __restrict__ Ys) {
  __shared__ double tile[32][33];
  const int64_t k0 = (int64_t)blockIdx.x * 32;
  const int n0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
  for (int r = ty; r < 32; r += 8) {
    const int64_t i = k0 + r;
    const int n = n0 + tx;
    tile[r][tx] = (i < k && n < ncol) ? Y[i * ldy + n] : 0.0;
  }
  if (blockIdx.x == 0 && ty == 0 && n0 + tx < npad)
    eY[n0 + tx] = n0 + tx < ncol ? oz_exp_of(mx[n0 + tx]) : 0;
  __syncthreads();
  const int64_t plane = (int64_t)npad * kpitch;
  for (int r = ty; r < 32; r += 8) {
    const int n = n0 + r;
    const int64_t i = k0 + tx;
    if (n >= npad || i >= k) continue;
    MSK_CHECK_OR(n >= ncol || fabs(tile[tx][r]) < ldexp(1.0, oz_exp_of(mx[n])), kCheckSlice, continue);
    const long long X = n < ncol ? oz_fixed_f64(tile[tx][r], oz_exp_of(mx[n])) : 0;
    uint16_t sl[kOzSlices];
    oz_slices(X, sl);
    uint16_t* out = reinterpret_cast<uint16_t*>(Ys) + (int64_t)n * kpitch + i;
#pragma unroll
    for (int l = 0; l < kOzSlices; ++l) out[l * plane] = sl[l];
  }
}

// One CTA: tile (mt, nt) of Z, K slice sidx, G-slice group grp (ja = grp,
// jb = 7 - grp).  Warp 0 lane 0 streams the G tiles of slices ja and jb and
// the Y tiles of slices 0 .. 7 - ja with TMA through a ring of stages;
// warp 1 lane 0 issues the MMAs into the level accumulators (TMEM columns
// (level - ja) * NT); then all four warps read the 128 rows back.  Every
// mbarrier wait is bounded (1 s): on expiry the kernel sets *timeout_flag
// (the tensor-core kernels' flag, reported by msk_take_timeout),
// waits (bounded) for its copies in flight, frees its tensor memory and
// returns.
__global__ void __launch_bounds__(kOzThreads, 1)
    oz_gemm_kernel(const __grid_constant__ CUtensorMap tmG, const __grid_constant__ CUtensorMap tmY,
                   int p, int ncol, int NT, int KT, int kt_per, uint32_t idesc,
                   longlong2* __restrict__ part, int* timeout_flag) {
  extern __shared__ __align__(1024) unsigned char oz_smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(oz_smem_raw) + 1023) & ~uintptr_t(1023));
  const int grp = blockIdx.z % kOzGroups, sidx = blockIdx.z / kOzGroups;
  const int ja = grp, jb = kOzSlices - 1 - grp;
  const int ng = ja == jb ? 1 : 2;       // G tiles per stage
  const int ny = kOzSlices - ja;         // Y tiles per stage (slices 0 .. 7 - ja)
  const int nlev = kOzSlices - ja;       // levels ja .. 7
  const uint32_t a_bytes = kOzBM * kOzBK * 2;
  const uint32_t b_bytes = (uint32_t)NT * kOzBK * 2;
  const uint32_t stage_bytes = ng * a_bytes + ny * b_bytes;
  // the ring: as many stages as the launch's shared memory holds (<= 4)
  uint32_t dyn = 0;
  asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
  const int stages = max(1, min(4, (int)((dyn - 1024u - 256u) / stage_bytes)));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)stages * stage_bytes);
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bars + 2 * stages + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * kOzBM, n0 = blockIdx.y * NT;
  const int kt0 = sidx * kt_per;
  const int nk = min(KT, kt0 + kt_per) - kt0;
  constexpr uint32_t kCols = 512;

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
                 "r"(kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  if (warp == 0 && lane == 0) {
    int issued = 0;
    for (int it = 0; it < nk; ++it) {
      const int s = it % stages;
      if (it >= stages &&
          !mbar_wait(smem_u32(&bars[stages + s]), ((it / stages) & 1) ^ 1, timeout_flag)) {
        *abort_flag = 1;
        break;
      }
      if (*abort_flag) break;
      const uint32_t full = smem_u32(&bars[s]);
      mbar_expect_tx(full, stage_bytes);
      unsigned char* st = smem + (size_t)s * stage_bytes;
      const int kc = (kt0 + it) * kOzBK;
      tma_load_3d(smem_u32(st), &tmG, kc, m0, ja, full);
      if (ng == 2) tma_load_3d(smem_u32(st + a_bytes), &tmG, kc, m0, jb, full);
      for (int l = 0; l < ny; ++l)
        tma_load_3d(smem_u32(st + ng * a_bytes + l * b_bytes), &tmY, kc, n0, l, full);
      ++issued;
    }
    if (*abort_flag)
      for (int it = (issued > stages ? issued - stages : 0); it < issued; ++it)
        mbar_wait(smem_u32(&bars[it % stages]), (it / stages) & 1, timeout_flag);
  } else if (warp == 1 && lane == 0) {
    for (int it = 0; it < nk; ++it) {
      const int s = it % stages;
      if (!mbar_wait(smem_u32(&bars[s]), (it / stages) & 1, timeout_flag)) {
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      const uint32_t a0 = smem_u32(smem + (size_t)s * stage_bytes);
      const uint32_t b0 = a0 + ng * a_bytes;
#pragma unroll
      for (int kk = 0; kk < kOzBK / 16; ++kk) {
        // slice ja with Y slices 0 .. 7 - ja: levels ja .. 7 (first touch of
        // each accumulator at it = 0, kk = 0)
        const uint64_t ada = sw128_desc(a0 + kk * 32);
        for (int l = 0; l < ny; ++l)
          umma_f16(tmem + (uint32_t)(l * NT), ada, sw128_desc(b0 + l * b_bytes + kk * 32), idesc,
                   (it > 0 || kk > 0) ? 1u : 0u);
        if (ng == 2) {
          // slice jb with Y slices 0 .. 7 - jb: levels jb .. 7
          const uint64_t adb = sw128_desc(a0 + a_bytes + kk * 32);
          for (int l = 0; l <= kOzSlices - 1 - jb; ++l)
            umma_f16(tmem + (uint32_t)((jb + l - ja) * NT), adb,
                     sw128_desc(b0 + l * b_bytes + kk * 32), idesc, 1u);
        }
      }
      umma_commit(smem_u32(&bars[stages + s]));
    }
    umma_commit(smem_u32(&bars[2 * stages]));
  }
  __syncwarp();
  const bool done = mbar_wait(smem_u32(&bars[2 * stages]), 0, timeout_flag);
  tc_fence_after();
  if (__all_sync(0xffffffffu, done && !*abort_flag && nk > 0)) {
    // Level sums are exact integers below 2^24: combined exactly as
    // H = sum_{s<4} V_s 2^(8(3-s)) and L = sum_{s>=4} V_s 2^(8(7-s)) (each
    // below 2^49), so Z's entry is 2^(eG + eY - 70) (H 2^32 + L) summed over
    // all CTAs — integer work only (GB300's FP64 pipe would make this epilogue
    // the kernel's bottleneck).
    const int row = m0 + warp * 32 + lane;
    longlong2* out = part + (int64_t)blockIdx.z * p * ncol;
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    // 8 columns at a time: every level's load issued before one wait
    for (int c0 = 0; c0 < NT; c0 += 8) {
      uint32_t v[kOzSlices][8];
#pragma unroll
      for (int lev = 0; lev < kOzSlices; ++lev)
        if (lev < nlev) tmem_ld8_nowait(lane_base + (uint32_t)(lev * NT + c0), v[lev]);
      tmem_wait_ld();
      long long H[8], L[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) H[q] = L[q] = 0;
#pragma unroll
      for (int lev = 0; lev < kOzSlices; ++lev) {
        if (lev >= nlev) break;
        const int s = ja + lev;  // this accumulator's level
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const long long x = (long long)__float2int_rn(__uint_as_float(v[lev][q]));  // exact
          if (s < 4) H[q] += x * (1LL << (8 * (3 - s)));
          else L[q] += x * (1LL << (8 * (7 - s)));
        }
      }
      if (row < p) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int col = n0 + c0 + q;
          if (col < ncol) out[(int64_t)col * p + row] = make_longlong2(H[q], L[q]);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols)
                 : "memory");
}

// Z[r + c ldz] = 2^(eG + eY_c - 70) (H 2^32 + L) with H, L the sums of the
// S partials of entry e = c p + r.  Block 32 x 8: 32 consecutive entries, 8
// lanes over the partials.  The partial sums are exact 64-bit integers (below
// 2^49 S), so the result does not depend on the order of the sums; the one
// rounding is the conversion to FP64 at the end.
__global__ void oz_reduce_kernel(const longlong2* __restrict__ part, int S, int64_t p, int64_t ncol, int eG,
                                 const int* __restrict__ eY, double* __restrict__ Z, int64_t ldz) {
  __shared__ long long sh[8][32], sl[8][32];
  const int64_t total = p * ncol;
  const int64_t e = (int64_t)blockIdx.x * 32 + threadIdx.x;
  long long H = 0, L = 0;
  if (e < total)
    for (int q = threadIdx.y; q < S; q += 8) {
      const longlong2 v = part[(int64_t)q * total + e];
      H += v.x;
      L += v.y;
    }
  sh[threadIdx.y][threadIdx.x] = H;
  sl[threadIdx.y][threadIdx.x] = L;
  __syncthreads();
  if (threadIdx.y == 0 && e < total) {
#pragma unroll
    for (int q = 1; q < 8; ++q) {
      H += sh[q][threadIdx.x];
      L += sl[q][threadIdx.x];
    }
    const int64_t c = e / p, r = e - c * p;
    Z[r + c * ldz] = scalbn(fma((double)H, 0x1p32, (double)L), eG + eY[c] - 70);
  }
}

// ---------------------------------------------------------------------------
struct OzPlan {
  int npad, NT, Nt, Mt, KT, kt_per, S;
  int64_t kpitch;
};

static OzPlan oz_plan(int64_t p, int64_t k, int64_t ncol) {
  OzPlan t;
  t.npad = (int)((ncol + 15) / 16 * 16);
  t.Nt = (t.npad + kOzMaxNT - 1) / kOzMaxNT;
  t.NT = (int)(((t.npad + t.Nt - 1) / t.Nt + 15) / 16 * 16);
  t.Mt = (int)((p + kOzBM - 1) / kOzBM);
  t.KT = (int)((k + kOzBK - 1) / kOzBK);
  t.kt_per = (int)std::max<long long>(1, std::min<long long>(kOzMaxKtPer, tune_get("oz.kt_per", kOzMaxKtPer)));
  t.S = (t.KT + t.kt_per - 1) / t.kt_per;
  t.kpitch = (k + 7) / 8 * 8;
  return t;
}

bool oz_applicable(int64_t p, int64_t k, int64_t ncol) {
  return tune_get("gemm.f64_ozaki", 1) != 0 && k >= 1024 && k < (1LL << 31) && ncol <= 512 &&
         p <= (1LL << 20);
}

size_t oz_gemm_workspace(int64_t p, int64_t k, int64_t ncol) {
  const OzPlan t = oz_plan(p, k, ncol);
  Need nd;
  nd.add((size_t)kOzSlices * p * t.kpitch * 2);                // G slices
  nd.add((size_t)kOzSlices * t.npad * t.kpitch * 2);           // Y slices
  nd.add((size_t)kOzGroups * t.S * p * ncol * sizeof(longlong2));  // partials
  nd.add((size_t)ncol * sizeof(unsigned long long));           // column maxima
  nd.add((size_t)t.npad * sizeof(int));                        // column exponents
  return nd.used;
}

// Smallest e with 2^e above the bound of |G| = |N(0,1) sample| / sqrt_p.
static int oz_g_exponent(float sqrt_p) {
  const double B = kOzGaussBound / (double)sqrt_p;
  int e = (int)std::ceil(std::log2(B));
  while (std::ldexp(1.0, e) <= B) ++e;
  while (std::ldexp(1.0, e - 1) > B) --e;
  return e;
}

// The stage's pieces in the caller's workspace (the same for every call with
// these sizes, so that the G slices a preparing call leaves are found).
struct OzBufs {
  __nv_bfloat16 *Gs, *Ys;
  longlong2* part;
  unsigned long long* mx;
  int* eY;
};
static bool oz_carve(void* ws, size_t ws_bytes, const OzPlan& t, int64_t p, int64_t ncol, OzBufs* b) {
  Carve cv(ws, ws_bytes);
  b->Gs = static_cast<__nv_bfloat16*>(cv.take((size_t)kOzSlices * p * t.kpitch * 2));
  b->Ys = static_cast<__nv_bfloat16*>(cv.take((size_t)kOzSlices * t.npad * t.kpitch * 2));
  b->part = static_cast<longlong2*>(cv.take((size_t)kOzGroups * t.S * p * ncol * sizeof(longlong2)));
  b->mx = static_cast<unsigned long long*>(cv.take((size_t)ncol * sizeof(unsigned long long)));
  b->eY = static_cast<int*>(cv.take((size_t)t.npad * sizeof(int)));
  return b->Gs && b->Ys && b->part && b->mx && b->eY;
}

int launch_oz_prepare_g(uint64_t gkey, int64_t p, int64_t k, int64_t ncol, void* ws, size_t ws_bytes,
                        cudaStream_t st) {
  if (p < 1 || ncol < 1 || k < 1) return MSK_OK;
  const OzPlan t = oz_plan(p, k, ncol);
  OzBufs bf;
  if (!oz_carve(ws, ws_bytes, t, p, ncol, &bf)) return MSK_ENOMEM;
  const float sqrt_p = __builtin_sqrtf((float)p);
  const dim3 grid((unsigned)std::min<int64_t>((k + 255) / 256, 64), (unsigned)std::min<int64_t>(p, 65535));
  oz_split_g_kernel<<<grid, 256, 0, st>>>(gkey, p, k, sqrt_p, oz_g_exponent(sqrt_p), t.kpitch, bf.Gs);
  MSK_CHECK_LAUNCH("oz_split_g_kernel");
  return MSK_OK;
}

int launch_oz_gemm(uint64_t gkey, int64_t p, int64_t k, int64_t ncol, const double* Y, int64_t ldy,
                   double* Z, int64_t ldz, void* ws, size_t ws_bytes, cudaStream_t st, bool g_ready) {
  if (p < 1 || ncol < 1 || k < 1) return MSK_OK;
  const OzPlan t = oz_plan(p, k, ncol);
  OzBufs bf;
  if (!oz_carve(ws, ws_bytes, t, p, ncol, &bf)) return MSK_ENOMEM;
  __nv_bfloat16 *Gs = bf.Gs, *Ys = bf.Ys;
  longlong2* part = bf.part;
  unsigned long long* mx = bf.mx;
  int* eY = bf.eY;
  const int sms = num_sms();
  // G slices (independent of Y), unless a preparing call already wrote them
  const float sqrt_p = __builtin_sqrtf((float)p);
  const int eG = oz_g_exponent(sqrt_p);
  if (!g_ready) {
    const int rc = launch_oz_prepare_g(gkey, p, k, ncol, ws, ws_bytes, st);
    if (rc) return rc;
  }
  // column maxima of Y, then its slices
  MSK_CUDA(cudaMemsetAsync(mx, 0, (size_t)ncol * sizeof(unsigned long long), st));
  {
    const unsigned gy = (unsigned)std::max<int64_t>(1, std::min<int64_t>((k + 63) / 64, (int64_t)sms * 4));
    oz_colmax_kernel<<<dim3((unsigned)((ncol + 31) / 32), gy), 256, 0, st>>>(Y, ldy, k, (int)ncol, mx);
    MSK_CHECK_LAUNCH("oz_colmax_kernel");
    oz_split_y_kernel<<<dim3((unsigned)((k + 31) / 32), (unsigned)((t.npad + 31) / 32)), 256, 0, st>>>(
        Y, ldy, k, (int)ncol, t.npad, t.kpitch, mx, eY, Ys);
    MSK_CHECK_LAUNCH("oz_split_y_kernel");
  }
  auto enc = tensor_map_encoder();
  if (!enc) {
    set_error_text("cuTensorMapEncodeTiled entry point not available");
    return MSK_ECUDA;
  }
  CUtensorMap tmG, tmY;
  {
    cuuint64_t dims[3] = {(cuuint64_t)k, (cuuint64_t)p, (cuuint64_t)kOzSlices};
    cuuint64_t strides[2] = {(cuuint64_t)t.kpitch * 2, (cuuint64_t)p * t.kpitch * 2};
    cuuint32_t box[3] = {(cuuint32_t)kOzBK, (cuuint32_t)kOzBM, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    if (enc(&tmG, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, Gs, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
      set_error_text("cuTensorMapEncodeTiled failed for the G slices");
      return MSK_ECUDA;
    }
  }
  {
    cuuint64_t dims[3] = {(cuuint64_t)k, (cuuint64_t)t.npad, (cuuint64_t)kOzSlices};
    cuuint64_t strides[2] = {(cuuint64_t)t.kpitch * 2, (cuuint64_t)t.npad * t.kpitch * 2};
    cuuint32_t box[3] = {(cuuint32_t)kOzBK, (cuuint32_t)t.NT, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    if (enc(&tmY, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, Ys, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
      set_error_text("cuTensorMapEncodeTiled failed for the Y slices");
      return MSK_ECUDA;
    }
  }
  // kind::f16 instruction descriptor: FP32 accumulator, bf16 A and B, K-major
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(t.NT >> 3) << 17) |
                         ((uint32_t)(kOzBM >> 4) << 24);
  // shared memory: the largest group's stage ({0, 7}: two G tiles, eight Y
  // tiles) at least twice, up to the budget
  const size_t big = 2 * (size_t)kOzBM * kOzBK * 2 + (size_t)kOzSlices * t.NT * kOzBK * 2;
  const size_t smem = std::min<size_t>((size_t)kTcSmemBudget, std::max<size_t>(2 * big, 3 * big)) + 1024 + 256;
  MSK_ALLOW_SMEM(oz_gemm_kernel);
  int* tflag = nullptr;
  const int frc = tc_timeout_flag(&tflag);
  if (frc) return frc;
  dim3 grid((unsigned)t.Mt, (unsigned)t.Nt, (unsigned)(kOzGroups * t.S));
  oz_gemm_kernel<<<grid, kOzThreads, smem, st>>>(tmG, tmY, (int)p, (int)ncol, t.NT, t.KT, t.kt_per, idesc,
                                                 part, tflag);
  MSK_CHECK_LAUNCH("oz_gemm_kernel");
  const int64_t total = p * ncol;
  oz_reduce_kernel<<<(unsigned)((total + 31) / 32), dim3(32, 8), 0, st>>>(part, kOzGroups * t.S, p, ncol, eG, eY,
                                                                          Z, ldz);
  MSK_CHECK_LAUNCH("oz_reduce_kernel");
  return MSK_OK;
}

}  // namespace msk
