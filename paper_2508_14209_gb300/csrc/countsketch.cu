// countsketch.cu — the CountSketch Y = S [A b] (Definition 3 and its row form,
// Section 4) for column-major A, row-major Y.
//
// ATOMIC strategy (the scatter-add of Algorithm 2, rebuilt for GB300):
//   A tile of 32 consecutive rows x all columns is read with coalesced column
//   loads (lane = row), transposed through shared memory, and each row is added
//   to its bucket row Y[h(i), :] by one warp with coalesced L2 reductions
//   (lane = column), so every reduction instruction covers whole 32-byte
//   sectors of Y.  Bucket and sign are hashed on the fly (Section 8's hashed
//   CountSketch); nothing but A is read.  FP64 uses red.add.f64; FP32 uses
//   4-wide red.add.v4.f32 on 16-byte aligned rows of Y.
//   Two shared-memory buffers alternate, so one __syncthreads per tile
//   suffices; the grid is persistent over tiles.
//
// SORTED strategy (deterministic): a counting sort of the rows by bucket
//   (histogram, exclusive scan, scatter, then each bucket's row list sorted in
//   increasing row order), then one warp per bucket sums its rows in that
//   order, lane = column.  Same result bit for bit on every run.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "msk_device.cuh"
#include "msk_internal.h"

namespace msk {

// ---------------------------------------------------------------------------
// cs_hash hook: materialise h(i), s(i).
__global__ void cs_hash_kernel(uint64_t key, int64_t i0, int64_t count, uint32_t k,
                               uint32_t* __restrict__ h, int8_t* __restrict__ s) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count;
       t += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t z = draw(key, (uint64_t)(i0 + t));
    if (h) h[t] = bucket_of(z, k);
    if (s) s[t] = negative_of(z) ? (int8_t)-1 : (int8_t)1;
  }
}

int launch_cs_hash(uint64_t key, int64_t i0, int64_t count, uint32_t k, uint32_t* h,
                   int8_t* s, cudaStream_t st) {
  if (count == 0) return MSK_OK;
  int64_t blocks = std::min<int64_t>((count + 255) / 256, (int64_t)num_sms() * 16);
  cs_hash_kernel<<<(unsigned)blocks, 256, 0, st>>>(key, i0, count, k, h, s);
  MSK_CHECK_LAUNCH("cs_hash_kernel");
  return MSK_OK;
}

// ---------------------------------------------------------------------------
// ATOMIC strategy.
constexpr int kCsRows = 32;    // rows per tile (one per lane in the load phase)
constexpr int kCsWarps = 8;    // warps per CTA
constexpr int kCsThreads = kCsWarps * 32;
// Columns per launch (wider problems are split): two FP64 tiles of 32 rows x
// 385 columns, or two FP32 tiles of 32 x 516, fit in 227 KB of shared memory.
constexpr int kCsMaxColsF64 = 384;
constexpr int kCsMaxColsF32 = 512;


// Shared-memory tile layout: row r at r * pitch.  FP64: one column per
// store, odd pitch, so the 32 transposing stores of a warp (lane = row) and
// the row reads (lane = column) are both conflict-free.  FP32: a lane stores
// 4 consecutive columns of its row as one 16-byte vector and pitch/4 is odd,
// so the 8 lanes of each store wavefront hit 8 distinct 16-byte bank groups;
// the row reads are 16-byte vectors of consecutive chunks.
template <typename T>
__device__ __forceinline__ T load_col(const CsParams<T>& P, int64_t i, int j) {
  if (j < P.ncol_a) return __ldcs(P.A + i + (int64_t)j * P.lda);
  if (j < P.ncol) return (T)__ldcs(P.b + i);
  return (T)0;
}

// QMAX = column slots (FP64) or 4-column groups (FP32) per lane in the load
// phase.
template <typename T, int QMAX, bool VEC4>
__global__ void __launch_bounds__(kCsThreads) cs_atomic_kernel(const CsParams<T> P) {
  extern __shared__ __align__(16) unsigned char cs_smem[];
  T* tiles = reinterpret_cast<T*>(cs_smem);
  uint64_t* hz = reinterpret_cast<uint64_t*>(cs_smem + 2 * sizeof(T) * kCsRows * P.pitch);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ntiles = (P.d + kCsRows - 1) / kCsRows;
  constexpr bool kF32 = sizeof(T) == 4;
  const int ngroups = (P.ncol + 3) >> 2;
  int buf = 0;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, buf ^= 1) {
    const int64_t i0 = t * kCsRows;
    const int64_t i = i0 + lane;
    const bool row_ok = i < P.d;
    T* tile = tiles + buf * kCsRows * P.pitch;
    if constexpr (kF32) {
      // load phase: warp w fetches column groups w, w+8, ... (4 columns each)
      float4 v[QMAX];
#pragma unroll
      for (int q = 0; q < QMAX; ++q) {
        const int g = warp + q * kCsWarps;
        float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
        if (row_ok && g < ngroups) {
          x.x = load_col(P, i, 4 * g);
          x.y = load_col(P, i, 4 * g + 1);
          x.z = load_col(P, i, 4 * g + 2);
          x.w = load_col(P, i, 4 * g + 3);
        }
        v[q] = x;
      }
      if (warp == 0) hz[buf * kCsRows + lane] = row_ok ? draw(P.key, (uint64_t)(P.i0 + i)) : 0ull;
#pragma unroll
      for (int q = 0; q < QMAX; ++q) {
        const int g = warp + q * kCsWarps;
        if (g < ngroups) *reinterpret_cast<float4*>(&tile[lane * P.pitch + 4 * g]) = v[q];
      }
    } else {
      // load phase: warp w fetches columns w, w+8, ... for rows i0..i0+31
      T v[QMAX];
#pragma unroll
      for (int q = 0; q < QMAX; ++q) {
        const int j = warp + q * kCsWarps;
        v[q] = (row_ok && j < P.ncol) ? load_col(P, i, j) : (T)0;
      }
      if (warp == 0) hz[buf * kCsRows + lane] = row_ok ? draw(P.key, (uint64_t)(P.i0 + i)) : 0ull;
#pragma unroll
      for (int q = 0; q < QMAX; ++q) {
        const int j = warp + q * kCsWarps;
        if (j < P.ncol) tile[lane * P.pitch + j] = v[q];
      }
    }
    __syncthreads();
    // reduction phase: warp w adds rows w, w+8, w+16, w+24 into their buckets
#pragma unroll
    for (int rr = 0; rr < kCsRows / kCsWarps; ++rr) {
      const int r = warp + rr * kCsWarps;
      if (i0 + r >= P.d) break;
      const uint64_t z = hz[buf * kCsRows + r];
      MSK_CHECK_OR(bucket_of(z, P.k) < P.k, kCheckBucket, continue);
      T* yrow = P.Y + (int64_t)bucket_of(z, P.k) * P.ldy;
      const bool neg = negative_of(z);
      const T* trow = tile + r * P.pitch;
      if constexpr (VEC4) {
        const int full = P.ncol & ~3;
        for (int c = lane * 4; c < full; c += 128) {
          const float4 x = *reinterpret_cast<const float4*>(&trow[c]);
          if (neg)
            red_add_v4(reinterpret_cast<float*>(yrow) + c, -x.x, -x.y, -x.z, -x.w);
          else
            red_add_v4(reinterpret_cast<float*>(yrow) + c, x.x, x.y, x.z, x.w);
        }
        if (lane < P.ncol - full) {
          const T x = trow[full + lane];
          red_add(yrow + full + lane, neg ? -x : x);
        }
      } else {
        for (int c = lane; c < P.ncol; c += 32) {
          const T x = trow[c];
          red_add(yrow + c, neg ? -x : x);
        }
      }
    }
  }
}

template <typename T, int QMAX, bool VEC4>
static int launch_cs_atomic_t(const CsParams<T>& P, cudaStream_t st) {
  const size_t smem = 2 * sizeof(T) * kCsRows * P.pitch + 2 * kCsRows * sizeof(uint64_t);
  auto kern = cs_atomic_kernel<T, QMAX, VEC4>;
  MSK_ALLOW_SMEM(kern);
  int per_sm = 0;
  MSK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kCsThreads, smem));
  per_sm = std::max(per_sm, 1);
  const int64_t ntiles = (P.d + kCsRows - 1) / kCsRows;
  const int64_t grid = std::min<int64_t>(ntiles, (int64_t)num_sms() * per_sm);
  if (grid <= 0) return MSK_OK;
  kern<<<(unsigned)grid, kCsThreads, smem, st>>>(P);
  MSK_CHECK_LAUNCH("cs_atomic_kernel");
  return MSK_OK;
}

template <typename T>
static int cs_atomic_chunk(CsParams<T> P, cudaStream_t st) {
  if (sizeof(T) == 4) {
    const bool vec4 = (P.ldy % 4 == 0) && ((reinterpret_cast<uintptr_t>(P.Y) & 15) == 0);
    const int ngroups = (P.ncol + 3) / 4;
    P.pitch = 4 * (ngroups | 1);  // pitch / 4 odd
    const int q = (ngroups + kCsWarps - 1) / kCsWarps;
    if (vec4) {
      if (q <= 1) return launch_cs_atomic_t<T, 1, true>(P, st);
      if (q <= 2) return launch_cs_atomic_t<T, 2, true>(P, st);
      if (q <= 4) return launch_cs_atomic_t<T, 4, true>(P, st);
      if (q <= 9) return launch_cs_atomic_t<T, 9, true>(P, st);
      return launch_cs_atomic_t<T, 16, true>(P, st);
    }
    if (q <= 1) return launch_cs_atomic_t<T, 1, false>(P, st);
    if (q <= 2) return launch_cs_atomic_t<T, 2, false>(P, st);
    if (q <= 4) return launch_cs_atomic_t<T, 4, false>(P, st);
    if (q <= 9) return launch_cs_atomic_t<T, 9, false>(P, st);
    return launch_cs_atomic_t<T, 16, false>(P, st);
  }
  P.pitch = P.ncol | 1;  // odd pitch
  const int q = (P.ncol + kCsWarps - 1) / kCsWarps;
  if (q <= 1) return launch_cs_atomic_t<T, 1, false>(P, st);
  if (q <= 4) return launch_cs_atomic_t<T, 4, false>(P, st);
  if (q <= 8) return launch_cs_atomic_t<T, 8, false>(P, st);
  if (q <= 17) return launch_cs_atomic_t<T, 17, false>(P, st);
  if (q <= 33) return launch_cs_atomic_t<T, 33, false>(P, st);
  return launch_cs_atomic_t<T, 64, false>(P, st);
}

// FP64 variant with TMA bulk reductions: a lane loads two columns of its row,
// applies the row's sign and stores them as one 16-byte vector (pitch/2 odd:
// conflict-free); then warp 0 hands each row of the tile to the TMA unit with
// one cp.reduce.async.bulk .add.f64 (Y row = 16-byte aligned, length a
// multiple of 16 bytes), so the SM issues one instruction per row instead of
// one reduction per element.  A row buffer is rewritten two tiles later, after
// its bulk reads have drained (cp.async.bulk.wait_group.read 1, then a CTA
// barrier).  nbulk = columns handed to the bulk unit (even); an odd last
// column that may not be padded goes through a warp reduction.
template <int QMAX>
__global__ void __launch_bounds__(kCsThreads) cs_bulk_f64_kernel(const CsParams<double> P, int nbulk) {
  extern __shared__ __align__(16) unsigned char cs_smem[];
  double* tiles = reinterpret_cast<double*>(cs_smem);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int npairs = (P.ncol + 1) >> 1;
  const int64_t ntiles = (P.d + kCsRows - 1) / kCsRows;
  int buf = 0;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, buf ^= 1) {
    const int64_t i0 = t * kCsRows;
    const int64_t i = i0 + lane;
    const bool row_ok = i < P.d;
    const uint64_t z = row_ok ? draw(P.key, (uint64_t)(P.i0 + i)) : 0ull;
    const unsigned long long sgn = negative_of(z) ? 0x8000000000000000ull : 0ull;
    double* tile = tiles + buf * kCsRows * P.pitch;
    double2 v[QMAX];
#pragma unroll
    for (int q = 0; q < QMAX; ++q) {
      const int g = warp + q * kCsWarps;
      double2 x = make_double2(0.0, 0.0);
      if (row_ok && g < npairs) {
        x.x = load_col(P, i, 2 * g);
        x.y = load_col(P, i, 2 * g + 1);
      }
      x.x = __longlong_as_double(__double_as_longlong(x.x) ^ sgn);
      x.y = __longlong_as_double(__double_as_longlong(x.y) ^ sgn);
      v[q] = x;
    }
    if (warp == 0) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
    __syncthreads();  // buffer `buf` no longer read by the bulk unit
#pragma unroll
    for (int q = 0; q < QMAX; ++q) {
      const int g = warp + q * kCsWarps;
      if (g < npairs) *reinterpret_cast<double2*>(&tile[lane * P.pitch + 2 * g]) = v[q];
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
      bool bucket_ok = true;
      MSK_CHECK_OR(bucket_of(z, P.k) < P.k, kCheckBucket, bucket_ok = false);
      if (row_ok && bucket_ok) {
        double* yrow = P.Y + (int64_t)bucket_of(z, P.k) * P.ldy;
        const uint32_t src = (uint32_t)__cvta_generic_to_shared(tile + lane * P.pitch);
        if (nbulk > 0)
          asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.f64 [%0], [%1], %2;"
                       ::"l"(yrow), "r"(src), "r"(nbulk * 8)
                       : "memory");
        if (nbulk < P.ncol) red_add(yrow + nbulk, tile[lane * P.pitch + nbulk]);
      }
      asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    }
  }
  if (warp == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

template <int QMAX>
static int launch_cs_bulk_t(const CsParams<double>& P, int nbulk, cudaStream_t st) {
  const size_t smem = 2 * sizeof(double) * kCsRows * P.pitch;
  auto kern = cs_bulk_f64_kernel<QMAX>;
  MSK_ALLOW_SMEM(kern);
  int per_sm = 0;
  MSK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kCsThreads, smem));
  per_sm = std::max(per_sm, 1);
  const int64_t ntiles = (P.d + kCsRows - 1) / kCsRows;
  const int64_t grid = std::min<int64_t>(ntiles, (int64_t)num_sms() * per_sm);
  if (grid <= 0) return MSK_OK;
  kern<<<(unsigned)grid, kCsThreads, smem, st>>>(P, nbulk);
  MSK_CHECK_LAUNCH("cs_bulk_f64_kernel");
  return MSK_OK;
}

// Returns 1 when the bulk variant ran, 0 when it does not apply.
static int cs_bulk_f64_chunk(CsParams<double> P, bool pad_ok, cudaStream_t st, int* rc) {
  *rc = MSK_OK;
  if (tune_get("cs.f64.variant", 0) != 1) return 0;
  if ((reinterpret_cast<uintptr_t>(P.Y) & 15) != 0 || (P.ldy & 1) != 0) return 0;
  int nbulk = P.ncol & ~1;
  if ((P.ncol & 1) && pad_ok && P.ldy >= P.ncol + 1) nbulk = P.ncol + 1;
  const int npairs = (P.ncol + 1) >> 1;
  P.pitch = 2 * (npairs | 1);  // pitch/2 odd, pitch >= ncol (+1 pad column, zero)
  const int q = (npairs + kCsWarps - 1) / kCsWarps;
  if (q <= 1) *rc = launch_cs_bulk_t<1>(P, nbulk, st);
  else if (q <= 2) *rc = launch_cs_bulk_t<2>(P, nbulk, st);
  else if (q <= 4) *rc = launch_cs_bulk_t<4>(P, nbulk, st);
  else if (q <= 9) *rc = launch_cs_bulk_t<9>(P, nbulk, st);
  else if (q <= 17) *rc = launch_cs_bulk_t<17>(P, nbulk, st);
  else *rc = launch_cs_bulk_t<24>(P, nbulk, st);
  return 1;
}

// Fixed-width variants (NCA = A columns per launch, known at compile time,
// plus an optional b column): fully unrolled loads, the row's sign applied
// by XOR of the sign bit while transposing, fixed reduction offsets.  Same
// tile scheme as cs_atomic_kernel.  FP64: lane = column, red.add.f64.
// FP32: 4 columns per lane, red.add.v4.f32 (a row of 4*L columns takes L
// lanes; several rows per warp instruction when 4*L < 128).
// FP64 accumulation; A is FP64, or FP32 widened exactly (TA = float) — the
// FP64 sketch of a matrix stored in binary32.
// PF: the next tile's loads are issued right after the barrier, so they are
// in flight while this tile's reductions go out (one tile of A in registers
// ahead of the shared-memory tile); without PF a tile's loads start after the
// previous tile's reductions.  Knob "cs.f64.prefetch": 1 on, 0 off, unset =
// on from 128 columns up.
template <int NCA, bool HAS_B, typename TA, bool PF>
__global__ void __launch_bounds__(kCsThreads) cs_fixed_f64_kernel(const CsParams<double> P,
                                                               const TA* __restrict__ Aa) {
  constexpr int NCOL = NCA + (HAS_B ? 1 : 0);
  constexpr int PITCH = NCOL | 1;
  constexpr int Q = (NCA + kCsWarps - 1) / kCsWarps;
  __shared__ double tiles[2][kCsRows][PITCH];
  __shared__ uint64_t hz[2][kCsRows];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nca = P.ncol_a;  // <= NCA: the kernel serves any width up to NCA
  const int64_t ntiles = (P.d + kCsRows - 1) / kCsRows;
  double v[Q];
  double vb = 0.0;
  uint64_t zr = 0;
  auto load = [&](int64_t t) {
    const int64_t i = t * kCsRows + lane;
    const bool row_ok = i < P.d;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int j = warp + q * kCsWarps;
      v[q] = (row_ok && j < nca) ? (double)__ldcs(Aa + i + (int64_t)j * P.lda) : 0.0;
    }
    if (HAS_B && warp == kCsWarps - 1) vb = row_ok ? __ldcs(P.b + i) : 0.0;
    if (warp == 0) zr = row_ok ? draw(P.key, (uint64_t)(P.i0 + i)) : 0ull;
  };
  int buf = 0;
  if (PF && (int64_t)blockIdx.x < ntiles) load(blockIdx.x);
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, buf ^= 1) {
    if (!PF) load(t);
    const int64_t i0 = t * kCsRows;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int j = warp + q * kCsWarps;
      if (j < nca) tiles[buf][lane][j] = v[q];  // column nca is b's slot
    }
    if (HAS_B && warp == kCsWarps - 1) tiles[buf][lane][nca] = vb;
    if (warp == 0) hz[buf][lane] = zr;
    __syncthreads();
    if (PF && t + gridDim.x < ntiles) load(t + gridDim.x);
#pragma unroll
    for (int rr = 0; rr < kCsRows / kCsWarps; ++rr) {
      const int r = warp + rr * kCsWarps;
      if (i0 + r >= P.d) break;
      const uint64_t z = hz[buf][r];
      MSK_CHECK_OR(bucket_of(z, P.k) < P.k, kCheckBucket, continue);
      double* yrow = P.Y + (int64_t)bucket_of(z, P.k) * P.ldy;
      const unsigned long long sg = negative_of(z) ? 0x8000000000000000ull : 0ull;
#pragma unroll
      for (int c = lane; c < NCA; c += 32)
        if (c < nca) red_add(yrow + c, flip(tiles[buf][r][c], sg));
      if (HAS_B && lane == 0) red_add(yrow + nca, flip(tiles[buf][r][nca], sg));
    }
  }
}



// Narrow FP64 variant (at most 32 A columns): a 32-row tile of 16 or 32
// columns carries too few elements for its barrier, hash and address work,
// so a tile here is RB blocks of 32 rows (lane = row within a block in the
// load phase; warp rb < RB hashes block rb), and in the reduction phase
// NCA lanes cover a row, i.e. two rows per warp instruction at 16 columns.
// nrep > 1: CTA c adds into replica c % nrep of Y (P.Y + (c % nrep) *
// rep_stride): with k = 2n^2 the sketch of a narrow A has only a few hundred
// to a few thousand 128-byte lines, and the L2 serialises reductions to the
// same line; the replicas are summed into Y afterwards.
template <int NCA, bool HAS_B, typename TA, int RB>
__global__ void __launch_bounds__(kCsThreads) cs_narrow_f64_kernel(const CsParams<double> P,
                                                                const TA* __restrict__ Aa,
                                                                int nrep, int64_t rep_stride) {
  static_assert(NCA == 16 || NCA == 32, "narrow widths");
  static_assert(RB >= 1 && RB <= kCsWarps, "one hashing warp per row block");
  constexpr int ROWS = 32 * RB;
  constexpr int NCOL = NCA + (HAS_B ? 1 : 0);
  constexpr int PITCH = NCOL | 1;
  constexpr int Q = NCA / kCsWarps;  // columns per warp in the load phase
  constexpr int RPI = 32 / NCA;      // rows per warp instruction in the reduction
  __shared__ double tiles[2][ROWS][PITCH];
  __shared__ uint64_t hz[2][ROWS];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nca = P.ncol_a;  // <= NCA
  const int64_t ntiles = (P.d + ROWS - 1) / ROWS;
  double* const ybase = P.Y + (nrep > 1 ? (int64_t)(blockIdx.x % nrep) * rep_stride : 0);
  int buf = 0;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, buf ^= 1) {
    const int64_t i0 = t * ROWS;
    double v[RB][Q];
    double vb[RB];
    uint64_t zr = 0;
#pragma unroll
    for (int rb = 0; rb < RB; ++rb) {
      const int64_t i = i0 + rb * 32 + lane;
      const bool row_ok = i < P.d;
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const int j = warp + q * kCsWarps;
        v[rb][q] = (row_ok && j < nca) ? (double)__ldcs(Aa + i + (int64_t)j * P.lda) : 0.0;
      }
      vb[rb] = (HAS_B && warp == kCsWarps - 1 && row_ok) ? __ldcs(P.b + i) : 0.0;
      if (warp == rb) zr = row_ok ? draw(P.key, (uint64_t)(P.i0 + i)) : 0ull;
    }
#pragma unroll
    for (int rb = 0; rb < RB; ++rb) {
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const int j = warp + q * kCsWarps;
        if (j < nca) tiles[buf][rb * 32 + lane][j] = v[rb][q];
      }
      if (HAS_B && warp == kCsWarps - 1) tiles[buf][rb * 32 + lane][nca] = vb[rb];
    }
    if (warp < RB) hz[buf][warp * 32 + lane] = zr;
    __syncthreads();
    const int c = lane % NCA;
#pragma unroll
    for (int r0 = warp * RPI; r0 < ROWS; r0 += kCsWarps * RPI) {
      const int r = r0 + lane / NCA;
      if (i0 + r < P.d) {
        const uint64_t z = hz[buf][r];
        MSK_CHECK_OR(bucket_of(z, P.k) < P.k, kCheckBucket, continue);
        double* yrow = ybase + (int64_t)bucket_of(z, P.k) * P.ldy;
        const unsigned long long sg = negative_of(z) ? 0x8000000000000000ull : 0ull;
        if (c < nca) red_add(yrow + c, flip(tiles[buf][r][c], sg));
        if (HAS_B && c == 0) red_add(yrow + nca, flip(tiles[buf][r][nca], sg));
      }
    }
  }
}


template <int NCA, bool HAS_B>
struct CsF32Tile {
  static constexpr int NG = (NCA + 3) / 4;           // 4-column groups of A
  static constexpr int PITCH = 4 * ((NG + 1) | 1);   // room for b's group, pitch/4 odd
  static constexpr int QG = (NG + kCsWarps - 1) / kCsWarps;
  static constexpr int LPR = NCA / 4 < 32 ? NCA / 4 : 32;  // lanes per row (reductions)
  static constexpr int RPI = 32 / LPR;               // rows per warp instruction
  struct Smem {
    float tiles[2][kCsRows][PITCH];
    uint64_t hz[2][kCsRows];
  };
  // A tile's loads into registers (v: this lane's row, the warp's column
  // groups; vb: b by the last warp; zr: the row's hash draw by warp 0).
  struct Regs {
    float4 v[QG];
    float vb;
    uint64_t zr;
  };
  __device__ __forceinline__ static void load(const CsParams<float>& P, int64_t i0, Regs& g) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = i0 + lane;
    const bool row_ok = i < P.d;
#pragma unroll
    for (int q = 0; q < QG; ++q) {
      const int gi = warp + q * kCsWarps;
      float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
      if (row_ok && gi < NG) {
        const float* a = P.A + i + (int64_t)(4 * gi) * P.lda;
        x.x = __ldcs(a);
        x.y = __ldcs(a + P.lda);
        x.z = __ldcs(a + 2 * P.lda);
        x.w = __ldcs(a + 3 * P.lda);
      }
      g.v[q] = x;
    }
    g.vb = 0.f;
    if (HAS_B && warp == kCsWarps - 1) g.vb = row_ok ? (float)__ldcs(P.b + i) : 0.f;
    g.zr = 0ull;
    if (warp == 0) g.zr = row_ok ? draw(P.key, (uint64_t)(P.i0 + i)) : 0ull;
  }
  __device__ __forceinline__ static void store(const Regs& g, int buf, Smem& sm) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < QG; ++q) {
      const int gi = warp + q * kCsWarps;
      if (gi < NG) *reinterpret_cast<float4*>(&sm.tiles[buf][lane][4 * gi]) = g.v[q];
    }
    if (HAS_B && warp == kCsWarps - 1) sm.tiles[buf][lane][NCA] = g.vb;
    if (warp == 0) sm.hz[buf][lane] = g.zr;
  }
  // reduction phase: RPI rows per warp instruction, row groups spread over warps
  __device__ __forceinline__ static void reduce(const CsParams<float>& P, int64_t i0, int buf,
                                                Smem& sm) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int r0 = warp * RPI; r0 < kCsRows; r0 += kCsWarps * RPI) {
      const int r = r0 + lane / LPR;
      const int cl = lane % LPR;
      const bool ok = i0 + r < P.d;
      const uint64_t z = sm.hz[buf][r];
      MSK_CHECK_OR(bucket_of(z, P.k) < P.k, kCheckBucket, continue);
      float* yrow = P.Y + (int64_t)bucket_of(z, P.k) * P.ldy;
      const unsigned sg = negative_of(z) ? 0x80000000u : 0u;
      if (ok) {
#pragma unroll
        for (int c = 4 * cl; c < NCA; c += 4 * LPR) {
          const float4 x = *reinterpret_cast<const float4*>(&sm.tiles[buf][r][c]);
          red_add_v4(yrow + c, flip(x.x, sg), flip(x.y, sg), flip(x.z, sg), flip(x.w, sg));
        }
        if (HAS_B && cl == 0) red_add(yrow + NCA, flip(sm.tiles[buf][r][NCA], sg));
      }
    }
  }
  // One 32-row tile starting at row i0 of problem P into buffer `buf`.
  __device__ __forceinline__ static void run(const CsParams<float>& P, int64_t i0, int buf,
                                             Smem& sm) {
    Regs g;
    load(P, i0, g);
    store(g, buf, sm);
    __syncthreads();
    reduce(P, i0, buf, sm);
  }
};

// PF: the next tile's loads are issued right after the barrier (see
// cs_fixed_f64_kernel).  Knob "cs.f32.prefetch": 1 on, 0 off, unset = on at
// 128 columns only (measured +3% there, -2% at 256, -15% at 16).
template <int NCA, bool HAS_B, bool PF>
__global__ void __launch_bounds__(kCsThreads) cs_fixed_f32_kernel(const CsParams<float> P) {
  using Tl = CsF32Tile<NCA, HAS_B>;
  __shared__ __align__(16) typename Tl::Smem sm;
  const int64_t ntiles = (P.d + kCsRows - 1) / kCsRows;
  int buf = 0;
  if (!PF) {
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, buf ^= 1)
      Tl::run(P, t * kCsRows, buf, sm);
    return;
  }
  typename Tl::Regs g;
  if ((int64_t)blockIdx.x < ntiles) Tl::load(P, (int64_t)blockIdx.x * kCsRows, g);
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, buf ^= 1) {
    Tl::store(g, buf, sm);
    __syncthreads();
    if (t + gridDim.x < ntiles) Tl::load(P, (t + gridDim.x) * kCsRows, g);
    Tl::reduce(P, t * kCsRows, buf, sm);
  }
}

// Batched form: many problems of the same width in one persistent launch.
// Tiles of all problems are numbered consecutively (tile_begin[j] = first
// global tile of problem j, tile_begin[nprob] = total); a CTA walks global
// tiles and finds each tile's problem by binary search.
template <int NCA>
__global__ void __launch_bounds__(kCsThreads) cs_batch_f32_kernel(const CsParams<float>* __restrict__ Ps,
                                                               const int64_t* __restrict__ tile_begin,
                                                               int nprob) {
  __shared__ __align__(16) typename CsF32Tile<NCA, true>::Smem sm;
  const int64_t total = tile_begin[nprob];
  int buf = 0;
  for (int64_t t = blockIdx.x; t < total; t += gridDim.x, buf ^= 1) {
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tile_begin[mid] <= t) lo = mid; else hi = mid - 1;
    }
    const CsParams<float> P = Ps[lo];
    CsF32Tile<NCA, true>::run(P, (t - tile_begin[lo]) * kCsRows, buf, sm);
  }
}

template <typename KernT, typename ParT, typename... Extra>
static int launch_fixed_rows(KernT kern, int rows, const ParT& P, cudaStream_t st,
                             Extra... extra) {
  int per_sm = 0;
  MSK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kCsThreads, 0));
  per_sm = std::max(per_sm, 1);
  const int64_t ntiles = (P.d + rows - 1) / rows;
  const int64_t grid = std::min<int64_t>(ntiles, (int64_t)num_sms() * per_sm);
  if (grid <= 0) return MSK_OK;
  kern<<<(unsigned)grid, kCsThreads, 0, st>>>(P, extra...);
  MSK_CHECK_LAUNCH("cs_fixed_kernel");
  return MSK_OK;
}
template <typename KernT, typename ParT, typename... Extra>
static int launch_fixed(KernT kern, const ParT& P, cudaStream_t st, Extra... extra) {
  return launch_fixed_rows(kern, kCsRows, P, st, extra...);
}

// Batched FP32 CountSketch launch over `nprob` problems of A-width nca with a
// b column each (Ps, tile_begin in device memory; total tiles known here).
int launch_cs_batch_f32(int nca, const CsParams<float>* Ps, const int64_t* tile_begin, int nprob,
                        int64_t total_tiles, cudaStream_t st) {
  if (total_tiles <= 0 || nprob <= 0) return MSK_OK;
  auto go = [&](auto kern) -> int {
    int per_sm = 0;
    MSK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kCsThreads, 0));
    per_sm = std::max(per_sm, 1);
    const int64_t grid = std::min<int64_t>(total_tiles, (int64_t)num_sms() * per_sm);
    kern<<<(unsigned)grid, kCsThreads, 0, st>>>(Ps, tile_begin, nprob);
    MSK_CHECK_LAUNCH("cs_batch_f32_kernel");
    return MSK_OK;
  };
  switch (nca) {
    case 16: return go(cs_batch_f32_kernel<16>);
    case 32: return go(cs_batch_f32_kernel<32>);
    case 64: return go(cs_batch_f32_kernel<64>);
    case 128: return go(cs_batch_f32_kernel<128>);
    case 256: return go(cs_batch_f32_kernel<256>);
    default: return MSK_ENOTSUP;
  }
}

// Replicas of Y for the narrow FP64 kernel: doubled while the sketch has
// fewer than 8192 distinct 128-byte lines in all, at most 16; used only when
// that gives 8 or more (measured: 16 columns at k = 512, 1.7x; 32 columns at
// k = 2048 with 4 replicas, no gain).
static int cs_replicas(int64_t k, int64_t ncol) {
  const int64_t lines = k * ((ncol * 8 + 127) / 128);
  int r = 1;
  while (r < 16 && lines * r * 2 <= 16384) r *= 2;
  return r >= 8 ? r : 1;
}
size_t cs_replica_bytes(int64_t k, int64_t ncol) {
  if (ncol < 1 || ncol > 33) return 0;
  const int r = cs_replicas(k, ncol);
  return r > 1 ? (size_t)r * (size_t)k * (size_t)ncol * sizeof(double) : 0;
}

// Y[r][c] += sum over the replicas (in replica order) of rep[q][r][c] (Y
// holds zeros, or the sketch of earlier row blocks).
__global__ void cs_replica_sum_kernel(const double* __restrict__ rep, int nrep, int64_t stride,
                                      int64_t k, int ncol, double* __restrict__ Y, int64_t ldy) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < k * ncol;
       e += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < nrep; ++q) s += rep[q * stride + e];
    Y[(e / ncol) * ldy + e % ncol] += s;
  }
}

// Narrow FP64 launch (<= 32 A columns), into replicas of Y when `ws` has room.
template <int NCA, int RB, typename TA>
static int launch_narrow_f64(const CsParams<double>& P0, const TA* Aa, void* ws, size_t ws_bytes,
                             cudaStream_t st) {
  const bool hb = P0.b != nullptr;
  CsParams<double> P = P0;
  int nrep = 1;
  int64_t stride = 0;
  const int r = cs_replicas(P0.k, P0.ncol);
  if (r > 1 && ws && ws_bytes >= (size_t)r * P0.k * P0.ncol * sizeof(double) &&
      tune_get("cs.f64.replicas", 1) != 0) {
    nrep = r;
    stride = (int64_t)P0.k * P0.ncol;
    P.Y = static_cast<double*>(ws);
    P.ldy = P0.ncol;
    MSK_CUDA(cudaMemsetAsync(ws, 0, (size_t)nrep * stride * sizeof(double), st));
  }
  int rc = hb ? launch_fixed_rows(cs_narrow_f64_kernel<NCA, true, TA, RB>, 32 * RB, P, st, Aa, nrep,
                                  stride)
              : launch_fixed_rows(cs_narrow_f64_kernel<NCA, false, TA, RB>, 32 * RB, P, st, Aa, nrep,
                                  stride);
  if (rc || nrep == 1) return rc;
  const int64_t total = (int64_t)P0.k * P0.ncol;
  cs_replica_sum_kernel<<<(unsigned)std::min<int64_t>((total + 255) / 256, num_sms() * 8), 256, 0,
                          st>>>(static_cast<const double*>(ws), nrep, stride, P0.k, P0.ncol, P0.Y,
                                P0.ldy);
  MSK_CHECK_LAUNCH("cs_replica_sum_kernel");
  return MSK_OK;
}

// Returns 1 when a fixed-width kernel covered this chunk.
// FP32 CountSketch with the sketch privatised in shared memory, for few
// buckets (k <= kCsPrivMaxK).  There the tile kernels' reductions queue on
// the L2, which reduces one element per slot whatever its width (an FP32
// element costs the slot of an FP64 one for half the bytes).  Measured on
// 16777216 rows: k = 128, 8 columns + b: 0.54 ms against 1.49 ms for the tile
// kernel; at k = 512 (16 columns) and 2048 (32) it lost (1.59 vs 0.58 ms,
// 1.55 vs 0.68 ms), so larger sketches keep the tile kernels.  CTA
// (chunk, slice) owns rows [chunk R, (chunk + 1) R) and the columns
// [slice cs, slice cs + cs) of Y; it adds its rows into a private k x cs copy
// with shared-memory atomic adds (thread = row: each column's loads are
// coalesced), then adds the copy's nonzero entries into Y (one global
// reduction each).  Every row's bucket and sign are drawn once per slice.
constexpr int kCsPrivThreads = 256;
constexpr size_t kCsPrivBytes = 72 * 1024;  // private copy per CTA (three CTAs per SM)
constexpr int64_t kCsPrivMaxK = 256;

__global__ void __launch_bounds__(kCsPrivThreads) cs_priv_f32_kernel(const CsParams<float> P, int cs,
                                                                  int nslices, int64_t rows) {
  extern __shared__ float ys[];  // k x cs
  const int slice = (int)(blockIdx.x % (unsigned)nslices);
  const int64_t chunk = blockIdx.x / (unsigned)nslices;
  const int c0 = slice * cs, w = min(P.ncol, c0 + cs) - c0;
  const int64_t r0 = chunk * rows, r1 = min(P.d, r0 + rows);
  const int nk = (int)P.k;
  for (int e = threadIdx.x; e < nk * cs; e += kCsPrivThreads) ys[e] = 0.f;
  __syncthreads();
  for (int64_t i = r0 + threadIdx.x; i < r1; i += kCsPrivThreads) {
    const uint64_t z = draw(P.key, (uint64_t)(P.i0 + i));
    const uint32_t bk = bucket_of(z, P.k);
    MSK_CHECK_OR(bk < P.k, kCheckBucket, continue);
    const unsigned sg = negative_of(z) ? 0x80000000u : 0u;
    float* yr = ys + (size_t)bk * cs;
    // eight columns' loads in flight before their shared-memory adds (the
    // compiler keeps loads behind earlier atomics)
    for (int cb = 0; cb < w; cb += 8) {
      float v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int col = c0 + cb + q;
        v[q] = cb + q >= w ? 0.f
                           : (col < P.ncol_a ? __ldcs(P.A + i + (int64_t)col * P.lda) : (float)__ldcs(P.b + i));
      }
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (cb + q < w) atomicAdd(yr + cb + q, flip(v[q], sg));
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nk * w; e += kCsPrivThreads) {
    const int bk = e / w, c = e - bk * w;
    const float v = ys[(size_t)bk * cs + c];
    if (v != 0.f) red_add(P.Y + (int64_t)bk * P.ldy + c0 + c, v);
  }
}

// The privatised kernel for k <= kCsPrivMaxK when it fits (k x cs floats
// within kCsPrivBytes for some cs >= 4) and the rows amortise the copy (every
// CTA >= 8 k rows): returns 1 when it ran.  Knob "cs.f32.priv": 0 off, 2 at
// any k that fits.
static int cs_priv_chunk(const CsParams<float>& P, cudaStream_t st, int* rc) {
  *rc = MSK_OK;
  const long long knob = tune_get("cs.f32.priv", 1);
  if (knob == 0) return 0;
  const int64_t k = P.k;
  if (k < 1 || P.ncol < 1 || P.ncol > 64 || (knob == 1 && k > kCsPrivMaxK)) return 0;
  const int64_t cap = (int64_t)(kCsPrivBytes / sizeof(float)) / k;  // columns that fit
  if (cap < 4 && cap < P.ncol) return 0;
  const int cs = (int)std::min<int64_t>(P.ncol, cap);
  const int nslices = (P.ncol + cs - 1) / cs;
  const int64_t min_rows = 8 * k;
  if (P.d < 2 * min_rows) return 0;
  const size_t smem = (size_t)k * cs * sizeof(float);
  int per_sm = 0;
  if (smem > 48 * 1024)
    MSK_CUDA(cudaFuncSetAttribute(cs_priv_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  MSK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cs_priv_f32_kernel, kCsPrivThreads, smem));
  if (per_sm < 1) return 0;
  const int64_t target = (int64_t)per_sm * num_sms();
  int64_t chunks = std::max<int64_t>(1, target / nslices);
  chunks = std::min<int64_t>(chunks, P.d / min_rows);
  const int64_t rows = (P.d + chunks - 1) / chunks;
  chunks = (P.d + rows - 1) / rows;
  cs_priv_f32_kernel<<<(unsigned)(chunks * nslices), kCsPrivThreads, smem, st>>>(P, cs, nslices, rows);
  MSK_CHECK_LAUNCH("cs_priv_f32_kernel");
  return 1;
}

template <typename T>
static int cs_fixed_chunk(const CsParams<T>& P, cudaStream_t st, int* rc, void* ws = nullptr,
                          size_t ws_bytes = 0) {
  *rc = MSK_OK;
  if (tune_get("cs.fixed", 1) == 0) return 0;
  const bool hb = P.b != nullptr;
  if (P.ncol != P.ncol_a + (hb ? 1 : 0)) return 0;
  const int nca = P.ncol_a;
  if constexpr (sizeof(T) == 8) {
    // register prefetch of the next tile: measured faster from 128 columns
    // up (more loads per thread to hide), slower at 64 and below
    const long long pf_knob = tune_get("cs.f64.prefetch", -1);
#define MSK_FIX64(N)                                                                          \
  if (nca <= N) {                                                                             \
    if (pf_knob > 0 || (pf_knob < 0 && N >= 128))                                             \
      *rc = hb ? launch_fixed(cs_fixed_f64_kernel<N, true, double, true>, P, st, P.A)         \
               : launch_fixed(cs_fixed_f64_kernel<N, false, double, true>, P, st, P.A);       \
    else                                                                                      \
      *rc = hb ? launch_fixed(cs_fixed_f64_kernel<N, true, double, false>, P, st, P.A)        \
               : launch_fixed(cs_fixed_f64_kernel<N, false, double, false>, P, st, P.A);      \
    return 1;                                                                                 \
  }
    if (nca <= 16 && tune_get("cs.f64.narrow", 1) != 0) {
      *rc = launch_narrow_f64<16, 4>(P, P.A, ws, ws_bytes, st);
      return 1;
    }
    if (nca <= 32 && tune_get("cs.f64.narrow", 1) != 0) {
      *rc = launch_narrow_f64<32, 2>(P, P.A, ws, ws_bytes, st);
      return 1;
    }
    MSK_FIX64(16) MSK_FIX64(32) MSK_FIX64(64) MSK_FIX64(128) MSK_FIX64(256)
#undef MSK_FIX64
  } else {
    // v4 reductions need 16-byte aligned Y rows
    if ((P.ldy % 4) != 0 || (reinterpret_cast<uintptr_t>(P.Y) & 15) != 0) return 0;
    const long long pf32 = tune_get("cs.f32.prefetch", -1);
#define MSK_FIX32(N)                                                                  \
  if (nca == N) {                                                                     \
    if (pf32 > 0 || (pf32 < 0 && N == 128))                                           \
      *rc = hb ? launch_fixed(cs_fixed_f32_kernel<N, true, true>, P, st)              \
               : launch_fixed(cs_fixed_f32_kernel<N, false, true>, P, st);            \
    else                                                                              \
      *rc = hb ? launch_fixed(cs_fixed_f32_kernel<N, true, false>, P, st)             \
               : launch_fixed(cs_fixed_f32_kernel<N, false, false>, P, st);           \
    return 1;                                                                         \
  }
    MSK_FIX32(16) MSK_FIX32(32) MSK_FIX32(64) MSK_FIX32(128) MSK_FIX32(256)
#undef MSK_FIX32
  }
  return 0;
}

// FP64 CountSketch of an FP32-stored A (each value widened exactly): the
// fixed-width FP64 kernels with runtime widths, in column chunks of <= 256
// (and L2-resident Y slices).
int launch_cs_f32a_f64y(const float* A, int64_t d, int64_t n, int64_t lda, const double* b,
                        uint32_t k, uint64_t key, double* Y, int64_t ldy, int64_t maxc,
                        cudaStream_t st, int64_t i0) {
  const int64_t nchunks = n > 0 ? (n + maxc - 1) / maxc : 1;
  for (int64_t ch = 0; ch < nchunks; ++ch) {
    const int64_t c0 = ch * maxc, c1 = std::min<int64_t>(n, c0 + maxc);
    const bool last = ch == nchunks - 1;
    CsParams<double> P{};
    P.A = nullptr;
    P.d = d;
    P.lda = lda;
    P.ncol_a = (int)(c1 - c0);
    P.b = (b && last) ? b : nullptr;
    P.ncol = P.ncol_a + (P.b ? 1 : 0);
    if (P.ncol == 0) continue;
    P.k = k;
    P.key = key;
    P.Y = Y + c0;
    P.ldy = ldy;
    P.i0 = i0;
    const float* Ac = A + c0 * lda;
    const bool hb = P.b != nullptr;
    const int w = P.ncol_a;
    int rc;
#define MSK_FIXF(N)                                                                     \
    if (w <= N) {                                                                       \
      rc = hb ? launch_fixed(cs_fixed_f64_kernel<N, true, float, (N >= 128)>, P, st, Ac) \
              : launch_fixed(cs_fixed_f64_kernel<N, false, float, (N >= 128)>, P, st, Ac); \
      if (rc) return rc;                                                                \
      continue;                                                                         \
    }
    if (w <= 16) {
      rc = launch_narrow_f64<16, 4>(P, Ac, nullptr, 0, st);
      if (rc) return rc;
      continue;
    }
    if (w <= 32) {
      rc = launch_narrow_f64<32, 2>(P, Ac, nullptr, 0, st);
      if (rc) return rc;
      continue;
    }
    MSK_FIXF(64) MSK_FIXF(128) MSK_FIXF(256)
#undef MSK_FIXF
    return MSK_ENOTSUP;
  }
  return MSK_OK;
}

template <typename T>
static int cs_atomic_typed(const T* A, int64_t d, int64_t n, int64_t lda, const double* b,
                           uint32_t k, uint64_t key, T* Y, int64_t ldy, bool pad_ok,
                           void* ws, size_t ws_bytes, bool zero, int64_t i0, cudaStream_t st) {
  const int64_t ncol = n + (b ? 1 : 0);
  if (zero) MSK_CUDA(zero_rows(Y, ldy, ncol, k, sizeof(T), st));
  if (d == 0 || ncol == 0) return MSK_OK;
  // Column chunks of at most kCsMaxColsF64/F32; b rides with the last chunk.
  // Column chunks: at most the shared-memory limit, and narrow enough that the
  // chunk's slice of Y (k x chunk) stays resident in L2 (about 40% of it) —
  // reductions that miss L2 turn into DRAM read-modify-writes.  A is still read
  // once: each chunk reads only its own columns.
  int64_t maxc = sizeof(T) == 8 ? kCsMaxColsF64 : kCsMaxColsF32;
  {
    static int l2_bytes = 0;
    if (l2_bytes == 0) {
      int dev = 0;
      if (cudaGetDevice(&dev) != cudaSuccess ||
          cudaDeviceGetAttribute(&l2_bytes, cudaDevAttrL2CacheSize, dev) != cudaSuccess ||
          l2_bytes <= 0)
        l2_bytes = 64 << 20;
    }
    const int64_t budget = tune_get("cs.l2_budget_bytes", (long long)l2_bytes * 2 / 5);
    int64_t fit = budget / ((int64_t)k * (int64_t)sizeof(T));
    // prefer the fixed-width kernels' widths (multiples of 64, or 32/16)
    fit = fit >= 64 ? fit / 64 * 64 : fit >= 32 ? 32 : 16;
    if (fit < maxc) maxc = fit;
  }
  // chunks of A columns; b rides with the last one
  const int64_t nchunks = n > 0 ? (n + maxc - 1) / maxc : 1;
  for (int64_t ch = 0; ch < nchunks; ++ch) {
    const int64_t c0 = ch * maxc, c1 = std::min<int64_t>(n, c0 + maxc);
    const bool last = ch == nchunks - 1;
    CsParams<T> P{};
    P.A = A + c0 * lda;
    P.d = d;
    P.lda = lda;
    P.ncol_a = (int)(c1 - c0);
    P.b = (b && last) ? b : nullptr;
    P.ncol = P.ncol_a + (P.b ? 1 : 0);
    if (P.ncol == 0) continue;
    P.k = k;
    P.key = key;
    P.Y = Y + c0;
    P.ldy = ldy;
    P.i0 = i0;
    int rc = MSK_OK;
    if constexpr (sizeof(T) == 4) {
      if (cs_priv_chunk(P, st, &rc)) {
        if (rc) return rc;
        continue;
      }
    }
    if (cs_fixed_chunk<T>(P, st, &rc, ws, ws_bytes)) {
      if (rc) return rc;
      continue;
    }
    if constexpr (sizeof(T) == 8) {
      if (cs_bulk_f64_chunk(P, pad_ok && last, st, &rc)) {
        if (rc) return rc;
        continue;
      }
    }
    rc = cs_atomic_chunk<T>(P, st);
    if (rc) return rc;
  }
  return MSK_OK;
}

int launch_cs_atomic(const void* A, int dtype, int64_t d, int64_t n, int64_t lda,
                     const double* b, uint32_t k, uint64_t key, void* Y, int64_t ldy,
                     bool pad_ok, cudaStream_t st, void* ws, size_t ws_bytes, bool zero,
                     int64_t i0) {
  if (dtype == MSK_F64)
    return cs_atomic_typed<double>(static_cast<const double*>(A), d, n, lda, b, k, key,
                                   static_cast<double*>(Y), ldy, pad_ok, ws, ws_bytes, zero, i0,
                                   st);
  return cs_atomic_typed<float>(static_cast<const float*>(A), d, n, lda, b, k, key,
                                static_cast<float*>(Y), ldy, pad_ok, nullptr, 0, zero, i0, st);
}

// ---------------------------------------------------------------------------
// SORTED strategy (deterministic).
//   ws layout: count[k] (u32), offs[k+1] (u32), cursor[k] (u32), perm[d] (u32)
size_t cs_sorted_workspace(int64_t d, int64_t k) {
  Need n;
  n.add((size_t)k * 4);
  n.add((size_t)(k + 1) * 4);
  n.add((size_t)k * 4);
  n.add((size_t)std::max<int64_t>(d, 1) * 4);
  return n.used;
}

__global__ void cs_hist_kernel(uint64_t key, int64_t d, uint32_t k, uint32_t* __restrict__ count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d;
       i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&count[bucket_of(draw(key, (uint64_t)i), k)], 1u);
}

// Single-CTA exclusive scan of count[0..k) into offs[0..k] (offs[k] = d).
__global__ void cs_scan_kernel(const uint32_t* __restrict__ count, uint32_t k,
                               uint32_t* __restrict__ offs) {
  __shared__ uint32_t part[1024];
  const uint32_t per = (k + blockDim.x - 1) / blockDim.x;
  const uint32_t lo = threadIdx.x * per, hi = min(k, lo + per);
  uint32_t s = 0;
  for (uint32_t m = lo; m < hi; ++m) s += count[m];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < (int)blockDim.x; off <<= 1) {
    uint32_t x = threadIdx.x >= (unsigned)off ? part[threadIdx.x - off] : 0u;
    __syncthreads();
    part[threadIdx.x] += x;
    __syncthreads();
  }
  uint32_t run = part[threadIdx.x] - s;  // exclusive prefix of this thread's range
  for (uint32_t m = lo; m < hi; ++m) {
    offs[m] = run;
    run += count[m];
  }
  if (threadIdx.x == blockDim.x - 1) offs[k] = part[threadIdx.x];
}

__global__ void cs_scatter_kernel(uint64_t key, int64_t d, uint32_t k,
                                  const uint32_t* __restrict__ offs, uint32_t* __restrict__ cursor,
                                  uint32_t* __restrict__ perm) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t m = bucket_of(draw(key, (uint64_t)i), k);
    perm[offs[m] + atomicAdd(&cursor[m], 1u)] = (uint32_t)i;
  }
}

// Sort each bucket's row list ascending (launched with 256 threads): bitonic
// sort in shared memory for lists up to kSortCap, selection sort otherwise.
constexpr int kSortCap = 2048;
__global__ void cs_segsort_kernel(const uint32_t* __restrict__ offs, uint32_t k,
                                  uint32_t* __restrict__ perm) {
  __shared__ uint32_t keys[kSortCap];
  for (uint32_t m = blockIdx.x; m < k; m += gridDim.x) {
    const uint32_t lo = offs[m], len = offs[m + 1] - offs[m];
    if (len <= 1) continue;
    if (len <= (uint32_t)kSortCap) {
      uint32_t P2 = 1;
      while (P2 < len) P2 <<= 1;
      for (uint32_t t = threadIdx.x; t < P2; t += blockDim.x)
        keys[t] = t < len ? perm[lo + t] : 0xFFFFFFFFu;
      __syncthreads();
      for (uint32_t size = 2; size <= P2; size <<= 1)
        for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
          for (uint32_t t = threadIdx.x; t < P2; t += blockDim.x) {
            const uint32_t u = t ^ stride;
            if (u > t) {
              const bool up = (t & size) == 0;
              const uint32_t a = keys[t], c = keys[u];
              if ((a > c) == up) {
                keys[t] = c;
                keys[u] = a;
              }
            }
          }
          __syncthreads();
        }
      for (uint32_t t = threadIdx.x; t < len; t += blockDim.x) perm[lo + t] = keys[t];
      __syncthreads();
    } else {
      // long list: selection sort, one block-wide argmin per position
      __shared__ uint32_t rb[256], ra[256];
      for (uint32_t pos = 0; pos + 1 < len; ++pos) {
        uint32_t best = 0xFFFFFFFFu, best_at = pos;
        for (uint32_t t = pos + threadIdx.x; t < len; t += blockDim.x) {
          const uint32_t x = perm[lo + t];
          if (x < best) {
            best = x;
            best_at = t;
          }
        }
        rb[threadIdx.x] = best;
        ra[threadIdx.x] = best_at;
        __syncthreads();
        for (int off = blockDim.x / 2; off > 0; off >>= 1) {
          if ((int)threadIdx.x < off && rb[threadIdx.x + off] < rb[threadIdx.x]) {
            rb[threadIdx.x] = rb[threadIdx.x + off];
            ra[threadIdx.x] = ra[threadIdx.x + off];
          }
          __syncthreads();
        }
        if (threadIdx.x == 0) {
          const uint32_t at = ra[0];
          const uint32_t tmp = perm[lo + pos];
          perm[lo + pos] = perm[lo + at];
          perm[lo + at] = tmp;
        }
        __syncthreads();
      }
    }
  }
}

// One warp per bucket: Y[m, c] = sum over the bucket's rows (ascending) of
// s(i) [A b][i, c]; lane = column.
template <typename T>
__global__ void cs_bucket_sum_kernel(const T* __restrict__ A, int64_t lda, int64_t n,
                                     const double* __restrict__ b, int ncol, uint32_t k,
                                     uint64_t key, const uint32_t* __restrict__ offs,
                                     const uint32_t* __restrict__ perm, T* __restrict__ Y,
                                     int64_t ldy) {
  const int lane = threadIdx.x & 31;
  const int64_t warp_g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t m = warp_g; m < k; m += nwarps) {
    const uint32_t lo = offs[m], hi = offs[m + 1];
    for (int c0 = 0; c0 < ncol; c0 += 32) {
      const int c = c0 + lane;
      T acc = 0;
      for (uint32_t t = lo; t < hi; ++t) {
        const uint32_t i = perm[t];
        const bool neg = negative_of(draw(key, (uint64_t)i));
        if (c < ncol) {
          const T x = c < n ? A[(int64_t)i + (int64_t)c * lda] : (T)b[i];
          acc += neg ? -x : x;
        }
      }
      if (c < ncol) Y[m * ldy + c] = acc;
    }
  }
}

// Counting sort of the draws 0..count-1 of stream `key` by
// bucket_of(draw, nb): offs[0..nb] the exclusive prefix of the bucket sizes,
// perm[0..count) the draw indices grouped by bucket (in no fixed order within
// a bucket).  cnt, cursor: nb words of scratch each.
int launch_draw_bucket_sort(uint64_t key, int64_t count, uint32_t nb, uint32_t* offs,
                            uint32_t* perm, uint32_t* cnt, uint32_t* cursor, cudaStream_t st) {
  MSK_CUDA(cudaMemsetAsync(cnt, 0, (size_t)nb * 4, st));
  MSK_CUDA(cudaMemsetAsync(cursor, 0, (size_t)nb * 4, st));
  const unsigned gb =
      (unsigned)std::max<int64_t>(1, std::min<int64_t>((count + 255) / 256, num_sms() * 16));
  if (count > 0) {
    cs_hist_kernel<<<gb, 256, 0, st>>>(key, count, nb, cnt);
    MSK_CHECK_LAUNCH("cs_hist_kernel");
  }
  cs_scan_kernel<<<1, 1024, 0, st>>>(cnt, nb, offs);
  MSK_CHECK_LAUNCH("cs_scan_kernel");
  if (count > 0) {
    cs_scatter_kernel<<<gb, 256, 0, st>>>(key, count, nb, offs, cursor, perm);
    MSK_CHECK_LAUNCH("cs_scatter_kernel");
  }
  return MSK_OK;
}

int launch_cs_sorted(const void* A, int dtype, int64_t d, int64_t n, int64_t lda,
                     const double* b, uint32_t k, uint64_t key, void* Y, int64_t ldy,
                     void* ws, size_t ws_bytes, cudaStream_t st) {
  Carve cv(ws, ws_bytes);
  uint32_t* count = static_cast<uint32_t*>(cv.take((size_t)k * 4));
  uint32_t* offs = static_cast<uint32_t*>(cv.take((size_t)(k + 1) * 4));
  uint32_t* cursor = static_cast<uint32_t*>(cv.take((size_t)k * 4));
  uint32_t* perm = static_cast<uint32_t*>(cv.take((size_t)std::max<int64_t>(d, 1) * 4));
  if (!count || !offs || !cursor || !perm) return MSK_ENOMEM;
  const int ncol = (int)(n + (b ? 1 : 0));
  MSK_CUDA(cudaMemsetAsync(count, 0, (size_t)k * 4, st));
  MSK_CUDA(cudaMemsetAsync(cursor, 0, (size_t)k * 4, st));
  const int sms = num_sms();
  const unsigned gb = (unsigned)std::max<int64_t>(1, std::min<int64_t>((d + 255) / 256, sms * 16));
  if (d > 0) {
    cs_hist_kernel<<<gb, 256, 0, st>>>(key, d, k, count);
    MSK_CHECK_LAUNCH("cs_hist_kernel");
  }
  cs_scan_kernel<<<1, 1024, 0, st>>>(count, k, offs);
  MSK_CHECK_LAUNCH("cs_scan_kernel");
  if (d > 0) {
    cs_scatter_kernel<<<gb, 256, 0, st>>>(key, d, k, offs, cursor, perm);
    MSK_CHECK_LAUNCH("cs_scatter_kernel");
    cs_segsort_kernel<<<(unsigned)std::min<int64_t>(k, sms * 8), 256, 0, st>>>(offs, k, perm);
    MSK_CHECK_LAUNCH("cs_segsort_kernel");
  }
  const unsigned gw = (unsigned)std::max<int64_t>(1, std::min<int64_t>((k + 7) / 8, sms * 16));
  if (dtype == MSK_F64)
    cs_bucket_sum_kernel<double><<<gw, 256, 0, st>>>(static_cast<const double*>(A), lda, n, b,
                                                     ncol, k, key, offs, perm,
                                                     static_cast<double*>(Y), ldy);
  else
    cs_bucket_sum_kernel<float><<<gw, 256, 0, st>>>(static_cast<const float*>(A), lda, n, b,
                                                    ncol, k, key, offs, perm,
                                                    static_cast<float*>(Y), ldy);
  MSK_CHECK_LAUNCH("cs_bucket_sum_kernel");
  return MSK_OK;
}

}  // namespace msk
