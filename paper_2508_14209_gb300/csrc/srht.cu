// srht.cu — the subsampled randomized Hadamard transform of Section 5 applied
// to a column-major [A b] with d = 2^m rows:
//     Y = (1/sqrt(k)) P H_d D [A b]
//   D   : d_ii = -1 when bit 0 of draw i of stream tag 5 is set, else +1;
//   H_d : the Hadamard matrix of the recursive definition,
//         H_d[i][j] = (-1)^popcount(i & j), applied by the fast Walsh-Hadamard
//         transform: one butterfly stage per bit of the row index; the stages
//         commute, so they may run in any order;
//   P   : row l of P picks row j_l = bucket_of(draw l of stream tag 6, d) of
//         H D [A b], uniformly and with replacement (the row-sampling reading
//         of the definition);
//   Y[l][c] = (H D x_c)[j_l] / sqrt(k), row-major k x (n+1) with ldy, like
//   cs_sketch's output.
// Butterflies are radix 4 as in Algorithm 3 (two stages per sweep of shared
// memory): x, y, z, t at stride s become (x+z)+(y+t), (x+z)-(y+t),
// (x-z)+(y-t), (x-z)-(y-t); an odd number of stages ends with one radix-2
// stage.  Up to 2^13 rows a column is transformed whole in shared memory
// (one pass: D applied while loading, P while storing).  Longer columns take
// two passes over a d x (n+1) FP64 scratch:
//   pass 1: D and the stages of the high h = m - 13 bits of the row index, on
//           tiles of 2^h rows x L = 2^(13-h) consecutive low indices (every
//           global access is an L*8-byte segment);
//   pass 2: the stages of the low 13 bits on contiguous tiles of 2^13 rows,
//           storing only the sampled rows of each tile (the k samples are
//           counting-sorted by tile first).
// One FP64 add per element and stage: the FP64 pipe bounds both passes on
// GB300.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <type_traits>

#include "msk_device.cuh"
#include "msk_internal.h"

namespace msk {

constexpr int kSrTileBits = 13;               // 2^13 FP64 = 64 KB of shared memory per tile
constexpr int kSrThreads = 512;
constexpr int kSrMaxBits = kSrTileBits + 13;  // d <= 2^26 (pass-1 tiles down to L = 1)

template <typename TA>
__device__ __forceinline__ double sr_x(const TA* A, int64_t lda, int64_t n, const double* b,
                                       int64_t i, int64_t c) {
  return c < n ? (double)A[i + c * lda] : b[i];
}

// The butterfly stages of `bits` index bits on 2^bits rows of L contiguous
// elements (element (h, l) at s[h * L + l]), radix 4 then one radix-2 stage
// for an odd count.  Ends with a barrier.
__device__ __forceinline__ void sr_fwht_smem(double* s, int bits, int L) {
  const int nrow = 1 << bits;
  int q = 0;
  for (; q + 1 < bits; q += 2) {
    const int st = 1 << q;
    const int sl = st * L;
    const int nbf = (nrow >> 2) * L;
    for (int u = threadIdx.x; u < nbf; u += blockDim.x) {
      const int l = u % L, hq = u / L;
      const int h0 = ((hq >> q) << (q + 2)) | (hq & (st - 1));
      double* p = s + h0 * L + l;
      const double x = p[0], y = p[sl], z = p[2 * sl], t = p[3 * sl];
      const double X = x + z, Y = y + t, Z = x - z, T = y - t;
      p[0] = X + Y;
      p[sl] = X - Y;
      p[2 * sl] = Z + T;
      p[3 * sl] = Z - T;
    }
    __syncthreads();
  }
  if (q < bits) {
    const int st = 1 << q;
    const int sl = st * L;
    const int nbf = (nrow >> 1) * L;
    for (int u = threadIdx.x; u < nbf; u += blockDim.x) {
      const int l = u % L, hq = u / L;
      const int h0 = ((hq >> q) << (q + 1)) | (hq & (st - 1));
      double* p = s + h0 * L + l;
      const double x = p[0], y = p[sl];
      p[0] = x + y;
      p[sl] = x - y;
    }
    __syncthreads();
  }
}

// Pass 1 of a two-pass transform: CTA (lb, c) takes rows
// (h << tbits) + lb * L + l, h < 2^hbits, l < L, of column c of [A b], applies
// D and the stages of the high bits, and writes them to the scratch T.
template <typename TA>
__global__ void __launch_bounds__(kSrThreads) srht_high_kernel(const TA* __restrict__ A,
                                                            int64_t lda, int64_t n,
                                                            const double* __restrict__ b,
                                                            int64_t d, int tbits, int hbits,
                                                            uint64_t dkey, double* __restrict__ T) {
  extern __shared__ double sr_s[];
  const int L = (1 << tbits) >> hbits;
  const int64_t lb = blockIdx.x, c = blockIdx.y;
  const int nel = (1 << hbits) * L;
  for (int e = threadIdx.x; e < nel; e += blockDim.x) {
    const int h = e / L, l = e % L;
    const int64_t g = ((int64_t)h << tbits) + lb * L + l;
    const double x = sr_x(A, lda, n, b, g, c);
    sr_s[e] = negative_of(draw(dkey, (uint64_t)g)) ? -x : x;
  }
  __syncthreads();
  sr_fwht_smem(sr_s, hbits, L);
  double* Tc = T + c * d;
  for (int e = threadIdx.x; e < nel; e += blockDim.x) {
    const int h = e / L, l = e % L;
    Tc[((int64_t)h << tbits) + lb * L + l] = sr_s[e];
  }
}

// Last pass: CTA (q, c) transforms rows [q 2^tbits, (q+1) 2^tbits) of column
// c along the low tbits bits — from the scratch T (two passes) or straight
// from [A b] with D (one pass) — and stores the sampled rows of the tile:
// samples perm[offs[q] .. offs[q+1]).  The 8 lowest bits go in registers and
// warp shuffles (their strides, 1 to 128 elements, conflict in shared memory).
template <typename TA, bool FROM_A>
__global__ void __launch_bounds__(kSrThreads) srht_low_kernel(
    const TA* __restrict__ A, int64_t lda, int64_t n, const double* __restrict__ b, int64_t d,
    int tbits, uint64_t dkey, const double* __restrict__ T, uint64_t pkey,
    const uint32_t* __restrict__ offs, const uint32_t* __restrict__ perm, double sqrt_k,
    double* __restrict__ Y, int64_t ldy) {
  extern __shared__ double sr_s[];
  const int64_t q = blockIdx.x, c = blockIdx.y;
  const int nel = 1 << tbits;
  const int64_t g0 = q << tbits;
  const double* Tc = FROM_A ? nullptr : T + c * d + g0;
  auto load = [&](int e) -> double {
    if (FROM_A) {
      const int64_t g = g0 + e;
      const double x = sr_x(A, lda, n, b, g, c);
      return negative_of(draw(dkey, (uint64_t)g)) ? -x : x;
    }
    return Tc[e];
  };
  if (tbits >= 8) {
    // the 8 low bits in registers: a warp takes 256 consecutive rows, lane =
    // bits 0-4 (butterflies by shuffle), register j = bits 5-7 (butterflies
    // within the thread); then the stages of the higher bits in shared
    // memory on rows of 256 contiguous elements (conflict-free)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nw = (int)(blockDim.x >> 5);
    for (int w = warp; w < (nel >> 8); w += nw) {
      const int base = w << 8;
      double x[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) x[j] = load(base + j * 32 + lane);
#pragma unroll
      for (int t = 0; t < 3; ++t)
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (!(j & (1 << t))) {
            const double a = x[j], v = x[j | (1 << t)];
            x[j] = a + v;
            x[j | (1 << t)] = a - v;
          }
#pragma unroll
      for (int bt = 0; bt < 5; ++bt) {
        // lo + hi on the lane whose bit is clear, lo - hi on its partner: one
        // exact-product FMA either way (x * -1 + o is o - x exactly)
        const double sg = (lane & (1 << bt)) ? -1.0 : 1.0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const double o = __shfl_xor_sync(0xffffffffu, x[j], 1 << bt);
          x[j] = fma(x[j], sg, o);
        }
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) sr_s[base + j * 32 + lane] = x[j];
    }
    __syncthreads();
    sr_fwht_smem(sr_s, tbits - 8, 256);
  } else {
    for (int e = threadIdx.x; e < nel; e += blockDim.x) sr_s[e] = load(e);
    __syncthreads();
    sr_fwht_smem(sr_s, tbits, 1);
  }
  for (uint32_t u = offs[q] + threadIdx.x; u < offs[q + 1]; u += blockDim.x) {
    const uint32_t l = perm[u];
    const uint32_t j = bucket_of(draw(pkey, (uint64_t)l), (uint32_t)d);
    Y[(int64_t)l * ldy + c] = sr_s[j - (uint32_t)g0] / sqrt_k;
  }
}

struct SrhtPlan {
  int m, tbits, hbits;
  int64_t ntiles;  // tiles of the last pass per column (= 2^hbits)
};

static bool srht_plan(int64_t d, SrhtPlan* p) {
  if (d < 2 || (d & (d - 1)) != 0) return false;
  int m = 0;
  while ((int64_t(1) << m) < d) ++m;
  if (m > kSrMaxBits) return false;
  p->m = m;
  p->tbits = std::min(m, kSrTileBits);
  p->hbits = m - p->tbits;
  p->ntiles = int64_t(1) << p->hbits;
  return true;
}

size_t srht_workspace(int64_t d, int64_t ncol, int64_t k) {
  SrhtPlan p;
  if (!srht_plan(d, &p)) return 0;
  Need nd;
  if (p.hbits > 0) nd.add((size_t)d * ncol * sizeof(double));  // scratch
  nd.add((size_t)(p.ntiles + 1) * 4);                          // offs
  nd.add((size_t)p.ntiles * 4);                                 // counts
  nd.add((size_t)p.ntiles * 4);                                 // cursors
  nd.add((size_t)std::max<int64_t>(k, 1) * 4);                  // perm
  return nd.used;
}

int launch_srht(const void* A, int dtype, int64_t d, int64_t n, int64_t lda, const double* b,
                int64_t k, uint64_t seed, double* Y, int64_t ldy, void* ws, size_t ws_bytes,
                cudaStream_t st) {
  SrhtPlan p;
  if (!srht_plan(d, &p)) return MSK_ENOTSUP;
  const int64_t ncol = n + (b ? 1 : 0);
  if (ncol < 1 || ncol > 65535 || k < 1 || k > 0xFFFFFFFFLL) return MSK_ENOTSUP;
  Carve cv(ws, ws_bytes);
  double* T = p.hbits > 0 ? static_cast<double*>(cv.take((size_t)d * ncol * sizeof(double)))
                          : nullptr;
  uint32_t* offs = static_cast<uint32_t*>(cv.take((size_t)(p.ntiles + 1) * 4));
  uint32_t* cnt = static_cast<uint32_t*>(cv.take((size_t)p.ntiles * 4));
  uint32_t* cursor = static_cast<uint32_t*>(cv.take((size_t)p.ntiles * 4));
  uint32_t* perm = static_cast<uint32_t*>(cv.take((size_t)std::max<int64_t>(k, 1) * 4));
  if ((p.hbits > 0 && !T) || !offs || !cnt || !cursor || !perm) return MSK_ENOMEM;
  const uint64_t dkey = stream_key(seed, kTagSrhtSign), pkey = stream_key(seed, kTagSrhtRow);
  // samples by tile of the last pass: tile of j_l = bucket_of(z, d) >> tbits
  // = bucket_of(z, 2^hbits) for the power-of-two d
  int rc = launch_draw_bucket_sort(pkey, k, (uint32_t)p.ntiles, offs, perm, cnt, cursor, st);
  if (rc) return rc;
  const size_t smem = (size_t)sizeof(double) << p.tbits;
  const double sq = std::sqrt((double)k);
  auto run = [&](auto* Ap) -> int {
    using TA = std::remove_const_t<std::remove_pointer_t<decltype(Ap)>>;
    if (p.hbits > 0) {
      MSK_ALLOW_SMEM(srht_high_kernel<TA>);
      dim3 g1((unsigned)p.ntiles, (unsigned)ncol);
      srht_high_kernel<TA><<<g1, kSrThreads, smem, st>>>(Ap, lda, n, b, d, p.tbits, p.hbits, dkey, T);
      MSK_CHECK_LAUNCH("srht_high_kernel");
      MSK_ALLOW_SMEM((srht_low_kernel<TA, false>));
      dim3 g2((unsigned)p.ntiles, (unsigned)ncol);
      srht_low_kernel<TA, false><<<g2, kSrThreads, smem, st>>>(Ap, lda, n, b, d, p.tbits, dkey, T,
                                                              pkey, offs, perm, sq, Y, ldy);
      MSK_CHECK_LAUNCH("srht_low_kernel");
    } else {
      MSK_ALLOW_SMEM((srht_low_kernel<TA, true>));
      dim3 g2(1u, (unsigned)ncol);
      srht_low_kernel<TA, true><<<g2, kSrThreads, smem, st>>>(Ap, lda, n, b, d, p.tbits, dkey,
                                                             nullptr, pkey, offs, perm, sq, Y, ldy);
      MSK_CHECK_LAUNCH("srht_low_kernel");
    }
    return MSK_OK;
  };
  if (dtype == MSK_F64) return run(static_cast<const double*>(A));
  return run(static_cast<const float*>(A));
}

}  // namespace msk
