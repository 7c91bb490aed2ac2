// rcq.cu — the tall steps of randomized Cholesky QR (Algorithms 4 and 5):
// preconditioning Q0 = A R0^{-1} and, for the explicit factor, Q = Q0 R1^{-1},
// both as a product of the tall column-major operand with an explicit upper-
// triangular inverse; and the small product R = R1 R0.
//
// trmm_upper_kernel: X (d x n, FP64 or FP32 values, ldx) times U (n x n
// upper triangular, FP64, column-major, zeros below the diagonal) into Y
// (d x n, FP64, ldy).  A CTA owns 32-row tiles (persistent grid): the tile of
// X is staged in shared memory (all n columns, odd pitch), U is staged 32 of
// its rows at a time, and each of the 8 warps accumulates 4 rows x NJ column
// groups (lane = column within a group of 32) in registers.  Row blocks of U
// below a column group's diagonal block are zero and skipped, so the work is
// n^2/2 FMAs per row plus half of the 32x32 diagonal blocks.  The finished
// tile goes back through shared memory and is written with lane = row
// (coalesced); all reads of a tile precede its writes, so Y may alias X when
// both are FP64 with the same leading dimension.  The FP64 pipe bounds it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "msk_internal.h"

namespace msk {

constexpr int kTmRows = 32;              // rows per tile
constexpr int kTmThreads = 256;          // 8 warps x 4 rows
constexpr int kTmMaxN = 416;             // 13 column groups of 32

template <int NJ, typename TX>
__global__ void __launch_bounds__(kTmThreads) trmm_upper_kernel(const TX* X, int64_t ldx, int64_t d,
                                                               int n, const double* __restrict__ U,
                                                               double* Y, int64_t ldy) {
  extern __shared__ double tm_smem[];
  const int pitch = n | 1;
  double* xt = tm_smem;                    // kTmRows x pitch: the tile, then the result
  double* us = tm_smem + kTmRows * pitch;  // 32 rows of U x pitch
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t ntiles = (d + kTmRows - 1) / kTmRows;
  const int nlb = (n + 31) / 32;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t i0 = t * kTmRows;
    __syncthreads();  // the previous tile's result has been written out
    for (int e = threadIdx.x; e < kTmRows * n; e += kTmThreads) {
      const int r = e % kTmRows, c = e / kTmRows;
      const int64_t i = i0 + r;
      xt[r * pitch + c] = i < d ? (double)X[i + (int64_t)c * ldx] : 0.0;
    }
    double acc[4][NJ];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int q = 0; q < NJ; ++q) acc[r][q] = 0.0;
    for (int lb = 0; lb < nlb; ++lb) {
      __syncthreads();  // previous block of U consumed (and the tile staged)
      for (int e = threadIdx.x; e < 32 * n; e += kTmThreads) {
        const int l = e % 32, c = e / 32;
        const int lr = lb * 32 + l;
        us[l * pitch + c] = (lr < n && lr <= c) ? U[lr + (int64_t)c * n] : 0.0;
      }
      __syncthreads();
      const int lend = min(32, n - lb * 32);
      for (int ll = 0; ll < lend; ++ll) {
        const int l = lb * 32 + ll;
        double a[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) a[r] = xt[(warp * 4 + r) * pitch + l];
#pragma unroll
        for (int q = 0; q < NJ; ++q) {
          if (q < lb) continue;  // U rows of this block are zero for these columns
          const int c = q * 32 + lane;
          const double u = c < n ? us[ll * pitch + c] : 0.0;
#pragma unroll
          for (int r = 0; r < 4; ++r) acc[r][q] = fma(a[r], u, acc[r][q]);
        }
      }
    }
    __syncthreads();  // every warp is done reading the tile
#pragma unroll
    for (int q = 0; q < NJ; ++q) {
      const int c = q * 32 + lane;
      if (c < n)
#pragma unroll
        for (int r = 0; r < 4; ++r) xt[(warp * 4 + r) * pitch + c] = acc[r][q];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kTmRows * n; e += kTmThreads) {
      const int r = e % kTmRows, c = e / kTmRows;
      const int64_t i = i0 + r;
      if (i < d) Y[i + (int64_t)c * ldy] = xt[r * pitch + c];
    }
  }
}

size_t trmm_upper_smem(int64_t n) { return (size_t)2 * kTmRows * (size_t)(n | 1) * sizeof(double); }

template <typename TX>
static int trmm_dispatch(const TX* X, int64_t ldx, int64_t d, int64_t n, const double* U, double* Y,
                         int64_t ldy, cudaStream_t st) {
  if (d <= 0) return MSK_OK;
  if (n < 1 || n > kTmMaxN) return MSK_ENOTSUP;
  const size_t smem = trmm_upper_smem(n);
  auto go = [&](auto kern) -> int {
    MSK_ALLOW_SMEM(kern);
    int per_sm = 0;
    MSK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTmThreads, smem));
    per_sm = std::max(per_sm, 1);
    const int64_t ntiles = (d + kTmRows - 1) / kTmRows;
    const int64_t grid = std::min<int64_t>(ntiles, (int64_t)num_sms() * per_sm);
    kern<<<(unsigned)grid, kTmThreads, smem, st>>>(X, ldx, d, (int)n, U, Y, ldy);
    MSK_CHECK_LAUNCH("trmm_upper_kernel");
    return MSK_OK;
  };
  if (n <= 32) return go(trmm_upper_kernel<1, TX>);
  if (n <= 64) return go(trmm_upper_kernel<2, TX>);
  if (n <= 128) return go(trmm_upper_kernel<4, TX>);
  if (n <= 256) return go(trmm_upper_kernel<8, TX>);
  return go(trmm_upper_kernel<13, TX>);
}

int launch_trmm_upper(const void* X, int dtype, int64_t ldx, int64_t d, int64_t n, const double* U,
                      double* Y, int64_t ldy, cudaStream_t st) {
  if (dtype == MSK_F64)
    return trmm_dispatch(static_cast<const double*>(X), ldx, d, n, U, Y, ldy, st);
  return trmm_dispatch(static_cast<const float*>(X), ldx, d, n, U, Y, ldy, st);
}

// R = R1 R0 for upper-triangular R1 (ld1) and R0 (ld0), n x n, into R (ldr,
// zeros below the diagonal): R[i][j] = sum_{i <= l <= j} R1[i][l] R0[l][j].
__global__ void tri_mul_upper_kernel(const double* __restrict__ R1, int64_t ld1,
                                     const double* __restrict__ R0, int64_t ld0, int n,
                                     double* __restrict__ R, int64_t ldr) {
  const int64_t total = (int64_t)n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % n), j = (int)(e / n);
    double s = 0.0;
    for (int l = i; l <= j; ++l) s = fma(R1[i + (int64_t)l * ld1], R0[l + (int64_t)j * ld0], s);
    R[i + (int64_t)j * ldr] = i <= j ? s : 0.0;
  }
}

int launch_tri_mul_upper(const double* R1, int64_t ld1, const double* R0, int64_t ld0, int64_t n,
                         double* R, int64_t ldr, cudaStream_t st) {
  const int64_t total = n * n;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 1024);
  tri_mul_upper_kernel<<<blocks, 256, 0, st>>>(R1, ld1, R0, ld0, (int)n, R, ldr);
  MSK_CHECK_LAUNCH("tri_mul_upper_kernel");
  return MSK_OK;
}

}  // namespace msk
