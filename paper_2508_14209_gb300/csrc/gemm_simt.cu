// gemm_simt.cu — the Gaussian stage Z = G Y on CUDA cores, in FP64 (G widened
// exactly from binary32) or FP32 (Section 1 "Count-Gauss"; Section 6.1 does
// this with a cuBLAS GEMM).  The output is tiny (p x ncol) and K = k is long,
// so the K dimension is split across CTAs: CTA (mt, nt, s) computes a 64 x 64
// tile of the partial product over K-slice s and writes it to the workspace;
// a second kernel sums the slices in a fixed order (deterministic).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "msk_device.cuh"
#include "msk_internal.h"

namespace msk {

constexpr int kGBM = 64, kGBK = 32, kGThreads = 256;

// Column-tile width 16 * nc (nc = 2, 3 or 4 columns per thread): the one that
// computes the fewest padded columns (ties to the wider tile).  The FP64 pipe
// bounds these kernels, so padding costs in proportion: at 129 columns 64-wide
// tiles compute 192 columns, 48-wide ones 144.
static int gemm_nc(int64_t ncol) {
  int best = 4;
  int64_t best_cols = (ncol + 63) / 64 * 64;
  for (int nc = 3; nc >= 2; --nc) {
    const int64_t w = 16 * nc, cols = (ncol + w - 1) / w * w;
    if (cols < best_cols) {
      best = nc;
      best_cols = cols;
    }
  }
  return best;
}

struct GemmSplit {
  int mt, nt, s, nc;
  int64_t kchunk;
};

static GemmSplit gemm_split(int64_t p, int64_t k, int64_t ncol) {
  GemmSplit g;
  g.nc = gemm_nc(ncol);
  g.mt = (int)((p + kGBM - 1) / kGBM);
  g.nt = (int)((ncol + 16 * g.nc - 1) / (16 * g.nc));
  const int64_t target = 2LL * num_sms();
  int64_t s = std::max<int64_t>(1, target / std::max(1, g.mt * g.nt));
  s = std::min<int64_t>(s, std::max<int64_t>(1, (k + kGBK - 1) / kGBK));
  int64_t chunk = (k + s - 1) / s;
  chunk = (chunk + kGBK - 1) / kGBK * kGBK;
  g.kchunk = std::max<int64_t>(chunk, kGBK);
  g.s = (int)((k + g.kchunk - 1) / g.kchunk);
  if (g.s < 1) g.s = 1;
  return g;
}

size_t gemm_simt_workspace(int64_t p, int64_t k, int64_t ncol, bool /*f64*/) {
  GemmSplit g = gemm_split(p, k, ncol);
  Need n;
  n.add((size_t)g.s * p * ncol * sizeof(double));
  return n.used;
}

// Partial tile: part[s][c * p + r] = sum_{m in slice s} G[r, m] Y[m, c].
template <typename T, typename TY, int NC>
__global__ void __launch_bounds__(kGThreads) gemm_simt_kernel(const float* __restrict__ G, int64_t ldg,
                                                           const TY* __restrict__ Y, int64_t ldy,
                                                           int64_t p, int64_t k, int64_t ncol,
                                                           int64_t kchunk, double* __restrict__ part) {
  __shared__ T Gs[kGBK][kGBM + 1];
  constexpr int kGBN = 16 * NC;
  __shared__ T Ys[kGBK][kGBN];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t m0 = (int64_t)blockIdx.x * kGBM, n0 = (int64_t)blockIdx.y * kGBN;
  const int64_t kb = (int64_t)blockIdx.z * kchunk, ke = (kb + kchunk < k) ? kb + kchunk : k;
  T acc[4][NC];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[a][c] = (T)0;
  for (int64_t k0 = kb; k0 < ke; k0 += kGBK) {
#pragma unroll
    for (int q = 0; q < (kGBM * kGBK) / kGThreads; ++q) {
      const int e = threadIdx.x + q * kGThreads;
      const int r = e / kGBK, kk = e % kGBK;
      const int64_t gr = m0 + r, gk = k0 + kk;
      Gs[kk][r] = (gr < p && gk < ke) ? (T)G[gr * ldg + gk] : (T)0;
    }
#pragma unroll
    for (int q = 0; q < (kGBN * kGBK) / kGThreads; ++q) {
      const int e = threadIdx.x + q * kGThreads;
      const int kk = e / kGBN, c = e % kGBN;
      const int64_t gk = k0 + kk, gc = n0 + c;
      Ys[kk][c] = (gk < ke && gc < ncol) ? (T)Y[gk * ldy + gc] : (T)0;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < kGBK; ++kk) {
      T av[4], bv[NC];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = Gs[kk][ty + 16 * a];
#pragma unroll
      for (int c = 0; c < NC; ++c) bv[c] = Ys[kk][tx + 16 * c];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[a][c] = fma(av[a], bv[c], acc[a][c]);
    }
    __syncthreads();
  }
  double* out = part + (int64_t)blockIdx.z * p * ncol;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const int64_t r = m0 + ty + 16 * a, cc = n0 + tx + 16 * c;
      if (r < p && cc < ncol) out[cc * p + r] = (double)acc[a][c];
    }
}

// Z[r + c*ldz] = sum_{s=0}^{S-1} part[s][c*p + r], slices added in order.
__global__ void splitk_reduce_kernel(const double* __restrict__ part, int S, int64_t p, int64_t ncol,
                                     double* __restrict__ Z, int64_t ldz) {
  const int64_t total = p * ncol;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < S; ++q) s += part[(int64_t)q * total + e];
    const int64_t c = e / p, r = e - c * p;
    Z[r + c * ldz] = s;
  }
}

int launch_gemm_simt(const float* G, int64_t ldg, const void* Y, bool y_f64, int64_t ldy, bool f64,
                     int64_t p, int64_t k, int64_t ncol, double* Z, int64_t ldz, void* ws,
                     size_t ws_bytes, cudaStream_t st) {
  if (p == 0 || ncol == 0) return MSK_OK;
  GemmSplit g = gemm_split(p, k, ncol);
  Carve cv(ws, ws_bytes);
  double* part = static_cast<double*>(cv.take((size_t)g.s * p * ncol * sizeof(double)));
  if (!part) return MSK_ENOMEM;
  dim3 grid(g.mt, g.nt, g.s);
  auto go = [&](auto nc_tag) {
    constexpr int NC = decltype(nc_tag)::value;
    if (f64 && y_f64)
      gemm_simt_kernel<double, double, NC><<<grid, kGThreads, 0, st>>>(
          G, ldg, static_cast<const double*>(Y), ldy, p, k, ncol, g.kchunk, part);
    else if (f64)
      gemm_simt_kernel<double, float, NC><<<grid, kGThreads, 0, st>>>(
          G, ldg, static_cast<const float*>(Y), ldy, p, k, ncol, g.kchunk, part);
    else if (y_f64)
      gemm_simt_kernel<float, double, NC><<<grid, kGThreads, 0, st>>>(
          G, ldg, static_cast<const double*>(Y), ldy, p, k, ncol, g.kchunk, part);
    else
      gemm_simt_kernel<float, float, NC><<<grid, kGThreads, 0, st>>>(
          G, ldg, static_cast<const float*>(Y), ldy, p, k, ncol, g.kchunk, part);
  };
  if (g.nc == 2) go(std::integral_constant<int, 2>{});
  else if (g.nc == 3) go(std::integral_constant<int, 3>{});
  else go(std::integral_constant<int, 4>{});
  MSK_CHECK_LAUNCH("gemm_simt_kernel");
  const int64_t total = p * ncol;
  splitk_reduce_kernel<<<(unsigned)std::min<int64_t>((total + 255) / 256, num_sms() * 8), 256, 0,
                         st>>>(part, g.s, p, ncol, Z, ldz);
  MSK_CHECK_LAUNCH("splitk_reduce_kernel");
  return MSK_OK;
}

// Gaussian-only sketch of a column-major [A b] (the Gaussian sketch-and-solve
// of Section 6.3, S = G with no CountSketch): Z = G [A b] with G the p x d
// matrix of the multisketch's Gaussian definition at k = d (entry (r, i) is
// standard normal number r*d + i of stream tag 2, divided by sqrt(p) in
// binary32).  G is generated tile by tile inside the product instead of being
// stored (p*d entries: 17 GB at d = 2^23, p = 512); its binary32 arithmetic
// is a few percent of the FP64 products it feeds.  Split over row slices of A
// like gemm_simt_kernel, FP64 accumulation, partials reduced in order.
template <typename TA, int NC>
__global__ void __launch_bounds__(kGThreads) gauss_gemm_kernel(uint64_t gkey, float sqrt_p,
                                                            const TA* __restrict__ A, int64_t lda,
                                                            int64_t d, int64_t n,
                                                            const double* __restrict__ b, int64_t p,
                                                            int64_t kchunk,
                                                            double* __restrict__ part) {
  __shared__ double Gs[kGBK][kGBM + 1];
  constexpr int kGBN = 16 * NC;
  __shared__ double Ys[kGBK][kGBN + 1];
  const int64_t ncol = n + 1;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t m0 = (int64_t)blockIdx.x * kGBM, n0 = (int64_t)blockIdx.y * kGBN;
  const int64_t kb = (int64_t)blockIdx.z * kchunk, ke = (kb + kchunk < d) ? kb + kchunk : d;
  double acc[4][NC];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[a][c] = 0.0;
  for (int64_t k0 = kb; k0 < ke; k0 += kGBK) {
#pragma unroll
    for (int q = 0; q < (kGBM * kGBK) / kGThreads; ++q) {
      const int e = threadIdx.x + q * kGThreads;
      const int r = e / kGBK, kk = e % kGBK;
      const int64_t gr = m0 + r, gk = k0 + kk;
      Gs[kk][r] = (gr < p && gk < ke)
                      ? (double)__fdiv_rn(gauss_std(gkey, (uint64_t)(gr * d + gk)), sqrt_p)
                      : 0.0;
    }
#pragma unroll
    for (int q = 0; q < (kGBN * kGBK) / kGThreads; ++q) {
      const int e = threadIdx.x + q * kGThreads;
      const int kk = e % kGBK, c = e / kGBK;
      const int64_t gk = k0 + kk, gc = n0 + c;
      double v = 0.0;
      if (gk < ke && gc < ncol) v = gc < n ? (double)A[gk + gc * lda] : b[gk];
      Ys[kk][c] = v;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < kGBK; ++kk) {
      double av[4], bv[NC];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = Gs[kk][ty + 16 * a];
#pragma unroll
      for (int c = 0; c < NC; ++c) bv[c] = Ys[kk][tx + 16 * c];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[a][c] = fma(av[a], bv[c], acc[a][c]);
    }
    __syncthreads();
  }
  double* out = part + (int64_t)blockIdx.z * p * ncol;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const int64_t r = m0 + ty + 16 * a, cc = n0 + tx + 16 * c;
      if (r < p && cc < ncol) out[cc * p + r] = acc[a][c];
    }
}

size_t gauss_gemm_workspace(int64_t p, int64_t d, int64_t ncol) {
  return gemm_simt_workspace(p, d, ncol, true);
}

int launch_gauss_gemm(uint64_t gkey, int64_t p, const void* A, int dtype, int64_t d, int64_t n,
                      int64_t lda, const double* b, double* Z, int64_t ldz, void* ws,
                      size_t ws_bytes, cudaStream_t st) {
  const int64_t ncol = n + 1;
  if (p == 0 || d == 0) return MSK_OK;
  GemmSplit g = gemm_split(p, d, ncol);
  Carve cv(ws, ws_bytes);
  double* part = static_cast<double*>(cv.take((size_t)g.s * p * ncol * sizeof(double)));
  if (!part) return MSK_ENOMEM;
  const float sqrt_p = __builtin_sqrtf((float)p);  // exact rounding of sqrt(p), p < 2^24
  dim3 grid(g.mt, g.nt, g.s);
  auto go = [&](auto nc_tag) {
    constexpr int NC = decltype(nc_tag)::value;
    if (dtype == MSK_F64)
      gauss_gemm_kernel<double, NC><<<grid, kGThreads, 0, st>>>(
          gkey, sqrt_p, static_cast<const double*>(A), lda, d, n, b, p, g.kchunk, part);
    else
      gauss_gemm_kernel<float, NC><<<grid, kGThreads, 0, st>>>(
          gkey, sqrt_p, static_cast<const float*>(A), lda, d, n, b, p, g.kchunk, part);
  };
  if (g.nc == 2) go(std::integral_constant<int, 2>{});
  else if (g.nc == 3) go(std::integral_constant<int, 3>{});
  else go(std::integral_constant<int, 4>{});
  MSK_CHECK_LAUNCH("gauss_gemm_kernel");
  const int64_t total = p * ncol;
  splitk_reduce_kernel<<<(unsigned)std::min<int64_t>((total + 255) / 256, num_sms() * 8), 256, 0,
                         st>>>(part, g.s, p, ncol, Z, ldz);
  MSK_CHECK_LAUNCH("splitk_reduce_kernel");
  return MSK_OK;
}

}  // namespace msk
