// msk_refine.cuh — device bodies of the refinement (sketch-and-precondition)
// passes and small vector steps, shared by ms_lstsq and the batched engine.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "msk_device.cuh"

namespace msk {

// ---------------------------------------------------------------------------
// Row-tiled FP64 passes over A (tiles of kPR rows, whole rows in shared memory,
// stored in A's own type — FP32 A is exact in binary32 — and widened on use).
//   RESID = true : r_i = b_i - A_i x; accumulates g = A^T r, ||r||^2, ||b||^2.
//   RESID = false: w_i = A_i p;       accumulates v = A^T w, ||w||^2.
// Dot phase: 4 threads per row (columns q, q+4, ...), combined by shuffles;
// column phase: thread j accumulates column j over the tile's rows.
// Per-CTA partials part[cta][0..n) (vector), part[cta][n], part[cta][n+1]
// (scalars); summed in a fixed order by pass_reduce_kernel.
constexpr int kPR = 64, kPThreads = 256;

template <typename TA, bool RESID>
__device__ __forceinline__ void pass_body(const TA* __restrict__ A, int64_t lda, int64_t d, int n,
                                          int pitch, const double* __restrict__ b,
                                          const double* __restrict__ vin,
                                          double* __restrict__ part, int cta, int nctas,
                                          unsigned char* pk_smem) {
  double* vs = reinterpret_cast<double*>(pk_smem);  // n (x or p)
  double* ws = vs + n;                              // kPR (row results)
  TA* tile = reinterpret_cast<TA*>(ws + kPR);       // kPR x pitch
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int j = threadIdx.x; j < n; j += kPThreads) vs[j] = vin[j];
  double accv[2] = {0.0, 0.0};  // columns threadIdx.x and threadIdx.x + 256 (n <= 512)
  double s1 = 0.0, s2 = 0.0;
  const int64_t ntiles = (d + kPR - 1) / kPR;
  for (int64_t t = cta; t < ntiles; t += nctas) {
    const int64_t i0 = t * kPR;
    __syncthreads();
    // load: warp w takes columns w, w+8, ...; lanes cover rows lane, lane+32
    for (int j = warp; j < n; j += kPThreads / 32) {
      const TA* col = A + (int64_t)j * lda;
#pragma unroll
      for (int h = 0; h < kPR / 32; ++h) {
        const int r = lane + 32 * h;
        const int64_t i = i0 + r;
        tile[r * pitch + j] = i < d ? __ldcs(col + i) : (TA)0;
      }
    }
    __syncthreads();
    {
      const int r = threadIdx.x >> 2, q = threadIdx.x & 3;
      const TA* row = tile + r * pitch;
      double w = 0.0;
      for (int j = q; j < n; j += 4) w = fma((double)row[j], vs[j], w);
      w += __shfl_xor_sync(0xffffffffu, w, 1);
      w += __shfl_xor_sync(0xffffffffu, w, 2);
      const int64_t i = i0 + r;
      if (q == 0) {
        if (i < d) {
          if (RESID) {
            const double bi = b[i];
            const double ri = bi - w;
            ws[r] = ri;
            s1 += ri * ri;
            s2 += bi * bi;
          } else {
            ws[r] = w;
            s1 += w * w;
          }
        } else {
          ws[r] = 0.0;
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int j = threadIdx.x + c * kPThreads;
      if (j < n) {
        double acc = accv[c];
        for (int r = 0; r < kPR; ++r) acc = fma((double)tile[r * pitch + j], ws[r], acc);
        accv[c] = acc;
      }
    }
  }
  double* out = part + (int64_t)cta * (n + 2);
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const int j = threadIdx.x + c * kPThreads;
    if (j < n) out[j] = accv[c];
  }
  __shared__ double red[2][kPThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  }
  if (lane == 0) {
    red[0][warp] = s1;
    red[1][warp] = s2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, c = 0.0;
    for (int w = 0; w < kPThreads / 32; ++w) {
      a += red[0][w];
      c += red[1][w];
    }
    out[n] = a;
    out[n + 1] = c;
  }
}

// out[j] = sum over CTAs of part[cta][j] (j < len), fixed order: block b
// covers outputs 32b .. 32b+31 (lane = output); warp w sums CTAs w, w+8, ...;
// the 8 warp sums are added in warp order.
__device__ __forceinline__ void pass_reduce_body(const double* __restrict__ part, int nctas, int len,
                                                 double* __restrict__ out, int blk) {
  __shared__ double ws[8][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = blk * 32 + lane;
  double s = 0.0;
  if (j < len)
    for (int q = warp; q < nctas; q += 8) s += part[(int64_t)q * len + j];
  ws[warp][lane] = s;
  __syncthreads();
  if (warp == 0 && j < len) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += ws[w][lane];
    out[j] = t;
  }
}

// ---------------------------------------------------------------------------
// Double-single pass for FP32 A (see the comment above the launcher).
// Tile: kPR rows x pitch floats, pitch = 4 (mod 32) so that 16-byte stores of
// 4 columns (lane = row) and the row reads of the dot phase are conflict-free.
__device__ __forceinline__ void pass_ds_body(const float* __restrict__ A, int64_t lda, int64_t d,
                                             int n, int pitch, const double* __restrict__ vin,
                                             double* __restrict__ part, int cta, int nctas,
                                             unsigned char* ds_smem) {
  float* tile = reinterpret_cast<float*>(ds_smem);  // kPR x pitch
  float* ph = tile + kPR * pitch;                   // n: p hi
  float* pl = ph + n;                               // n: p lo
  float* wh = pl + n;                               // kPR: w hi
  float* wl = wh + kPR;                             // kPR: w lo
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int j = threadIdx.x; j < n; j += kPThreads) {
    const double x = vin[j];
    const float h = (float)x;
    ph[j] = h;
    pl[j] = (float)(x - (double)h);
  }
  DS acc[2] = {{0.f, 0.f}, {0.f, 0.f}};
  const int ngroups = (n + 3) >> 2;
  const int64_t ntiles = (d + kPR - 1) / kPR;
  for (int64_t t = cta; t < ntiles; t += nctas) {
    const int64_t i0 = t * kPR;
    __syncthreads();
    // load: lane = row (two row halves), warp w takes 4-column groups w, w+8, ...
    for (int g = warp; g < ngroups; g += kPThreads / 32) {
#pragma unroll
      for (int h = 0; h < kPR / 32; ++h) {
        const int r = lane + 32 * h;
        const int64_t i = i0 + r;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < d) {
          const int j = 4 * g;
          v.x = __ldcs(A + i + (int64_t)j * lda);
          if (j + 1 < n) v.y = __ldcs(A + i + (int64_t)(j + 1) * lda);
          if (j + 2 < n) v.z = __ldcs(A + i + (int64_t)(j + 2) * lda);
          if (j + 3 < n) v.w = __ldcs(A + i + (int64_t)(j + 3) * lda);
        }
        *reinterpret_cast<float4*>(&tile[r * pitch + 4 * g]) = v;
      }
    }
    __syncthreads();
    // dot phase: 4 threads per row, thread q takes columns q, q+4, ...
    {
      const int r = threadIdx.x >> 2, q = threadIdx.x & 3;
      const float* row = tile + r * pitch;
      DS w{0.f, 0.f};
      for (int j = q; j < n; j += 4) w = ds_fma(w, row[j], ph[j], pl[j]);
      DS o = ds_shfl_xor(w, 1);
      w = ds_add(w, o.hi, o.lo);
      o = ds_shfl_xor(w, 2);
      w = ds_add(w, o.hi, o.lo);
      if (q == 0) {
        const bool ok = i0 + r < d;
        wh[r] = ok ? w.hi : 0.f;
        wl[r] = ok ? w.lo : 0.f;
      }
    }
    __syncthreads();
    // column phase: v_j += sum_r A[r][j] w_r
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int j = threadIdx.x + c * kPThreads;
      if (j < n) {
        DS a = acc[c];
        for (int r = 0; r < kPR; ++r) a = ds_fma(a, tile[r * pitch + j], wh[r], wl[r]);
        acc[c] = a;
      }
    }
  }
  double* out = part + (int64_t)cta * (n + 2);
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const int j = threadIdx.x + c * kPThreads;
    if (j < n) out[j] = (double)acc[c].hi + (double)acc[c].lo;
  }
  if (threadIdx.x == 0) {
    out[n] = 0.0;
    out[n + 1] = 0.0;
  }
}

// ---------------------------------------------------------------------------
// Small FP64 vector kernels of the refinement (single CTA; n <= 512).

// Explicit inverse of the upper-triangular R (n x n, ldr) into Ri (n x n,
// column-major): column c of Ri solves R y = e_c; one warp per column.
__device__ __forceinline__ void tri_inverse_body(const double* __restrict__ R, int n, int64_t ldr,
                                                 double* __restrict__ Ri, int blk, int nblk) {
  const int lane = threadIdx.x & 31;
  const int warp_g = (blk * blockDim.x + threadIdx.x) >> 5;
  const int nw = (nblk * blockDim.x) >> 5;
  for (int c = warp_g; c < n; c += nw) {
    double* y = Ri + (int64_t)c * n;
    for (int r = lane; r < n; r += 32) y[r] = 0.0;
    __syncwarp();
    // back substitution restricted to rows <= c
    for (int i = c; i >= 0; --i) {
      double s = (i == c) ? 1.0 : 0.0;
      double part = 0.0;
      for (int j = i + 1 + lane; j <= c; j += 32) part += R[i + (int64_t)j * ldr] * y[j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
      if (lane == 0) y[i] = (s - part) / R[i + (int64_t)i * ldr];
      __syncwarp();
    }
  }
}

// State of the refinement, all device FP64 (n-vectors unless noted):
//   x, dlt (correction), p (search dir), res (normal-eq. residual), z,
//   sc[0] = rho.
struct RefState {
  double *x, *dlt, *p, *res, *z, *sc;
};

// z = Ri (Ri^T v): the preconditioner M^{-1} v with M = R^T R.
__device__ __forceinline__ void apply_minv(const double* __restrict__ Ri, int n, const double* v, double* tmp,
                           double* z) {
  // tmp = Ri^T v  (tmp[j] = sum_{i<=j} Ri[i][j] v[i])
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double* col = Ri + (int64_t)j * n;
    double s = 0.0;
    for (int i = 0; i <= j; ++i) s += col[i] * v[i];
    tmp[j] = s;
  }
  __syncthreads();
  // z = Ri tmp  (z[i] = sum_{j>=i} Ri[i][j] tmp[j])
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double s = 0.0;
    for (int j = i; j < n; ++j) s += Ri[i + (int64_t)j * n] * tmp[j];
    z[i] = s;
  }
  __syncthreads();
}

// Start of an inner solve: res = g (from the FP64 pass), dlt = 0,
// z = M^{-1} res, p = z, rho = res.z.
__device__ __forceinline__ void pcg_start_body(const double* __restrict__ Ri, int n,
                                               const double* __restrict__ g, RefState s) {
  __shared__ double tmp[512];
  __shared__ double red[32];
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    s.res[j] = g[j];
    s.dlt[j] = 0.0;
  }
  __syncthreads();
  apply_minv(Ri, n, s.res, tmp, s.z);
  double part = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    s.p[j] = s.z[j];
    part += s.res[j] * s.z[j];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += red[w];
    s.sc[0] = r;
  }
}

// One CG update after the pass produced v = A^T A p (pv[0..n)), pv[n] = p.v:
//   alpha = rho / p.v; dlt += alpha p; res -= alpha v; z = M^{-1} res;
//   rho' = res.z; p = z + (rho'/rho) p.
__device__ __forceinline__ void pcg_update_body(const double* __restrict__ Ri, int n,
                                                const double* __restrict__ pv, RefState s) {
  __shared__ double tmp[512];
  __shared__ double red[32];
  __shared__ double alpha_s, beta_s;
  // p.v from the vector itself (more accurate than ||A p||^2 in FP32)
  double part = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) part += s.p[j] * pv[j];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double pAp = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) pAp += red[w];
    alpha_s = pAp > 0.0 ? s.sc[0] / pAp : 0.0;
  }
  __syncthreads();
  const double alpha = alpha_s;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    s.dlt[j] += alpha * s.p[j];
    s.res[j] -= alpha * pv[j];
  }
  __syncthreads();
  apply_minv(Ri, n, s.res, tmp, s.z);
  part = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) part += s.res[j] * s.z[j];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double rho = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) rho += red[w];
    beta_s = s.sc[0] > 0.0 ? rho / s.sc[0] : 0.0;
    s.sc[1] = alpha_s * s.sc[0];  // decrease of ||b - A x||^2 by this step (CG identity)
    s.sc[0] = rho;
  }
  __syncthreads();
  const double beta = beta_s;
  for (int j = threadIdx.x; j < n; j += blockDim.x) s.p[j] = s.z[j] + beta * s.p[j];
}


// Inner CG per outer (FP64 residual) step: at most kMaxInner iterations; the
// gain-based stopping rule (kDecFrac) is in ms_lstsq.
}  // namespace msk
