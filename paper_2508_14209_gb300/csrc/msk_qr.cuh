// msk_qr.cuh — device bodies of the FP64 Householder QR (one thread-block
// cluster per matrix) and of the upper-triangular solve, shared by the
// single-problem and the batched kernels.
#pragma once
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace msk {
namespace cg = cooperative_groups;

constexpr int kQrThreads = 256;
constexpr int kQrMaxRows = 2048;
constexpr int kQrMaxCols = 512;
constexpr int kTrsvMax = 4096;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum (all threads get the result).  `red` holds >= 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < nw; ++w) s += red[w];
  return s;
}

// The owner of column j publishes (v0, tau) in its shared memory slot
// pub[j & 1]; the other CTAs read it through distributed shared memory after
// the cluster barrier.  Two slots: slot j & 1 is rewritten at step j + 2 only,
// after a barrier every reader of step j has passed.  Columns owned by other
// CTAs are read with L1-bypassing loads.
__device__ __forceinline__ void qr_cluster_body(double* __restrict__ W, int m, int c, int64_t ldw) {
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int CL = (int)cluster.num_blocks();
  __shared__ double vbuf[kQrMaxRows];
  __shared__ double red[32];
  __shared__ double pub[2][2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int steps = min(m, c);
  for (int j = 0; j < steps; ++j) {
    const int owner = j % CL;
    double* colj = W + (int64_t)j * ldw;
    if (rank == owner) {
      double s = 0.0;
      for (int i = j + threadIdx.x; i < m; i += blockDim.x) s += colj[i] * colj[i];
      const double norm2 = block_sum(s, red);
      if (threadIdx.x == 0) {
        const double x0 = colj[j];
        const double alpha = sqrt(norm2);
        const double sgn = x0 >= 0.0 ? 1.0 : -1.0;
        const double v0 = x0 + sgn * alpha;
        const double vtv = norm2 - x0 * x0 + v0 * v0;
        pub[j & 1][0] = v0;
        pub[j & 1][1] = vtv > 0.0 ? 2.0 / vtv : 0.0;
        colj[j] = -sgn * alpha;
      }
    }
    __threadfence();
    cluster.sync();
    // stage v = (v0, W[j+1:m, j]) and apply the reflector to owned columns
    const double* opub = cluster.map_shared_rank(&pub[j & 1][0], owner);
    const double v0 = opub[0], tau = opub[1];
    // v = (v0, W[j+1:m, j]); staged in shared memory when it fits, else read
    // from W's column j (L2) where it is needed (no CTA writes that column
    // below the diagonal during the step)
    const bool staged = m - j <= kQrMaxRows;
    if (staged)
      for (int i = j + threadIdx.x; i < m; i += blockDim.x) vbuf[i - j] = (i == j) ? v0 : __ldcg(colj + i);
    __syncthreads();
    if (tau != 0.0) {
      // owned columns > j: first owned column index >= j+1 with col % CL == rank
      int first = j + 1 + ((rank - (j + 1) % CL) + CL) % CL;
      for (int col = first + warp * CL; col < c; col += nwarps * CL) {
        double* w = W + (int64_t)col * ldw;
        double s = 0.0;
        if (staged) {
          for (int i = j + lane; i < m; i += 32) s += vbuf[i - j] * w[i];
          s = warp_sum(s) * tau;
          for (int i = j + lane; i < m; i += 32) w[i] -= s * vbuf[i - j];
        } else {
          for (int i = j + lane; i < m; i += 32) s += (i == j ? v0 : __ldcg(colj + i)) * w[i];
          s = warp_sum(s) * tau;
          for (int i = j + lane; i < m; i += 32) w[i] -= s * (i == j ? v0 : __ldcg(colj + i));
        }
      }
    }
    __syncthreads();
  }
  cluster.sync();
  // zero the strictly lower part of owned columns
  for (int col = rank; col < c; col += CL) {
    double* w = W + (int64_t)col * ldw;
    for (int i = col + 1 + threadIdx.x; i < m; i += blockDim.x) w[i] = 0.0;
  }
}

// Shared-memory form of the cluster QR, blocked by panels of kQrPanel
// columns, for matrices whose owned columns fit on chip (qr_smem_fits).
// Panel P (columns P b .. P b + b - 1) belongs to CTA P mod CL, which keeps
// its panels in shared memory for the whole factorisation.
//   panel P: its owner factors the panel alone (b Householder steps: the
//     reflector v = x + sign(x0)||x|| e0, tau = 2 / v^T v of each column from
//     ||x||^2, which the warp that last updated the column accumulated on the
//     way, then the panel's later columns updated one warp per column), writes
//     the b reflectors into W's panel columns in global memory (those columns
//     are broadcast slots until the final write-back) and publishes the taus;
//   one cluster barrier per panel (not per column); every CTA reads the
//     panel's reflectors from L2 and applies them, in order, to each of its
//     columns after the panel, one warp per column; the warp that updates the
//     first column of the next panel also sums its squares below the pivot.
// Every column receives the same reflectors in the same order and the same
// arithmetic as the unblocked algorithm, so R is the same.  The taus use two
// slots alternating by panel: slot P & 1 is rewritten at panel P + 2, after
// every CTA has passed the barrier of panel P + 1.  The factor goes back to W
// at the end, zeros below the diagonal.
constexpr int kQrPanel = 8;
// Columns held by the CTA owning the most (panels cyclic over the cluster).
__host__ __device__ __forceinline__ int qr_owned_cols(int c, int CL, int rank) {
  const int npan = (c + kQrPanel - 1) / kQrPanel;
  int n = 0;
  for (int P = rank; P < npan; P += CL) n += min(kQrPanel, c - P * kQrPanel);
  return n;
}
// Dynamic shared memory: the owned columns of the busiest CTA (stored panel
// after panel; only a CTA's last panel can be narrower than kQrPanel, so
// panel q starts at local column q kQrPanel) and the current panel's
// reflectors, m doubles per column, plus the owned columns' norms.
__host__ __device__ __forceinline__ size_t qr_smem_bytes(int m, int c, int CL) {
  int own = 0;
  for (int r = 0; r < CL; ++r) own = max(own, qr_owned_cols(c, CL, r));
  return sizeof(double) * ((size_t)(own + kQrPanel) * (size_t)m + (size_t)own);
}
constexpr size_t kQrSmemMax = 205 * 1024;  // 1024 x 257 on a 16-CTA cluster: 200 KB
__host__ __device__ __forceinline__ bool qr_smem_fits(int m, int c, int CL) {
  return qr_smem_bytes(m, c, CL) <= kQrSmemMax;
}

__device__ __forceinline__ void qr_cluster_smem_body(double* __restrict__ W, int m, int c,
                                                     int64_t ldw, double* sm) {
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int CL = (int)cluster.num_blocks();
  constexpr int b = kQrPanel;
  const int npan = (c + b - 1) / b;
  int own = 0;
  for (int r = 0; r < CL; ++r) own = max(own, qr_owned_cols(c, CL, r));
  const int myp = (npan - rank + CL - 1) / CL;  // panels rank, rank + CL, ...
  double* cols = sm;                            // panel q, column t: cols[(q b + t) m + i]
  double* vl = sm + (size_t)own * m;            // the current panel's reflectors, b x m
  double* cnorm = vl + (size_t)b * m;           // per owned column: ||column below its pivot||^2
  __shared__ double taus[2][kQrPanel];
  __shared__ double rdiag[kQrPanel];
  __shared__ double red[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  auto width = [&](int P) { return min(b, c - P * b); };
  for (int q = 0; q < myp; ++q) {
    const int P = rank + q * CL;
    for (int t = 0; t < width(P); ++t) {
      const double* src = W + (int64_t)(P * b + t) * ldw;
      for (int i = threadIdx.x; i < m; i += blockDim.x) cols[(size_t)(q * b + t) * m + i] = src[i];
    }
  }
  __syncthreads();
  if (rank == 0) {  // ||column 0||^2
    double s = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) s += cols[i] * cols[i];
    s = block_sum(s, red);
    if (threadIdx.x == 0) cnorm[0] = s;
  }
  for (int P = 0; P < npan; ++P) {
    const int owner = P % CL, slot = P & 1, c0 = P * b, wP = width(P);
    __syncthreads();  // the panel's columns and first norm are final; vl is free
    if (rank == owner) {
      double* pc = cols + (size_t)(P / CL) * b * m;
      for (int t = 0; t < wP; ++t) {
        const int j = c0 + t;
        double* x = pc + (size_t)t * m;
        if (threadIdx.x == 0) {
          const double norm2 = cnorm[(P / CL) * b + t];
          const double x0 = x[j];
          const double alpha = sqrt(norm2);
          const double sgn = x0 >= 0.0 ? 1.0 : -1.0;
          const double v0 = x0 + sgn * alpha;
          const double vtv = norm2 - x0 * x0 + v0 * v0;
          taus[slot][t] = vtv > 0.0 ? 2.0 / vtv : 0.0;
          rdiag[t] = -sgn * alpha;
          x[j] = v0;  // column j holds v from row j down until the panel is published
        }
        __syncthreads();
        const double tau = taus[slot][t];
        for (int u = t + 1 + warp; u < wP; u += nwarps) {
          double* w = pc + (size_t)u * m;
          double s = 0.0;
          for (int i = j + lane; i < m; i += 32) s += x[i] * w[i];
          s = warp_sum(s) * tau;
          if (u == t + 1) {  // the panel's next pivot column: update and sum squares
            double s2 = 0.0;
            for (int i = j + lane; i < m; i += 32) {
              const double wi = w[i] - s * x[i];
              w[i] = wi;
              if (i > j) s2 += wi * wi;
            }
            s2 = warp_sum(s2);
            if (lane == 0) cnorm[(P / CL) * b + u] = s2;
          } else {
            for (int i = j + lane; i < m; i += 32) w[i] -= s * x[i];
          }
        }
        __syncthreads();
      }
      // publish the reflectors (zeros above each pivot), then R's diagonal
      for (int t = 0; t < wP; ++t) {
        double* g = W + (int64_t)(c0 + t) * ldw;
        const double* x = pc + (size_t)t * m;
        for (int i = threadIdx.x; i < m; i += blockDim.x) g[i] = i < c0 + t ? 0.0 : x[i];
      }
      __syncthreads();
      if (threadIdx.x < wP) pc[(size_t)threadIdx.x * m + c0 + threadIdx.x] = rdiag[threadIdx.x];
      __threadfence();
    }
    cluster.sync();
    if (P + 1 == npan) break;  // no column after the last panel
    // the panel's reflectors (rows from c0 down) and taus
    for (int t = 0; t < wP; ++t) {
      const double* g = W + (int64_t)(c0 + t) * ldw;
      for (int i = c0 + threadIdx.x; i < m; i += blockDim.x) vl[(size_t)t * m + i] = __ldcg(g + i);
    }
    double tau[kQrPanel];
    const double* otau = cluster.map_shared_rank(&taus[slot][0], owner);
#pragma unroll
    for (int t = 0; t < kQrPanel; ++t) tau[t] = t < wP ? otau[t] : 0.0;
    __syncthreads();
    // owned columns after the panel, one warp per column: the panel's
    // reflectors in order
    const int q0 = (P + 1 - rank + CL - 1) / CL;  // first owned panel after P
    const int nfirst = (P + 1) * b;               // the next panel's first column
    int lc = 0;
    for (int q = q0; q < myp; ++q) lc += width(rank + q * CL);
    for (int g = warp; g < lc; g += nwarps) {
      int q = q0, t = g;
      while (t >= width(rank + q * CL)) t -= width(rank + q * CL), ++q;
      const int col = (rank + q * CL) * b + t;
      double* w = cols + (size_t)(q * b + t) * m;
      for (int r = 0; r < wP; ++r) {
        const int j = c0 + r;
        const double* v = vl + (size_t)r * m;
        double s = 0.0;
        for (int i = j + lane; i < m; i += 32) s += v[i] * w[i];
        s = warp_sum(s) * tau[r];
        for (int i = j + lane; i < m; i += 32) w[i] -= s * v[i];
      }
      if (col == nfirst) {  // the next pivot column: its squares below the pivot
        double s2 = 0.0;
        for (int i = nfirst + lane; i < m; i += 32) s2 += w[i] * w[i];
        s2 = warp_sum(s2);
        if (lane == 0) cnorm[q * b + t] = s2;
      }
    }
  }
  __syncthreads();
  for (int q = 0; q < myp; ++q) {
    const int P = rank + q * CL;
    for (int t = 0; t < width(P); ++t) {
      const int col = P * b + t;
      double* dst = W + (int64_t)col * ldw;
      const double* src = cols + (size_t)(q * b + t) * m;
      for (int i = threadIdx.x; i < m; i += blockDim.x) dst[i] = i <= col ? src[i] : 0.0;
    }
  }
  __threadfence();
  cluster.sync();
}

// R x = rhs, R upper (column-major, ldr).  x may alias rhs.
__device__ __forceinline__ void trsv_upper_body(const double* __restrict__ R, int n, int64_t ldr,
                                                const double* rhs, double* x, int* status,
                                                double* xs) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) xs[i] = rhs[i];
  __syncthreads();
  for (int i = n - 1; i >= 0; --i) {
    if (threadIdx.x == 0) {
      const double rii = R[i + (int64_t)i * ldr];
      if (rii == 0.0 && status && status[0] == 0) status[0] = i + 1;
      xs[i] = xs[i] / rii;
    }
    __syncthreads();
    const double xi = xs[i];
    const double* col = R + (int64_t)i * ldr;
    for (int r = threadIdx.x; r < i; r += blockDim.x) xs[r] -= col[r] * xi;
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = xs[i];
}

}  // namespace msk
