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

// Shared-memory form of the cluster QR, for matrices whose owned columns fit
// on chip (qr_smem_fits): CTA `rank` keeps columns rank, rank + CL, ... of W
// in its shared memory for the whole factorisation.
//   step j: the owner of column j forms the reflector v = x + sign(x0)||x|| e0,
//     tau = 2 / v^T v from ||x||^2, which the warp that last updated column j
//     accumulated on the way (no block reduction); it writes v into W's
//     column j in global memory (that column is only a broadcast slot until
//     the final write-back), publishes tau, and writes R_jj into row j of its
//     own copy.
//   one cluster barrier; every CTA reads v from L2 (an L1-bypassing copy is
//     faster than a pull through distributed shared memory) and applies the
//     reflector to its owned columns > j, one warp per column; the warp that
//     updates column j + 1 also sums its new squares below row j.
// (v0, tau) use two slots alternating by step: slot j & 1 is rewritten at step
// j + 2, after every CTA has passed the barrier of step j + 1.  The factor
// goes back to W at the end, zeros below the diagonal.
// Dynamic shared memory: (ceil(c / CL) + 1) * m doubles + ceil(c / CL) norms.
__host__ __device__ __forceinline__ size_t qr_smem_bytes(int m, int c, int CL) {
  const size_t own = (size_t)((c + CL - 1) / CL);
  return sizeof(double) * ((own + 1) * (size_t)m + own);
}
constexpr size_t kQrSmemMax = 160 * 1024;  // 1024 x 257 on a 16-CTA cluster: 148 KB
__host__ __device__ __forceinline__ bool qr_smem_fits(int m, int c, int CL) {
  return qr_smem_bytes(m, c, CL) <= kQrSmemMax;
}

__device__ __forceinline__ void qr_cluster_smem_body(double* __restrict__ W, int m, int c,
                                                     int64_t ldw, double* sm) {
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int CL = (int)cluster.num_blocks();
  const int own = (c + CL - 1) / CL;
  const int nown = (c - rank + CL - 1) / CL;  // columns rank, rank + CL, ...
  double* cols = sm;                           // own x m
  double* vl = sm + (size_t)own * m;           // m: local copy of the step's v
  double* cnorm = vl + m;                      // own: ||column below the pivot row||^2
  __shared__ double vsc[2][2];
  __shared__ double red[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int lj = 0; lj < nown; ++lj) {
    const double* src = W + (int64_t)(rank + lj * CL) * ldw;
    for (int i = threadIdx.x; i < m; i += blockDim.x) cols[(size_t)lj * m + i] = src[i];
  }
  __syncthreads();
  if (rank == 0) {  // ||column 0||^2
    double s = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) s += cols[i] * cols[i];
    s = block_sum(s, red);
    if (threadIdx.x == 0) cnorm[0] = s;
  }
  const int steps = min(m, c);
  for (int j = 0; j < steps; ++j) {
    const int owner = j % CL, slot = j & 1;
    __syncthreads();  // column j and its norm are final; vl is free
    if (rank == owner) {
      double* x = cols + (size_t)(j / CL) * m;
      double* gcol = W + (int64_t)j * ldw;  // W's column j: a broadcast slot until write-back
      if (threadIdx.x == 0) {
        const double norm2 = cnorm[j / CL];
        const double x0 = x[j];
        const double alpha = sqrt(norm2);
        const double sgn = x0 >= 0.0 ? 1.0 : -1.0;
        const double v0 = x0 + sgn * alpha;
        const double vtv = norm2 - x0 * x0 + v0 * v0;
        gcol[j] = v0;
        vsc[slot][1] = vtv > 0.0 ? 2.0 / vtv : 0.0;
        x[j] = -sgn * alpha;
      }
      for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) gcol[i] = x[i];
      __threadfence();
    }
    cluster.sync();
    const double* gv = W + (int64_t)j * ldw;
    for (int i = j + threadIdx.x; i < m; i += blockDim.x) vl[i] = __ldcg(gv + i);
    const double tau = *cluster.map_shared_rank(&vsc[slot][1], owner);
    __syncthreads();
    // owned columns > j: local index from the first one after j
    const int lj0 = (j + CL - rank) / CL;
    for (int lj = lj0 + warp; lj < nown; lj += nwarps) {
      double* w = cols + (size_t)lj * m;
      double t = 0.0;
      for (int i = j + lane; i < m; i += 32) t += vl[i] * w[i];
      t = warp_sum(t) * tau;
      if (rank + lj * CL == j + 1) {  // the next pivot column: update and sum squares
        double s2 = 0.0;
        for (int i = j + lane; i < m; i += 32) {
          const double wi = w[i] - t * vl[i];
          w[i] = wi;
          if (i > j) s2 += wi * wi;
        }
        s2 = warp_sum(s2);
        if (lane == 0) cnorm[lj] = s2;
      } else {
        for (int i = j + lane; i < m; i += 32) w[i] -= t * vl[i];
      }
    }
  }
  __syncthreads();
  for (int lj = 0; lj < nown; ++lj) {
    const int col = rank + lj * CL;
    double* dst = W + (int64_t)col * ldw;
    for (int i = threadIdx.x; i < m; i += blockDim.x) dst[i] = i <= col ? cols[(size_t)lj * m + i] : 0.0;
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
