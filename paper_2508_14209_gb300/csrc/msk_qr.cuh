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
    for (int i = j + threadIdx.x; i < m; i += blockDim.x) vbuf[i - j] = (i == j) ? v0 : __ldcg(colj + i);
    __syncthreads();
    if (tau != 0.0) {
      // owned columns > j: first owned column index >= j+1 with col % CL == rank
      int first = j + 1 + ((rank - (j + 1) % CL) + CL) % CL;
      for (int col = first + warp * CL; col < c; col += nwarps * CL) {
        double* w = W + (int64_t)col * ldw;
        double s = 0.0;
        for (int i = j + lane; i < m; i += 32) s += vbuf[i - j] * w[i];
        s = warp_sum(s) * tau;
        for (int i = j + lane; i < m; i += 32) w[i] -= s * vbuf[i - j];
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
