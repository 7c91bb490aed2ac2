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
//   step j: every CTA waits for reflector j (v = x + sign(x0)||x|| e0,
//     tau = 2 / v^T v) to be published, copies v from W's column j in L2
//     (that column is only a broadcast slot until the final write-back) and
//     tau from the owner's shared memory, and applies I - tau v v^T to its
//     owned columns > j, one warp per column;
//   look-ahead: the owner of column j + 1 updates that column first (warp 0,
//     its other warps waiting so that the SM's FP64 pipe serves it alone),
//     summing its squares below the pivot on the way, and publishes
//     reflector j + 1 before it updates its other columns.
// The steps are chained by the split cluster barrier: a thread arrives at
// phase j + 1 as soon as it has read reflector j (warp 0 of the next owner
// only after publishing reflector j + 1) and waits for phase j + 1 when it
// needs that reflector, so the publication of reflector j + 1 overlaps the
// updates of step j.  v is copied into one of two buffers by step parity and
// tau sits in one of two slots: both are rewritten two steps later, after
// every thread of the cluster has arrived at the phase in between (and so has
// finished with them).  The factor goes back to W at the end, zeros below the
// diagonal.
// Dynamic shared memory: (ceil(c / CL) + 2) * m doubles.
__host__ __device__ __forceinline__ size_t qr_smem_bytes(int m, int c, int CL) {
  const size_t own = (size_t)((c + CL - 1) / CL);
  return sizeof(double) * ((own + 2) * (size_t)m);
}
constexpr size_t kQrSmemMax = 160 * 1024;  // 1024 x 257 on a 16-CTA cluster: 152 KB
__host__ __device__ __forceinline__ bool qr_smem_fits(int m, int c, int CL) {
  return qr_smem_bytes(m, c, CL) <= kQrSmemMax;
}

__device__ __forceinline__ void cluster_arrive_release() {
  asm volatile("barrier.cluster.arrive.release;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait_acquire() {
  asm volatile("barrier.cluster.wait.acquire;" ::: "memory");
}

// Reflector j from the owner's copy x of column j (norm2 = ||x[j:]||^2), by
// one whole warp: tau into the slot of step j, v into W's column j (v0 at the
// pivot, then x below it), R[j][j] into x[j].
__device__ __forceinline__ void qr_publish_reflector(double* __restrict__ x, double* __restrict__ gcol,
                                                     int j, int m, double norm2, double* tau_slot) {
  const int lane = threadIdx.x & 31;
  if (lane == 0) {
    const double x0 = x[j];
    const double alpha = sqrt(norm2);
    const double sgn = x0 >= 0.0 ? 1.0 : -1.0;
    const double v0 = x0 + sgn * alpha;
    const double vtv = norm2 - x0 * x0 + v0 * v0;
    *tau_slot = vtv > 0.0 ? 2.0 / vtv : 0.0;
    gcol[j] = v0;
    x[j] = -sgn * alpha;
  }
  for (int i = j + 1 + lane; i < m; i += 32) gcol[i] = x[i];
  __threadfence();
  __syncwarp();
}

__device__ __forceinline__ void qr_cluster_smem_body(double* __restrict__ W, int m, int c,
                                                     int64_t ldw, double* sm) {
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int CL = (int)cluster.num_blocks();
  const int own = (c + CL - 1) / CL;
  const int nown = (c - rank + CL - 1) / CL;  // columns rank, rank + CL, ...
  double* cols = sm;                           // own x m
  double* vl = sm + (size_t)own * m;           // 2 x m: the step's v, by step parity
  __shared__ double vsc[2];                    // tau, by step parity
  __shared__ double red[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int lj = 0; lj < nown; ++lj) {
    const double* src = W + (int64_t)(rank + lj * CL) * ldw;
    for (int i = threadIdx.x; i < m; i += blockDim.x) cols[(size_t)lj * m + i] = src[i];
  }
  __syncthreads();
  const int steps = min(m, c);
  if (rank == 0 && steps > 0) {  // reflector 0
    double s = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) s += cols[i] * cols[i];
    s = block_sum(s, red);
    if (warp == 0) qr_publish_reflector(cols, W, 0, m, s, &vsc[0]);
  }
  cluster_arrive_release();  // phase 0: reflector 0 published
  for (int j = 0; j < steps; ++j) {
    const int owner = j % CL, slot = j & 1;
    cluster_wait_acquire();  // phase j: reflector j published, buffers of step j - 2 free
    double* v = vl + (size_t)slot * m;
    const double* gv = W + (int64_t)j * ldw;
    for (int i = j + threadIdx.x; i < m; i += blockDim.x) v[i] = __ldcg(gv + i);
    const double tau = *cluster.map_shared_rank(&vsc[slot], owner);
    __syncthreads();
    const int lj0 = (j + CL - rank) / CL;  // first owned column after j
    const bool pivot = j + 1 < steps && rank == (j + 1) % CL;  // then lj0 is column j + 1
    if (pivot && warp == 0) {
      double* w = cols + (size_t)lj0 * m;
      double t = 0.0;
      for (int i = j + lane; i < m; i += 32) t += v[i] * w[i];
      t = warp_sum(t) * tau;
      double s2 = 0.0;
      for (int i = j + lane; i < m; i += 32) {
        const double wi = w[i] - t * v[i];
        w[i] = wi;
        if (i > j) s2 += wi * wi;
      }
      s2 = warp_sum(s2);
      qr_publish_reflector(w, W + (int64_t)(j + 1) * ldw, j + 1, m, s2, &vsc[slot ^ 1]);
    }
    cluster_arrive_release();  // phase j + 1
    // the FP64 pipe is the SM's scarcest resource: in the pivot's CTA the
    // other warps start their updates only once reflector j + 1 is out
    if (pivot) __syncthreads();
    for (int lj = lj0 + (pivot ? 1 : 0) + warp; lj < nown; lj += nwarps) {
      double* w = cols + (size_t)lj * m;
      double t = 0.0;
      for (int i = j + lane; i < m; i += 32) t += v[i] * w[i];
      t = warp_sum(t) * tau;
      for (int i = j + lane; i < m; i += 32) w[i] -= t * v[i];
    }
  }
  cluster_wait_acquire();  // every CTA has read the last reflector
  __syncthreads();
  for (int lj = 0; lj < nown; ++lj) {
    const int col = rank + lj * CL;
    double* dst = W + (int64_t)col * ldw;
    for (int i = threadIdx.x; i < m; i += blockDim.x) dst[i] = i <= col ? cols[(size_t)lj * m + i] : 0.0;
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
