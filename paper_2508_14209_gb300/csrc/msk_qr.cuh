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
//   step j: every CTA waits for reflector j to be published: x below the
//     pivot in W's column j in L2 (that column is only a broadcast slot until
//     the final write-back) and (x0, ||x||^2) in the owner's shared memory;
//     it copies x into its v buffer, forms v0 = x0 + sign(x0)||x|| and
//     tau = 2 / v^T v itself, and applies I - tau v v^T to its owned columns
//     > j, one warp per column;
//   look-ahead: the owner of column j + 1 updates that column first and
//     publishes reflector j + 1 before it updates its other columns; the
//     owner of column j + 2 likewise updates that column first, so that the
//     next step can start on it at once.  Both spread the column over warps
//     0-3, one per SM sub-partition: on GB300 each sub-partition issues FP64
//     at a quarter of the SM's 2 lanes per clock, so one warp alone would run
//     at a quarter of the pipe; warp 4 forms (v0, tau) meanwhile (the square
//     root and the division cost about 0.7 us), and the other warps wait so
//     that the FP64 pipe serves the chain alone.  The pivot writes the column
//     below the new pivot to W as it goes and sums its squares; R[j+1][j+1]
//     is written after the publication.
// The steps are chained by the split cluster barrier: a thread arrives at
// phase j + 1 as soon as it has read reflector j (warp 0 of the next owner
// only after publishing reflector j + 1) and waits for phase j + 1 when it
// needs that reflector, so the publication of reflector j + 1 overlaps the
// updates of step j.  v is copied into one of two buffers by step parity and
// (x0, ||x||^2) and tau sit in slots by step parity: they are rewritten two
// steps later at the earliest, after every thread of the cluster has arrived
// at the phase in between (and so has finished with them).  Dot products run
// four independent FP64 chains.  The factor goes back to W at the end, zeros
// below the diagonal.
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
// named barrier `id` over the first `nthreads` threads (whole warps)
__device__ __forceinline__ void qr_bar_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// (v0, tau) of the reflector of x, from x0 = x[j] and norm2 = ||x[j:]||^2:
// v = x + sign(x0) ||x|| e0 (v0 its pivot entry), tau = 2 / v^T v (0 for a
// zero column).
__device__ __forceinline__ void qr_reflector_coeffs(double x0, double norm2, double& v0, double& tau) {
  const double alpha = sqrt(norm2);
  const double sgn = x0 >= 0.0 ? 1.0 : -1.0;
  v0 = x0 + sgn * alpha;
  const double vtv = norm2 - x0 * x0 + v0 * v0;
  tau = vtv > 0.0 ? 2.0 / vtv : 0.0;
}

// sum over i = i0 + lane + 32 q < m of a[i] b[i], summed over the warp: four
// independent FP64 chains (a dependent DFMA costs about 35 ns on GB300, so a
// single chain of 16 would cost more than the warp's whole share of the pipe).
__device__ __forceinline__ double qr_warp_dot(const double* a, const double* b, int i0, int m) {
  const int lane = threadIdx.x & 31;
  double t0 = 0.0, t1 = 0.0, t2 = 0.0, t3 = 0.0;
  int i = i0 + lane;
  for (; i + 96 < m; i += 128) {
    t0 = fma(a[i], b[i], t0);
    t1 = fma(a[i + 32], b[i + 32], t1);
    t2 = fma(a[i + 64], b[i + 64], t2);
    t3 = fma(a[i + 96], b[i + 96], t3);
  }
  for (; i < m; i += 32) t0 = fma(a[i], b[i], t0);
  return warp_sum((t0 + t1) + (t2 + t3));
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
  __shared__ double vsc[2][2];                 // (x0, norm2) this CTA published, by step parity
  __shared__ double vtau[2];                   // the step's tau, by step parity
  __shared__ double qcoef[2], qpart[4], qpart2[4];  // the pivot warps' exchange
  __shared__ double red[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int lj = 0; lj < nown; ++lj) {
    const double* src = W + (int64_t)(rank + lj * CL) * ldw;
    for (int i = threadIdx.x; i < m; i += blockDim.x) cols[(size_t)lj * m + i] = src[i];
  }
  __syncthreads();
  const int steps = min(m, c);
  if (rank == 0 && steps > 0) {  // reflector 0: (x0, norm2) to the slot, x below the pivot to W
    double s = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) s += cols[i] * cols[i];
    s = block_sum(s, red);
    for (int i = 1 + threadIdx.x; i < m; i += blockDim.x) W[i] = cols[i];
    if (threadIdx.x == 0) {
      vsc[0][0] = cols[0];
      vsc[0][1] = s;
    }
    __threadfence();
    __syncthreads();
  }
  cluster_arrive_release();  // phase 0: reflector 0 published
  if (rank == 0 && steps > 0 && threadIdx.x == 0)  // R[0][0], off the chain
    cols[0] = -(vsc[0][0] >= 0.0 ? 1.0 : -1.0) * sqrt(vsc[0][1]);
  for (int j = 0; j < steps; ++j) {
    const int owner = j % CL, slot = j & 1;
    cluster_wait_acquire();  // phase j: reflector j published, buffers of step j - 2 free
    double* v = vl + (size_t)slot * m;
    const double* gv = W + (int64_t)j * ldw;
    const double* opub = cluster.map_shared_rank(&vsc[slot][0], owner);
    const double x0 = opub[0], nrm = opub[1];
    for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) v[i] = __ldcg(gv + i);
    const int lj0 = (j + CL - rank) / CL;  // first owned column after j
    const int pc = rank + lj0 * CL;        // ... its global index
    // this CTA's first column after j is the next pivot (j + 1: apply
    // reflector j, publish reflector j + 1) or the one after (j + 2: apply
    // reflector j now, so that the next step can start on it at once)
    const bool pivot = lj0 < nown && pc == j + 1 && j + 1 < steps;
    const bool prep = lj0 < nown && pc == j + 2 && j + 2 < steps;
    __syncthreads();
    if ((pivot || prep) && warp < 5) {
      // that column by warps 0-3, one per SM sub-partition (a warp issues
      // FP64 at a quarter of the SM's rate), rows j + 1 + 32 (4 q + warp) +
      // lane; reflector j's (v0, tau) by warp 4 meanwhile.  The pivot writes
      // x below the new pivot to W as it goes and publishes (x0, norm2) once
      // the partial norms meet.
      double* w = cols + (size_t)lj0 * m;
      if (warp == 4) {
        cluster_arrive_release();  // phase j + 1 (nothing of its own to publish)
        if (lane == 0) {
          double v0, tau;
          qr_reflector_coeffs(x0, nrm, v0, tau);
          qcoef[0] = v0;
          qcoef[1] = tau;
        }
        qr_bar_sync(1, 160);
      } else {
        if (prep) cluster_arrive_release();  // phase j + 1: reflector j has been read
        const double wj = w[j];
        double p0 = 0.0, p1 = 0.0;
        for (int i = j + 1 + 32 * warp + lane; i < m; i += 256) {
          p0 = fma(v[i], w[i], p0);
          if (i + 128 < m) p1 = fma(v[i + 128], w[i + 128], p1);
        }
        const double p = warp_sum(p0 + p1);
        if (lane == 0) qpart[warp] = p;
        qr_bar_sync(1, 160);
        const double v0 = qcoef[0], tau = qcoef[1];
        const double t = tau * fma(v0, wj, (qpart[0] + qpart[1]) + (qpart[2] + qpart[3]));
        double* gcol = W + (int64_t)(j + 1) * ldw;
        double s0 = 0.0, s1 = 0.0;
        for (int i = j + 1 + 32 * warp + lane; i < m; i += 256) {
          const double w0 = w[i] - t * v[i];
          w[i] = w0;
          if (pivot) {
            if (i > j + 1) gcol[i] = w0;
            s0 = fma(w0, w0, s0);
          }
          if (i + 128 < m) {
            const double w1 = w[i + 128] - t * v[i + 128];
            w[i + 128] = w1;
            if (pivot) {
              gcol[i + 128] = w1;
              s1 = fma(w1, w1, s1);
            }
          }
        }
        if (warp == 0 && lane == 0) {
          w[j] = wj - t * v0;
          v[j] = v0;
          vtau[slot] = tau;
        }
        if (pivot) {
          const double s2 = warp_sum(s0 + s1);
          if (lane == 0) qpart2[warp] = s2;
          qr_bar_sync(2, 128);
          if (warp == 0 && lane == 0) {
            vsc[slot ^ 1][0] = w[j + 1];
            vsc[slot ^ 1][1] = (qpart2[0] + qpart2[1]) + (qpart2[2] + qpart2[3]);
          }
          __threadfence();
          __syncwarp();
          cluster_arrive_release();  // phase j + 1: reflector j + 1 published
        }
      }
    } else {
      cluster_arrive_release();  // phase j + 1: reflector j has been read
    }
    // off the chain: reflector j's (v0, tau) in the other CTAs; in the
    // pivot's CTA the other warps start their updates only once reflector
    // j + 1 is out (the FP64 pipe serves the chain alone)
    if (!pivot && !prep && threadIdx.x == 0) {
      double v0, tau;
      qr_reflector_coeffs(x0, nrm, v0, tau);
      v[j] = v0;
      vtau[slot] = tau;
    }
    __syncthreads();
    if (pivot && threadIdx.x == 0)  // R[j+1][j+1]
      cols[(size_t)lj0 * m + j + 1] = -(vsc[slot ^ 1][0] >= 0.0 ? 1.0 : -1.0) * sqrt(vsc[slot ^ 1][1]);
    const double tau = vtau[slot];
    for (int lj = lj0 + (pivot || prep ? 1 : 0) + warp; lj < nown; lj += nwarps) {
      double* w = cols + (size_t)lj * m;
      const double t = qr_warp_dot(v, w, j, m) * tau;
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

// ---------------------------------------------------------------------------
// Flow form of the on-chip cluster QR: no cluster-wide step barrier.  Each
// reflector j has its own mbarrier in every CTA of the cluster (count 1, one
// phase); its producer, the warp that owns column j, writes v below the pivot
// into W's column j (a broadcast slot until the final write-back) and (v0,
// tau) into its CTA's slot j, then arrives remotely on mbarrier j of every
// CTA.  Warp w of a CTA owns the CTA's local columns w, w + 8, ... and walks
// the reflectors in order, waiting for each on its own CTA's mbarrier,
// applying it to its columns after j (the next pivot, column j + 1, first)
// and publishing reflector j + 1 when it owns column j + 1.  So a column's
// owner needs only the reflectors before it: warps and CTAs run ahead or
// behind each other, the chain of the factorisation is producer -> consumer
// only, and the updates of columns far from the pivot fill the FP64 pipe in
// its shadow.  Every wait is bounded (kQrWaitNs); a warp whose wait expires
// sets *tflag and stops, and the others then expire in turn.
constexpr uint64_t kQrWaitNs = 1000000000ull;

__device__ __forceinline__ unsigned qr_smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void qr_mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(qr_smem_u32(bar)), "r"(count) : "memory");
}
// arrive (release at cluster scope) on the mbarrier at bar's offset in CTA `rank`
__device__ __forceinline__ void qr_mbar_arrive_remote(uint64_t* bar, unsigned rank) {
  unsigned remote;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(qr_smem_u32(bar)), "r"(rank));
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(remote) : "memory");
}
__device__ __forceinline__ bool qr_mbar_try(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(qr_smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t qr_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait for phase 0 of bar: false (and *tflag = 1) once kQrWaitNs
// have passed.
__device__ __forceinline__ bool qr_mbar_wait(uint64_t* bar, int* tflag) {
  if (qr_mbar_try(bar, 0)) return true;
  const uint64_t t0 = qr_ns();
  while (qr_ns() - t0 <= kQrWaitNs)
    if (qr_mbar_try(bar, 0)) return true;
  if (tflag) atomicExch(tflag, 1);
  return false;
}

// Dynamic shared memory of the flow form: the owned columns, then per
// reflector one mbarrier and one (v0, tau) slot.
__host__ __device__ __forceinline__ size_t qr_flow_smem_bytes(int m, int c, int CL) {
  const size_t own = (size_t)((c + CL - 1) / CL);
  const size_t steps = (size_t)(m < c ? m : c);
  return sizeof(double) * own * (size_t)m + 24 * steps;
}
__host__ __device__ __forceinline__ bool qr_flow_fits(int m, int c, int CL) {
  return qr_flow_smem_bytes(m, c, CL) <= kQrSmemMax;
}

// Reflector j from the owner's copy x of column j (norm2 = ||x[j:]||^2), by
// one whole warp: (v0, tau) into slot, R[j][j] into x[j], v below the pivot
// into W's column gcol; then the release of all that to the cluster by one
// remote arrival on mbarrier j (bar) of each of the CL CTAs.
__device__ __forceinline__ void qr_flow_publish(double* __restrict__ x, double* __restrict__ gcol, int j,
                                                int m, double norm2, double* slot, uint64_t* bar, int CL) {
  const int lane = threadIdx.x & 31;
  if (lane == 0) {
    const double x0 = x[j];
    const double alpha = sqrt(norm2);
    const double sgn = x0 >= 0.0 ? 1.0 : -1.0;
    const double v0 = x0 + sgn * alpha;
    const double vtv = norm2 - x0 * x0 + v0 * v0;
    slot[0] = v0;
    slot[1] = vtv > 0.0 ? 2.0 / vtv : 0.0;
    x[j] = -sgn * alpha;
  }
  for (int i = j + 1 + lane; i < m; i += 32) gcol[i] = x[i];
  __threadfence();
  __syncwarp();
  for (int r = lane; r < CL; r += 32) qr_mbar_arrive_remote(bar, (unsigned)r);
}

__device__ __forceinline__ void qr_cluster_flow_body(double* __restrict__ W, int m, int c, int64_t ldw,
                                                     double* sm, int* tflag) {
  constexpr int VR = 16;  // v below the pivot in registers: VR rows per lane (m - j - 1 <= 32 VR)
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int CL = (int)cluster.num_blocks();
  const int own = (c + CL - 1) / CL;
  const int nown = (c - rank + CL - 1) / CL;  // columns rank, rank + CL, ...
  const int steps = min(m, c);
  double* cols = sm;                                                    // own x m
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + (size_t)own * m);  // steps
  double* pub = reinterpret_cast<double*>(bars + steps);                // steps x (v0, tau)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int lj = 0; lj < nown; ++lj) {
    const double* src = W + (int64_t)(rank + lj * CL) * ldw;
    for (int i = threadIdx.x; i < m; i += blockDim.x) cols[(size_t)lj * m + i] = __ldcg(src + i);
  }
  for (int j = threadIdx.x; j < steps; j += blockDim.x) qr_mbar_init(&bars[j], 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncthreads();
  cluster.sync();  // every CTA's mbarriers exist before the first remote arrival
  // reflector 0: column 0 is local column 0 of rank 0, owned by its warp 0
  if (rank == 0 && warp == 0 && steps > 0) {
    double s = 0.0;
    for (int i = lane; i < m; i += 32) s = fma(cols[i], cols[i], s);
    qr_flow_publish(cols, W, 0, m, warp_sum(s), &pub[0], &bars[0], CL);
  }
  // this warp's columns: local lj = warp + q nwarps, global rank + lj CL
  int last = -1;
  for (int lj = warp; lj < nown; lj += nwarps) last = rank + lj * CL;
  const int jend = min(last, steps);  // reflectors 0 .. jend - 1 reach its columns
  for (int j = 0; j < jend; ++j) {
    if (!qr_mbar_wait(&bars[j], tflag)) break;
    const double* opub = cluster.map_shared_rank(&pub[2 * j], j % CL);
    const double v0 = opub[0], tau = opub[1];
    const double* gv = W + (int64_t)j * ldw;  // v below the pivot (L2: never cached stale)
    // first local column after j, then this warp's first one from there
    const int lj0 = j >= rank ? (j - rank) / CL + 1 : 0;
    int lj = lj0 + ((warp - lj0) % nwarps + nwarps) % nwarps;
    if (lj >= nown || tau == 0.0) {
      // nothing of this warp's to update (or the identity reflector); a
      // pivot column still publishes its reflector
      if (lj < nown && rank + lj * CL == j + 1 && j + 1 < steps) {
        double* w = cols + (size_t)lj * m;
        double s2 = 0.0;
        for (int i = j + 1 + lane; i < m; i += 32) s2 = fma(w[i], w[i], s2);
        qr_flow_publish(w, W + (int64_t)(j + 1) * ldw, j + 1, m, warp_sum(s2), &pub[2 * (j + 1)],
                        &bars[j + 1], CL);
      }
      continue;
    }
    const bool in_regs = m - (j + 1) <= 32 * VR;
    double vr[VR];
    if (in_regs) {
#pragma unroll
      for (int q = 0; q < VR; ++q) {
        const int i = j + 1 + lane + 32 * q;
        vr[q] = i < m ? __ldcg(gv + i) : 0.0;
      }
    }
    for (; lj < nown; lj += nwarps) {
      const int col = rank + lj * CL;
      double* w = cols + (size_t)lj * m;
      const bool pivot = col == j + 1 && j + 1 < steps;
      double t0 = lane == 0 ? v0 * w[j] : 0.0, t1 = 0.0;
      if (in_regs) {
#pragma unroll
        for (int q = 0; q < VR; q += 2) {
          const int i = j + 1 + lane + 32 * q;
          if (i < m) t0 = fma(vr[q], w[i], t0);
          if (i + 32 < m) t1 = fma(vr[q + 1], w[i + 32], t1);
        }
      } else {
        for (int i = j + 1 + lane; i < m; i += 64) {
          t0 = fma(__ldcg(gv + i), w[i], t0);
          if (i + 32 < m) t1 = fma(__ldcg(gv + i + 32), w[i + 32], t1);
        }
      }
      const double t = warp_sum(t0 + t1) * tau;
      if (lane == 0) w[j] -= t * v0;
      double s2 = 0.0;
      if (in_regs) {
#pragma unroll
        for (int q = 0; q < VR; ++q) {
          const int i = j + 1 + lane + 32 * q;
          if (i < m) {
            const double wi = w[i] - t * vr[q];
            w[i] = wi;
            s2 = fma(wi, wi, s2);
          }
        }
      } else {
        for (int i = j + 1 + lane; i < m; i += 32) {
          const double wi = w[i] - t * __ldcg(gv + i);
          w[i] = wi;
          s2 = fma(wi, wi, s2);
        }
      }
      // the next pivot: publish reflector j + 1 before the other columns
      if (pivot)
        qr_flow_publish(w, W + (int64_t)(j + 1) * ldw, j + 1, m, warp_sum(s2), &pub[2 * (j + 1)],
                        &bars[j + 1], CL);
    }
  }
  __syncthreads();
  cluster.sync();  // every read of W's broadcast columns and of the slots is done
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
