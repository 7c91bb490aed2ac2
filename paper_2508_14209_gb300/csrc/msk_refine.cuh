// msk_refine.cuh — device bodies of the refinement (sketch-and-precondition)
// passes and small vector steps, shared by ms_lstsq and the batched engine.
#pragma once
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "msk_device.cuh"

namespace msk {

// The refinement's convergence tests count only while the inner CG
// iterations so far stay within kStallIters * n: CG ends in at most n steps
// in exact arithmetic and a well-preconditioned solve takes far fewer; after
// more, the preconditioner is too poor for a stall or a small CG gain to
// show that x sits at the minimiser, and the solve stops unconverged.
constexpr int kStallIters = 4;

// ---------------------------------------------------------------------------
// Row-tiled FP64 passes over an FP64 A (tiles of kPR rows, whole rows in
// shared memory).  Passes over an FP32 A are in msk_pass.cuh.
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
// Entries j < nsum are summed over the CTAs, the rest (nonnegative column
// maxima) reduced by max.
__device__ __forceinline__ void pass_reduce_body(const double* __restrict__ part, int nctas, int len,
                                                 int nsum, double* __restrict__ out, int blk) {
  __shared__ double ws[8][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = blk * 32 + lane;
  const bool sum = j < nsum;
  double s = 0.0;
  if (j < len)
    for (int q = warp; q < nctas; q += 8) {
      const double v = part[(int64_t)q * len + j];
      s = sum ? s + v : fmax(s, v);
    }
  ws[warp][lane] = s;
  __syncthreads();
  if (warp == 0 && j < len) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t = sum ? t + ws[w][lane] : fmax(t, ws[w][lane]);
    out[j] = t;
  }
}

// ---------------------------------------------------------------------------
// Small FP64 vector kernels of the refinement (single CTA; n <= 512).

// Explicit inverse of the upper-triangular R (n x n, ldr) into Ri (n x n,
// column-major; rows below the diagonal zero).  Column c of Ri is R^{-1} e_c,
// computed by one warp with the column-oriented back substitution
//   t = e_c;  for j = c .. 0:  y_j = t_j / R_jj;  t_i -= y_j R_ij  (i < j),
// so every step reads a contiguous piece of R's column j; t lives in shared
// memory (all lanes read t_j as a broadcast) and 1/R_jj is formed once.
// Shared memory: kTriMaxN reciprocals + kTriMaxN per warp (blockDim <= 256).
constexpr int kTriMaxN = 512;
__device__ __forceinline__ void tri_inverse_body(const double* __restrict__ R, int n, int64_t ldr,
                                                 double* __restrict__ Ri, int blk, int nblk) {
  __shared__ double rinv[kTriMaxN];
  __shared__ double tw[8][kTriMaxN];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwb = (int)(blockDim.x >> 5);
  const int warp_g = blk * nwb + warp, nw = nblk * nwb;
  for (int j = threadIdx.x; j < n; j += blockDim.x) rinv[j] = 1.0 / R[j + (int64_t)j * ldr];
  __syncthreads();
  double* t = tw[warp];
  for (int c = warp_g; c < n; c += nw) {
    double* y = Ri + (int64_t)c * n;
    for (int i = lane; i <= c; i += 32) t[i] = (i == c) ? 1.0 : 0.0;
    for (int i = c + 1 + lane; i < n; i += 32) y[i] = 0.0;
    __syncwarp();
    for (int j = c; j >= 0; --j) {
      const double yj = t[j] * rinv[j];
      if (lane == 0) y[j] = yj;
      const double* col = R + (int64_t)j * ldr;
      for (int i = lane; i < j; i += 32) t[i] = fma(-yj, __ldg(col + i), t[i]);
      __syncwarp();
    }
  }
}

// x = Ri c with Ri = R^{-1} upper triangular (n x n, column-major): the
// sketch-and-solve start x0 = R11^{-1} R[0:n, n] when R^{-1} is formed anyway
// (refinement).  One CTA: G = blockDim / n thread groups split the sum over
// j >= i (reads of Ri[i + j n] contiguous across a group); partial sums added
// in group order.  scratch: blockDim doubles of shared memory.
__device__ __forceinline__ void tri_matvec_body(const double* __restrict__ Ri, int n,
                                                const double* __restrict__ c, double* __restrict__ x,
                                                double* scratch) {
  const int G = (int)blockDim.x >= 2 * n ? (int)blockDim.x / n : 1;
  for (int idx = threadIdx.x; idx < n * G; idx += blockDim.x) {
    const int i = idx % n, g = idx / n;
    double s = 0.0;
    for (int j = i + g; j < n; j += G) s += Ri[i + (int64_t)j * n] * c[j];
    scratch[idx] = s;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double s = 0.0;
    for (int g = 0; g < G; ++g) s += scratch[g * n + i];
    x[i] = s;
  }
}

// State of the refinement, all device FP64 (n-vectors unless noted):
//   x, dlt (correction), p (search dir), res (normal-eq. residual), z,
//   sc[0] = rho.
struct RefState {
  double *x, *dlt, *p, *res, *z, *sc;
};

// z = Ri (Ri^T v): the preconditioner M^{-1} v with M = R^T R (one CTA).
//   tmp = Ri^T v : warp w takes columns w, w + nwarps, ...; its lanes read the
//                  column contiguously and are summed by shuffles;
//   z = Ri tmp   : G = blockDim / n thread groups split the sum over j
//                  (j = i + g, i + g + G, ...); reads of Ri[i + j n] are
//                  contiguous across the threads of a group; partial sums are
//                  added in group order.
// scratch: at least max(n, blockDim) + n doubles of shared memory.
__device__ __forceinline__ void apply_minv(const double* __restrict__ Ri, int n, const double* v,
                                           double* tmp, double* z, double* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = warp; j < n; j += nw) {
    const double* col = Ri + (int64_t)j * n;
    double s = 0.0;
    for (int i = lane; i <= j; i += 32) s += col[i] * v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) tmp[j] = s;
  }
  __syncthreads();
  const int G = (int)blockDim.x >= 2 * n ? (int)blockDim.x / n : 1;
  for (int idx = threadIdx.x; idx < n * G; idx += blockDim.x) {
    const int i = idx % n, g = idx / n;
    double s = 0.0;
    for (int j = i + g; j < n; j += G) s += Ri[i + (int64_t)j * n] * tmp[j];
    scratch[idx] = s;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double s = 0.0;
    for (int g = 0; g < G; ++g) s += scratch[g * n + i];
    z[i] = s;
  }
  __syncthreads();
}

// Start of an inner solve: res = g (from the FP64 pass), dlt = 0,
// z = M^{-1} res, p = z, rho = res.z.
__device__ __forceinline__ void pcg_start_body(const double* __restrict__ Ri, int n,
                                               const double* __restrict__ g, RefState s) {
  __shared__ double tmp[512];
  __shared__ double scr[1024];
  __shared__ double red[32];
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    s.res[j] = g[j];
    s.dlt[j] = 0.0;
  }
  __syncthreads();
  apply_minv(Ri, n, s.res, tmp, s.z, scr);
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

// Refinement scalars (sc, FP64):
//   [0] rho = res.z            [1] gain of the last step (alpha rho)
//   [2] active (1 while the inner solve runs)
//   [3] floor: a step gaining no more than this ends the inner solve
//   [4] inner steps taken      [5] 1 if the very first step was below the floor
//   [6] sum of the gains       [7] 1 if the solve ended by the gain rule
//                                  (rather than by the step limit)
constexpr int kScCount = 8;

// Start-of-solve bookkeeping (thread 0, after pcg_start_body).
__device__ __forceinline__ void pcg_arm(double* sc, double floor) {
  sc[1] = 0.0;
  sc[2] = 1.0;
  sc[3] = floor;
  sc[4] = 0.0;
  sc[5] = 0.0;
  sc[6] = 0.0;
  sc[7] = 0.0;
}

// Stopping rule after a CG step (one thread, after the step): returns
// true when this step ended the inner solve.
__device__ __forceinline__ bool pcg_stop_check(double* sc, int max_steps) {
  sc[4] += 1.0;
  sc[6] += sc[1];
  const bool by_rule = !(sc[1] > sc[3]) || !(sc[0] > 0.0);
  if (by_rule || sc[4] >= (double)max_steps) {
    if (by_rule && sc[4] == 1.0) sc[5] = 1.0;
    sc[7] = by_rule ? 1.0 : 0.0;
    sc[2] = 0.0;
    return true;
  }
  return false;
}
// ---------------------------------------------------------------------------
// One CG step fused with the reduction of the pass partials, on a cluster of
// kUpdCL CTAs (kUpdThreads threads each; n <= kUpdMaxN).  CTA r owns the
// slice j0 = r*sl .. j0+sl-1 of the n-vectors (sl = ceil(n / CL)):
//   1. v_j = sum over pass CTAs of part[c][j] (j in the slice; fixed order),
//      and the slice's share of p.v;
//   -- barrier: alpha = rho / p.v from the CL shares, summed in rank order;
//   2. dlt_j += alpha p_j, res_j -= alpha v_j; res_j to every CTA (DSMEM);
//   -- barrier: tmp_j = (Ri^T res)_j for the slice (one warp per column);
//      tmp_j to every CTA;
//   -- barrier: z_i = (Ri tmp)_i for the slice and its share of rho' = res.z;
//   -- barrier: rho' from the shares; beta = rho' / rho; p_i = z_i + beta p_i.
// The FP64 work of M^{-1} (2 n^2 operations, a few microseconds on one SM at
// GB300's FP64 rate) is split CL ways.  Returns true in CTA 0, thread 0 when
// this step ended the inner solve (pcg_stop_check).  All CTAs of the cluster
// see the same sc[2] on entry, so they return together when the solve has
// already stopped.
constexpr int kUpdCL = 8, kUpdThreads = 256, kUpdMaxN = 512;
constexpr int kUpdMaxSlice = kUpdMaxN / kUpdCL;

__device__ __forceinline__ bool pcg_cluster_update_body(const double* __restrict__ part, int nchunks,
                                                        int stride, const double* __restrict__ Ri,
                                                        int n, RefState s, int max_steps) {
  namespace cgr = cooperative_groups;
  cgr::cluster_group cluster = cgr::this_cluster();
  const int CL = (int)cluster.num_blocks(), rank = (int)cluster.block_rank();
  __shared__ double resg[kUpdMaxN], tmpg[kUpdMaxN];
  __shared__ double pr[kUpdThreads];
  __shared__ double vsl[kUpdMaxSlice], zsl[kUpdMaxSlice];
  __shared__ double dotp[kUpdCL], dotr[kUpdCL];
  __shared__ double red[32];
  if (s.sc[2] == 0.0) return false;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nw = blockDim.x >> 5;
  const int sl = (n + CL - 1) / CL;
  const int j0 = rank * sl, ns = max(0, min(n, j0 + sl) - j0);
  const double rho_old = s.sc[0];
  auto block_total = [&](double v) -> double {  // all threads get the sum (fixed order)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double r = 0.0;
    for (int w = 0; w < nw; ++w) r += red[w];
    return r;
  };
  // 1. v on the slice from the pass partials; share of p.v
  const int G = ns > 0 ? (int)blockDim.x / ns : 1;
  if (ns > 0 && t < G * ns) {
    const int jj = t % ns, g = t / ns;
    double a0 = 0.0, a1 = 0.0;
    int c = g;
    for (; c + G < nchunks; c += 2 * G) {
      a0 += part[(int64_t)c * stride + j0 + jj];
      a1 += part[(int64_t)(c + G) * stride + j0 + jj];
    }
    if (c < nchunks) a0 += part[(int64_t)c * stride + j0 + jj];
    pr[t] = a0 + a1;
  }
  __syncthreads();
  double pv = 0.0;
  if (t < ns) {
    double v = 0.0;
    for (int g = 0; g < G; ++g) v += pr[g * ns + t];
    vsl[t] = v;
    pv = s.p[j0 + t] * v;
  }
  pv = block_total(pv);
  if (t < CL) *cluster.map_shared_rank(&dotp[rank], t) = pv;
  cluster.sync();
  double pAp = 0.0;
  for (int r = 0; r < CL; ++r) pAp += dotp[r];
  const double alpha = pAp > 0.0 ? rho_old / pAp : 0.0;
  // 2. dlt, res on the slice; res to every CTA
  if (t < ns) {
    const int j = j0 + t;
    s.dlt[j] += alpha * s.p[j];
    const double rj = s.res[j] - alpha * vsl[t];
    s.res[j] = rj;
    for (int r = 0; r < CL; ++r) *cluster.map_shared_rank(&resg[j], r) = rj;
  }
  cluster.sync();
  // 3. tmp = Ri^T res on the slice (column j of Ri is contiguous)
  for (int jj = warp; jj < ns; jj += nw) {
    const int j = j0 + jj;
    const double* col = Ri + (int64_t)j * n;
    double a = 0.0;
    for (int i = lane; i <= j; i += 32) a += col[i] * resg[i];
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane < CL) *cluster.map_shared_rank(&tmpg[j], lane) = a;
  }
  cluster.sync();
  // 4. z = Ri tmp on the slice: thread (ii, g) sums j = i + g, i + g + G, ...
  if (ns > 0 && t < G * ns) {
    const int ii = t % ns, g = t / ns, i = j0 + ii;
    double a = 0.0;
    for (int j = i + g; j < n; j += G) a += Ri[i + (int64_t)j * n] * tmpg[j];
    pr[t] = a;
  }
  __syncthreads();
  double rz = 0.0;
  if (t < ns) {
    double z = 0.0;
    for (int g = 0; g < G; ++g) z += pr[g * ns + t];
    zsl[t] = z;
    s.z[j0 + t] = z;
    rz = resg[j0 + t] * z;
  }
  rz = block_total(rz);
  if (t < CL) *cluster.map_shared_rank(&dotr[rank], t) = rz;
  cluster.sync();
  double rho = 0.0;
  for (int r = 0; r < CL; ++r) rho += dotr[r];
  const double beta = rho_old > 0.0 ? rho / rho_old : 0.0;
  if (t < ns) s.p[j0 + t] = zsl[t] + beta * s.p[j0 + t];
  bool stopped = false;
  if (rank == 0 && t == 0) {
    s.sc[1] = alpha * rho_old;  // decrease of ||b - A x||^2 by this step (CG identity)
    s.sc[0] = rho;
    stopped = pcg_stop_check(s.sc, max_steps);
  }
  return stopped;
}

}  // namespace msk
