// lstsq.cu — least-squares solvers built on the multisketch:
//   * ms_lstsq, refine = 0: sketch-and-solve (Algorithm 1, Section 2):
//       Z = G S [A b] (p x (n+1)), Householder QR of Z, x = R11^{-1} R[0:n, n].
//   * ms_lstsq, refine = 1: sketch-and-precondition refinement (the iterative
//       route Section 6 cites).  Outer loop: true residual r = b - A x and
//       g = A^T r in FP64 (one pass over A).  Inner loop: conjugate gradients
//       on A^T A d = g preconditioned by M = R11^T R11, each iteration one pass
//       over A computing A^T (A p) — in FP64 for FP64 A, in double-single
//       arithmetic on the FP32 units for FP32 A (binary32 alone fails: with
//       kappa(A) * 2^-24 > 1 the products A p cancel to noise) — until a step
//       lowers ||b - A x||^2 by less than 0.05 tol ||r||^2 (CG on the normal
//       equations lowers it by alpha*rho per step).  Then x += d and a new
//       FP64 residual.  Converged when that residual confirms the decrease
//       the CG recurrences predicted (to tol * ||r||^2), when the relative
//       residual changes by at most tol * relres between outer steps, or when
//       the first inner step already gains less than the floor.
//   * ne_lstsq: normal equations (Section 6.3): [A b]^T [A b] in one FP64
//       pass (split over row slices, partials summed in a fixed order),
//       Cholesky, two triangular solves.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "msk_device.cuh"
#include "msk_internal.h"
#include "msk_pass.cuh"
#include "msk_refine.cuh"

namespace msk {

// ---------------------------------------------------------------------------
// Gram matrix of [A b] (FP64): C[a][c] = sum_i X[i][a] X[i][c] for the
// (n+1)-column X = [A b], upper 64x64 tiles only, split over row slices.
constexpr int kGrT = 64, kGrK = 32, kGrThreads = 256;

template <typename TA>
__device__ __forceinline__ double x_at(const TA* A, int64_t lda, int64_t n, const double* b,
                                       int64_t i, int64_t c) {
  return c < n ? (double)A[i + c * lda] : b[i];
}

template <typename TA>
__global__ void __launch_bounds__(kGrThreads) gram_kernel(const TA* __restrict__ A, int64_t lda,
                                                       int64_t d, int64_t n,
                                                       const double* __restrict__ b, int64_t rchunk,
                                                       const int2* __restrict__ tiles,
                                                       double* __restrict__ part) {
  __shared__ double Xa[kGrK][kGrT + 1];
  __shared__ double Xc[kGrK][kGrT + 1];
  const int64_t ncol = n + 1;
  const int2 t = tiles[blockIdx.x];
  const int64_t a0 = (int64_t)t.x * kGrT, c0 = (int64_t)t.y * kGrT;
  const int64_t r0 = (int64_t)blockIdx.y * rchunk, r1 = min(d, r0 + rchunk);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4] = {};
  for (int64_t k0 = r0; k0 < r1; k0 += kGrK) {
    for (int e = threadIdx.x; e < kGrK * kGrT; e += kGrThreads) {
      const int kk = e % kGrK, cc = e / kGrK;
      const int64_t i = k0 + kk;
      Xa[kk][cc] = (i < r1 && a0 + cc < ncol) ? x_at(A, lda, n, b, i, a0 + cc) : 0.0;
      Xc[kk][cc] = (i < r1 && c0 + cc < ncol) ? x_at(A, lda, n, b, i, c0 + cc) : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kGrK; ++kk) {
      double av[4], cv[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) av[q] = Xa[kk][ty + 16 * q];
#pragma unroll
      for (int q = 0; q < 4; ++q) cv[q] = Xc[kk][tx + 16 * q];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(av[u], cv[v], acc[u][v]);
    }
    __syncthreads();
  }
  // part[slice][c * ncol + a] (column-major (n+1) x (n+1)); only a <= c kept
  double* out = part + (int64_t)blockIdx.y * ncol * ncol;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int64_t a = a0 + ty + 16 * u, c = c0 + tx + 16 * v;
      if (a < ncol && c < ncol && a <= c) out[c * ncol + a] = acc[u][v];
    }
}

// Sum the slices and mirror the upper triangle: one warp per entry, lane l
// adds slices l, l+32, ... in order, then a fixed shuffle tree (the same
// order on every run).
__global__ void gram_reduce_kernel(const double* __restrict__ part, int S, int64_t ncol,
                                   double* __restrict__ C) {
  const int64_t total = ncol * ncol;
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t e = w0; e < total; e += nw) {
    const int64_t c = e / ncol, a = e % ncol;
    const int64_t src = a <= c ? c * ncol + a : a * ncol + c;
    double s = 0.0;
    for (int q = lane; q < S; q += 32) s += part[(int64_t)q * total + src];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) C[e] = s;
  }
}

static void launch_gram_reduce(const double* part, int S, int64_t ncol, double* C, cudaStream_t st) {
  const int64_t warps = ncol * ncol;
  gram_reduce_kernel<<<(unsigned)std::min<int64_t>((warps + 7) / 8, 4096), 256, 0, st>>>(part, S,
                                                                                       ncol, C);
}

// Gram of [A b] by 2x2 blocks of the upper triangle (up to kGtMaxCol
// columns).  GB300's FP64 pipe (about 1.75 DFMA per clock per SM) is the
// bound, so what counts is how many products are computed: blocks of 2x2
// cover the upper triangle with half of each diagonal block to spare (1.02x
// the needed products at 129 columns, where 64x64 tiles computed 2.9x).  A
// CTA "panel" owns a contiguous run of the blocks (row-major order over the
// upper triangle), each thread kGtBpt of them with their four accumulators
// in registers; K rows of its row slice of [A b] are staged in shared memory
// (zero-padded to an even column count), and a block takes two 16-byte loads
// per four DFMAs.  Partials per row slice, reduced in a fixed order.
constexpr int kGtK = 32, kGtBpt = 8, kGtMaxThreads = 512, kGtMaxCol = 513;

__device__ __forceinline__ void gt_cp8(double* dst, const double* src, int bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(bytes)
               : "memory");
}

// nbuf = 2: the next K rows are copied (cp.async) while this K-row tile is
// multiplied; nbuf = 1 when two tiles do not fit in shared memory.
// BPT: blocks (slots) per thread.  A CTA of blockDim = G * tpanel threads runs
// G row groups over the same panel: group g takes rows kk = g, g + G, ... of
// each staged tile with its own accumulators and writes its own partial slice
// (blockIdx.y * G + g).  Narrow panels (few 2x2 blocks) use BPT = 2 and G > 1,
// so that an SM holds enough independent FP64 accumulation chains.
template <int BPT>
__global__ void __launch_bounds__(kGtMaxThreads) gram_tri_kernel(
    const double* __restrict__ A, int64_t lda, int64_t d, int64_t n, const double* __restrict__ b,
    int64_t rchunk, int nb, int per_panel, int nbuf, int tpanel, double* __restrict__ part) {
  extern __shared__ __align__(16) double gt_x[];
  const int64_t ncol = n + 1;
  const int pitch = 2 * nb + 2;
  const int64_t nblk = (int64_t)nb * (nb + 1) / 2;
  const int64_t bfirst = (int64_t)blockIdx.x * per_panel;
  const int64_t blast = min(nblk, bfirst + per_panel);
  const int G = (int)blockDim.x / tpanel;
  const int grp = (int)threadIdx.x / tpanel, tl = (int)threadIdx.x % tpanel;
  int ai[BPT], cj[BPT];
#pragma unroll
  for (int s = 0; s < BPT; ++s) {
    const int64_t q = bfirst + tl + (int64_t)s * tpanel;
    int i = 0, j = 0;
    if (q < blast) {
      int64_t r = q;
      while (r >= nb - i) {
        r -= nb - i;
        ++i;
      }
      j = i + (int)r;
    }
    ai[s] = q < blast ? 2 * i : -1;  // -1: no block in this slot
    cj[s] = 2 * j;
  }
  const int64_t r0 = (int64_t)blockIdx.y * rchunk, r1 = min(d, r0 + rchunk);
  double acc[BPT][4] = {};
  const int width = 2 * nb;  // staged columns (ncol, or ncol + 1 zero column)
  // rows k0 .. k0+K-1 of [A b] into buf (zero past r1 and in the pad column)
  auto stage = [&](int64_t k0, double* buf) {
    for (int e = threadIdx.x; e < kGtK * width; e += blockDim.x) {
      const int kk = e % kGtK, cc = e / kGtK;
      const int64_t i = k0 + kk;
      const bool ok = i < r1 && cc < ncol;
      const double* src = !ok ? A : (cc < n ? A + i + cc * lda : b + i);
      gt_cp8(buf + kk * pitch + cc, src, ok ? 8 : 0);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  const int tsz = kGtK * pitch;  // doubles per staged tile
  if (r0 < r1) stage(r0, gt_x);
  int it = 0;
  for (int64_t k0 = r0; k0 < r1; k0 += kGtK, ++it) {
    double* cur = gt_x + (nbuf == 2 ? (it & 1) * tsz : 0);
    if (nbuf == 2 && k0 + kGtK < r1) {
      stage(k0 + kGtK, gt_x + ((it + 1) & 1) * tsz);
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();
    // (8-slot panels have one row group: their loop keeps a unit stride)
    const int kk0 = BPT == 2 ? grp : 0, kstep = BPT == 2 ? G : 1;
#pragma unroll 2
    for (int kk = kk0; kk < kGtK; kk += kstep) {
      const double* row = cur + kk * pitch;
#pragma unroll
      for (int s = 0; s < BPT; ++s) {
        if (ai[s] < 0) continue;
        const double2 av = *reinterpret_cast<const double2*>(row + ai[s]);
        const double2 cv = *reinterpret_cast<const double2*>(row + cj[s]);
        acc[s][0] = fma(av.x, cv.x, acc[s][0]);
        acc[s][1] = fma(av.x, cv.y, acc[s][1]);
        acc[s][2] = fma(av.y, cv.x, acc[s][2]);
        acc[s][3] = fma(av.y, cv.y, acc[s][3]);
      }
    }
    __syncthreads();  // cur is free for the copies issued next
    if (nbuf == 1 && k0 + kGtK < r1) stage(k0 + kGtK, gt_x);
  }
  // part[slice][c * ncol + a] (column-major (n+1) x (n+1)); only a <= c kept
  double* out = part + ((int64_t)blockIdx.y * G + grp) * ncol * ncol;
#pragma unroll
  for (int s = 0; s < BPT; ++s) {
    if (ai[s] < 0) continue;
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int v = 0; v < 2; ++v) {
        const int64_t a = ai[s] + u, c = cj[s] + v;
        if (a < ncol && c < ncol && a <= c) out[c * ncol + a] = acc[s][2 * u + v];
      }
  }
}

struct GramPlan {
  bool tri;              // gram_tri_kernel (else 64x64 tiles of gram_kernel)
  int ntile, npairs;     // tiles: tiles per side, upper tile pairs
  int nb, per_panel, npanels, threads, nbuf;  // tri: 2x2 blocks per side, blocks per CTA panel
  int bpt, tpanel, groups;  // tri: slots per thread, threads per panel copy, row groups per CTA
  int slices;
  int parts;                // partial slices written: slices * groups
  int64_t rchunk;
  size_t smem;
};

static GramPlan gram_plan(int64_t d, int64_t n) {
  GramPlan g{};
  const int64_t ncol = n + 1;
  g.tri = ncol <= kGtMaxCol;
  int64_t groups;  // CTAs per row slice
  int64_t kstep;
  int64_t target = 2LL * num_sms();  // CTAs in all
  if (g.tri) {
    g.nb = (int)((ncol + 1) / 2);
    const int64_t nblk = (int64_t)g.nb * (g.nb + 1) / 2;
    // narrow panels: 2 slots per thread and up to 8 row groups per CTA
    g.bpt = nblk <= 512 ? 2 : kGtBpt;
    const int64_t cap = (int64_t)(g.bpt == 2 ? 256 : kGtMaxThreads) * g.bpt;
    g.npanels = (int)((nblk + cap - 1) / cap);
    g.per_panel = (int)((nblk + g.npanels - 1) / g.npanels);
    g.tpanel = (int)(((g.per_panel + g.bpt - 1) / g.bpt + 31) / 32 * 32);
    g.groups = g.bpt == 2 ? std::max(1, std::min(8, 256 / g.tpanel)) : 1;
    g.threads = g.tpanel * g.groups;
    const size_t tile = (size_t)kGtK * (2 * g.nb + 2) * sizeof(double);
    g.nbuf = 2 * tile <= (size_t)160 * 1024 ? 2 : 1;
    g.smem = g.nbuf * tile;
    // The FP64 pipe needs many independent accumulation chains per SM (one
    // warp's chain of dependent DFMAs issues far below the pipe's rate):
    // about 16 warps of 8-slot panels, or 48 of narrow 2-slot ones, as
    // occupancy allows, by giving panels more row slices.
    const void* kfn = g.bpt == 2 ? reinterpret_cast<const void*>(gram_tri_kernel<2>)
                                 : reinterpret_cast<const void*>(gram_tri_kernel<kGtBpt>);
    int occ = 0;
    if (allow_max_smem(kfn) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kfn, g.threads, g.smem) != cudaSuccess)
      occ = 1;
    const int warps = g.threads / 32;
    const int want = g.bpt == 2 ? 48 : 16;
    const int per_sm = std::max(1, std::min(occ, std::max(2, (want + warps - 1) / warps)));
    target = (int64_t)num_sms() * per_sm;
    groups = g.npanels;
    kstep = kGtK;
  } else {
    g.ntile = (int)((ncol + kGrT - 1) / kGrT);
    g.npairs = g.ntile * (g.ntile + 1) / 2;
    groups = g.npairs;
    kstep = kGrK;
  }
  int64_t s = std::max<int64_t>(1, target / groups);
  s = std::min<int64_t>(s, std::max<int64_t>(1, (d + kstep - 1) / kstep));
  g.rchunk = ((d + s - 1) / s + kstep - 1) / kstep * kstep;
  if (g.rchunk < kstep) g.rchunk = kstep;
  g.slices = (int)std::max<int64_t>(1, (d + g.rchunk - 1) / g.rchunk);
  g.parts = g.slices * (g.tri ? g.groups : 1);
  return g;
}

static size_t gram_workspace(int64_t d, int64_t n) {
  GramPlan g = gram_plan(d, n);
  const int64_t ncol = n + 1;
  Need nd;
  nd.add((size_t)std::max(g.npairs, 1) * sizeof(int2));
  nd.add((size_t)g.parts * ncol * ncol * sizeof(double));
  return nd.used;
}

// Partials of the Gram of [A b] (FP64 A) into part[slices][ncol][ncol]
// (upper entries a <= c); `tiles` is workspace for the 64x64-tile plan.
static int launch_gram(const GramPlan& g, const double* A, int64_t lda, int64_t d, int64_t n,
                       const double* b, int2* tiles, double* part, cudaStream_t st) {
  if (g.tri) {
    dim3 grid(g.npanels, g.slices);
    if (g.bpt == 2) {
      MSK_ALLOW_SMEM(gram_tri_kernel<2>);
      gram_tri_kernel<2><<<grid, g.threads, g.smem, st>>>(A, lda, d, n, b, g.rchunk, g.nb,
                                                          g.per_panel, g.nbuf, g.tpanel, part);
    } else {
      MSK_ALLOW_SMEM(gram_tri_kernel<kGtBpt>);
      gram_tri_kernel<kGtBpt><<<grid, g.threads, g.smem, st>>>(A, lda, d, n, b, g.rchunk, g.nb,
                                                               g.per_panel, g.nbuf, g.tpanel, part);
    }
    MSK_CHECK_LAUNCH("gram_tri_kernel");
    return MSK_OK;
  }
  std::vector<int2> hp;
  for (int a = 0; a < g.ntile; ++a)
    for (int c = a; c < g.ntile; ++c) hp.push_back(make_int2(a, c));
  MSK_CUDA(cudaMemcpyAsync(tiles, hp.data(), hp.size() * sizeof(int2), cudaMemcpyHostToDevice, st));
  dim3 grid(g.npairs, g.slices);
  gram_kernel<double><<<grid, kGrThreads, 0, st>>>(A, lda, d, n, b, g.rchunk, tiles, part);
  MSK_CHECK_LAUNCH("gram_kernel");
  return MSK_OK;
}

// Thin kernels over the bodies in msk_refine.cuh.
// `active` (optional): the inner solve's running flag; the inner-iteration
// kernels return at once when it is 0, so that a round of several iterations
// can be queued without a host round trip per iteration.
template <typename TA, bool RESID>
__global__ void __launch_bounds__(kPThreads) pass_kernel(const TA* __restrict__ A, int64_t lda,
                                                      int64_t d, int n, int pitch,
                                                      const double* __restrict__ b,
                                                      const double* __restrict__ vin,
                                                      double* __restrict__ part,
                                                      const double* __restrict__ active) {
  if (active && *active == 0.0) return;
  extern __shared__ __align__(16) unsigned char pk_smem[];
  pass_body<TA, RESID>(A, lda, d, n, pitch, b, vin, part, blockIdx.x, gridDim.x, pk_smem);
}
__global__ void __launch_bounds__(256) pass_reduce_kernel(const double* __restrict__ part, int nctas,
                                                          int len, int nsum, double* __restrict__ out,
                                                          const double* __restrict__ active) {
  if (active && *active == 0.0) return;
  pass_reduce_body(part, nctas, len, nsum, out, blockIdx.x);
}
template <int NC, bool RESID>
__global__ void __launch_bounds__(kP32Threads, pass32_ctas_per_sm(NC))
    pass32_kernel(const float* __restrict__ A, int64_t lda, int64_t d, int n, int cw,
                  const double* __restrict__ b, const double* __restrict__ vin,
                  const double* __restrict__ cmax, double* __restrict__ part,
                  const double* __restrict__ active) {
  if (active && *active == 0.0) return;
  extern __shared__ __align__(16) unsigned char p32_smem[];
  if constexpr (NC == 0)
    pass32g_body<RESID>(A, lda, d, n, cw == 4, b, vin, part, blockIdx.x, gridDim.x, p32_smem);
  else
    pass32n_body<NC, RESID>(A, lda, d, n, cw, b, vin, cmax, part, blockIdx.x, gridDim.x, p32_smem);
}
__global__ void __launch_bounds__(512) x0_kernel(const double* __restrict__ Ri, int n,
                                                 const double* __restrict__ c, double* __restrict__ x) {
  __shared__ double scr[512];
  tri_matvec_body(Ri, n, c, x, scr);
}
__global__ void tri_inverse_kernel(const double* __restrict__ R, int n, int64_t ldr,
                                   double* __restrict__ Ri) {
  tri_inverse_body(R, n, ldr, Ri, blockIdx.x, gridDim.x);
}
__global__ void pcg_start_kernel(const double* __restrict__ Ri, int n, const double* __restrict__ g,
                                 RefState s, double floor) {
  pcg_start_body(Ri, n, g, s);
  __syncthreads();
  if (threadIdx.x == 0) pcg_arm(s.sc, floor);
}

// One CG step fused with the reduction of the pass partials (one cluster).
__global__ void __launch_bounds__(kUpdThreads) pcg_cluster_kernel(const double* __restrict__ part,
                                                                 int nchunks, int stride,
                                                                 const double* __restrict__ Ri, int n,
                                                                 RefState s, int max_steps) {
  pcg_cluster_update_body(part, nchunks, stride, Ri, n, s, max_steps);
}
// x += dlt
__global__ void axpy_kernel(int n, const double* __restrict__ dlt, double* __restrict__ x) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
    x[j] += dlt[j];
}

static int pass_grid(int64_t d) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((d + kPR - 1) / kPR, 3LL * num_sms()));
}

// out == nullptr: leave the per-CTA partials unreduced (the fused CG step
// reduces them); *grid_out receives the number of partials.
template <typename TA, bool RESID>
static int launch_pass_t(const TA* A, int64_t lda, int64_t d, int n, const double* b,
                         const double* vin, double* part, double* out, const double* active,
                         cudaStream_t st, int* grid_out) {
  const int pitch = n | 1;  // odd: conflict-free transposing stores and row reads
  const size_t smem = sizeof(double) * ((size_t)n + kPR) + sizeof(TA) * (size_t)kPR * pitch;
  auto kern = pass_kernel<TA, RESID>;
  MSK_ALLOW_SMEM(kern);
  const int grid = pass_grid(d);
  kern<<<grid, kPThreads, smem, st>>>(A, lda, d, n, pitch, b, vin, part, active);
  MSK_CHECK_LAUNCH("pass_kernel");
  if (grid_out) *grid_out = grid;
  if (!out) return MSK_OK;
  pass_reduce_kernel<<<(n + 2 + 31) / 32, 256, 0, st>>>(part, grid, n + 2, n + 2, out, active);
  MSK_CHECK_LAUNCH("pass_reduce_kernel");
  return MSK_OK;
}

// Passes over an FP32 A (msk_pass.cuh): the FP64 residual pass and the
// double-single operator pass of the inner iterations.  Persistent CTAs, at
// most kPassCtasPerSm per SM (the occupancy of the 70 KB shared-memory tile
// pipeline), each walking every nctas-th tile of R rows.
constexpr int kPassCtasPerSm = 3;

static int pass32_grid(int64_t d, int n) {
  const int R = pass32_rows(n);
  return (int)std::max<int64_t>(1, std::min<int64_t>((d + R - 1) / R, (int64_t)kPassCtasPerSm * num_sms()));
}

// cmax: the column maxima of |A| from an earlier residual pass (inner passes
// of the specialised bodies).
template <int NC, bool RESID>
static int launch_pass32_nc(const float* A, int64_t lda, int64_t d, int n, const double* b,
                            const double* vin, const double* cmax, double* part, double* out,
                            const double* active, cudaStream_t st, int* grid_out) {
  const size_t smem = pass32_smem(n);
  auto kern = pass32_kernel<NC, RESID>;
  MSK_ALLOW_SMEM(kern);
  int per_sm = 0;
  MSK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kP32Threads, smem));
  per_sm = std::max(1, std::min<int>(per_sm, (int)std::min<long long>(kPassCtasPerSm, tune_get("pass.ctas_per_sm", kPassCtasPerSm))));
  const int R = pass32_rows(n);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((d + R - 1) / R, (int64_t)per_sm * num_sms()));
  if (!RESID && NC != 0 && !cmax) return MSK_ENOTSUP;  // no residual pass before
  kern<<<grid, kP32Threads, smem, st>>>(A, lda, d, n, pass32_copy_width(A, lda), b, vin, cmax, part,
                                        active);
  MSK_CHECK_LAUNCH("pass32_kernel");
  if (grid_out) *grid_out = grid;
  if (!out) return MSK_OK;
  const int len = RESID && NC != 0 ? (int)pass_out_len(n) : n + 2;
  pass_reduce_kernel<<<(len + 31) / 32, 256, 0, st>>>(part, grid, len, n + 2, out, active);
  MSK_CHECK_LAUNCH("pass_reduce_kernel");
  return MSK_OK;
}

template <bool RESID>
static int launch_pass32(const float* A, int64_t lda, int64_t d, int n, const double* b,
                         const double* vin, const double* cmax, double* part, double* out,
                         const double* active, cudaStream_t st, int* grid_out) {
  if (n > 2 * kP32Threads) return MSK_ENOTSUP;
#define MSK_PASS32_NC(NCV) \
  launch_pass32_nc<NCV, RESID>(A, lda, d, n, b, vin, cmax, part, out, active, st, grid_out)
  switch (pass32_class(n)) {
    case 16: return MSK_PASS32_NC(16);
    case 32: return MSK_PASS32_NC(32);
    case 64: return MSK_PASS32_NC(64);
    case 128: return MSK_PASS32_NC(128);
    case 256: return MSK_PASS32_NC(256);
    default: return MSK_PASS32_NC(0);
  }
#undef MSK_PASS32_NC
}

// RESID: out = [A^T r (n), ||r||^2, ||b||^2, column maxima of |A| (n; FP32 A,
// n <= 256)] with r = b - A x (FP64; for FP32 A the sum A^T r in
// double-single): out holds pass_out_len(n) doubles.
// else : out = [A^T A p (n), ., .] (FP64 for FP64 A, double-single for FP32 A,
// which reads the column maxima at cmax = the residual pass's out + n + 2).
static int launch_pass(const void* A, int dtype, int64_t lda, int64_t d, int n, const double* b,
                       const double* vin, bool resid, double* part, double* out,
                       const double* active, cudaStream_t st, int* grid_out = nullptr,
                       const double* cmax = nullptr) {
  if (dtype == MSK_F64) {
    if (resid)
      return launch_pass_t<double, true>(static_cast<const double*>(A), lda, d, n, b, vin, part,
                                         out, nullptr, st, grid_out);
    return launch_pass_t<double, false>(static_cast<const double*>(A), lda, d, n, b, vin, part, out,
                                        active, st, grid_out);
  }
  if (resid)
    return launch_pass32<true>(static_cast<const float*>(A), lda, d, n, b, vin, nullptr, part, out,
                               nullptr, st, grid_out);
  return launch_pass32<false>(static_cast<const float*>(A), lda, d, n, nullptr, vin, cmax, part, out,
                              active, st, grid_out);
}

static size_t pass_workspace(int64_t d, int64_t n) {
  return (size_t)std::max(pass_grid(d), pass32_grid(d, (int)n)) * pass_out_len(n) * sizeof(double);
}

constexpr int kMaxInner = 200;
constexpr double kDecFrac = 0.05;
constexpr int kInnerRound = 4;  // inner iterations queued per host check

}  // namespace msk

using namespace msk;

namespace {

bool is_tensor_prec_l(int prec) {
  return prec == MSK_GEMM_BF16 || prec == MSK_GEMM_F16 || prec == MSK_GEMM_BF16X3;
}



// Column-major W (m x c, ldw) from row-major Y (m x c, ldy): 32 x 32 tiles
// through shared memory (the CountSketch writes bucket rows; the QR reads
// columns).
__global__ void transpose_rm_to_cm_kernel(const double* __restrict__ Y, int64_t ldy, int64_t m,
                                          int64_t c, double* __restrict__ W, int64_t ldw) {
  __shared__ double t[32][33];
  const int64_t r0 = (int64_t)blockIdx.x * 32, c0 = (int64_t)blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 256 threads: 8 rows per pass
  for (int i = ty; i < 32; i += 8) {
    const int64_t r = r0 + i, cc = c0 + tx;
    t[i][tx] = (r < m && cc < c) ? Y[r * ldy + cc] : 0.0;
  }
  __syncthreads();
  for (int j = ty; j < 32; j += 8) {
    const int64_t cc = c0 + j, r = r0 + tx;
    if (r < m && cc < c) W[r + cc * ldw] = t[tx][j];
  }
}

// ---------------------------------------------------------------------------
// Randomized Cholesky QR (Algorithms 4 and 5).  Shared front: Y = S A (the
// multisketch of A alone), R0 from its Householder QR, the explicit R0^{-1}.
struct RcqFront {
  double* Z;    // p x n: R0 in its upper n x n
  double* Ri0;  // n x n: R0^{-1}
};

static size_t rcq_front_workspace(int64_t d, int64_t n, int64_t k, int64_t p, int dtype,
                                  int gemm_prec) {
  Need nd;
  nd.add(msk_ms_workspace(d, n, 0, k, p, dtype, gemm_prec, MSK_CS_ATOMIC));
  nd.add((size_t)p * n * sizeof(double));  // Z
  nd.add((size_t)n * n * sizeof(double));  // R0^{-1}
  return nd.used;
}

// Returns MSK_OK, an error, or j+1 when R0[j][j] == 0 (synchronises then).
static int rcq_front(const void* A, int dtype, int64_t d, int64_t n, int64_t lda, int64_t k,
                     int64_t p, uint64_t seed, int gemm_prec, Carve& cv, RcqFront* f,
                     void* stream) {
  cudaStream_t st = as_stream(stream);
  const size_t ms_ws = msk_ms_workspace(d, n, 0, k, p, dtype, gemm_prec, MSK_CS_ATOMIC);
  void* msw = cv.take(ms_ws);
  f->Z = static_cast<double*>(cv.take((size_t)p * n * sizeof(double)));
  f->Ri0 = static_cast<double*>(cv.take((size_t)n * n * sizeof(double)));
  if (!f->Z || !f->Ri0) return MSK_ENOMEM;
  // 1. Y = S A (Z = G C A)
  int rc = ms_sketch(A, dtype, d, n, lda, nullptr, k, p, seed, gemm_prec, f->Z, p, MSK_CS_ATOMIC,
                     msw, ms_ws, stream);
  if (rc) return rc;
  // 2. R0 = R of qr(Y, 0)
  rc = launch_householder_qr(f->Z, p, n, p, st);
  if (rc) return rc;
  const int piv = first_zero_pivot(f->Z, n, p, st);
  if (piv) return piv;
  // 3. (Q0 = A R0^{-1} through) the explicit inverse
  tri_inverse_kernel<<<(unsigned)std::max<int64_t>(1, (n + 7) / 8), 256, 0, st>>>(f->Z, (int)n, p,
                                                                                 f->Ri0);
  MSK_CHECK_LAUNCH("tri_inverse_kernel");
  return MSK_OK;
}

// C (ncol x ncol, ld ncol) = X^T X for X = [Q0[:, 0:m] col] (m + 1 columns).
static size_t rcq_gram_workspace(int64_t d, int64_t m) {
  return gram_workspace(d, m) + (size_t)(m + 1) * (m + 1) * sizeof(double) + 256;
}
static int rcq_gram(const double* Q0, int64_t ldq, int64_t d, int64_t m, const double* col,
                    Carve& cv, double** Cout, cudaStream_t st) {
  GramPlan g = gram_plan(d, m);
  const int64_t ncol = m + 1;
  int2* tiles = static_cast<int2*>(cv.take((size_t)std::max(g.npairs, 1) * sizeof(int2)));
  double* part = static_cast<double*>(cv.take((size_t)g.parts * ncol * ncol * sizeof(double)));
  double* C = static_cast<double*>(cv.take((size_t)ncol * ncol * sizeof(double)));
  if (!tiles || !part || !C) return MSK_ENOMEM;
  int rc = launch_gram(g, Q0, ldq, d, m, col, tiles, part, st);
  if (rc) return rc;
  launch_gram_reduce(part, g.parts, ncol, C, st);
  MSK_CHECK_LAUNCH("gram_reduce_kernel");
  *Cout = C;
  return MSK_OK;
}

static int rcq_args(const void* A, int dtype, int64_t d, int64_t n, int64_t lda, int64_t k,
                    int64_t p, int gemm_prec) {
  if (!A) return -1;
  if (dtype != MSK_F64 && dtype != MSK_F32) return -2;
  if (d < n) return -3;
  if (n < 1 || n > 400) return -4;
  if (lda < d) return -5;
  if (k < n + 1) return -7;
  if (p < n + 1 || p > k || p > 2048) return -8;
  if (gemm_prec < MSK_GEMM_F64 || gemm_prec > MSK_GEMM_BF16X3) return -10;
  if (is_tensor_prec_l(gemm_prec) && dtype != MSK_F32) return MSK_ENOTSUP;
  return MSK_OK;
}

// Fill x with NaN (a failed factorisation), then report status.
static int rcq_fail(double* x, int64_t n, int status, cudaStream_t st) {
  std::vector<double> nanv((size_t)n, std::nan(""));
  MSK_CUDA(cudaMemcpyAsync(x, nanv.data(), (size_t)n * sizeof(double), cudaMemcpyHostToDevice, st));
  MSK_CUDA(cudaStreamSynchronize(st));
  return status;
}

}  // namespace

extern "C" {

size_t msk_lstsq_workspace(int64_t d, int64_t n, int64_t k, int64_t p, int dtype, int gemm_prec,
                           int refine) {
  Need nd;
  nd.add(msk_ms_workspace(d, n, 1, k, p, dtype, gemm_prec, MSK_CS_ATOMIC));
  nd.add((size_t)p * (n + 1) * sizeof(double));  // Z
  nd.add(pass_workspace(d, n));                     // pass partials
  nd.add((size_t)pass_out_len(n) * sizeof(double));         // pass result
  if (refine) {
    nd.add((size_t)n * n * sizeof(double));  // R^{-1}
    nd.add((size_t)5 * n * sizeof(double));  // dlt, p, res, z, g copy
    nd.add(64);                              // scalars
  }
  return nd.used;
}

int ms_lstsq(const void* A, int dtype, int64_t d, int64_t n, int64_t lda, const double* b,
             int64_t k, int64_t p, uint64_t seed, int gemm_prec, int refine, double tol,
             int32_t max_iter, double* x, msk_lstsq_info* info, void* ws, size_t ws_bytes,
             void* stream) {
  StageRange nvtx_range_("ms_lstsq");
  if (!A) return -1;
  if (dtype != MSK_F64 && dtype != MSK_F32) return -2;
  if (d < n) return -3;
  if (n < 1 || n > 400) return -4;
  if (lda < d) return -5;
  if (!b) return -6;
  if (k < n + 1) return -7;
  if (p < n + 1 || p > k || p > 2048) return -8;
  if (gemm_prec < MSK_GEMM_F64 || gemm_prec > MSK_GEMM_BF16X3) return -10;
  if (refine != 0 && refine != 1) return -11;
  if (!x) return -14;
  if (ws_bytes < msk_lstsq_workspace(d, n, k, p, dtype, gemm_prec, refine)) return MSK_ENOMEM;
  if (is_tensor_prec_l(gemm_prec) && dtype != MSK_F32) return MSK_ENOTSUP;
  cudaStream_t st = as_stream(stream);
  Carve cv(ws, ws_bytes);
  const size_t ms_ws = msk_ms_workspace(d, n, 1, k, p, dtype, gemm_prec, MSK_CS_ATOMIC);
  void* msw = cv.take(ms_ws);
  double* Z = static_cast<double*>(cv.take((size_t)p * (n + 1) * sizeof(double)));
  double* part = static_cast<double*>(cv.take(pass_workspace(d, n)));
  double* pout = static_cast<double*>(cv.take((size_t)pass_out_len(n) * sizeof(double)));
  if (!Z || !part || !pout) return MSK_ENOMEM;
  // 1. Z = G S [A b]
  int rc = ms_sketch(A, dtype, d, n, lda, b, k, p, seed, gemm_prec, Z, p, MSK_CS_ATOMIC, msw, ms_ws,
                     stream);
  if (rc) return rc;
  // 2. Householder QR of Z (in place): R = Z[0:n+1, 0:n+1]
  rc = launch_householder_qr(Z, p, n + 1, p, st);
  if (rc) return rc;
  // 3. x0 = R11^{-1} R[0:n, n]: a triangular solve, or with refinement the
  //    product with the explicit inverse formed for the preconditioner
  if (!refine) {
    rc = launch_trsv_upper(Z, n, p, Z + n * p, x, nullptr, false, st);
    if (rc) return rc;
  }
  double relres_sns = -1.0, relres = -1.0, bnorm2 = 0.0;
  int iters = 0, converged = 1, inner_total = 0;
  int status = MSK_OK;
  if (refine) {
    double* Ri = static_cast<double*>(cv.take((size_t)n * n * sizeof(double)));
    double* vec = static_cast<double*>(cv.take((size_t)5 * n * sizeof(double)));
    double* sc = static_cast<double*>(cv.take(kScCount * sizeof(double)));
    if (!Ri || !vec || !sc) return MSK_ENOMEM;
    RefState s{x, vec, vec + n, vec + 2 * n, vec + 3 * n, sc};
    double* gsave = vec + 4 * n;
    tri_inverse_kernel<<<(unsigned)std::max<int64_t>(1, (n + 7) / 8), 256, 0, st>>>(Z, (int)n, p, Ri);
    MSK_CHECK_LAUNCH("tri_inverse_kernel");
    x0_kernel<<<1, 512, 0, st>>>(Ri, (int)n, Z + n * p, x);
    MSK_CHECK_LAUNCH("x0_kernel");
    converged = 0;
    // FP64 true residual pass: pout = [A^T r, ||r||^2, ||b||^2]; rr = ||r||^2
    double rr = 0.0;
    auto residual = [&]() -> int {
      int e = launch_pass(A, dtype, lda, d, (int)n, b, x, true, part, pout, nullptr, st);
      if (e) return e;
      double h[2];
      MSK_CUDA(cudaMemcpyAsync(h, pout + n, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
      MSK_CUDA(cudaStreamSynchronize(st));
      rr = std::max(h[0], 0.0);
      bnorm2 = h[1];
      relres = std::sqrt(rr / (bnorm2 > 0.0 ? bnorm2 : 1.0));
      return MSK_OK;
    };
    rc = residual();
    if (rc) return rc;
    relres_sns = relres;
    for (int outer = 0; outer < max_iter; ++outer) {
      // Inner PCG on A^T A d = g (double-single passes for FP32 A).  Each CG
      // step lowers ||b - A x||^2 by alpha*rho; the solve ends once a step
      // gains no more than kDecFrac * tol * ||r||^2 (the geometric tail is then
      // below ~2x that).  Iterations are queued kInnerRound at a time; the
      // kernels of a stopped solve return at once.
      MSK_CUDA(cudaMemcpyAsync(gsave, pout, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
      pcg_start_kernel<<<1, 512, 0, st>>>(Ri, (int)n, gsave, s, kDecFrac * tol * rr);
      MSK_CHECK_LAUNCH("pcg_start_kernel");
      double active = 1.0;
      cudaLaunchConfig_t ucfg = {};
      ucfg.gridDim = dim3(kUpdCL, 1, 1);
      ucfg.blockDim = dim3(kUpdThreads, 1, 1);
      ucfg.stream = st;
      cudaLaunchAttribute uat[1];
      uat[0].id = cudaLaunchAttributeClusterDimension;
      uat[0].val.clusterDim.x = kUpdCL;
      uat[0].val.clusterDim.y = 1;
      uat[0].val.clusterDim.z = 1;
      ucfg.attrs = uat;
      ucfg.numAttrs = 1;
      for (int queued = 0; active != 0.0 && queued < kMaxInner; queued += kInnerRound) {
        for (int r = 0; r < kInnerRound; ++r) {
          int nparts = 0;
          rc = launch_pass(A, dtype, lda, d, (int)n, nullptr, s.p, false, part, nullptr, sc + 2, st,
                           &nparts, pout + n + 2);
          if (rc) return rc;
          MSK_CUDA(cudaLaunchKernelEx(&ucfg, pcg_cluster_kernel, (const double*)part, nparts,
                                      (int)n + 2, (const double*)Ri, (int)n, s, (int)kMaxInner));
        }
        MSK_CUDA(cudaMemcpyAsync(&active, sc + 2, sizeof(double), cudaMemcpyDeviceToHost, st));
        MSK_CUDA(cudaStreamSynchronize(st));
      }
      double h[kScCount];
      MSK_CUDA(cudaMemcpyAsync(h, sc, sizeof(h), cudaMemcpyDeviceToHost, st));
      MSK_CUDA(cudaStreamSynchronize(st));
      inner_total += (int)h[4];
      // every convergence test below is trusted only while the inner
      // iterations stay within kStallIters * n; beyond that the solve stops
      // unconverged when a test fires
      const bool trusted = inner_total <= kStallIters * n;
      if (h[5] != 0.0) {
        // even the first step gains no more than the floor: x is the
        // minimiser to within tol; keep it (relres is its FP64 residual)
        converged = trusted ? 1 : 0;
        break;
      }
      axpy_kernel<<<1, 512, 0, st>>>((int)n, s.dlt, x);
      MSK_CHECK_LAUNCH("axpy_kernel");
      const double rr_prev = rr, relres_prev = relres;
      rc = residual();
      if (rc) return rc;
      // Converged when the solve ended by its gain rule and the true FP64
      // residual confirms the decrease the CG recurrences predicted (no loss
      // to the inner arithmetic), or when the relative residual no longer
      // moves by more than tol, in either case while the inner iterations
      // so far stay within kStallIters * n.  After more, the preconditioner
      // is too poor to trust either test: stop, unconverged.
      const double predicted = rr_prev - h[6];
      if ((h[7] != 0.0 && std::fabs(rr - predicted) <= tol * rr) ||
          std::fabs(relres_prev - relres) <= tol * relres) {
        converged = trusted ? 1 : 0;
        break;
      }
    }
    iters = inner_total;
    if (!converged) status = MSK_ENOCONV;
  } else if (info) {
    rc = launch_pass(A, dtype, lda, d, (int)n, b, x, true, part, pout, nullptr, st);
    if (rc) return rc;
    double host[2];
    MSK_CUDA(cudaMemcpyAsync(host, pout + n, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    MSK_CUDA(cudaStreamSynchronize(st));
    relres = std::sqrt(std::max(host[0], 0.0) / (host[1] > 0.0 ? host[1] : 1.0));
    relres_sns = relres;
  }
  if (info) {
    const int piv = first_zero_pivot(Z, n, p, st);
    if (piv > 0 && piv < 1000) status = piv;
    info->iters = iters;
    info->converged = converged;
    info->relres = relres;
    info->relres_sns = relres_sns;
  }
  return status;
}

size_t msk_sns_workspace(int64_t d, int64_t n, int kind, int64_t k, int64_t p, int dtype) {
  if (kind == MSK_SKETCH_MULTI) return msk_lstsq_workspace(d, n, k, p, dtype, MSK_GEMM_F64, 0);
  const int64_t ncol = n + 1;
  Need nd;
  if (kind == MSK_SKETCH_COUNT || kind == MSK_SKETCH_SRHT) {
    nd.add((size_t)k * ((ncol + 1) / 2 * 2) * sizeof(double));  // Y, row-major
    nd.add((size_t)k * ncol * sizeof(double));                  // W, column-major
    if (kind == MSK_SKETCH_SRHT) nd.add(srht_workspace(d, ncol, k));
  } else {
    nd.add((size_t)p * ncol * sizeof(double));  // Z
    nd.add(gauss_gemm_workspace(p, d, ncol));
  }
  nd.add(pass_workspace(d, n));
  nd.add((size_t)pass_out_len(n) * sizeof(double));
  return nd.used;
}

int sns_lstsq(const void* A, int dtype, int64_t d, int64_t n, int64_t lda, const double* b,
              int kind, int64_t k, int64_t p, uint64_t seed, double* x, msk_lstsq_info* info,
              void* ws, size_t ws_bytes, void* stream) {
  StageRange nvtx_range_("sns_lstsq");
  if (kind == MSK_SKETCH_MULTI)
    return ms_lstsq(A, dtype, d, n, lda, b, k, p, seed, MSK_GEMM_F64, 0, 0.0, 0, x, info, ws,
                    ws_bytes, stream);
  if (!A) return -1;
  if (dtype != MSK_F64 && dtype != MSK_F32) return -2;
  if (d < n) return -3;
  if (n < 1 || n > 400) return -4;
  if (lda < d) return -5;
  if (!b) return -6;
  if (kind != MSK_SKETCH_COUNT && kind != MSK_SKETCH_GAUSS && kind != MSK_SKETCH_SRHT) return -7;
  // the QR of the k x (n+1) sketch indexes rows in 32 bits
  if ((kind == MSK_SKETCH_COUNT || kind == MSK_SKETCH_SRHT) && (k < n + 1 || k > 0x7FFFFFFFLL))
    return -8;
  if (kind == MSK_SKETCH_SRHT && (d < 2 || (d & (d - 1)) != 0 || d > (int64_t(1) << 26)))
    return MSK_ENOTSUP;
  if (kind == MSK_SKETCH_GAUSS && (p < n + 1 || p > 2048)) return -9;
  if (!x) return -11;
  if (ws_bytes < msk_sns_workspace(d, n, kind, k, p, dtype)) return MSK_ENOMEM;
  cudaStream_t st = as_stream(stream);
  Carve cv(ws, ws_bytes);
  const int64_t ncol = n + 1;
  double* W;  // the sketched [SA Sb], column-major m x ncol
  int64_t m;
  int rc;
  if (kind == MSK_SKETCH_COUNT || kind == MSK_SKETCH_SRHT) {
    // S = C: the k x (n+1) CountSketch itself (Definition 3), FP64; or the
    // SRHT (Section 5)
    const int64_t ldy = (ncol + 1) / 2 * 2;
    double* Y = static_cast<double*>(cv.take((size_t)k * ldy * sizeof(double)));
    W = static_cast<double*>(cv.take((size_t)k * ncol * sizeof(double)));
    if (!Y || !W) return MSK_ENOMEM;
    if (kind == MSK_SKETCH_COUNT) {
      rc = count_sketch_f64y(A, dtype, d, n, lda, b, k, seed, Y, ldy, st);
    } else {
      const size_t sws = srht_workspace(d, ncol, k);
      void* sw = cv.take(sws);
      if (!sw) return MSK_ENOMEM;
      rc = launch_srht(A, dtype, d, n, lda, b, k, seed, Y, ldy, sw, sws, st);
    }
    if (rc) return rc;
    dim3 grid((unsigned)((k + 31) / 32), (unsigned)((ncol + 31) / 32));
    transpose_rm_to_cm_kernel<<<grid, 256, 0, st>>>(Y, ldy, k, ncol, W, k);
    MSK_CHECK_LAUNCH("transpose_rm_to_cm_kernel");
    m = k;
  } else {
    // S = G: the p x d Gaussian sketch (Section 1), generated inside the product
    W = static_cast<double*>(cv.take((size_t)p * ncol * sizeof(double)));
    const size_t gws = gauss_gemm_workspace(p, d, ncol);
    void* gw = cv.take(gws);
    if (!W || !gw) return MSK_ENOMEM;
    rc = launch_gauss_gemm(stream_key(seed, kTagGauss), p, A, dtype, d, n, lda, b, W, p, gw, gws,
                           st);
    if (rc) return rc;
    m = p;
  }
  double* part = static_cast<double*>(cv.take(pass_workspace(d, n)));
  double* pout = static_cast<double*>(cv.take((size_t)pass_out_len(n) * sizeof(double)));
  if (!part || !pout) return MSK_ENOMEM;
  // Algorithm 1 steps 2-3: Householder QR of the sketched [A b], then TRSV
  rc = launch_householder_qr(W, m, ncol, m, st);
  if (rc) return rc;
  rc = launch_trsv_upper(W, n, m, W + n * m, x, nullptr, false, st);
  if (rc) return rc;
  int status = MSK_OK;
  if (info) {
    rc = launch_pass(A, dtype, lda, d, (int)n, b, x, true, part, pout, nullptr, st);
    if (rc) return rc;
    double h[2];
    MSK_CUDA(cudaMemcpyAsync(h, pout + n, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    MSK_CUDA(cudaStreamSynchronize(st));
    info->iters = 0;
    info->converged = 1;
    info->relres = std::sqrt(std::max(h[0], 0.0) / (h[1] > 0.0 ? h[1] : 1.0));
    info->relres_sns = info->relres;
    const int piv = first_zero_pivot(W, n, m, st);
    if (piv > 0) status = piv;
  }
  return status;
}

size_t msk_rcq_workspace(int64_t d, int64_t n, int64_t k, int64_t p, int dtype, int gemm_prec,
                         int want_q) {
  Need nd;
  nd.add(rcq_front_workspace(d, n, k, p, dtype, gemm_prec));
  nd.add((size_t)n * n * sizeof(double));  // R1
  nd.add(64);                              // status
  if (want_q) {
    nd.add(rcq_gram_workspace(d, n - 1));    // Gram of Q0
    nd.add((size_t)n * n * sizeof(double));  // R1^{-1}
  } else {
    nd.add((size_t)d * n * sizeof(double));  // Q0
    nd.add(rcq_gram_workspace(d, n));        // Gram of [Q0 b]
    nd.add((size_t)n * n * sizeof(double));  // R
    nd.add((size_t)n * sizeof(double));      // y
    nd.add(pass_workspace(d, n));            // residual pass partials
    nd.add((size_t)pass_out_len(n) * sizeof(double));
  }
  return nd.used;
}

int rcq_lstsq(const void* A, int dtype, int64_t d, int64_t n, int64_t lda, const double* b,
              int64_t k, int64_t p, uint64_t seed, int gemm_prec, double* x, msk_lstsq_info* info,
              void* ws, size_t ws_bytes, void* stream) {
  StageRange nvtx_range_("rcq_lstsq");
  int rc = rcq_args(A, dtype, d, n, lda, k, p, gemm_prec);
  if (rc) return rc;
  if (!b) return -6;
  if (!x) return -11;
  if (ws_bytes < msk_rcq_workspace(d, n, k, p, dtype, gemm_prec, 0)) return MSK_ENOMEM;
  cudaStream_t st = as_stream(stream);
  Carve cv(ws, ws_bytes);
  RcqFront f;
  rc = rcq_front(A, dtype, d, n, lda, k, p, seed, gemm_prec, cv, &f, stream);
  if (rc > 0 && rc < 1000) return rcq_fail(x, n, rc, st);
  if (rc) return rc;
  double* R1 = static_cast<double*>(cv.take((size_t)n * n * sizeof(double)));
  int* status = static_cast<int*>(cv.take(64));
  double* Q0 = static_cast<double*>(cv.take((size_t)d * n * sizeof(double)));
  if (!R1 || !status || !Q0) return MSK_ENOMEM;
  // Q0 = A R0^{-1}
  rc = launch_trmm_upper(A, dtype, lda, d, n, f.Ri0, Q0, d, st);
  if (rc) return rc;
  // G = Q0^T Q0 and z = Q0^T b: the Gram of [Q0 b] (C[0:n, n] = z)
  double* C = nullptr;
  rc = rcq_gram(Q0, d, d, n, b, cv, &C, st);
  if (rc) return rc;
  double* R = static_cast<double*>(cv.take((size_t)n * n * sizeof(double)));
  double* y = static_cast<double*>(cv.take((size_t)n * sizeof(double)));
  double* part = static_cast<double*>(cv.take(pass_workspace(d, n)));
  double* pout = static_cast<double*>(cv.take((size_t)pass_out_len(n) * sizeof(double)));
  if (!R || !y || !part || !pout) return MSK_ENOMEM;
  const int64_t ncol = n + 1;
  MSK_CUDA(cudaMemsetAsync(status, 0, sizeof(int), st));
  // R1 = chol(G); R = R1 R0; y = R1^{-T} z; x = R^{-1} y
  rc = launch_cholesky(C, n, ncol, R1, n, status, st);
  if (rc) return rc;
  rc = launch_tri_mul_upper(R1, n, f.Z, p, n, R, n, st);
  if (rc) return rc;
  rc = launch_trsv_upper(R1, n, n, C + n * ncol, y, nullptr, true, st);
  if (rc) return rc;
  rc = launch_trsv_upper(R, n, n, y, x, nullptr, false, st);
  if (rc) return rc;
  int hs = 0;
  MSK_CUDA(cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st));
  MSK_CUDA(cudaStreamSynchronize(st));
  if (hs > 0) return rcq_fail(x, n, hs, st);
  if (info) {
    rc = launch_pass(A, dtype, lda, d, (int)n, b, x, true, part, pout, nullptr, st);
    if (rc) return rc;
    double h[2];
    MSK_CUDA(cudaMemcpyAsync(h, pout + n, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    MSK_CUDA(cudaStreamSynchronize(st));
    info->iters = 0;
    info->converged = 1;
    info->relres = std::sqrt(std::max(h[0], 0.0) / (h[1] > 0.0 ? h[1] : 1.0));
    info->relres_sns = -1.0;
  }
  return MSK_OK;
}

int rcq_qr(const void* A, int dtype, int64_t d, int64_t n, int64_t lda, int64_t k, int64_t p,
           uint64_t seed, int gemm_prec, double* Q, int64_t ldq, double* R, int64_t ldr, void* ws,
           size_t ws_bytes, void* stream) {
  StageRange nvtx_range_("rcq_qr");
  int rc = rcq_args(A, dtype, d, n, lda, k, p, gemm_prec);
  if (rc) return rc;
  if (!Q) return -10;
  if (ldq < d) return -11;
  if (!R) return -12;
  if (ldr < n) return -13;
  if (ws_bytes < msk_rcq_workspace(d, n, k, p, dtype, gemm_prec, 1)) return MSK_ENOMEM;
  cudaStream_t st = as_stream(stream);
  Carve cv(ws, ws_bytes);
  RcqFront f;
  rc = rcq_front(A, dtype, d, n, lda, k, p, seed, gemm_prec, cv, &f, stream);
  if (rc) return rc;
  double* R1 = static_cast<double*>(cv.take((size_t)n * n * sizeof(double)));
  int* status = static_cast<int*>(cv.take(64));
  if (!R1 || !status) return MSK_ENOMEM;
  // Q0 = A R0^{-1}, into Q
  rc = launch_trmm_upper(A, dtype, lda, d, n, f.Ri0, Q, ldq, st);
  if (rc) return rc;
  // G = Q0^T Q0: the Gram of [Q0[:, 0:n-1] Q0[:, n-1]]
  double* C = nullptr;
  rc = rcq_gram(Q, ldq, d, n - 1, Q + (n - 1) * ldq, cv, &C, st);
  if (rc) return rc;
  double* Ri1 = static_cast<double*>(cv.take((size_t)n * n * sizeof(double)));
  if (!Ri1) return MSK_ENOMEM;
  MSK_CUDA(cudaMemsetAsync(status, 0, sizeof(int), st));
  rc = launch_cholesky(C, n, n, R1, n, status, st);
  if (rc) return rc;
  int hs = 0;
  MSK_CUDA(cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st));
  MSK_CUDA(cudaStreamSynchronize(st));
  if (hs > 0) return hs;
  // Q = Q0 R1^{-1} (in place), R = R1 R0
  tri_inverse_kernel<<<(unsigned)std::max<int64_t>(1, (n + 7) / 8), 256, 0, st>>>(R1, (int)n, n, Ri1);
  MSK_CHECK_LAUNCH("tri_inverse_kernel");
  rc = launch_trmm_upper(Q, MSK_F64, ldq, d, n, Ri1, Q, ldq, st);
  if (rc) return rc;
  rc = launch_tri_mul_upper(R1, n, f.Z, p, n, R, ldr, st);
  if (rc) return rc;
  MSK_CUDA(cudaStreamSynchronize(st));
  return MSK_OK;
}

size_t msk_ne_workspace(int64_t d, int64_t n) {
  Need nd;
  nd.add(gram_workspace(d, n));
  nd.add((size_t)(n + 1) * (n + 1) * sizeof(double));  // C = [A b]^T [A b]
  nd.add((size_t)n * n * sizeof(double));              // R
  nd.add((size_t)n * sizeof(double));                  // y
  nd.add(64);                                          // status
  return nd.used;
}

int ne_lstsq(const double* A, int64_t d, int64_t n, int64_t lda, const double* b, double* x,
             void* ws, size_t ws_bytes, void* stream) {
  StageRange nvtx_range_("ne_lstsq");
  if (!A) return -1;
  if (d < n) return -2;
  if (n < 1 || n > 4096) return -3;
  if (lda < d) return -4;
  if (!b) return -5;
  if (!x) return -6;
  if (ws_bytes < msk_ne_workspace(d, n)) return MSK_ENOMEM;
  cudaStream_t st = as_stream(stream);
  Carve cv(ws, ws_bytes);
  GramPlan g = gram_plan(d, n);
  const int64_t ncol = n + 1;
  int2* tiles = static_cast<int2*>(cv.take((size_t)std::max(g.npairs, 1) * sizeof(int2)));
  double* part = static_cast<double*>(cv.take((size_t)g.parts * ncol * ncol * sizeof(double)));
  double* C = static_cast<double*>(cv.take((size_t)ncol * ncol * sizeof(double)));
  double* R = static_cast<double*>(cv.take((size_t)n * n * sizeof(double)));
  double* y = static_cast<double*>(cv.take((size_t)n * sizeof(double)));
  int* status = static_cast<int*>(cv.take(64));
  if (!tiles || !part || !C || !R || !y || !status) return MSK_ENOMEM;
  MSK_CUDA(cudaMemsetAsync(status, 0, sizeof(int), st));
  {
    const int rc = launch_gram(g, A, lda, d, n, b, tiles, part, st);
    if (rc) return rc;
  }
  launch_gram_reduce(part, g.parts, ncol, C, st);
  MSK_CHECK_LAUNCH("gram_reduce_kernel");
  // C[0:n,0:n] = A^T A, C[0:n, n] = A^T b.  Cholesky overwrites C's upper part.
  int rc = launch_cholesky(C, n, ncol, R, n, status, st);
  if (rc) return rc;
  rc = launch_trsv_upper(R, n, n, C + n * ncol, y, nullptr, true, st);  // R^T y = A^T b
  if (rc) return rc;
  rc = launch_trsv_upper(R, n, n, y, x, nullptr, false, st);            // R x = y
  if (rc) return rc;
  int hs = 0;
  MSK_CUDA(cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st));
  MSK_CUDA(cudaStreamSynchronize(st));
  if (hs > 0) {
    // x is meaningless after a failed factorisation: make that visible
    std::vector<double> nanv((size_t)n, std::nan(""));
    MSK_CUDA(cudaMemcpyAsync(x, nanv.data(), (size_t)n * sizeof(double), cudaMemcpyHostToDevice, st));
    MSK_CUDA(cudaStreamSynchronize(st));
    return hs;
  }
  return MSK_OK;
}

size_t msk_normal_apply_workspace(int64_t d, int64_t n) {
  if (d < 1 || n < 1 || n > 2 * kP32Threads) return 0;
  Need nd;
  nd.add((size_t)d * sizeof(double));                  // b = 0 of the residual pass
  nd.add((size_t)n * sizeof(double));                  // x = 0
  nd.add(pass_workspace(d, n));                        // pass partials
  nd.add((size_t)pass_out_len(n) * sizeof(double));    // residual-pass result (column maxima)
  nd.add((size_t)(n + 2) * sizeof(double));            // operator-pass result
  return nd.used;
}

int msk_normal_apply(const float* A, int64_t d, int64_t n, int64_t lda, const double* p, double* v,
                     void* ws, size_t ws_bytes, void* stream) {
  StageRange nvtx_range_("msk_normal_apply");
  if (!A || !p || !v) return -1;
  if (d < 1) return -2;
  if (n < 1 || n > 2 * kP32Threads) return -3;
  if (lda < d) return -4;
  if (ws_bytes < msk_normal_apply_workspace(d, n)) return MSK_ENOMEM;
  cudaStream_t st = as_stream(stream);
  Carve cv(ws, ws_bytes);
  double* b0 = static_cast<double*>(cv.take((size_t)d * sizeof(double)));
  double* x0 = static_cast<double*>(cv.take((size_t)n * sizeof(double)));
  double* part = static_cast<double*>(cv.take(pass_workspace(d, n)));
  double* pout = static_cast<double*>(cv.take((size_t)pass_out_len(n) * sizeof(double)));
  double* vout = static_cast<double*>(cv.take((size_t)(n + 2) * sizeof(double)));
  if (!b0 || !x0 || !part || !pout || !vout) return MSK_ENOMEM;
  MSK_CUDA(cudaMemsetAsync(b0, 0, (size_t)d * sizeof(double), st));
  MSK_CUDA(cudaMemsetAsync(x0, 0, (size_t)n * sizeof(double), st));
  int rc = launch_pass(A, MSK_F32, lda, d, (int)n, b0, x0, true, part, pout, nullptr, st);
  if (rc) return rc;
  rc = launch_pass(A, MSK_F32, lda, d, (int)n, nullptr, p, false, part, vout, nullptr, st, nullptr,
                   pout + n + 2);
  if (rc) return rc;
  MSK_CUDA(cudaMemcpyAsync(v, vout, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  return MSK_OK;
}

}  // extern "C"

