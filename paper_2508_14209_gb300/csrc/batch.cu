// batch.cu — many least-squares solves of uneven sizes in one set of launches
// (msk_batch_lstsq), the engine under the request server.
//
// Path per problem (the mixed-precision multisketch of the configurations):
// FP32 CountSketch of [A b] to k = 2n^2 rows (Section 6.2), Gaussian stage to
// p = 4n rows as split-BF16 products on the tensor cores with draining FP32
// accumulators, FP64 Householder QR and triangular solve (Algorithm 1), then
// sketch-and-precondition refinement (FP64 residual passes, double-single CG
// passes).  Every stage is ONE launch over all problems of the batch:
//   CountSketch   one persistent launch per width class (tiles of all problems
//                 numbered consecutively);
//   Gaussian, split, GEMM, split-K reduction: one launch each, per-problem
//                 descriptors (the GEMM reads its tensor maps from global
//                 memory);
//   QR (+ solve)  one launch, one thread-block cluster per problem; with
//                 refinement, x0 = R^{-1} c after the explicit inverse;
//   refinement    an FP64 residual pass, then an outer loop on the device: CG
//                 start, an inner loop of kRound (knob "batch.round") CG
//                 iterations per trip (a pass per width class, then the CG
//                 step fused with the partials' reduction on one 8-CTA
//                 cluster per problem) until every problem has met its
//                 stopping rule, x += d, the FP64 residual of the corrected
//                 problems and the convergence tests, until every problem has
//                 converged or max_iter outer steps are done.
// The whole chain is ONE CUDA-graph launch: the straight segments are
// captured, the two loops are while nodes (the inner one nested in the outer
// one's body) whose conditions kernels set on the device, so the host waits
// once, for the results.  Instantiated graphs are cached per device and host
// thread, keyed by every value their launches bake in.
// Problems that stop early are skipped by the later launches (device flags).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "msk_device.cuh"
#include "msk_internal.h"
#include "msk_pass.cuh"
#include "msk_qr.cuh"
#include "msk_refine.cuh"

namespace msk {

constexpr int kBatchKtPer = 16;   // K tiles per CTA of the batched GEMM (knob "batch.kt_per")
constexpr int kRound = 4;         // CG iterations per captured graph round
constexpr int kBatchMaxInner = 200;
constexpr double kBatchDecFrac = 0.05;

// Per-problem device descriptor (pointers into the caller's workspace).
struct BatchJob {
  const float* A;
  const double* b;
  double* x;
  int64_t d, lda;
  int n, k, p, ncol;
  uint64_t gkey;
  float* Y;
  int ldy;
  uint16_t* G;
  uint16_t* Yt;
  int64_t kpitch;
  int npad;
  double* part;  // GEMM partials (S x p x ncol)
  int S;
  double* Z;     // p x ncol, then R
  // refinement
  double* Ri;
  double* vec;   // dlt, p, res, z, g: 5n
  double* sc;    // [0] rho, [1] gain, [2] active, [3] floor, [4] inner iters, [5] bb, [6] rr0
  double* ppart; // pass partials: nchunks x pass_out_len(n) (inner passes: stride n + 2)
  double* pout;  // reduced pass result: pass_out_len(n) (A^T r, ||r||^2, ||b||^2, column maxima of |A|)
  int nchunks;      // CTAs of this problem in the refinement passes
  int chunk_begin;  // its first CTA in the batch-wide pass grid
  int cw;           // floats per tile copy (pass32_copy_width: 4, 2 or 1)
};

__global__ void batch_zero_kernel(const BatchJob* __restrict__ jobs) {
  const BatchJob& J = jobs[blockIdx.y];
  const int64_t total = (int64_t)J.k * J.ldy;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x)
    J.Y[e] = 0.f;
}

__global__ void batch_gaussian_kernel(const BatchJob* __restrict__ jobs) {
  const BatchJob& J = jobs[blockIdx.y];
  const int64_t total = (int64_t)J.p * J.k;
  const float sqrt_p = __fsqrt_rn((float)J.p);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / J.k, c = e - r * J.k;
    const float g = __fdiv_rn(gauss_std(J.gkey, (uint64_t)e), sqrt_p);
    J.G[r * J.kpitch + c] = __bfloat16_as_ushort(__float2bfloat16_rn(g));
  }
}

// Yt[t][n][kk] = bf16 split of Y[kk][n] (3 parts), 32x32 transposed tiles.
__global__ void batch_split_kernel(const BatchJob* __restrict__ jobs) {
  const BatchJob& J = jobs[blockIdx.z];
  const int64_t k0 = (int64_t)blockIdx.x * 32;
  const int n0 = blockIdx.y * 32;
  if (k0 >= J.k || n0 >= J.npad) return;
  __shared__ float tile[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int r = ty; r < 32; r += 8) {
    const int64_t kk = k0 + r;
    const int n = n0 + tx;
    tile[r][tx] = (kk < J.k && n < J.ncol) ? J.Y[kk * J.ldy + n] : 0.0f;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int n = n0 + r;
    const int64_t kk = k0 + tx;
    if (n >= J.npad || kk >= J.k) continue;
    float y = tile[tx][r];
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      const __nv_bfloat16 h = __float2bfloat16_rn(y);
      J.Yt[((int64_t)t * J.npad + n) * J.kpitch + kk] = __bfloat16_as_ushort(h);
      y = y - __bfloat162float(h);
    }
  }
}

__global__ void batch_gemm_reduce_kernel(const BatchJob* __restrict__ jobs) {
  const BatchJob& J = jobs[blockIdx.y];
  const int64_t total = (int64_t)J.p * J.ncol;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < J.S; ++q) s += J.part[(int64_t)q * total + e];
    const int64_t c = e / J.p, r = e - c * J.p;
    J.Z[r + c * J.p] = s;  // Z column-major p x ncol
  }
}

// One cluster per problem: Householder QR of Z (p x (n+1)), then
// x0 = R11^{-1} R[0:n, n] by the cluster's first CTA.
// QR of every problem's sketch; with solve, also x0 = R11^{-1} R[0:n, n] by
// the cluster's first CTA (the refined path forms x0 = R^{-1} c after the
// explicit inverse instead).
__global__ void __launch_bounds__(kQrThreads) batch_qr_kernel(const BatchJob* __restrict__ jobs,
                                                             size_t smem_cap, int solve, int flow,
                                                             int* tflag) {
  extern __shared__ __align__(16) double bqr_dyn[];
  const BatchJob& J = jobs[blockIdx.y];
  const int CL = (int)cg::this_cluster().num_blocks();
  if (flow && qr_flow_smem_bytes(J.p, J.ncol, CL) <= smem_cap)
    qr_cluster_flow_body(J.Z, J.p, J.ncol, J.p, bqr_dyn, tflag);
  else if (qr_smem_bytes(J.p, J.ncol, CL) <= smem_cap)
    qr_cluster_smem_body(J.Z, J.p, J.ncol, J.p, bqr_dyn);
  else
    qr_cluster_body(J.Z, J.p, J.ncol, J.p);
  if (!solve) return;
  cg::this_cluster().sync();
  if (cg::this_cluster().block_rank() == 0) {
    __shared__ double xs[512];  // n <= 256 in a batch
    trsv_upper_body(J.Z, J.n, J.p, J.Z + (int64_t)J.n * J.p, J.x, nullptr, xs);
  }
}

// x0 = R^{-1} c from the explicit inverse (c = R[0:n, n]).
__global__ void __launch_bounds__(512) batch_x0_kernel(const BatchJob* __restrict__ jobs) {
  __shared__ double scr[512];
  const BatchJob& J = jobs[blockIdx.x];
  tri_matvec_body(J.Ri, J.n, J.Z + (int64_t)J.n * J.p, J.x, scr);
}

__global__ void batch_tri_inverse_kernel(const BatchJob* __restrict__ jobs) {
  const BatchJob& J = jobs[blockIdx.y];
  tri_inverse_body(J.Z, J.n, J.p, J.Ri, blockIdx.x, gridDim.x);
}

// Refinement passes, one launch per width class NC: a 1-D grid over the
// class's problems mem[0..nmem), problem mem[m] owning CTAs
// [chunk_begin, chunk_begin + nchunks) (found by binary search).  RESID passes
// run for the problems with only[j] != 0 (all when only is null); the inner
// passes for the problems whose solve is still active.
template <int NC, bool RESID>
__global__ void __launch_bounds__(kP32Threads, pass32_ctas_per_sm(NC))
    batch_pass_kernel(const BatchJob* __restrict__ jobs, const int* __restrict__ mem, int nmem,
                      const int* __restrict__ only) {
  extern __shared__ __align__(16) unsigned char bp_smem[];
  const int c = blockIdx.x;
  int lo = 0, hi = nmem - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mem[mid]].chunk_begin <= c) lo = mid;
    else hi = mid - 1;
  }
  const int j = mem[lo];
  const BatchJob& J = jobs[j];
  MSK_CHECK_OR(lo >= 0 && lo < nmem && J.chunk_begin <= c, kCheckBatch, return);
  const int lc = c - J.chunk_begin;
  if (lc >= J.nchunks) return;
  if (RESID) {
    if (only && !only[j]) return;
    pass32n_body<NC, true>(J.A, J.lda, J.d, J.n, J.cw, J.b, J.x, nullptr, J.ppart, lc, J.nchunks,
                           bp_smem);
  } else {
    if (J.sc[2] == 0.0) return;  // problem already stopped
    pass32n_body<NC, false>(J.A, J.lda, J.d, J.n, J.cw, nullptr, J.vec + J.n, J.pout + J.n + 2, J.ppart, lc,
                            J.nchunks, bp_smem);
  }
}

// Sum of the residual pass's per-CTA partials (problems with only[j] set).
__global__ void __launch_bounds__(256) batch_pass_reduce_kernel(const BatchJob* __restrict__ jobs,
                                                                const int* __restrict__ only) {
  const BatchJob& J = jobs[blockIdx.y];
  if (only && !only[blockIdx.y]) return;
  if ((int64_t)blockIdx.x * 32 >= pass_out_len(J.n)) return;
  pass_reduce_body(J.ppart, J.nchunks, (int)pass_out_len(J.n), J.n + 2, J.pout, blockIdx.x);
}

__device__ __forceinline__ RefState ref_state(const BatchJob& J) {
  return RefState{J.x, J.vec, J.vec + J.n, J.vec + 2 * J.n, J.vec + 3 * J.n, J.sc};
}

// After an FP64 residual pass: start CG on A^T A d = g for every problem that
// is still refining; its stopping floor is kBatchDecFrac * tol * ||r||^2.
__global__ void batch_pcg_start_kernel(const BatchJob* __restrict__ jobs, double tol,
                                       int* __restrict__ active_count) {
  const BatchJob& J = jobs[blockIdx.x];
  const double rr = J.pout[J.n];
  if (J.sc[2] == 0.0) return;
  double* g = J.vec + 4 * J.n;
  for (int j = threadIdx.x; j < J.n; j += blockDim.x) g[j] = J.pout[j];
  __syncthreads();
  pcg_start_body(J.Ri, J.n, g, ref_state(J));
  __syncthreads();
  if (threadIdx.x == 0) {
    pcg_arm(J.sc, kBatchDecFrac * tol * rr);
    atomicAdd(active_count, 1);
  }
}

// One CG step of every problem, fused with the reduction of its pass
// partials: one kUpdCL-CTA cluster per problem (blockIdx.y).
__global__ void __launch_bounds__(kUpdThreads) batch_pcg_cluster_kernel(const BatchJob* __restrict__ jobs,
                                                                       int* __restrict__ active_count,
                                                                       int* __restrict__ refining) {
  const BatchJob& J = jobs[blockIdx.y];
  if (pcg_cluster_update_body(J.ppart, J.nchunks, J.n + 2, J.Ri, J.n, ref_state(J), kBatchMaxInner)) {
    if (J.sc[5] != 0.0) refining[blockIdx.y] = 0;
    atomicSub(active_count, 1);
  }
}

// x += dlt for the problems that refined in this outer step; re-arm them.
__global__ void batch_axpy_kernel(const BatchJob* __restrict__ jobs, const int* __restrict__ refining) {
  const BatchJob& J = jobs[blockIdx.x];
  if (!refining[blockIdx.x]) return;
  for (int j = threadIdx.x; j < J.n; j += blockDim.x) J.x[j] += J.vec[j];
}

// Doubles per problem in the result buffer copied back to the host.
constexpr int kGather = 6;

// Per-problem state of the refinement loop that runs on the device.
struct BatchCtl {
  double rr, relres, rr_prev, relres_prev, relres_sns, gain;
  int iters, conv, ref, by_rule;
  int stop;  // stalled without the evidence of convergence: no more steps
};

// After the first FP64 residual pass: ||r||^2 and the relative residual of
// the start (the sketch-and-solve x0), counters cleared; with refinement,
// the outer loop's condition: some problem to refine and max_iter > 0.
__global__ void __launch_bounds__(256) batch_ref_init_kernel(const BatchJob* __restrict__ jobs, int nitems,
                                                             BatchCtl* __restrict__ ctl, int refine,
                                                             int max_iter, int* __restrict__ flags,
                                                             cudaGraphConditionalHandle h) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int j = threadIdx.x; j < nitems; j += blockDim.x) {
    const BatchJob& J = jobs[j];
    const double rr = fmax(J.pout[J.n], 0.0), bb = J.pout[J.n + 1];
    BatchCtl& c = ctl[j];
    c.rr = rr;
    c.relres = sqrt(rr / (bb > 0.0 ? bb : 1.0));
    c.relres_sns = c.relres;
    c.rr_prev = rr;
    c.relres_prev = c.relres;
    c.gain = 0.0;
    c.iters = 0;
    c.conv = refine ? 0 : 1;
    c.ref = 0;
    c.by_rule = 0;
    c.stop = 0;
    if (!c.conv) any = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    flags[2] = 0;  // outer steps taken
    if (refine) cudaGraphSetConditional(h, (any && max_iter > 0) ? 1u : 0u);
  }
}

// Top of an outer step: every problem not yet converged refines (CG scalars
// cleared, sc[2] = 1); the device loop's counters cleared.
__global__ void batch_outer_arm_kernel(const BatchJob* __restrict__ jobs, int nitems,
                                       BatchCtl* __restrict__ ctl, int* __restrict__ refining,
                                       int* __restrict__ active) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nitems; j += gridDim.x * blockDim.x) {
    const BatchJob& J = jobs[j];
    BatchCtl& c = ctl[j];
    c.ref = (c.conv || c.stop) ? 0 : 1;
    refining[j] = c.ref;
    for (int q = 0; q < kScCount; ++q) J.sc[q] = 0.0;
    J.sc[2] = c.ref ? 1.0 : 0.0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    active[0] = 0;  // problems still iterating (pcg_start counts them in)
    active[1] = 0;  // CG iterations run by the device loop
  }
}

// Before the inner loop: run it only if some problem started iterating.
__global__ void batch_inner_arm_kernel(cudaGraphConditionalHandle h, const int* __restrict__ active) {
  cudaGraphSetConditional(h, active[0] > 0 ? 1u : 0u);
}

// End of one inner-loop trip: continue while a problem is still iterating,
// and never beyond kBatchMaxInner iterations in all (every problem also stops
// itself at kBatchMaxInner steps).
__global__ void batch_loop_cond_kernel(cudaGraphConditionalHandle h, int* __restrict__ active) {
  const int it = ++active[1];
  cudaGraphSetConditional(h, (active[0] > 0 && it < kBatchMaxInner) ? 1u : 0u);
}

// After the inner solve: count its steps; a problem whose first step already
// gained less than the floor sits at the minimiser (its last relres stands);
// the others get a new FP64 residual (recheck) against the decrease the CG
// recurrences predicted.
__global__ void batch_post_inner_kernel(const BatchJob* __restrict__ jobs, int nitems,
                                        BatchCtl* __restrict__ ctl, int* __restrict__ recheck) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nitems; j += gridDim.x * blockDim.x) {
    BatchCtl& c = ctl[j];
    recheck[j] = 0;
    if (!c.ref) continue;
    const BatchJob& J = jobs[j];
    c.iters += (int)J.sc[4];
    if (J.sc[5] != 0.0) {
      if (c.iters <= kStallIters * J.n) c.conv = 1;
      else c.stop = 1;
    } else {
      recheck[j] = 1;
      c.rr_prev = c.rr;
      c.relres_prev = c.relres;
      c.gain = J.sc[6];
      c.by_rule = J.sc[7] != 0.0 ? 1 : 0;
    }
  }
}

// End of an outer step: the rechecked problems' new residuals; converged
// when the solve ended by its gain rule and the FP64 residual confirms the
// predicted decrease to tol * ||r||^2, or when the relative residual moved
// by at most tol, in either case while the inner iterations so far stay
// within kStallIters * n (after more, a preconditioner too poor to trust
// either test: the problem stops unconverged); then the outer loop's
// condition (some problem left, fewer than max_iter steps taken).
__global__ void __launch_bounds__(256) batch_outer_check_kernel(const BatchJob* __restrict__ jobs,
                                                                int nitems, BatchCtl* __restrict__ ctl,
                                                                const int* __restrict__ recheck, double tol,
                                                                int max_iter, int* __restrict__ flags,
                                                                cudaGraphConditionalHandle h) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int j = threadIdx.x; j < nitems; j += blockDim.x) {
    BatchCtl& c = ctl[j];
    if (recheck[j]) {
      const BatchJob& J = jobs[j];
      const double rr = fmax(J.pout[J.n], 0.0), bb = J.pout[J.n + 1];
      const double relres = sqrt(rr / (bb > 0.0 ? bb : 1.0));
      const double predicted = c.rr_prev - c.gain;
      c.rr = rr;
      c.relres = relres;
      if ((c.by_rule && fabs(rr - predicted) <= tol * rr) || fabs(c.relres_prev - relres) <= tol * relres) {
        if (c.iters <= kStallIters * J.n) c.conv = 1;
        else c.stop = 1;
      }
    }
    if (!c.conv && !c.stop) any = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int outer = ++flags[2];
    cudaGraphSetConditional(h, (any && outer < max_iter) ? 1u : 0u);
  }
}

// out[kGather j + (0..3)] = inner iterations, converged, relres, relres_sns.
__global__ void batch_final_kernel(int nitems, const BatchCtl* __restrict__ ctl, double* __restrict__ out) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nitems; j += gridDim.x * blockDim.x) {
    const BatchCtl& c = ctl[j];
    double* o = out + kGather * j;
    o[0] = (double)c.iters;
    o[1] = (double)c.conv;
    o[2] = c.relres;
    o[3] = c.relres_sns;
  }
}

// Instantiated whole-batch graphs, per device and host thread, keyed by
// every value the capture baked in (pointers into the workspace, grid sizes,
// tolerance, step limits); the problems themselves are read from the
// workspace at run time, so a batch of a shape seen before on the same
// workspace skips capture and instantiation.
struct GraphCache {
  cudaStream_t cap = nullptr;  // private capture stream of this device
  std::vector<std::pair<std::vector<int64_t>, cudaGraphExec_t>> entries;  // most recent last
  ~GraphCache() {
    for (auto& e : entries) cudaGraphExecDestroy(e.second);
  }
};
constexpr size_t kGraphCacheMax = 64;
constexpr int kMaxDevices = 64;

struct BatchPlan {
  std::vector<BatchJob> jobs;
  std::vector<TcJob> tc;
  std::vector<TcShape> shapes;
  std::vector<int> widths;  // CountSketch width classes present
  std::vector<std::vector<CsParams<float>>> cs;
  std::vector<std::vector<int64_t>> cs_tiles;
  std::vector<size_t> cs_off, tiles_off;
  size_t jobs_off = 0, tc_off = 0, flags_off = 0, gather_off = 0, ctl_off = 0;
  int total_items = 0, max_nt = 16, max_npad = 16, max_n = 1;
  // refinement-pass launches, one per width class present
  std::vector<int> pass_nc, pass_chunks;
  std::vector<std::vector<int>> pass_mem;
  std::vector<size_t> pass_mem_off;
  int64_t max_k = 1, max_pk = 1, max_yk = 1;
  size_t bytes = 0;
};

static bool width_ok(int64_t n) {
  return n == 16 || n == 32 || n == 64 || n == 128 || n == 256;
}

// Sizes and places every piece of the batch in the workspace (offsets from
// its base; with base == nullptr only the sizes are computed).
static void plan_batch(const msk_batch_item* items, int nitems, int refine, char* base,
                       BatchPlan* P) {
  Need nd;
  auto take = [&](size_t bytes) -> size_t {
    const size_t off = align_up(nd.used, 256);
    nd.used = off + bytes;
    return off;
  };
  auto ptr = [&](size_t off) -> char* { return base ? base + off : nullptr; };
  P->jobs_off = take(sizeof(BatchJob) * (size_t)nitems);
  P->tc_off = take(sizeof(TcJob) * (size_t)nitems);
  // flags: [0] problems iterating, [1] inner iterations, [2] outer steps,
  // then refining[nitems] and recheck[nitems]
  P->flags_off = take(sizeof(int) * (size_t)(2 * nitems + 8));
  P->gather_off = take(sizeof(double) * kGather * (size_t)nitems);
  P->ctl_off = take(sizeof(BatchCtl) * (size_t)nitems);
  P->jobs.resize(nitems);
  P->tc.resize(nitems);
  P->shapes.resize(nitems);
  const int kt_per = (int)std::min<long long>(64, std::max<long long>(1, tune_get("batch.kt_per", kBatchKtPer)));
  for (int j = 0; j < nitems; ++j) {
    const msk_batch_item& it = items[j];
    BatchJob& J = P->jobs[j];
    J.A = it.A;
    J.b = it.b;
    J.x = it.x;
    J.d = it.d;
    J.lda = it.lda;
    J.n = (int)it.n;
    J.k = (int)(2 * it.n * it.n);
    J.p = (int)(4 * it.n);
    J.ncol = J.n + 1;
    J.gkey = stream_key(it.seed, kTagGauss);
    J.ldy = (J.ncol + 3) / 4 * 4;
    TcShape& sh = P->shapes[j];
    tc_ds_shape(J.p, J.k, J.ncol, kt_per, &sh);
    J.kpitch = sh.kpitch;
    J.npad = sh.npad;
    J.S = sh.S;
    J.Y = reinterpret_cast<float*>(ptr(take((size_t)J.k * J.ldy * 4)));
    J.G = reinterpret_cast<uint16_t*>(ptr(take((size_t)J.p * sh.kpitch * 2)));
    J.Yt = reinterpret_cast<uint16_t*>(ptr(take((size_t)3 * sh.npad * sh.kpitch * 2)));
    J.part = reinterpret_cast<double*>(ptr(take((size_t)sh.S * J.p * J.ncol * 8)));
    J.Z = reinterpret_cast<double*>(ptr(take((size_t)J.p * J.ncol * 8)));
    J.Ri = reinterpret_cast<double*>(ptr(take(refine ? (size_t)J.n * J.n * 8 : 0)));
    J.vec = reinterpret_cast<double*>(ptr(take(refine ? (size_t)5 * J.n * 8 : 0)));
    J.sc = reinterpret_cast<double*>(ptr(take(kScCount * 8)));
    J.pout = reinterpret_cast<double*>(ptr(take((size_t)pass_out_len(J.n) * 8)));
    P->max_nt = std::max(P->max_nt, sh.NT);
    P->max_npad = std::max(P->max_npad, sh.npad);
    P->max_n = std::max(P->max_n, J.n);
    P->max_k = std::max<int64_t>(P->max_k, J.k);
    P->max_pk = std::max<int64_t>(P->max_pk, (int64_t)J.p * J.k);
    P->max_yk = std::max<int64_t>(P->max_yk, (int64_t)J.k * J.ldy);
  }
  // Refinement passes: one launch per width class present, each sized to
  // fill the GPU (pass32_ctas_per_sm CTAs per SM) and shared out among the
  // class's problems in proportion to their row tiles (every CTA then walks
  // about the same number of tiles), at least one CTA per problem.
  for (int nc : {16, 32, 64, 128, 256}) {
    std::vector<int> mem;
    int64_t total_tiles = 0;
    for (int j = 0; j < nitems; ++j)
      if (pass32_class(P->jobs[j].n) == nc) {
        mem.push_back(j);
        total_tiles += (P->jobs[j].d + pass32_rows(nc) - 1) / pass32_rows(nc);
      }
    if (mem.empty()) continue;
    const int64_t per_sm = std::min<long long>(pass32_ctas_per_sm(nc),
                                               std::max<long long>(1, tune_get("pass.ctas_per_sm", 3)));
    const int64_t cap = per_sm * num_sms();
    int begin = 0;
    for (int j : mem) {
      BatchJob& J = P->jobs[j];
      const int64_t tiles = (J.d + pass32_rows(nc) - 1) / pass32_rows(nc);
      const int64_t share = (cap * tiles + total_tiles - 1) / total_tiles;
      J.nchunks = (int)std::max<int64_t>(1, std::min<int64_t>(share, tiles));
      J.chunk_begin = begin;
      begin += J.nchunks;
      J.cw = pass32_copy_width(J.A, J.lda);
      J.ppart = reinterpret_cast<double*>(ptr(take((size_t)J.nchunks * pass_out_len(J.n) * 8)));
    }
    P->pass_nc.push_back(nc);
    P->pass_chunks.push_back(begin);
    P->pass_mem_off.push_back(take(sizeof(int) * mem.size()));
    P->pass_mem.push_back(mem);
  }
  for (int w : {16, 32, 64, 128, 256}) {
    std::vector<CsParams<float>> ps;
    std::vector<int64_t> tb(1, 0);
    for (int j = 0; j < nitems; ++j) {
      const BatchJob& J = P->jobs[j];
      if (J.n != w) continue;
      CsParams<float> c{};
      c.A = J.A;
      c.d = J.d;
      c.lda = J.lda;
      c.ncol_a = J.n;
      c.b = J.b;
      c.ncol = J.ncol;
      c.k = (uint32_t)J.k;
      c.key = stream_key(items[j].seed, kTagHash);
      c.Y = J.Y;
      c.ldy = J.ldy;
      ps.push_back(c);
      tb.push_back(tb.back() + (J.d + 31) / 32);
    }
    if (ps.empty()) continue;
    P->widths.push_back(w);
    P->cs_off.push_back(take(sizeof(CsParams<float>) * ps.size()));
    P->tiles_off.push_back(take(sizeof(int64_t) * tb.size()));
    P->cs.push_back(ps);
    P->cs_tiles.push_back(tb);
  }
  P->bytes = nd.used;
}

}  // namespace msk

using namespace msk;

extern "C" {

size_t msk_batch_workspace(const msk_batch_item* items, int nitems, int refine) {
  if (!items || nitems <= 0) return 0;
  BatchPlan P;
  plan_batch(items, nitems, refine, nullptr, &P);
  return P.bytes;
}

// Every piece plan_batch takes for this item, each with its alignment slack,
// its refinement pass at the most CTAs it can receive, its entries of the
// batch-wide arrays, and 4 KiB towards the per-batch remainder (alignment of
// the five batch arrays, 256 bytes each, and of a width class's three
// tables, 776 bytes: a batch with c classes has at least c items).
size_t msk_batch_item_bound(const msk_batch_item* item, int refine) {
  if (!item || !width_ok(item->n)) return 0;
  const int64_t n = item->n, k = 2 * n * n, p = 4 * n, ncol = n + 1;
  const int kt_per = (int)std::min<long long>(64, std::max<long long>(1, tune_get("batch.kt_per", kBatchKtPer)));
  TcShape sh;
  tc_ds_shape(p, k, ncol, kt_per, &sh);
  const int64_t ldy = (ncol + 3) / 4 * 4;
  const int nc = pass32_class((int)n);
  const int64_t tiles = (item->d + pass32_rows(nc) - 1) / pass32_rows(nc);
  const int64_t cap = (int64_t)pass32_ctas_per_sm(nc) * num_sms();
  const int64_t nchunks = std::max<int64_t>(1, std::min<int64_t>(cap, tiles));
  size_t b = 4096;
  auto piece = [&](size_t bytes) { b += bytes + 255; };
  piece(sizeof(BatchJob) + sizeof(TcJob) + 2 * sizeof(int) + kGather * sizeof(double) + sizeof(BatchCtl));
  piece((size_t)k * ldy * 4);                          // Y
  piece((size_t)p * sh.kpitch * 2);                    // G
  piece((size_t)3 * sh.npad * sh.kpitch * 2);          // Yt
  piece((size_t)sh.S * p * ncol * 8);                  // GEMM partials
  piece((size_t)p * ncol * 8);                         // Z
  piece(refine ? (size_t)n * n * 8 : 0);               // R^{-1}
  piece(refine ? (size_t)5 * n * 8 : 0);               // CG vectors
  piece((size_t)kScCount * 8);                         // CG scalars
  piece((size_t)pass_out_len(n) * 8);                  // pass result
  piece((size_t)nchunks * pass_out_len(n) * 8);        // pass partials
  piece(sizeof(int) + sizeof(CsParams<float>) + sizeof(int64_t));  // class tables
  return b;
}

int msk_batch_lstsq(const msk_batch_item* items, int nitems, int refine, double tol,
                    int32_t max_iter, msk_lstsq_info* infos, void* ws, size_t ws_bytes,
                    void* stream) {
  StageRange nvtx_range_("msk_batch_lstsq");
  if (!items) return -1;
  if (nitems < 1) return -2;
  if (refine != 0 && refine != 1) return -3;
  for (int j = 0; j < nitems; ++j) {
    const msk_batch_item& it = items[j];
    if (!it.A || !it.b || !it.x || !width_ok(it.n) || it.d < 4 * it.n || it.lda < it.d)
      return -1;
  }
  char* base = static_cast<char*>(ws);
  BatchPlan P;
  plan_batch(items, nitems, refine, base, &P);
  if (!ws || ws_bytes < P.bytes || (reinterpret_cast<uintptr_t>(ws) & 255) != 0) return MSK_ENOMEM;
  cudaStream_t st = as_stream(stream);
  BatchJob* jobs_dev = reinterpret_cast<BatchJob*>(base + P.jobs_off);
  TcJob* tc_dev = reinterpret_cast<TcJob*>(base + P.tc_off);
  double* gather = reinterpret_cast<double*>(base + P.gather_off);
  int item = 0;
  int rc = MSK_OK;
  for (int j = 0; j < nitems; ++j) {
    const BatchJob& J = P.jobs[j];
    rc = tc_ds_make_job(J.p, J.k, J.ncol, P.shapes[j], J.G, J.Yt, J.part, item, &P.tc[j]);
    if (rc) return rc;
    item += P.shapes[j].items;
  }
  P.total_items = item;
  MSK_CUDA(cudaMemcpyAsync(jobs_dev, P.jobs.data(), sizeof(BatchJob) * nitems, cudaMemcpyHostToDevice, st));
  MSK_CUDA(cudaMemcpyAsync(tc_dev, P.tc.data(), sizeof(TcJob) * nitems, cudaMemcpyHostToDevice, st));
  for (size_t c = 0; c < P.pass_nc.size(); ++c)
    MSK_CUDA(cudaMemcpyAsync(base + P.pass_mem_off[c], P.pass_mem[c].data(), sizeof(int) * P.pass_mem[c].size(),
                             cudaMemcpyHostToDevice, st));
  for (size_t c = 0; c < P.widths.size(); ++c) {
    MSK_CUDA(cudaMemcpyAsync(base + P.cs_off[c], P.cs[c].data(), sizeof(CsParams<float>) * P.cs[c].size(),
                             cudaMemcpyHostToDevice, st));
    MSK_CUDA(cudaMemcpyAsync(base + P.tiles_off[c], P.cs_tiles[c].data(),
                             sizeof(int64_t) * P.cs_tiles[c].size(), cudaMemcpyHostToDevice, st));
  }
  const int sms = num_sms();
  int* flags = reinterpret_cast<int*>(base + P.flags_off);
  int* active = flags;                // [0] iterating, [1] inner iterations, [2] outer steps
  int* refining = flags + 8;          // per problem
  int* recheck = flags + 8 + nitems;  // per problem
  BatchCtl* ctl = reinterpret_cast<BatchCtl*>(base + P.ctl_off);
  const bool fp64_start = refine || infos;  // an FP64 residual pass of the start
  const int round_len = (int)std::min<long long>(16, std::max<long long>(1, tune_get("batch.round", kRound)));
  const unsigned gblocks = (unsigned)((nitems + 255) / 256);
  const dim3 rgrid((unsigned)((pass_out_len(P.max_n) + 31) / 32), nitems);
  // cluster QR: the flow form where it fits (knob "qr.flow"), else the
  // look-ahead on-chip form, else the global-memory form
  const int qflow = tune_get("qr.flow", 0) != 0 ? 1 : 0;
  size_t qsm = 0;
  for (const BatchJob& J : P.jobs) {
    if (qflow && qr_flow_fits(J.p, J.ncol, 16)) qsm = std::max(qsm, qr_flow_smem_bytes(J.p, J.ncol, 16));
    else if (qr_smem_fits(J.p, J.ncol, 16)) qsm = std::max(qsm, qr_smem_bytes(J.p, J.ncol, 16));
  }
  int* qtflag = nullptr;
  if (qflow) {
    const int frc = tc_timeout_flag(&qtflag);
    if (frc) return frc;
  }
  // Function attributes before any capture begins.
  MSK_CUDA(cudaFuncSetAttribute(batch_qr_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  if (qsm) MSK_ALLOW_SMEM(batch_qr_kernel);
  MSK_ALLOW_SMEM((batch_pass_kernel<16, true>));
  MSK_ALLOW_SMEM((batch_pass_kernel<32, true>));
  MSK_ALLOW_SMEM((batch_pass_kernel<64, true>));
  MSK_ALLOW_SMEM((batch_pass_kernel<128, true>));
  MSK_ALLOW_SMEM((batch_pass_kernel<256, true>));
  MSK_ALLOW_SMEM((batch_pass_kernel<16, false>));
  MSK_ALLOW_SMEM((batch_pass_kernel<32, false>));
  MSK_ALLOW_SMEM((batch_pass_kernel<64, false>));
  MSK_ALLOW_SMEM((batch_pass_kernel<128, false>));
  MSK_ALLOW_SMEM((batch_pass_kernel<256, false>));

  // The whole batch is ONE graph launch: every stage below, and with
  // refinement the outer loop (a while node) whose body holds the inner CG
  // loop (a nested while node), steered by device-side convergence tests.
  // Graphs are cached by every value their launches bake in.
  std::vector<int64_t> key;
  {
    int dev = 0;
    MSK_CUDA(cudaGetDevice(&dev));
    auto push = [&](int64_t v) { key.push_back(v); };
    auto pushp = [&](const void* q) { key.push_back((int64_t)reinterpret_cast<uintptr_t>(q)); };
    push(dev), pushp(base), push(nitems), push(refine), push(fp64_start), push(max_iter), push(round_len);
    int64_t tb;
    std::memcpy(&tb, &tol, sizeof(tb));
    push(tb);
    push(P.max_yk), push(P.max_pk), push(P.max_k), push(P.max_npad), push(P.max_n), push(P.max_nt);
    push(P.total_items), push((int64_t)qsm), push(sms), push(qflow);
    push((int64_t)P.widths.size());
    for (size_t c = 0; c < P.widths.size(); ++c)
      push(P.widths[c]), push((int64_t)P.cs_off[c]), push((int64_t)P.tiles_off[c]), push((int64_t)P.cs[c].size()),
          push(P.cs_tiles[c].back());
    push((int64_t)P.pass_nc.size());
    for (size_t c = 0; c < P.pass_nc.size(); ++c)
      push(P.pass_nc[c]), push(P.pass_chunks[c]), push((int64_t)P.pass_mem_off[c]),
          push((int64_t)P.pass_mem[c].size());
    push((int64_t)P.jobs_off), push((int64_t)P.tc_off), push((int64_t)P.flags_off), push((int64_t)P.gather_off),
        push((int64_t)P.ctl_off);
  }

  // one pass over every problem (a launch per width class): the FP64 residual
  // pass (resid, problems with only[j] set, all when null) or a CG pass
  auto passes = [&](bool resid, const int* only, cudaStream_t s) {
    for (size_t c = 0; c < P.pass_nc.size(); ++c) {
      const int nc = P.pass_nc[c];
      const unsigned g = (unsigned)P.pass_chunks[c];
      const size_t sm = pass32_smem(nc);
      const int* mem = reinterpret_cast<const int*>(base + P.pass_mem_off[c]);
      const int nm = (int)P.pass_mem[c].size();
#define MSK_BATCH_PASS(NCV)                                                                     \
  if (nc == NCV) {                                                                              \
    if (resid) batch_pass_kernel<NCV, true><<<g, kP32Threads, sm, s>>>(jobs_dev, mem, nm, only);  \
    else batch_pass_kernel<NCV, false><<<g, kP32Threads, sm, s>>>(jobs_dev, mem, nm, only);      \
  }
      MSK_BATCH_PASS(16)
      MSK_BATCH_PASS(32)
      MSK_BATCH_PASS(64)
      MSK_BATCH_PASS(128)
      MSK_BATCH_PASS(256)
#undef MSK_BATCH_PASS
    }
  };
  auto fp64_pass = [&](const int* only, cudaStream_t s) -> int {
    passes(true, only, s);
    MSK_CHECK_LAUNCH("batch_pass_kernel");
    batch_pass_reduce_kernel<<<rgrid, 256, 0, s>>>(jobs_dev, only);
    MSK_CHECK_LAUNCH("batch_pass_reduce_kernel");
    return MSK_OK;
  };
  // Stages 1-4 and the start of the refinement, on stream s.
  auto stages = [&](cudaStream_t s, cudaGraphConditionalHandle h_out) -> int {
    // 1. CountSketch: zero every Y, then one launch per width class
    batch_zero_kernel<<<dim3((unsigned)std::min<int64_t>((P.max_yk + 255) / 256, 64), nitems), 256, 0, s>>>(jobs_dev);
    MSK_CHECK_LAUNCH("batch_zero_kernel");
    for (size_t c = 0; c < P.widths.size(); ++c) {
      const int e = launch_cs_batch_f32(P.widths[c], reinterpret_cast<const CsParams<float>*>(base + P.cs_off[c]),
                                        reinterpret_cast<const int64_t*>(base + P.tiles_off[c]),
                                        (int)P.cs[c].size(), P.cs_tiles[c].back(), s);
      if (e) return e;
    }
    // 2. Gaussian (bfloat16) and the 3-part bfloat16 split of Y
    batch_gaussian_kernel<<<dim3((unsigned)std::min<int64_t>((P.max_pk + 255) / 256, 8 * sms), nitems), 256, 0, s>>>(jobs_dev);
    MSK_CHECK_LAUNCH("batch_gaussian_kernel");
    batch_split_kernel<<<dim3((unsigned)((P.max_k + 31) / 32), (unsigned)((P.max_npad + 31) / 32), nitems), 256, 0, s>>>(jobs_dev);
    MSK_CHECK_LAUNCH("batch_split_kernel");
    // 3. tensor-core Gaussian stage and its split-K reduction
    int e = launch_tc_ds_batch(tc_dev, nitems, P.total_items, P.max_nt, s);
    if (e) return e;
    batch_gemm_reduce_kernel<<<dim3(64, nitems), 256, 0, s>>>(jobs_dev);
    MSK_CHECK_LAUNCH("batch_gemm_reduce_kernel");
    // 4. QR (+ triangular solve without refinement), one 16-CTA cluster per problem
    {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(16, nitems, 1);
      cfg.blockDim = dim3(kQrThreads, 1, 1);
      cfg.dynamicSmemBytes = qsm;
      cfg.stream = s;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = 16;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      MSK_CUDA(cudaLaunchKernelEx(&cfg, batch_qr_kernel, (const BatchJob*)jobs_dev, qsm, refine ? 0 : 1, qflow,
                                  qtflag));
    }
    if (refine) {  // R^{-1} (the preconditioner) and from it x0 = R^{-1} c
      batch_tri_inverse_kernel<<<dim3((P.max_n + 7) / 8, nitems), 256, 0, s>>>(jobs_dev);
      MSK_CHECK_LAUNCH("batch_tri_inverse_kernel");
      batch_x0_kernel<<<nitems, 512, 0, s>>>(jobs_dev);
      MSK_CHECK_LAUNCH("batch_x0_kernel");
    }
    if (fp64_start) {
      e = fp64_pass(nullptr, s);
      if (e) return e;
      batch_ref_init_kernel<<<1, 256, 0, s>>>(jobs_dev, nitems, ctl, refine, max_iter, flags, h_out);
      MSK_CHECK_LAUNCH("batch_ref_init_kernel");
    }
    return MSK_OK;
  };
  // Top of an outer step: arm, start CG, and the inner loop's condition.
  auto outer_head = [&](cudaStream_t s, cudaGraphConditionalHandle h_in) -> int {
    batch_outer_arm_kernel<<<gblocks, 256, 0, s>>>(jobs_dev, nitems, ctl, refining, active);
    MSK_CHECK_LAUNCH("batch_outer_arm_kernel");
    batch_pcg_start_kernel<<<nitems, 512, 0, s>>>(jobs_dev, tol, active);
    MSK_CHECK_LAUNCH("batch_pcg_start_kernel");
    batch_inner_arm_kernel<<<1, 1, 0, s>>>(h_in, active);
    MSK_CHECK_LAUNCH("batch_inner_arm_kernel");
    return MSK_OK;
  };
  // One trip of the inner loop: round_len CG iterations (passes per width
  // class, then the CG step fused with the partials' reduction on one 8-CTA
  // cluster per problem), then the loop's condition.
  auto inner_trip = [&](cudaStream_t s, cudaGraphConditionalHandle h_in) -> int {
    cudaLaunchConfig_t ucfg = {};
    ucfg.gridDim = dim3(kUpdCL, nitems, 1);
    ucfg.blockDim = dim3(kUpdThreads, 1, 1);
    ucfg.stream = s;
    cudaLaunchAttribute uat[1];
    uat[0].id = cudaLaunchAttributeClusterDimension;
    uat[0].val.clusterDim.x = kUpdCL;
    uat[0].val.clusterDim.y = 1;
    uat[0].val.clusterDim.z = 1;
    ucfg.attrs = uat;
    ucfg.numAttrs = 1;
    for (int r = 0; r < round_len; ++r) {
      passes(false, nullptr, s);
      MSK_CHECK_LAUNCH("batch_pass_kernel");
      MSK_CUDA(cudaLaunchKernelEx(&ucfg, batch_pcg_cluster_kernel, (const BatchJob*)jobs_dev, active, refining));
    }
    batch_loop_cond_kernel<<<1, 1, 0, s>>>(h_in, active);
    MSK_CHECK_LAUNCH("batch_loop_cond_kernel");
    return MSK_OK;
  };
  // Bottom of an outer step: x += d, the FP64 residual of the corrected
  // problems, the convergence tests and the outer loop's condition.
  auto outer_tail = [&](cudaStream_t s, cudaGraphConditionalHandle h_out) -> int {
    batch_axpy_kernel<<<nitems, 256, 0, s>>>(jobs_dev, refining);
    MSK_CHECK_LAUNCH("batch_axpy_kernel");
    batch_post_inner_kernel<<<gblocks, 256, 0, s>>>(jobs_dev, nitems, ctl, recheck);
    MSK_CHECK_LAUNCH("batch_post_inner_kernel");
    const int e = fp64_pass(recheck, s);
    if (e) return e;
    batch_outer_check_kernel<<<1, 256, 0, s>>>(jobs_dev, nitems, ctl, recheck, tol, max_iter, flags, h_out);
    MSK_CHECK_LAUNCH("batch_outer_check_kernel");
    return MSK_OK;
  };

  thread_local GraphCache caches[kMaxDevices];
  int dev = 0;
  MSK_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return MSK_ENOTSUP;
  GraphCache& cache = caches[dev];
  if (!cache.cap) MSK_CUDA(cudaStreamCreateWithFlags(&cache.cap, cudaStreamNonBlocking));
  cudaGraphExec_t exec = nullptr;
  for (size_t e = 0; e < cache.entries.size(); ++e)
    if (cache.entries[e].first == key) {
      exec = cache.entries[e].second;
      auto hit = cache.entries[e];
      cache.entries.erase(cache.entries.begin() + (long)e);
      cache.entries.push_back(hit);
      break;
    }
  if (!exec) {
    // Build: capture each straight segment into its graph (recording work
    // without running it, on the private stream) and add the while nodes
    // between the segments.
    cudaStream_t cap = cache.cap;
    cudaGraph_t top = nullptr;
    MSK_CUDA(cudaGraphCreate(&top, 0));
    std::vector<cudaGraphNode_t> tail;
    auto begin = [&](cudaGraph_t g, const std::vector<cudaGraphNode_t>& deps) {
      return cudaStreamBeginCaptureToGraph(cap, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(),
                                           cudaStreamCaptureModeThreadLocal);
    };
    // end a segment; `out` receives its last nodes
    auto end = [&](std::vector<cudaGraphNode_t>* out) {
      cudaStreamCaptureStatus cs;
      const cudaGraphNode_t* deps = nullptr;
      size_t nd = 0;
      cudaError_t e1 = cudaStreamGetCaptureInfo(cap, &cs, nullptr, nullptr, &deps, nullptr, &nd);
      if (e1 == cudaSuccess) out->assign(deps, deps + nd);
      cudaGraph_t g = nullptr;
      cudaError_t e2 = cudaStreamEndCapture(cap, &g);
      return e1 != cudaSuccess ? e1 : e2;
    };
    auto add_while = [&](cudaGraph_t g, const std::vector<cudaGraphNode_t>& deps, cudaGraphConditionalHandle h,
                         cudaGraphNode_t* node, cudaGraph_t* body) {
      cudaGraphNodeParams cp = {};
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = h;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      cudaError_t e = cudaGraphAddNode(node, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(), &cp);
      if (e == cudaSuccess) *body = cp.conditional.phGraph_out[0];
      return e;
    };
    cudaError_t ce = cudaSuccess;
    int brc = MSK_OK;
    cudaGraphConditionalHandle h_out = 0, h_in = 0;
    if (refine) ce = cudaGraphConditionalHandleCreate(&h_out, top, 0, 0);
    if (ce == cudaSuccess) ce = begin(top, tail);
    if (ce == cudaSuccess) {
      brc = stages(cap, h_out);
      ce = end(&tail);
    }
    if (ce == cudaSuccess && !brc && refine) {
      cudaGraphNode_t onode = nullptr, inode = nullptr;
      cudaGraph_t obody = nullptr, ibody = nullptr;
      std::vector<cudaGraphNode_t> t2, t3, t4;
      ce = add_while(top, tail, h_out, &onode, &obody);
      if (ce == cudaSuccess) ce = cudaGraphConditionalHandleCreate(&h_in, obody, 0, 0);
      if (ce == cudaSuccess) ce = begin(obody, {});
      if (ce == cudaSuccess) {
        brc = outer_head(cap, h_in);
        ce = end(&t2);
      }
      if (ce == cudaSuccess && !brc) ce = add_while(obody, t2, h_in, &inode, &ibody);
      if (ce == cudaSuccess && !brc) ce = begin(ibody, {});
      if (ce == cudaSuccess && !brc) {
        brc = inner_trip(cap, h_in);
        ce = end(&t3);
      }
      if (ce == cudaSuccess && !brc) ce = begin(obody, {inode});
      if (ce == cudaSuccess && !brc) {
        brc = outer_tail(cap, h_out);
        ce = end(&t4);
      }
      tail.assign(1, onode);
    }
    if (ce == cudaSuccess && !brc && fp64_start) {
      ce = begin(top, tail);
      if (ce == cudaSuccess) {
        batch_final_kernel<<<gblocks, 256, 0, cap>>>(nitems, ctl, gather);
        ce = cudaGetLastError();
        std::vector<cudaGraphNode_t> t5;
        const cudaError_t ce2 = end(&t5);
        if (ce == cudaSuccess) ce = ce2;
      }
    }
    if (ce == cudaSuccess && !brc) ce = cudaGraphInstantiate(&exec, top, 0);
    cudaGraphDestroy(top);
    if (brc) return brc;
    if (ce != cudaSuccess) return cuda_fail(ce, "batch graph");
    if (cache.entries.size() >= kGraphCacheMax) {
      cudaGraphExecDestroy(cache.entries.front().second);
      cache.entries.erase(cache.entries.begin());
    }
    cache.entries.push_back({key, exec});
  }
  MSK_CUDA(cudaGraphLaunch(exec, st));
  std::vector<double> hg(kGather * (size_t)nitems);
  if (fp64_start)
    MSK_CUDA(cudaMemcpyAsync(hg.data(), gather, sizeof(double) * kGather * nitems, cudaMemcpyDeviceToHost, st));
  MSK_CUDA(cudaStreamSynchronize(st));  // also: the uploads above read host vectors
  int status = MSK_OK;
  for (int j = 0; j < nitems; ++j) {
    const bool conv = fp64_start ? hg[kGather * j + 1] != 0.0 : true;
    if (refine && !conv) status = MSK_ENOCONV;
    if (infos) {
      infos[j].iters = (int32_t)hg[kGather * j];
      infos[j].converged = conv ? 1 : 0;
      infos[j].relres = hg[kGather * j + 2];
      infos[j].relres_sns = hg[kGather * j + 3];
    }
  }
  return status;
}

}  // extern "C"
