// qr.cu — the small dense FP64 steps of sketch-and-solve (Algorithm 1 steps
// 2-3; GeQRF/OrMQR/TRSV in Section 6.1) and of the normal equations
// (POTRF + two TRSV, Section 6.3).
//
// Householder QR of the sketched m x c matrix (m = p rows, c = n+1 columns):
// one thread-block cluster (up to 16 CTAs on 16 SMs) factors one matrix.
// Column j belongs to CTA j mod CL (cyclic, so the shrinking trailing matrix
// stays balanced).  Step j: the owner builds the reflector of column j
// (v = x + sign(x0)||x|| e0, tau = 2 / v^T v, R[j][j] = -sign(x0)||x||) and
// publishes it; every CTA then applies I - tau v v^T to the columns it owns,
// one warp per column.  On chip (qr_cluster_smem_body) the owned columns stay
// in shared memory and the steps overlap through a split cluster barrier with
// one column of look-ahead; in global memory (larger matrices) one full
// cluster barrier per column, v staged in each CTA's shared memory.  FP64
// throughout: GB300's FP64 rate (2 FMAs per clock per SM) over the cluster's
// 16 SMs bounds the factorisation at 2 m c^2 flops.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "msk_internal.h"
#include "msk_qr.cuh"

namespace msk {


// smem_cap: dynamic shared memory of the launch; flow != 0: the flow form
// (sized for it); else the look-ahead on-chip form when the owned columns
// fit in smem_cap, the global-memory form otherwise.  tflag: set when a
// bounded wait of the flow form expires.
__global__ void __launch_bounds__(kQrThreads) qr_cluster_kernel(double* __restrict__ W, int m, int c,
                                                              int64_t ldw, size_t smem_cap, int flow,
                                                              int* tflag) {
  extern __shared__ __align__(16) double qr_dyn[];
  const int CL = (int)cg::this_cluster().num_blocks();
  if (flow)
    qr_cluster_flow_body(W, m, c, ldw, qr_dyn, tflag);
  else if (qr_smem_bytes(m, c, CL) <= smem_cap)
    qr_cluster_smem_body(W, m, c, ldw, qr_dyn);
  else
    qr_cluster_body(W, m, c, ldw);
}

// The flow form (knob "qr.flow", default off: measured slower) when its
// shared memory fits.
bool qr_use_flow(int64_t m, int64_t c, int CL) {
  return tune_get("qr.flow", 0) != 0 && qr_flow_fits((int)m, (int)c, CL);
}

int launch_householder_qr(double* W, int64_t m, int64_t c, int64_t ldw, cudaStream_t st) {
  static int cluster_size = 0;
  if (cluster_size == 0) {
    cudaError_t e = cudaFuncSetAttribute(qr_cluster_kernel,
                                         cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    int cs = 8;
    if (e == cudaSuccess) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(16, 1, 1);
      cfg.blockDim = dim3(kQrThreads, 1, 1);
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = 16;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int ncl = 0;
      if (cudaOccupancyMaxActiveClusters(&ncl, qr_cluster_kernel, &cfg) == cudaSuccess && ncl > 0)
        cs = 16;
    }
    cudaGetLastError();
    cluster_size = cs;
  }
  int CL = (int)std::min<int64_t>(cluster_size, c);
  if (CL < 1) CL = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CL, 1, 1);
  cfg.blockDim = dim3(kQrThreads, 1, 1);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const bool flow = qr_use_flow(m, c, CL);
  const size_t smem = flow ? qr_flow_smem_bytes((int)m, (int)c, CL)
                           : (qr_smem_fits((int)m, (int)c, CL) ? qr_smem_bytes((int)m, (int)c, CL) : 0);
  int* tflag = nullptr;
  if (flow) {
    const int frc = tc_timeout_flag(&tflag);
    if (frc) return frc;
  }
  if (smem) MSK_ALLOW_SMEM(qr_cluster_kernel);
  cfg.dynamicSmemBytes = smem;
  MSK_CUDA(cudaLaunchKernelEx(&cfg, qr_cluster_kernel, W, (int)m, (int)c, ldw, smem, flow ? 1 : 0,
                              tflag));
  return MSK_OK;
}

// ---------------------------------------------------------------------------
// Triangular solves (single CTA; n <= 4096).  status[0] <- j+1 for the first
// zero pivot met (0 when none).

// R x = rhs, R upper (column-major, ldr).  x may alias rhs.
__global__ void trsv_upper_kernel(const double* __restrict__ R, int n, int64_t ldr,
                                  const double* rhs, double* x, int* status) {
  __shared__ double xs[kTrsvMax];
  trsv_upper_body(R, n, ldr, rhs, x, status, xs);
}

// R^T y = rhs, R upper (so R^T lower).  y may alias rhs.
__global__ void trsv_upper_t_kernel(const double* __restrict__ R, int n, int64_t ldr,
                                    const double* rhs, double* y, int* status) {
  __shared__ double ys[kTrsvMax];
  for (int i = threadIdx.x; i < n; i += blockDim.x) ys[i] = rhs[i];
  __syncthreads();
  for (int i = 0; i < n; ++i) {
    if (threadIdx.x == 0) {
      const double rii = R[i + (int64_t)i * ldr];
      if (rii == 0.0 && status && status[0] == 0) status[0] = i + 1;
      ys[i] = ys[i] / rii;
    }
    __syncthreads();
    const double yi = ys[i];
    for (int r = i + 1 + threadIdx.x; r < n; r += blockDim.x) ys[r] -= R[i + (int64_t)r * ldr] * yi;
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) y[i] = ys[i];
}

int launch_trsv_upper(const double* R, int64_t n, int64_t ldr, const double* rhs, double* x,
                      int* status, bool transposed, cudaStream_t st) {
  if (n <= 0) return MSK_OK;
  if (n > kTrsvMax) return MSK_ENOTSUP;
  if (transposed)
    trsv_upper_t_kernel<<<1, 256, 0, st>>>(R, (int)n, ldr, rhs, x, status);
  else
    trsv_upper_kernel<<<1, 256, 0, st>>>(R, (int)n, ldr, rhs, x, status);
  MSK_CHECK_LAUNCH("trsv_kernel");
  return MSK_OK;
}

// ---------------------------------------------------------------------------
// Cholesky of the symmetric n x n matrix Gm (column-major, ldg; upper part
// used) into upper R (column-major, ldr) with R^T R = Gm: right-looking, one
// CTA.  Gm is overwritten (trailing updates).  status[0] <- j+1 when pivot j is
// not positive.
__global__ void cholesky_kernel(double* __restrict__ Gm, int n, int64_t ldg, double* __restrict__ R,
                                int64_t ldr, int* status) {
  __shared__ double piv;
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
    const int r = i % n, c = i / n;
    if (r > c) R[r + (int64_t)c * ldr] = 0.0;
  }
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      const double s = Gm[j + (int64_t)j * ldg];
      if (!(s > 0.0)) {
        bad = 1;
        if (status) status[0] = j + 1;
      } else {
        piv = sqrt(s);
        R[j + (int64_t)j * ldr] = piv;
      }
    }
    __syncthreads();
    if (bad) return;
    const double rjj = piv;
    for (int c = j + 1 + threadIdx.x; c < n; c += blockDim.x)
      R[j + (int64_t)c * ldr] = Gm[j + (int64_t)c * ldg] / rjj;
    __syncthreads();
    // trailing update of the upper triangle: Gm[a][c] -= R[j][a] R[j][c], j < a <= c
    const int t = n - j - 1;
    for (int e = threadIdx.x; e < t * t; e += blockDim.x) {
      const int a = j + 1 + e % t, c = j + 1 + e / t;
      if (a <= c) Gm[a + (int64_t)c * ldg] -= R[j + (int64_t)a * ldr] * R[j + (int64_t)c * ldr];
    }
    __syncthreads();
  }
}

// Host-side check of an upper-triangular factor's diagonal: synchronises the
// stream, returns j+1 for the first exactly-zero R[j][j], else MSK_OK.
int first_zero_pivot(const double* R, int64_t n, int64_t ldr, cudaStream_t st) {
  if (n <= 0) return MSK_OK;
  std::vector<double> diag((size_t)n);
  MSK_CUDA(cudaMemcpy2DAsync(diag.data(), sizeof(double), R, (size_t)(ldr + 1) * sizeof(double),
                             sizeof(double), (size_t)n, cudaMemcpyDeviceToHost, st));
  MSK_CUDA(cudaStreamSynchronize(st));
  for (int64_t j = 0; j < n; ++j)
    if (diag[(size_t)j] == 0.0) return (int)(j + 1);
  return MSK_OK;
}

int launch_cholesky(double* Gm, int64_t n, int64_t ldg, double* R, int64_t ldr, int* status,
                    cudaStream_t st) {
  cholesky_kernel<<<1, 1024, 0, st>>>(Gm, (int)n, ldg, R, ldr, status);
  MSK_CHECK_LAUNCH("cholesky_kernel");
  return MSK_OK;
}

}  // namespace msk

using namespace msk;

extern "C" {

int msk_householder_qr(double* W, int64_t m, int64_t c, int64_t ldw, void* stream) {
  StageRange nvtx_range_("msk_householder_qr");
  if (!W) return -1;
  if (m < c || m > 0x7fffffffLL) return -2;
  if (c < 1 || c > kQrMaxCols) return -3;
  if (ldw < m) return -4;
  return launch_householder_qr(W, m, c, ldw, as_stream(stream));
}

int msk_trsv_upper(const double* R, int64_t n, int64_t ldr, const double* rhs, double* x,
                   void* stream) {
  if (!R) return -1;
  if (n < 0 || n > kTrsvMax) return -2;
  if (ldr < (n > 1 ? n : 1)) return -3;
  if (!rhs && n > 0) return -4;
  if (!x && n > 0) return -5;
  cudaStream_t st = as_stream(stream);
  int rc = launch_trsv_upper(R, n, ldr, rhs, x, nullptr, false, st);
  if (rc) return rc;
  return first_zero_pivot(R, n, ldr, st);
}

}  // extern "C"
