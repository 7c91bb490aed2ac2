// api.cu — the extern "C" entry points of libmsketch for the sketching steps
// (hash hook, Gaussian hook, CountSketch, multisketch, Gaussian-stage GEMM):
// argument checks, workspace carving, and the launch sequence on the caller's
// stream.  Every numeric step runs in this library's kernels.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <algorithm>

#include "msk_device.cuh"
#include "msk_internal.h"

namespace msk {

static thread_local char g_last_error[256] = {0};

int cuda_fail(cudaError_t e, const char* where) {
  std::snprintf(g_last_error, sizeof(g_last_error), "%s: %s", where, cudaGetErrorString(e));
  return MSK_ECUDA;
}

void set_error_text(const char* msg) {
  std::snprintf(g_last_error, sizeof(g_last_error), "%s", msg);
}

int smem_optin_max() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || v <= 0)
    return 48 * 1024;
  return v;
}

cudaError_t zero_rows(void* Y, int64_t ldy, int64_t ncol, int64_t k, size_t esz, cudaStream_t st) {
  if (k <= 0 || ncol <= 0) return cudaSuccess;
  if (ldy == ncol) return cudaMemsetAsync(Y, 0, (size_t)k * (size_t)ncol * esz, st);
  return cudaMemset2DAsync(Y, (size_t)ldy * esz, 0, (size_t)ncol * esz, (size_t)k, st);
}

cudaError_t allow_max_smem(const void* func) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, func);
  if (e != cudaSuccess) return e;
  const int dyn = smem_optin_max() - (int)fa.sharedSizeBytes;
  return cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn > 0 ? dyn : 0);
}

int num_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
  return sms > 0 ? sms : 1;
}

static size_t dtype_size(int dtype) { return dtype == MSK_F64 ? 8 : 4; }

// Row pitch of the CountSketch Y inside ms_sketch's workspace: FP32 rows are
// padded to 4 elements so the vector reductions stay 16-byte aligned.
static int64_t ws_ldy(int64_t ncol, int dtype) {
  return dtype == MSK_F32 ? (ncol + 3) / 4 * 4 : (ncol + 1) / 2 * 2;
}

static bool is_tensor_prec(int prec) {
  return prec == MSK_GEMM_BF16 || prec == MSK_GEMM_F16 || prec == MSK_GEMM_BF16X3;
}

// Element type of the CountSketch inside ms_sketch: the FP64 Gaussian stage
// gets an FP64-accumulated sketch even from FP32 A (the plain FP64 path);
// the tensor-core stages take an FP32 sketch; otherwise A's type.
static int ms_y_dtype(int dtype, int gemm_prec) {
  if (gemm_prec == MSK_GEMM_F64) return MSK_F64;
  if (is_tensor_prec(gemm_prec)) return MSK_F32;
  return dtype;
}

}  // namespace msk

namespace msk {
// First failed index check of a checked build (its site), 0 otherwise; the
// kernels of other files reach it only in checked builds (relocatable device
// code).
__device__ int g_msk_check = 0;
size_t tc_gemm_workspace(int64_t p, int64_t k, int64_t ncol, int prec);
// Z = G Y for a Y of element type y_dtype (FP64 or FP32); the tensor-core
// precisions take FP32 Y only.
// A side stream (and its fork/join events) per device and host thread.
struct SideStream {
  cudaStream_t s = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};
static int side_stream(SideStream** out) {
  constexpr int kMaxDev = 64;
  thread_local SideStream sides[kMaxDev];
  int dev = 0;
  MSK_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDev) return MSK_ENOTSUP;
  SideStream& sd = sides[dev];
  if (!sd.s) {
    MSK_CUDA(cudaStreamCreateWithFlags(&sd.s, cudaStreamNonBlocking));
    MSK_CUDA(cudaEventCreateWithFlags(&sd.fork, cudaEventDisableTiming));
    MSK_CUDA(cudaEventCreateWithFlags(&sd.join, cudaEventDisableTiming));
  }
  *out = &sd;
  return MSK_OK;
}

// Events the next ms_sketch call of this thread records around its
// CountSketch (msk_stage_events), then forgets.
struct StageEvents {
  cudaEvent_t before_cs = nullptr, after_cs = nullptr;
};
static StageEvents& stage_events() {
  thread_local StageEvents ev;
  return ev;
}

bool gemm_stage_sliced(int64_t p, int64_t k, int64_t ncol, int y_dtype, int gemm_prec, size_t ws_bytes) {
  return gemm_prec == MSK_GEMM_F64 && y_dtype == MSK_F64 && oz_applicable(p, k, ncol) &&
         ws_bytes >= oz_gemm_workspace(p, k, ncol);
}

int gemm_stage(uint64_t seed, int64_t p, int64_t k, int64_t ncol, const void* Y, int y_dtype,
               int64_t ldy, int gemm_prec, double* Z, int64_t ldz, void* ws, size_t ws_bytes,
               cudaStream_t st, bool g_ready) {
  StageRange nvtx_range_("gemm_stage");
  const uint64_t gkey = stream_key(seed, kTagGauss);
  if (is_tensor_prec(gemm_prec)) {
    if (y_dtype != MSK_F32) return MSK_ENOTSUP;
    return launch_tc_gemm(gkey, p, k, ncol, static_cast<const float*>(Y), ldy, gemm_prec, Z, ldz,
                          ws, ws_bytes, st);
  }
  // FP64 Y and FP64 arithmetic: the exact-slicing tensor-core stage where it
  // applies and the workspace holds it, else the FP64 SIMT kernel
  if (gemm_stage_sliced(p, k, ncol, y_dtype, gemm_prec, ws_bytes))
    return launch_oz_gemm(gkey, p, k, ncol, static_cast<const double*>(Y), ldy, Z, ldz, ws, ws_bytes,
                          st, g_ready);
  Carve cv(ws, ws_bytes);
  float* G = static_cast<float*>(cv.take((size_t)p * k * sizeof(float)));
  if (!G) return MSK_ENOMEM;
  int rc = launch_gaussian(gkey, p, k, MSK_GEMM_F32, G, k, st);
  if (rc) return rc;
  const size_t rest_off = align_up(cv.used, 256);
  if (rest_off > ws_bytes) return MSK_ENOMEM;
  return launch_gemm_simt(G, k, Y, y_dtype == MSK_F64, ldy, gemm_prec == MSK_GEMM_F64, p, k, ncol,
                          Z, ldz, cv.base + rest_off, ws_bytes - rest_off, st);
}
}  // namespace msk

using namespace msk;

extern "C" {

const char* msk_version(void) { return "msketch 0.1 (sm_103a)"; }

int msk_stage_events(void* before_cs, void* after_cs) {
  StageEvents& ev = stage_events();
  ev.before_cs = static_cast<cudaEvent_t>(before_cs);
  ev.after_cs = static_cast<cudaEvent_t>(after_cs);
  return MSK_OK;
}

int msk_checked_build(void) {
#ifdef MSK_CHECKED
  return 1;
#else
  return 0;
#endif
}

int msk_check_status(void* stream) {
  MSK_CUDA(cudaStreamSynchronize(as_stream(stream)));
  int h = 0, zero = 0;
  MSK_CUDA(cudaMemcpyFromSymbol(&h, g_msk_check, sizeof(int)));
  if (h) MSK_CUDA(cudaMemcpyToSymbol(g_msk_check, &zero, sizeof(int)));
  return h;
}

const char* msk_last_error(void) { return g_last_error; }

int msk_take_timeout(void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return tc_take_timeout(st);
}

int msk_selftest_wait(void* stream) {
  return launch_tc_wait_selftest(static_cast<cudaStream_t>(stream));
}

int cs_hash(uint64_t seed, int64_t i0, int64_t count, int64_t k, uint32_t* h, int8_t* s,
            void* stream) {
  if (count < 0) return -3;
  if (k < 1 || k > 0xFFFFFFFFLL) return -4;
  if (i0 < 0) return -2;
  return launch_cs_hash(stream_key(seed, kTagHash), i0, count, (uint32_t)k, h, s,
                        as_stream(stream));
}

int ms_gaussian(uint64_t seed, int64_t p, int64_t k, int out_prec, void* G, int64_t ldg,
                void* stream) {
  if (p < 1 || p >= (1LL << 24)) return -2;
  if (k < 1) return -3;
  if (out_prec < MSK_GEMM_F64 || out_prec > MSK_GEMM_F16) return -4;
  if (!G) return -5;
  if (ldg < k) return -6;
  return launch_gaussian(stream_key(seed, kTagGauss), p, k, out_prec, G, ldg, as_stream(stream));
}

size_t msk_srht_workspace(int64_t d, int64_t n, int with_b, int64_t k) {
  return srht_workspace(d, n + (with_b ? 1 : 0), k);
}

int srht_sketch(const void* A, int dtype, int64_t d, int64_t n, int64_t lda, const double* b,
                int64_t k, uint64_t seed, double* Y, int64_t ldy, void* ws, size_t ws_bytes,
                void* stream) {
  StageRange nvtx_range_("srht_sketch");
  if (!A) return -1;
  if (dtype != MSK_F64 && dtype != MSK_F32) return -2;
  if (d < 2 || (d & (d - 1)) != 0 || d > (int64_t(1) << 26)) return -3;
  if (n < 0 || n + (b ? 1 : 0) < 1 || n + (b ? 1 : 0) > 65535) return -4;
  if (lda < d) return -5;
  if (k < 1 || k > 0xFFFFFFFFLL) return -7;
  if (!Y) return -9;
  if (ldy < n + (b ? 1 : 0)) return -10;
  if (ws_bytes < msk_srht_workspace(d, n, b ? 1 : 0, k)) return MSK_ENOMEM;
  return launch_srht(A, dtype, d, n, lda, b, k, seed, Y, ldy, ws, ws_bytes, as_stream(stream));
}

size_t msk_cs_workspace(int64_t d, int64_t n, int64_t k, int dtype, int strategy) {
  if (strategy == MSK_CS_SORTED) return cs_sorted_workspace(d, k);
  if (dtype != MSK_F64) return 0;
  // replicas of Y for narrow FP64 sketches (with or without the b column)
  return std::max(cs_replica_bytes(k, n), cs_replica_bytes(k, n + 1));
}

int cs_sketch(const void* A, int dtype, int64_t d, int64_t n, int64_t lda, const double* b,
              int64_t k, uint64_t seed, void* Y, int64_t ldy, int strategy, void* ws,
              size_t ws_bytes, void* stream) {
  StageRange nvtx_range_("cs_sketch");
  return cs_sketch_internal(A, dtype, d, n, lda, b, k, seed, Y, ldy, strategy, ws, ws_bytes,
                            false, as_stream(stream));
}

}  // extern "C"

int msk::count_sketch_f64y(const void* A, int dtype, int64_t d, int64_t n, int64_t lda,
                           const double* b, int64_t k, uint64_t seed, double* Y, int64_t ldy,
                           cudaStream_t st, bool zero, int64_t i0) {
  if (dtype == MSK_F64)
    return launch_cs_atomic(A, dtype, d, n, lda, b, (uint32_t)k, stream_key(seed, kTagHash), Y, ldy,
                            false, st, nullptr, 0, zero, i0);
  const int64_t ncol = n + (b ? 1 : 0);
  if (zero) MSK_CUDA(zero_rows(Y, ldy, ncol, k, 8, st));
  int64_t maxc = 256;
  const int64_t fit = (int64_t)(tune_get("cs.l2_budget_bytes", 48ll << 20)) / (k * 8);
  if (fit >= 64 && fit / 64 * 64 < maxc) maxc = fit / 64 * 64;
  return launch_cs_f32a_f64y(static_cast<const float*>(A), d, n, lda, b, (uint32_t)k,
                             stream_key(seed, kTagHash), Y, ldy, maxc, st, i0);
}

int msk::cs_sketch_internal(const void* A, int dtype, int64_t d, int64_t n, int64_t lda,
                            const double* b, int64_t k, uint64_t seed, void* Y, int64_t ldy,
                            int strategy, void* ws, size_t ws_bytes, bool pad_ok,
                            cudaStream_t st) {
  if (!A && d > 0 && n > 0) return -1;
  if (dtype != MSK_F64 && dtype != MSK_F32) return -2;
  if (d < 0) return -3;
  if (n < 0) return -4;
  if (lda < (d > 1 ? d : 1)) return -5;
  if (k < 1 || k > 0xFFFFFFFFLL) return -7;
  const int64_t ncol = n + (b ? 1 : 0);
  if (!Y) return -9;
  if (ldy < ncol) return -10;
  if (strategy != MSK_CS_ATOMIC && strategy != MSK_CS_SORTED) return -11;
  const uint64_t key = stream_key(seed, kTagHash);
  if (strategy == MSK_CS_ATOMIC)
    return launch_cs_atomic(A, dtype, d, n, lda, b, (uint32_t)k, key, Y, ldy, pad_ok, st, ws,
                            ws_bytes);
  if (d >= (1LL << 31) || k >= (1LL << 31)) return MSK_ENOTSUP;
  if (ws_bytes < cs_sorted_workspace(d, k)) return MSK_ENOMEM;
  return launch_cs_sorted(A, dtype, d, n, lda, b, (uint32_t)k, key, Y, ldy, ws, ws_bytes, st);
}

extern "C" {

size_t msk_gemm_workspace(int64_t p, int64_t k, int64_t ncol, int gemm_prec) {
  Need nd;
  if (is_tensor_prec(gemm_prec)) {
    nd.add(tc_gemm_workspace(p, k, ncol, gemm_prec));
  } else {
    nd.add((size_t)p * k * sizeof(float));  // G in binary32
    nd.add(gemm_simt_workspace(p, k, ncol, gemm_prec == MSK_GEMM_F64));
    if (gemm_prec == MSK_GEMM_F64 && oz_applicable(p, k, ncol))
      return std::max(nd.used, oz_gemm_workspace(p, k, ncol));
  }
  return nd.used;
}

int msk_gemm(uint64_t seed, int64_t p, int64_t k, int64_t ncol, const void* Y, int64_t ldy,
             int gemm_prec, double* Z, int64_t ldz, void* ws, size_t ws_bytes, void* stream) {
  StageRange nvtx_range_("msk_gemm");
  if (p < 1 || p >= (1LL << 24)) return -2;
  if (k < 1) return -3;
  if (ncol < 1) return -4;
  if (!Y) return -5;
  if (ldy < ncol) return -6;
  if (gemm_prec < MSK_GEMM_F64 || gemm_prec > MSK_GEMM_BF16X3) return -7;
  if (!Z) return -8;
  if (ldz < p) return -9;
  if (ws_bytes < msk_gemm_workspace(p, k, ncol, gemm_prec)) return MSK_ENOMEM;
  const int y_dtype = gemm_prec == MSK_GEMM_F64 ? MSK_F64 : MSK_F32;
  return gemm_stage(seed, p, k, ncol, Y, y_dtype, ldy, gemm_prec, Z, ldz, ws, ws_bytes,
                    as_stream(stream));
}

size_t msk_ms_workspace(int64_t d, int64_t n, int with_b, int64_t k, int64_t p, int dtype,
                        int gemm_prec, int strategy) {
  const int64_t ncol = n + (with_b ? 1 : 0);
  const int ydt = ms_y_dtype(dtype, gemm_prec);
  Need nd;
  nd.add((size_t)k * ws_ldy(ncol, ydt) * dtype_size(ydt));  // Y
  nd.add(msk_cs_workspace(d, n, k, ydt, strategy));
  nd.add(msk_gemm_workspace(p, k, ncol, gemm_prec));
  return nd.used;
}

int ms_sketch(const void* A, int dtype, int64_t d, int64_t n, int64_t lda, const double* b,
              int64_t k, int64_t p, uint64_t seed, int gemm_prec, void* Z, int64_t ldz,
              int strategy, void* ws, size_t ws_bytes, void* stream) {
  StageRange nvtx_range_("ms_sketch");
  if (!A && d > 0 && n > 0) return -1;
  if (dtype != MSK_F64 && dtype != MSK_F32) return -2;
  if (d < 0) return -3;
  if (n < 0) return -4;
  if (lda < (d > 1 ? d : 1)) return -5;
  if (k < 1 || k > 0xFFFFFFFFLL) return -7;
  if (p < 1 || p >= (1LL << 24)) return -8;
  if (gemm_prec < MSK_GEMM_F64 || gemm_prec > MSK_GEMM_BF16X3) return -10;
  if (!Z) return -11;
  if (ldz < p) return -12;
  if (strategy != MSK_CS_ATOMIC && strategy != MSK_CS_SORTED) return -13;
  const int64_t ncol = n + (b ? 1 : 0);
  if (ncol < 1) return -4;
  if (ws_bytes < msk_ms_workspace(d, n, b ? 1 : 0, k, p, dtype, gemm_prec, strategy))
    return MSK_ENOMEM;
  // The tensor-core paths take an FP32 CountSketch (dtype F32).
  if (is_tensor_prec(gemm_prec) && dtype != MSK_F32) return MSK_ENOTSUP;
  cudaStream_t st = as_stream(stream);
  Carve cv(ws, ws_bytes);
  const int ydt = ms_y_dtype(dtype, gemm_prec);
  const int64_t ldy = ws_ldy(ncol, ydt);
  void* Y = cv.take((size_t)k * ldy * dtype_size(ydt));
  const size_t cs_ws = msk_cs_workspace(d, n, k, ydt, strategy);
  void* csw = cv.take(cs_ws);
  if (!Y) return MSK_ENOMEM;
  if (ydt == MSK_F64 && dtype == MSK_F32 && strategy != MSK_CS_ATOMIC) return MSK_ENOTSUP;
  const size_t rest_off = align_up(cv.used, 256);
  // The sliced FP64 stage's G slices depend on the seed only: with the knob
  // "ms.overlap_gauss" they are sampled on a side stream while the
  // CountSketch runs (the CountSketch is bound by L2 reductions, the sampler
  // by the SMs' issue slots).  Measured at 4194304 x 64: the step 0.552 ->
  // 0.546 ms, but the CountSketch itself 0.470 -> 0.485 ms (it shares the
  // SMs), so it is off by default.
  const bool fork = tune_get("ms.overlap_gauss", 0) != 0 &&
                    gemm_stage_sliced(p, k, ncol, ydt, gemm_prec, ws_bytes - rest_off) && d > 0;
  SideStream* side = nullptr;
  if (fork) {
    int rc = side_stream(&side);
    if (rc) return rc;
    MSK_CUDA(cudaEventRecord(side->fork, st));
    MSK_CUDA(cudaStreamWaitEvent(side->s, side->fork, 0));
    rc = launch_oz_prepare_g(stream_key(seed, kTagGauss), p, k, ncol, cv.base + rest_off, ws_bytes - rest_off,
                             side->s);
    if (rc) return rc;
    MSK_CUDA(cudaEventRecord(side->join, side->s));
  }
  StageEvents& sev = stage_events();
  if (sev.before_cs) MSK_CUDA(cudaEventRecord(sev.before_cs, st));
  int rc = MSK_OK;
  if (ydt == MSK_F64 && dtype == MSK_F32) {
    // FP64 sketch of the FP32-stored A
    rc = count_sketch_f64y(A, dtype, d, n, lda, b, k, seed, static_cast<double*>(Y), ldy, st);
  } else {
    rc = cs_sketch_internal(A, dtype, d, n, lda, b, k, seed, Y, ldy, strategy, csw, cs_ws, true,
                            st);
  }
  if (sev.after_cs) MSK_CUDA(cudaEventRecord(sev.after_cs, st));
  sev = StageEvents{};
  if (fork) MSK_CUDA(cudaStreamWaitEvent(st, side->join, 0));  // joined before any return
  if (rc) return rc;
  return gemm_stage(seed, p, k, ncol, Y, ydt, ldy, gemm_prec, static_cast<double*>(Z), ldz,
                    cv.base + rest_off, ws_bytes - rest_off, st, fork);
}

int ms_sketch_rows(const void* A, int dtype, int64_t d, int64_t n, int64_t lda, const double* b,
                   int64_t row0, int64_t k, int64_t p, uint64_t seed, int gemm_prec, double* Z,
                   int64_t ldz, void* ws, size_t ws_bytes, void* stream) {
  StageRange nvtx_range_("ms_sketch_rows");
  if (!A && d > 0 && n > 0) return -1;
  if (dtype != MSK_F64 && dtype != MSK_F32) return -2;
  if (d < 0) return -3;
  if (n < 0) return -4;
  if (lda < (d > 1 ? d : 1)) return -5;
  if (row0 < 0) return -7;
  if (k < 1 || k > 0xFFFFFFFFLL) return -8;
  if (p < 1 || p >= (1LL << 24)) return -9;
  if (gemm_prec < MSK_GEMM_F64 || gemm_prec > MSK_GEMM_BF16X3) return -11;
  if (!Z) return -12;
  if (ldz < p) return -13;
  const int64_t ncol = n + (b ? 1 : 0);
  if (ncol < 1) return -4;
  if (ws_bytes < msk_ms_workspace(d, n, b ? 1 : 0, k, p, dtype, gemm_prec, MSK_CS_ATOMIC))
    return MSK_ENOMEM;
  if (is_tensor_prec(gemm_prec) && dtype != MSK_F32) return MSK_ENOTSUP;
  cudaStream_t st = as_stream(stream);
  Carve cv(ws, ws_bytes);
  const int ydt = ms_y_dtype(dtype, gemm_prec);
  const int64_t ldy = ws_ldy(ncol, ydt);
  void* Y = cv.take((size_t)k * ldy * dtype_size(ydt));
  const size_t cs_ws = msk_cs_workspace(d, n, k, ydt, MSK_CS_ATOMIC);
  void* csw = cv.take(cs_ws);
  if (!Y) return MSK_ENOMEM;
  int rc;
  if (ydt == MSK_F64 && dtype == MSK_F32)
    rc = count_sketch_f64y(A, dtype, d, n, lda, b, k, seed, static_cast<double*>(Y), ldy, st, true,
                           row0);
  else
    rc = launch_cs_atomic(A, dtype, d, n, lda, b, (uint32_t)k, stream_key(seed, kTagHash), Y, ldy,
                          true, st, csw, cs_ws, true, row0);
  if (rc) return rc;
  const size_t rest_off = align_up(cv.used, 256);
  return gemm_stage(seed, p, k, ncol, Y, ydt, ldy, gemm_prec, Z, ldz, cv.base + rest_off,
                    ws_bytes - rest_off, st);
}

// Rows per staged block of ms_sketch_host: the caller's value, else blocks of
// about 256 MiB of A.
static int64_t host_chunk_rows(int64_t d, int64_t n, int dtype, int64_t chunk_rows) {
  if (chunk_rows > 0) return std::min<int64_t>(chunk_rows, std::max<int64_t>(d, 1));
  const int64_t esz = dtype == MSK_F64 ? 8 : 4;
  const int64_t rows = ((int64_t)256 << 20) / (std::max<int64_t>(n, 1) * esz);
  return std::max<int64_t>(1, std::min<int64_t>(std::max<int64_t>(d, 1), rows / 256 * 256));
}

size_t msk_ms_host_workspace(int64_t d, int64_t n, int with_b, int64_t k, int64_t p, int dtype,
                             int gemm_prec, int64_t chunk_rows) {
  const int64_t ncol = n + (with_b ? 1 : 0);
  const int64_t rows = host_chunk_rows(d, n, dtype, chunk_rows);
  const int ydt = ms_y_dtype(dtype, gemm_prec);
  Need nd;
  nd.add((size_t)k * ws_ldy(ncol, ydt) * dtype_size(ydt));  // Y
  nd.add(msk_cs_workspace(rows, n, k, ydt, MSK_CS_ATOMIC));  // replicas
  for (int j = 0; j < 2; ++j) {
    nd.add((size_t)rows * std::max<int64_t>(n, 1) * dtype_size(dtype));  // staged A rows
    if (with_b) nd.add((size_t)rows * sizeof(double));                    // staged b rows
  }
  nd.add((size_t)p * ncol * sizeof(double));  // Z on the device
  nd.add(msk_gemm_workspace(p, k, ncol, gemm_prec));
  return nd.used;
}

int ms_sketch_host(const void* A, int dtype, int64_t d, int64_t n, int64_t lda, const double* b,
                   int64_t k, int64_t p, uint64_t seed, int gemm_prec, double* Z, int64_t ldz,
                   int64_t chunk_rows, void* ws, size_t ws_bytes, void* stream) {
  StageRange nvtx_range_("ms_sketch_host");
  if (!A && d > 0 && n > 0) return -1;
  if (dtype != MSK_F64 && dtype != MSK_F32) return -2;
  if (d < 0) return -3;
  if (n < 0) return -4;
  if (lda < (d > 1 ? d : 1)) return -5;
  if (k < 1 || k > 0xFFFFFFFFLL) return -7;
  if (p < 1 || p >= (1LL << 24)) return -8;
  if (gemm_prec < MSK_GEMM_F64 || gemm_prec > MSK_GEMM_BF16X3) return -10;
  if (!Z) return -11;
  if (ldz < p) return -12;
  if (chunk_rows < 0) return -13;
  const int64_t ncol = n + (b ? 1 : 0);
  if (ncol < 1) return -4;
  if (ws_bytes < msk_ms_host_workspace(d, n, b ? 1 : 0, k, p, dtype, gemm_prec, chunk_rows))
    return MSK_ENOMEM;
  if (is_tensor_prec(gemm_prec) && dtype != MSK_F32) return MSK_ENOTSUP;
  cudaStream_t st = as_stream(stream);
  const int64_t rows = host_chunk_rows(d, n, dtype, chunk_rows);
  const int ydt = ms_y_dtype(dtype, gemm_prec);
  const int64_t ldy = ws_ldy(ncol, ydt);
  const size_t esz = dtype_size(dtype);
  Carve cv(ws, ws_bytes);
  void* Y = cv.take((size_t)k * ldy * dtype_size(ydt));
  const size_t cs_ws = msk_cs_workspace(rows, n, k, ydt, MSK_CS_ATOMIC);
  void* csw = cv.take(cs_ws);
  void* sa[2];
  double* sb[2] = {nullptr, nullptr};
  for (int j = 0; j < 2; ++j) {
    sa[j] = cv.take((size_t)rows * std::max<int64_t>(n, 1) * esz);
    if (b) sb[j] = static_cast<double*>(cv.take((size_t)rows * sizeof(double)));
  }
  double* Zd = static_cast<double*>(cv.take((size_t)p * ncol * sizeof(double)));
  if (!Y || !sa[0] || !sa[1] || (b && (!sb[0] || !sb[1])) || !Zd) return MSK_ENOMEM;
  // a copy stream and five events per host thread: block j of the rows is
  // copied into staging buffer j & 1 while block j - 1 is sketched on `st`
  // (a second copy stream for alternate blocks measured no faster: the
  // host link, ~200 GB/s, is the bound)
  // (kept per device: streams and events belong to the device current when
  // they were created)
  struct HostStreamSet {
    cudaStream_t cps = nullptr;
    cudaEvent_t ev[5];
  };
  constexpr int kMaxDevices = 64;
  thread_local HostStreamSet sets[kMaxDevices];
  int dev = 0;
  MSK_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return MSK_ENOTSUP;
  HostStreamSet& hs = sets[dev];
  if (!hs.cps) {
    MSK_CUDA(cudaStreamCreateWithFlags(&hs.cps, cudaStreamNonBlocking));
    for (auto& e : hs.ev) MSK_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  cudaStream_t cps = hs.cps;
  cudaEvent_t* ev = hs.ev;
  cudaEvent_t* ready = ev;      // ready[j]: block in buffer j copied
  cudaEvent_t* done = ev + 2;   // done[j]: buffer j's block sketched
  cudaEvent_t start = ev[4];    // earlier work on `st` (the caller's use of ws) finished
  MSK_CUDA(cudaEventRecord(start, st));
  MSK_CUDA(cudaStreamWaitEvent(cps, start, 0));
  MSK_CUDA(zero_rows(Y, ldy, ncol, k, dtype_size(ydt), st));
  const uint64_t key = stream_key(seed, kTagHash);
  const int64_t nblk = d > 0 ? (d + rows - 1) / rows : 0;
  for (int64_t j = 0; j < nblk; ++j) {
    const int u = (int)(j & 1);
    const int64_t r0 = j * rows, m = std::min<int64_t>(rows, d - r0);
    if (j >= 2) MSK_CUDA(cudaStreamWaitEvent(cps, done[u], 0));
    if (n > 0)
      MSK_CUDA(cudaMemcpy2DAsync(sa[u], (size_t)rows * esz,
                                 static_cast<const char*>(A) + (size_t)r0 * esz, (size_t)lda * esz,
                                 (size_t)m * esz, (size_t)n, cudaMemcpyHostToDevice, cps));
    if (b)
      MSK_CUDA(cudaMemcpyAsync(sb[u], b + r0, (size_t)m * sizeof(double), cudaMemcpyHostToDevice,
                               cps));
    MSK_CUDA(cudaEventRecord(ready[u], cps));
    MSK_CUDA(cudaStreamWaitEvent(st, ready[u], 0));
    int rc;
    if (ydt == MSK_F64 && dtype == MSK_F32)
      rc = count_sketch_f64y(sa[u], dtype, m, n, rows, sb[u], k, seed, static_cast<double*>(Y), ldy,
                             st, false, r0);
    else
      rc = launch_cs_atomic(sa[u], dtype, m, n, rows, sb[u], (uint32_t)k, key, Y, ldy, true, st, csw,
                            cs_ws, false, r0);
    if (rc) return rc;
    MSK_CUDA(cudaEventRecord(done[u], st));
  }
  const size_t rest_off = align_up(cv.used, 256);
  int rc = gemm_stage(seed, p, k, ncol, Y, ydt, ldy, gemm_prec, Zd, p, cv.base + rest_off,
                      ws_bytes - rest_off, st);
  if (rc) return rc;
  MSK_CUDA(cudaMemcpy2DAsync(Z, (size_t)ldz * sizeof(double), Zd, (size_t)p * sizeof(double),
                             (size_t)p * sizeof(double), (size_t)ncol, cudaMemcpyDeviceToHost, st));
  MSK_CUDA(cudaStreamSynchronize(st));
  return MSK_OK;
}

}  // extern "C"
