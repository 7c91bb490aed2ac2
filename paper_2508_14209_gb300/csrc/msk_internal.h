// msk_internal.h — host-side internals of libmsketch shared by the .cu files:
// status propagation, stream casts, workspace carving, launch declarations.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstddef>
#include <cstdint>

#include "../../include/msketch.h"

namespace msk {

// Records the CUDA error text for msk_last_error() and returns MSK_ECUDA.
int cuda_fail(cudaError_t e, const char* where);
// Records a plain message for msk_last_error().
void set_error_text(const char* msg);

#define MSK_CUDA(call)                                  \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return ::msk::cuda_fail(e_, #call); \
  } while (0)

#define MSK_CHECK_LAUNCH(where)                         \
  do {                                                  \
    cudaError_t e_ = cudaGetLastError();                \
    if (e_ != cudaSuccess) return ::msk::cuda_fail(e_, where); \
  } while (0)

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Named host range around an entry point or stage, for profilers that read
// NVTX (header-only; nothing happens unless such a tool is attached).
struct StageRange {
  explicit StageRange(const char* name) { nvtxRangePushA(name); }
  ~StageRange() { nvtxRangePop(); }
  StageRange(const StageRange&) = delete;
  StageRange& operator=(const StageRange&) = delete;
};

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Bump allocator over the caller's workspace (256-byte aligned pieces).
struct Carve {
  char* base;
  size_t cap;
  size_t used = 0;
  Carve(void* b, size_t c) : base(static_cast<char*>(b)), cap(c) {}
  // Returns nullptr when the piece does not fit (or base is null).
  void* take(size_t bytes) {
    size_t off = align_up(used, 256);
    if (bytes == 0) return base ? base + off : nullptr;
    if (!base || off + bytes > cap) return nullptr;
    used = off + bytes;
    return base + off;
  }
};
// Size accounting twin of Carve.
struct Need {
  size_t used = 0;
  void add(size_t bytes) { used = align_up(used, 256) + bytes; }
};

int num_sms();
// Zero the first `ncol` elements (esz bytes each) of k rows of pitch ldy
// elements: one contiguous memset when the rows are packed (ldy == ncol),
// a 2D memset otherwise.
cudaError_t zero_rows(void* Y, int64_t ldy, int64_t ncol, int64_t k, size_t esz, cudaStream_t st);
// Opt-in shared-memory limit per block of the current device (bytes).
int smem_optin_max();
// Allow `func` all the dynamic shared memory the device offers next to its
// static shared memory.  The value is the same for every caller, so
// concurrent launches from several host threads cannot race on it (occupancy
// follows the size passed at launch).
cudaError_t allow_max_smem(const void* func);
#define MSK_ALLOW_SMEM(kern) \
  MSK_CUDA(::msk::allow_max_smem(reinterpret_cast<const void*>(kern)))

// One CountSketch launch's problem: rows [0, d) of the A columns
// [c0, c0 + ncol_a) (A points at column c0) plus the optional b column,
// accumulated into Y (row-major, ldy; Y points at column c0).
template <typename T>
struct CsParams {
  const T* A;
  int64_t d, lda;
  int ncol_a;          // columns taken from A in this launch
  const double* b;     // extra column (after the A columns) or null
  int ncol;            // ncol_a + (b != null)
  uint32_t k;
  uint64_t key;
  T* Y;
  int64_t ldy;
  int pitch;           // shared-memory row pitch (elements)
  int64_t i0;          // hash index of row 0 (a row block of a taller A), 0 by default
};

// Tuning registry lookup (tune.cpp).
long long tune_get(const char* name, long long dflt);

// ---- kernels launched across translation units -------------------------
// countsketch.cu
int launch_cs_hash(uint64_t key, int64_t i0, int64_t count, uint32_t k, uint32_t* h,
                   int8_t* s, cudaStream_t st);
// pad_ok: the column after the last one of each Y row is scratch (ldy > ncol)
// and may receive +0.0 from a padded bulk reduction.
// ws (optional): room for the replicas of Y of the narrow FP64 kernels
// (cs_replica_bytes); without it those kernels add into Y directly.
// zero = false: add into Y as it is (a further row block); i0: hash index of
// A's row 0 (the row block's offset in the full matrix).
int launch_cs_atomic(const void* A, int dtype, int64_t d, int64_t n, int64_t lda,
                     const double* b, uint32_t k, uint64_t key, void* Y, int64_t ldy,
                     bool pad_ok, cudaStream_t st, void* ws = nullptr, size_t ws_bytes = 0,
                     bool zero = true, int64_t i0 = 0);
// Bytes of the replicas of Y the FP64 CountSketch of `ncol` columns uses (0: none).
size_t cs_replica_bytes(int64_t k, int64_t ncol);
// Internal CountSketch launch used by the multisketch (same checks as cs_sketch).
int cs_sketch_internal(const void* A, int dtype, int64_t d, int64_t n, int64_t lda,
                       const double* b, int64_t k, uint64_t seed, void* Y, int64_t ldy,
                       int strategy, void* ws, size_t ws_bytes, bool pad_ok, cudaStream_t st);
size_t cs_sorted_workspace(int64_t d, int64_t k);
int launch_cs_sorted(const void* A, int dtype, int64_t d, int64_t n, int64_t lda,
                     const double* b, uint32_t k, uint64_t key, void* Y, int64_t ldy,
                     void* ws, size_t ws_bytes, cudaStream_t st);
// gaussian.cu
int launch_gaussian(uint64_t key, int64_t p, int64_t k, int out_prec, void* G, int64_t ldg,
                    cudaStream_t st);
// gemm_simt.cu
size_t gemm_simt_workspace(int64_t p, int64_t k, int64_t ncol, bool f64);
int launch_gemm_simt(const float* G, int64_t ldg, const void* Y, bool y_f64, int64_t ldy, bool f64,
                     int64_t p, int64_t k, int64_t ncol, double* Z, int64_t ldz, void* ws,
                     size_t ws_bytes, cudaStream_t st);

// Z[r + c*ldz] = sum_s part[s][c*p + r] (FP64 partials, fixed order).
__global__ void splitk_reduce_kernel(const double* __restrict__ part, int S, int64_t p, int64_t ncol,
                                     double* __restrict__ Z, int64_t ldz);
// countsketch.cu: FP64 CountSketch of FP32 A (column chunks of <= maxc <= 256)
// (i0: hash index of A's row 0; Y is not zeroed here)
int launch_cs_f32a_f64y(const float* A, int64_t d, int64_t n, int64_t lda, const double* b,
                        uint32_t k, uint64_t key, double* Y, int64_t ldy, int64_t maxc,
                        cudaStream_t st, int64_t i0 = 0);
// countsketch.cu: batched FP32 CountSketch (problems of one A width + b)
int launch_cs_batch_f32(int nca, const CsParams<float>* Ps, const int64_t* tile_begin, int nprob,
                        int64_t total_tiles, cudaStream_t st);
// gemm_tc.cu: one problem of the batched draining BF16x3 GEMM.
struct alignas(64) TcJob {
  CUtensorMap mapA;  // G, 2D {k, p}
  CUtensorMap mapB;  // Yt parts, 3D {k, npad, 3}
  double* part;      // S x p x ncol FP64 partials
  int p, ncol, NT, KT, kt_per, Mt, Nt, S;
  uint32_t idesc;
  int item_begin;    // first work item (CTA) of this job
};
struct TcShape {
  int npad, NT, Nt, Mt, KT, kt_per, S, items;
  int64_t kpitch;
};
void tc_ds_shape(int64_t p, int64_t k, int64_t ncol, int kt_per, TcShape* s);
int tc_ds_make_job(int64_t p, int64_t k, int64_t ncol, const TcShape& s, const void* G,
                   const void* Yt, double* part, int item_begin, TcJob* job);
int launch_tc_ds_batch(const TcJob* jobs, int njobs, int total_items, int max_nt, cudaStream_t st);
int tc_take_timeout(cudaStream_t st);
// Device address of that flag (for the tensor-core kernels of other files).
int tc_timeout_flag(int** out);
int launch_tc_wait_selftest(cudaStream_t st);
// gemm_tc.cu (tcgen05 tensor-core Gaussian stage)
size_t tc_gemm_workspace(int64_t p, int64_t k, int64_t ncol, int prec);
int launch_tc_gemm(uint64_t gkey, int64_t p, int64_t k, int64_t ncol, const float* Y, int64_t ldy,
                   int prec, double* Z, int64_t ldz, void* ws, size_t ws_bytes, cudaStream_t st);
// gemm_oz.cu (FP64 Gaussian stage on the tensor cores by exact 8-bit slicing)
bool oz_applicable(int64_t p, int64_t k, int64_t ncol);
size_t oz_gemm_workspace(int64_t p, int64_t k, int64_t ncol);
// g_ready: a launch_oz_prepare_g with the same sizes and workspace already
// wrote G's slices (ordered before this call's kernels).
int launch_oz_gemm(uint64_t gkey, int64_t p, int64_t k, int64_t ncol, const double* Y, int64_t ldy,
                   double* Z, int64_t ldz, void* ws, size_t ws_bytes, cudaStream_t st,
                   bool g_ready = false);
// G's slices alone: the part of the sliced stage that depends on the seed only.
int launch_oz_prepare_g(uint64_t gkey, int64_t p, int64_t k, int64_t ncol, void* ws, size_t ws_bytes,
                        cudaStream_t st);
// qr.cu
int launch_householder_qr(double* W, int64_t m, int64_t c, int64_t ldw, cudaStream_t st);
// Whether the cluster QR of an m x c matrix on CL CTAs runs its flow form.
bool qr_use_flow(int64_t m, int64_t c, int CL);
int launch_trsv_upper(const double* R, int64_t n, int64_t ldr, const double* rhs, double* x,
                      int* status, bool transposed, cudaStream_t st);
int launch_cholesky(double* Gm, int64_t n, int64_t ldg, double* R, int64_t ldr, int* status,
                    cudaStream_t st);
int first_zero_pivot(const double* R, int64_t n, int64_t ldr, cudaStream_t st);
// countsketch.cu: counting sort of counter draws by bucket
int launch_draw_bucket_sort(uint64_t key, int64_t count, uint32_t nb, uint32_t* offs,
                            uint32_t* perm, uint32_t* cnt, uint32_t* cursor, cudaStream_t st);
// srht.cu (subsampled randomized Hadamard transform, Section 5)
size_t srht_workspace(int64_t d, int64_t ncol, int64_t k);
int launch_srht(const void* A, int dtype, int64_t d, int64_t n, int64_t lda, const double* b,
                int64_t k, uint64_t seed, double* Y, int64_t ldy, void* ws, size_t ws_bytes,
                cudaStream_t st);
// rcq.cu (randomized Cholesky QR's tall product and small triangular product)
size_t trmm_upper_smem(int64_t n);
int launch_trmm_upper(const void* X, int dtype, int64_t ldx, int64_t d, int64_t n, const double* U,
                      double* Y, int64_t ldy, cudaStream_t st);
int launch_tri_mul_upper(const double* R1, int64_t ld1, const double* R0, int64_t ld0, int64_t n,
                         double* R, int64_t ldr, cudaStream_t st);
// gemm_simt.cu: Gaussian-only sketch Z = G [A b] (G p x d generated in place)
size_t gauss_gemm_workspace(int64_t p, int64_t d, int64_t ncol);
int launch_gauss_gemm(uint64_t gkey, int64_t p, const void* A, int dtype, int64_t d, int64_t n,
                      int64_t lda, const double* b, double* Z, int64_t ldz, void* ws,
                      size_t ws_bytes, cudaStream_t st);
// api.cu
// FP64 CountSketch of [A b] (FP64 A, or FP32 A widened exactly) into
// row-major Y (k x ncol, ldy), atomic strategy; Y is zeroed first.
// zero = false: add into Y as it is; i0: hash index of A's row 0.
int count_sketch_f64y(const void* A, int dtype, int64_t d, int64_t n, int64_t lda,
                      const double* b, int64_t k, uint64_t seed, double* Y, int64_t ldy,
                      cudaStream_t st, bool zero = true, int64_t i0 = 0);
int gemm_stage(uint64_t seed, int64_t p, int64_t k, int64_t ncol, const void* Y, int y_dtype,
               int64_t ldy, int gemm_prec, double* Z, int64_t ldz, void* ws, size_t ws_bytes,
               cudaStream_t st, bool g_ready = false);
// Whether gemm_stage takes the sliced FP64 path for these arguments.
bool gemm_stage_sliced(int64_t p, int64_t k, int64_t ncol, int y_dtype, int gemm_prec, size_t ws_bytes);

}  // namespace msk
