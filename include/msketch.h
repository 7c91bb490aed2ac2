/*
 * msketch.h — C ABI of libmsketch: GPU CountSketch, Count-Gauss multisketch
 * and sketched least squares on one GB300 (sm_103a).
 *
 * The operations follow "A High Performance GPU CountSketch Implementation
 * and Its Application to Multisketching and Least Squares Problems"
 * (Higgins, Boman, Yamazaki, arXiv 2508.14209):
 *   - CountSketch, Definition 3 and its row form (Section 4), applied by a
 *     signed scatter-add of rows as in Algorithm 2;
 *   - the multisketch S2 (S1 x) with S1 a CountSketch and S2 a Gaussian
 *     sketch ("Count-Gauss", Section 1, Section 6.2);
 *   - sketch-and-solve least squares, Algorithm 1 (Section 2), with the
 *     Householder-QR solve of Section 6.1;
 *   - the normal-equations baseline of Section 6.3 (Gram matrix, Cholesky,
 *     two triangular solves).
 * The random sketch entries are not stored (Section 8 names an on-the-fly
 * hashed CountSketch as future work): bucket and sign of row i, and every
 * Gaussian entry, are recomputed from a 64-bit seed by a splitmix64 counter
 * generator, defined below, so that any party can regenerate them.
 *
 * Conventions for every entry point
 *   - Matrices are dense with a leading dimension.  A and Z are column-major;
 *     the CountSketch output Y is row-major (bucket-major, the layout in
 *     which Algorithm 2 accumulates rows, Section 6.1).
 *   - Array arguments are DEVICE pointers owned by the caller unless marked
 *     "host".  The library never allocates device memory: scratch space is
 *     the caller's `ws` buffer, sized by the matching *_workspace() query
 *     (ws may be NULL when the query returns 0).  ws must be 256-byte aligned.
 *   - Work is enqueued on `stream` (a cudaStream_t passed as void*; NULL is
 *     the legacy default stream) and is asynchronous, except where an entry
 *     point says it synchronises the stream to fill a host-side result.
 *   - Return value: MSK_OK (0); -i when argument i (1-based) is invalid;
 *     a positive MSK_E* code below; or, for numerical breakdown, the
 *     positive value documented at the entry point.
 *   - No entry point falls back to the CPU.
 *
 * Counter generator (splitmix64, Steele, Lea and Flood, OOPSLA 2014):
 *   mix(z):  z ^= z>>30; z *= 0xBF58476D1CE4E5B9; z ^= z>>27;
 *            z *= 0x94D049BB133111EB; z ^= z>>31
 *   key(seed, tag) = mix(seed ^ (tag * 0xD1B54A32D192ED03))
 *   draw(key, i)   = mix(key + (i+1) * 0x9E3779B97F4A7C15)   (mod 2^64)
 *   CountSketch (tag 0): z = draw(key(seed,0), i) for 0-based row i;
 *     bucket h(i) = ((z >> 32) * k) >> 32,  sign s(i) = (z & 1) ? -1 : +1.
 *   Gaussian (tag 2): entry (r, c) of the p x k matrix G is number r*k + c of
 *     the polar-method sampler in binary32 (attempt a uses draw index
 *     (r*k+c)*2^16 + a; U = z>>40, V = (z>>16) & 0xFFFFFF,
 *     u = (2U+1-2^24)*2^-24, v likewise; accept s = u*u+v*v < 1; result
 *     u*sqrt(-2*ln(s)/s) with ln(m*2^e) = e*ln2 + 2t(1 + t^2/3 + t^4/5 +
 *     t^6/7 + t^8/9), t = (m-1)/(m+1), m in [sqrt(1/2), sqrt(2)); every step
 *     one round-to-nearest binary32 operation), divided by sqrt(p) so the
 *     entries are N(0, 1/p).
 */
#ifndef MSKETCH_H
#define MSKETCH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Element type of A (and of the CountSketch output Y). */
typedef enum { MSK_F64 = 0, MSK_F32 = 1 } msk_dtype;

/* Arithmetic of the Gaussian stage Z = G Y.
 *   F64    : G widened exactly from binary32, FP64 multiply-add (CUDA cores).
 *   F32    : G and Y in binary32, FP32 multiply-add (CUDA cores).
 *   BF16   : G and Y rounded to bfloat16, tensor cores (tcgen05), FP32 accum.
 *   F16    : G and Y rounded to binary16, tensor cores, FP32 accumulation.
 *   BF16X3 : G rounded to bfloat16; Y split exactly into Y1+Y2+Y3 bfloat16
 *            parts (Henry, Tang, Heinecke, ARITH 2019); the three products
 *            accumulate in one FP32 tensor-memory accumulator.  Keeps Z at
 *            FP32 accuracy, which the least-squares preconditioner needs. */
typedef enum {
  MSK_GEMM_F64 = 0,
  MSK_GEMM_F32 = 1,
  MSK_GEMM_BF16 = 2,
  MSK_GEMM_F16 = 3,
  MSK_GEMM_BF16X3 = 4
} msk_gemm_prec;

/* CountSketch strategy.
 *   ATOMIC : rows streamed once, each added to its bucket row by L2
 *            reductions (Algorithm 2's atomics, coalesced per row).
 *   SORTED : rows grouped by bucket (counting sort on h(i), each bucket's
 *            rows in increasing order), then each bucket summed in
 *            increasing row order: deterministic, bitwise reproducible. */
typedef enum { MSK_CS_ATOMIC = 0, MSK_CS_SORTED = 1 } msk_cs_strategy;

/* Sketch of a sketch-and-solve (Section 6.3 compares the three):
 *   MULTI : S = G C, CountSketch C to k rows then Gaussian G to p rows;
 *   COUNT : S = C alone (k rows; the QR is of a k x (n+1) matrix);
 *   GAUSS : S = G alone, a p x d Gaussian with the entries of the
 *           multisketch's G at k = d (generated inside the product). */
typedef enum {
  MSK_SKETCH_MULTI = 0,
  MSK_SKETCH_COUNT = 1,
  MSK_SKETCH_GAUSS = 2,
  MSK_SKETCH_SRHT = 3 /* S = (1/sqrt(k)) P H D, k rows (d a power of two) */
} msk_sketch_kind;

#define MSK_OK 0
#define MSK_ENOCONV 1001  /* refinement stopped unconverged (x is returned) */
#define MSK_ENOMEM 1002   /* ws too small, or a request over the memory budget */
#define MSK_ETIMEOUT 1003 /* a bounded device wait gave up */
#define MSK_ECUDA 1004    /* a CUDA runtime call failed */
#define MSK_ENOTSUP 1005  /* unsupported combination (e.g. alignment) */
#define MSK_EBUSY 1006    /* server queue full */

/* Result summary of a least-squares solve (host struct). */
typedef struct {
  int32_t iters;      /* inner refinement iterations (= passes over A besides
                         the FP64 residual passes); 0 for plain SnS */
  int32_t converged;  /* 1 when the stopping test held */
  double relres;      /* ||b - A x|| / ||b|| of the returned x (FP64) */
  double relres_sns;  /* the same for the sketch-and-solve start x0 */
} msk_lstsq_info;

/* ---- Version / self description ---------------------------------------- */

/* Library version string (static storage). */
const char *msk_version(void);

/* Last CUDA error string seen by the library on this host thread (static
 * storage, empty when none). */
const char *msk_last_error(void);

/* Synchronises `stream` (a cudaStream_t, NULL = legacy default stream) and
 * reports whether a tensor-core Gaussian-stage kernel (the library's
 * mbarrier-pipelined kernels) gave up a bounded wait since the previous
 * call: MSK_ETIMEOUT (the results of that launch are not valid), else
 * MSK_OK.  Clears the record.  MSK_ECUDA if synchronising fails. */
int msk_take_timeout(void *stream);

/* Test hook for the bounded waits: launches one CTA whose thread waits, with
 * the pipelined kernels' bounded wait (1 s), on an mbarrier that nothing
 * arrives on; the wait expires and records a timeout that msk_take_timeout
 * then reports.  Returns the launch status (MSK_OK or MSK_ECUDA). */
int msk_selftest_wait(void *stream);

/* ---- Tuning registry (set by the autotuner, read by the launchers) ------- */

/* Named integer knobs that the launchers read (unset = launcher default):
 *   "cs.fixed"            1 = fixed-width CountSketch kernels (default), 0 = generic
 *   "cs.l2_budget_bytes"  bytes of Y a CountSketch column chunk keeps in L2
 *                         (default 2/5 of L2)
 *   "cs.f64.variant"      1 = FP64 CountSketch by TMA bulk reductions per row
 *   "cs.f64.prefetch"     FP64-output CountSketch loads the next tile during the
 *                         current one's reductions: 1 on, 0 off (default: on
 *                         from 128 columns up)
 *   "cs.f32.prefetch"     the same for the FP32 CountSketch (default: on at 128
 *                         columns only)
 *   "cs.f64.narrow"       0 = no narrow FP64 kernel for <= 32 columns (default on)
 *   "cs.f64.replicas"     0 = the narrow FP64 kernel adds into Y directly
 *                         (default: replicas from ws where they apply)
 *   "tc.drain"            0 = split-BF16 GEMM without draining accumulators
 *   "batch.kt_per"        K tiles per CTA of the batched tensor-core GEMM (16)
 *   "batch.round"         CG iterations per captured graph round (4)
 *   "pass.ctas_per_sm"    refinement-pass CTAs per SM (3, at most 3)
 * Process-wide and thread-safe; they change speed only, never results beyond
 * rounding order.  msk_autotune (below) sets them from measurements.
 * msk_tune_set returns -1 for an empty name; msk_tune_clear(NULL) clears all. */
int msk_tune_set(const char *name, long long value);
long long msk_tune_get(const char *name, long long dflt);
int msk_tune_clear(const char *name);

/* ---- Sketch randomness (test hooks) ------------------------------------ */

/* Bucket h(i) in [0, k) and sign s(i) in {-1, +1} of rows i0 .. i0+count-1,
 * from the counter generator above (Definition 3, Section 4; tag 0).
 *   h: device uint32[count]; s: device int8[count] (either may be NULL).
 * Errors: -3 count < 0, -4 k < 1 or k > 2^32-1. */
int cs_hash(uint64_t seed, int64_t i0, int64_t count, int64_t k, uint32_t *h,
            int8_t *s, void *stream);

/* The p x k Gaussian G of the multisketch's second stage (Section 1; N(0,1/p)
 * entries from the sampler above), written row-major with leading dimension
 * ldg >= k in the element type `out_prec`: MSK_GEMM_F64 (double),
 * MSK_GEMM_F32 (float), MSK_GEMM_BF16 (bfloat16, round-to-nearest-even of the
 * binary32 value), MSK_GEMM_F16 (binary16, likewise).
 * Errors: -2 p < 1, -3 k < 1, -4 bad out_prec, -6 ldg < k. */
int ms_gaussian(uint64_t seed, int64_t p, int64_t k, int out_prec, void *G,
                int64_t ldg, void *stream);

/* ---- CountSketch (Definition 3; Algorithm 2) --------------------------- */

/* Scratch bytes cs_sketch needs: for MSK_CS_SORTED the sort arrays; for
 * MSK_CS_ATOMIC with FP64 A, room for 8 or 16 replicas of Y when the sketch
 * has few 128-byte lines (k * ncol small, e.g. n = 16 at k = 512), else 0.
 * A smaller ws is allowed for MSK_CS_ATOMIC: the replicas are then skipped. */
size_t msk_cs_workspace(int64_t d, int64_t n, int64_t k, int dtype,
                        int strategy);

/* Y = S [A b]: the k x ncol CountSketch of the d x n matrix A, with the
 * optional column b appended (ncol = n + (b != NULL)), so that
 *   Y[m, j] = sum_{i : h(i) = m} s(i) [A b][i, j]       (Section 4).
 *   A : device, column-major d x n, leading dimension lda >= max(d,1), of
 *       type dtype (MSK_F64 double / MSK_F32 float); 16-byte aligned.
 *   b : device double[d] or NULL (rounded to float when dtype = MSK_F32).
 *   Y : device, row-major k x ncol, leading dimension ldy >= ncol, type dtype;
 *       overwritten (the kernel zeroes it first).  16-byte aligned.
 *   strategy : msk_cs_strategy; ws/ws_bytes : scratch (msk_cs_workspace).
 * Errors: -1 A NULL, -2 bad dtype, -3 d < 0, -4 n < 0, -5 lda < d,
 *   -7 k < 1, -9 Y NULL, -10 ldy < ncol, -11 bad strategy,
 *   MSK_ENOMEM ws too small, MSK_ENOTSUP d >= 2^31 for SORTED. */
int cs_sketch(const void *A, int dtype, int64_t d, int64_t n, int64_t lda,
              const double *b, int64_t k, uint64_t seed, void *Y, int64_t ldy,
              int strategy, void *ws, size_t ws_bytes, void *stream);

/* ---- Multisketch (Count-Gauss) ----------------------------------------- */

/* Scratch bytes ms_sketch needs for these sizes (ncol = n + with_b). */
size_t msk_ms_workspace(int64_t d, int64_t n, int with_b, int64_t k, int64_t p,
                        int dtype, int gemm_prec, int strategy);

/* Z = G (S [A b]): CountSketch to k rows, then the p x k Gaussian G
 * (Section 1 "Count-Gauss"; Section 6.2 uses k = 2n^2).  A, b, dtype, k,
 * seed, strategy as in cs_sketch; the Gaussian uses the same seed (tag 2).
 * With the FP64 Gaussian stage on the tensor cores (gemm_prec F64, k >=
 * 1024) and the tuning knob "ms.overlap_gauss" set, G's slices are sampled
 * on a library side stream while the CountSketch runs on `stream`, which
 * waits for them before the stage (the call stays ordered on `stream`, and
 * can be captured).
 *   gemm_prec : msk_gemm_prec, the arithmetic of Z = G Y.
 *   Z : device double, column-major p x ncol, leading dimension ldz >= p.
 * Errors: -1 A NULL (with d, n > 0), -2 bad dtype, -3 d < 0, -4 n < 0 or
 *   no column at all, -5 lda < d, -7 k < 1 or k >= 2^32, -8 p < 1 or
 *   p >= 2^24, -10 bad gemm_prec, -11 Z NULL, -12 ldz < p, -13 bad strategy,
 *   MSK_ENOMEM ws too small.  MSK_ENOTSUP in three cases only: a tensor-core
 *   gemm_prec (BF16, F16, BF16X3) with dtype MSK_F64 (those paths take the
 *   FP32 CountSketch); a tensor-core gemm_prec with ncol > 512; the sorted
 *   strategy for the FP64 sketch of FP32 A (gemm_prec F64 with dtype F32).
 *   Every other combination of dtype, gemm_prec and strategy is supported. */
int ms_sketch(const void *A, int dtype, int64_t d, int64_t n, int64_t lda,
              const double *b, int64_t k, int64_t p, uint64_t seed,
              int gemm_prec, void *Z, int64_t ldz, int strategy, void *ws,
              size_t ws_bytes, void *stream);

/* Profiling hook: the next ms_sketch call of the calling thread records
 * before_cs and after_cs (cudaEvent_t handles, or NULL) on its stream right
 * before and right after its CountSketch, so that the CountSketch's own time
 * can be read inside a timed loop of whole multisketch calls; the hook is
 * then cleared.  Always returns MSK_OK.  The paper has no counterpart. */
int msk_stage_events(void *before_cs, void *after_cs);

/* ms_sketch of a row block of a taller [A b] (Section 7's block-row
 * distribution): A, b hold rows row0 .. row0+d-1 of the full matrix, and
 * the CountSketch hashes them with their global indices, so the Z of the
 * blocks of a row partition add up to the Z of the whole matrix (up to the
 * order of the reductions).  Atomic strategy; workspace msk_ms_workspace.
 * Errors: -1 A NULL, -2 dtype, -3 d < 0, -4 n < 0, -5 lda < d, -7 row0 < 0,
 * -8 k < 1, -9 p < 1, -11 gemm_prec, -12 Z NULL, -13 ldz < p, MSK_ENOMEM,
 * MSK_ENOTSUP (tensor precisions need FP32 A). */
int ms_sketch_rows(const void *A, int dtype, int64_t d, int64_t n, int64_t lda,
                   const double *b, int64_t row0, int64_t k, int64_t p,
                   uint64_t seed, int gemm_prec, double *Z, int64_t ldz, void *ws,
                   size_t ws_bytes, void *stream);

/* Scratch bytes (device) ms_sketch_host needs; chunk_rows as there. */
size_t msk_ms_host_workspace(int64_t d, int64_t n, int with_b, int64_t k,
                             int64_t p, int dtype, int gemm_prec,
                             int64_t chunk_rows);

/* ms_sketch from HOST memory, streamed: A (host, column-major d x n, lda),
 * b (host double[d] or NULL) and Z (host double, column-major p x ncol,
 * ldz >= p) live on the host; only Y, two staging blocks of chunk_rows rows
 * and the Gaussian stage's scratch live on the device (ws), so d is not
 * limited by device memory.  Block j of the rows is copied (a second stream,
 * strided 2D copies) while block j-1 is CountSketched on `stream` with its
 * global row indices, which the CountSketch is additive over; then Z = G Y
 * and Z is copied back.  Same Z as ms_sketch (atomic strategy) up to the
 * order of the reductions.  A and b should be page-locked for the copies to
 * overlap the sketch.  chunk_rows = 0 picks blocks of about 256 MiB of A.
 * Synchronises `stream` before returning.
 * Errors as ms_sketch, plus -13 chunk_rows < 0. */
int ms_sketch_host(const void *A, int dtype, int64_t d, int64_t n, int64_t lda,
                   const double *b, int64_t k, int64_t p, uint64_t seed,
                   int gemm_prec, double *Z, int64_t ldz, int64_t chunk_rows,
                   void *ws, size_t ws_bytes, void *stream);

/* ---- Dense building blocks (Algorithm 1 steps 2-3) ----------------------- */

/* Scratch bytes msk_gemm needs. */
size_t msk_gemm_workspace(int64_t p, int64_t k, int64_t ncol, int gemm_prec);

/* Z = G Y with G the counter-generated p x k Gaussian of `seed` (generated
 * into ws) and Y given: the second stage of ms_sketch on its own.
 *   Y : device, row-major k x ncol (ldy), double when gemm_prec = F64, float
 *       otherwise; Z : device double column-major p x ncol (ldz). */
int msk_gemm(uint64_t seed, int64_t p, int64_t k, int64_t ncol, const void *Y,
             int64_t ldy, int gemm_prec, double *Z, int64_t ldz, void *ws,
             size_t ws_bytes, void *stream);

/* In-place Householder QR of the m x c column-major FP64 matrix W (ldw >= m,
 * m >= c): on return the upper triangle of W[0:c, 0:c] holds R with
 * R[j][j] = -sign(x_0) ||x|| (sign(0) = +1), the GeQRF step of Section 6.1;
 * the strictly lower part is overwritten with zeros.  One thread-block
 * cluster of up to 16 CTAs factors the matrix with the columns split across
 * the CTAs' shared memory (or, when they do not fit, in place in global
 * memory).  Limits: m < 2^31, c <= 512.
 * Errors: -2 m < c or m >= 2^31, -3 c < 1 or c > 512, -4 ldw < m. */
int msk_householder_qr(double *W, int64_t m, int64_t c, int64_t ldw,
                       void *stream);

/* Solve R x = rhs (upper triangular n x n, column-major, ldr; x may alias
 * rhs).  Returns j+1 (positive) on an exactly zero pivot R[j][j] — the value
 * is only known after the stream is synchronised, so this entry point
 * synchronises `stream`. */
int msk_trsv_upper(const double *R, int64_t n, int64_t ldr, const double *rhs,
                   double *x, void *stream);

/* ---- Checked builds ------------------------------------------------------ */

/* 1 when this library was built with device-side index checks (MSK_CHECKED:
 * CountSketch buckets, the sliced FP64 stage's fixed-point ranges, the batch
 * tables; a failed check skips the access and records its site), else 0.
 * The paper has no counterpart: this stands in for a memory checker. */
int msk_checked_build(void);

/* Synchronise `stream`; return and clear the site of the first failed index
 * check since the last call (1 CountSketch bucket, 2 fixed-point range of the
 * sliced FP64 stage, 3 batch tables), 0 when none failed (always 0 in builds
 * without checks), or MSK_ECUDA. */
int msk_check_status(void *stream);

/* Size of the fixed scratch array behind msk_gemm_noalloc (64 MiB). */
#define MSK_NOALLOC_SCRATCH_BYTES ((size_t)64 << 20)

/* msk_gemm without a caller workspace, for programs that may not allocate
 * device memory when they need the Gaussian stage (for instance a component
 * running under a host application whose allocator owns all device memory, or
 * a loop that cannot pay for the device-wide synchronisation an allocation can
 * cause).  The paper has no counterpart; this is a convenience of the library.
 *   Same arguments and result as msk_gemm, minus ws/ws_bytes.  The scratch (G
 *   or its slices, the slices of Y and the split-K partials) lives in one array of
 *   MSK_NOALLOC_SCRATCH_BYTES inside the library, reserved on every GPU that
 *   loads it until the process exits.  No device memory is allocated.
 *   The first call made on a device looks up the array's device address (once
 *   per device, with that device current); make that first call before any
 *   stream capture starts on the device.  A device reset (cudaDeviceReset)
 *   ends the context the address belongs to: the first call after it looks
 *   the address up again, and it too should come before any capture.
 *   All calls share the array and each call overwrites it: calls whose GPU
 *   work overlaps in time (e.g. on different streams) race and give wrong
 *   results; serialise them.  Nothing in the array needs to start at zero.
 * Errors: as msk_gemm; MSK_ENOMEM (with a message in msk_last_error) when
 *   msk_gemm_workspace(p, k, ncol, gemm_prec) exceeds the array. */
int msk_gemm_noalloc(uint64_t seed, int64_t p, int64_t k, int64_t ncol,
                     const void *Y, int64_t ldy, int gemm_prec, double *Z,
                     int64_t ldz, void *stream);

/* ---- Least squares -------------------------------------------------------- */

/* Scratch bytes ms_lstsq needs. */
size_t msk_lstsq_workspace(int64_t d, int64_t n, int64_t k, int64_t p,
                           int dtype, int gemm_prec, int refine);

/* Multisketched least squares min ||b - A x||.
 *   refine = 0 : sketch-and-solve, Algorithm 1: Z = G S [A b] (p x (n+1)),
 *     Householder QR of Z, x = R11^{-1} (Q^T z) with Q^T z = R[0:n, n].
 *   refine = 1 : then sketch-and-precondition refinement (the iterative
 *     route Section 6 cites, Blendenpik / LSRN).  Each outer step forms the
 *     residual r = b - A x and g = A^T r in FP64 (one pass over A), then runs
 *     conjugate gradients on A^T A d = g preconditioned by R11^T R11 (one pass
 *     over A per iteration; FP64 for FP64 A, double-single arithmetic on the
 *     FP32 units for FP32 A) until a step lowers ||r||^2 by no more than
 *     0.05 tol ||r||^2, and sets x += d.  Converged when the next FP64
 *     residual confirms the decrease the CG steps predicted (to tol ||r||^2),
 *     when the relative residual moves by at most tol * relres between outer
 *     steps, or when the first CG step already gains less than that floor;
 *     each test counts only within 4n inner iterations.  Stops unconverged
 *     when a test fires after more, or after max_iter outer steps.
 *   A : device column-major d x n (lda), dtype F64 or F32; b : device double[d].
 *   x : device double[n] (output).
 *   info : host msk_lstsq_info* or NULL; when non-NULL the stream is
 *     synchronised and relres fields are filled.
 * Returns MSK_OK; MSK_ENOCONV if refinement stopped unconverged; j+1 if R11 has an
 * exactly zero pivot at column j; negative for bad arguments (-1 A, -2 dtype,
 * -3 d < n, -4 n < 1, -5 lda, -6 b, -7 k < n+1, -8 p < n+1 or p > k,
 * -10 gemm_prec, -11 refine, -14 x, MSK_ENOMEM ws). */
int ms_lstsq(const void *A, int dtype, int64_t d, int64_t n, int64_t lda,
             const double *b, int64_t k, int64_t p, uint64_t seed,
             int gemm_prec, int refine, double tol, int32_t max_iter,
             double *x, msk_lstsq_info *info, void *ws, size_t ws_bytes,
             void *stream);

/* Scratch bytes ne_lstsq needs. */
size_t msk_ne_workspace(int64_t d, int64_t n);

/* Normal equations (Section 6.3): Gm = A^T A and y = A^T b in one FP64 pass,
 * Cholesky Gm = R^T R, x = R^{-1} (R^{-T} y).
 *   A : device double column-major d x n (lda); b : device double[d];
 *   x : device double[n].  Synchronises `stream` to read the Cholesky status.
 * Returns MSK_OK, or j+1 when pivot j of the Cholesky factorisation is not
 * positive (A^T A numerically not positive definite; x is then NaN). */
int ne_lstsq(const double *A, int64_t d, int64_t n, int64_t lda,
             const double *b, double *x, void *ws, size_t ws_bytes,
             void *stream);

/* ---- The refinement's operator (Section 6.3, preconditioned normal
 * equations): v = A^T (A p) for an FP32 A, as the conjugate-gradient steps of
 * ms_lstsq(refine = 1) and msk_batch_lstsq apply it. ------------------------ */

/* Scratch bytes of msk_normal_apply (0 for bad sizes). */
size_t msk_normal_apply_workspace(int64_t d, int64_t n);

/* v = A^T (A p) in double-single arithmetic.
 *   A : device float column-major d x n (lda >= d), 1 <= n <= 512;
 *   p : device double[n] (read as the pair fl32(p), fl32(p - fl32(p)));
 *   v : device double[n] (written).
 * Runs the refinement's FP64 residual pass first (with x = 0: it records the
 * column maxima of |A| that bound the terms of the operator pass), then one
 * operator pass: w = A p and v = A^T w, each product sum carried to about
 * 2^-44 of its terms' magnitude (n <= 256: an exact integer part on a grid
 * plus a binary32 rest; wider: compensated Dot2 sums).  Asynchronous on
 * `stream`.  Returns MSK_OK; -1 null pointer, -2 d < 1, -3 n outside
 * [1, 512], -4 lda < d, MSK_ENOMEM ws too small. */
int msk_normal_apply(const float *A, int64_t d, int64_t n, int64_t lda,
                     const double *p, double *v, void *ws, size_t ws_bytes,
                     void *stream);

/* ---- SRHT (Section 5: Definition of the SRHT, Algorithm 3) -------------- */

/* Scratch bytes of srht_sketch (d x ncol doubles when d > 8192, plus the
 * sample lists). */
size_t msk_srht_workspace(int64_t d, int64_t n, int with_b, int64_t k);

/* Subsampled randomized Hadamard transform of [A b]:
 *   Y = (1/sqrt(k)) P H_d D [A b],  d = 2^m (2 <= d <= 2^26),
 *   D   diagonal, d_ii = -1 when bit 0 of draw i of stream tag 5 is set;
 *   H_d the Hadamard matrix of the recursive definition
 *       (H_d[i][j] = (-1)^popcount(i & j)), by the fast Walsh-Hadamard
 *       transform with radix-4 butterflies (Algorithm 3);
 *   P   k x d row sampling: row l picks row ((z >> 32) * d) >> 32 of H D [A b],
 *       z = draw l of stream tag 6 (uniform, with replacement).
 *   A: device FP64 or FP32 (widened exactly), column-major d x n (lda >= d);
 *   b: device double[d] or NULL (then n >= 1);
 *   Y: device double, row-major k x ncol (ldy >= ncol), every entry written.
 * FP64 arithmetic.  Errors: -1 A NULL, -2 dtype, -3 d not a power of two in
 * [2, 2^26], -4 bad n, -5 lda < d, -7 k < 1, -9 Y NULL, -10 ldy < ncol,
 * MSK_ENOMEM ws too small. */
int srht_sketch(const void *A, int dtype, int64_t d, int64_t n, int64_t lda,
                const double *b, int64_t k, uint64_t seed, double *Y, int64_t ldy,
                void *ws, size_t ws_bytes, void *stream);

/* ---- Sketch-and-solve with one of the sketches (Section 6.3) ------------- */

/* Scratch bytes of sns_lstsq. */
size_t msk_sns_workspace(int64_t d, int64_t n, int kind, int64_t k, int64_t p,
                         int dtype);

/* Sketch-and-solve least squares (Algorithm 1) in FP64 with the sketch
 * `kind` (msk_sketch_kind): W = S [A b]; Householder QR of W; x = R11^{-1}
 * R[0:n, n].  MULTI is ms_lstsq with MSK_GEMM_F64 and no refinement.
 * COUNT uses k (n+1 <= k < 2^31; p is ignored): the FP64 CountSketch of [A b] (FP32
 * A widened exactly), transposed to column-major for the QR.  GAUSS uses p
 * (n+1 <= p <= 2048; k is ignored).  SRHT uses k (>= n+1) and needs d a
 * power of two (srht_sketch).  A, b, x, info and the return codes as
 * ms_lstsq (n <= 400); -7 unknown kind, -8 bad k (COUNT), -9 bad p (GAUSS).
 * info (optional, host): relres of x; relres_sns = relres. */
int sns_lstsq(const void *A, int dtype, int64_t d, int64_t n, int64_t lda,
              const double *b, int kind, int64_t k, int64_t p, uint64_t seed,
              double *x, msk_lstsq_info *info, void *ws, size_t ws_bytes,
              void *stream);

/* ---- Randomized Cholesky QR (Section 6.3, Algorithms 4 and 5) ----------- */

/* Scratch bytes of rcq_lstsq (want_q = 0) or rcq_qr (want_q = 1). */
size_t msk_rcq_workspace(int64_t d, int64_t n, int64_t k, int64_t p, int dtype,
                         int gemm_prec, int want_q);

/* rand_cholQR least squares (Algorithm 5) with the multisketch S = G C of
 * ms_sketch (CountSketch to k rows, Gaussian to p rows, gemm_prec as there):
 *   Y = S A;  R0 = R of the Householder QR of Y;  Q0 = A R0^{-1} (formed in
 *   FP64 through the explicit R0^{-1});  G = Q0^T Q0, z = Q0^T b (one pass);
 *   R1 = chol(G);  R = R1 R0;  y = R1^{-T} z;  x = R^{-1} y.
 * x is the least-squares minimiser with no sketching distortion, for
 * kappa(A) < 1/u.  Arguments and layouts as ms_lstsq (A FP64 or FP32 values,
 * column-major d x n, lda >= d; b, x device double); n <= 400,
 * n + 1 <= p <= min(k, 2048).  Needs d x n doubles of workspace for Q0.
 * info (optional, host): relres of x (an FP64 residual pass), iters = 0,
 * converged = 1, relres_sns = -1.  Synchronises `stream`.
 * Returns MSK_OK; -i for argument i; j+1 when R0[j][j] is zero or pivot j of
 * chol(G) is not positive (x is then NaN); MSK_ENOMEM / MSK_ENOTSUP / MSK_ECUDA
 * as ms_lstsq. */
int rcq_lstsq(const void *A, int dtype, int64_t d, int64_t n, int64_t lda,
              const double *b, int64_t k, int64_t p, uint64_t seed, int gemm_prec,
              double *x, msk_lstsq_info *info, void *ws, size_t ws_bytes,
              void *stream);

/* rand_cholQR (Algorithm 4): the QR factorisation A = Q R from the sketch's
 * R0 and one Cholesky step: Q0 = A R0^{-1}, R1 = chol(Q0^T Q0),
 * Q = Q0 R1^{-1}, R = R1 R0.
 *   Q : device double column-major d x n (ldq >= d), written; it may be A
 *       itself when A is FP64 with lda == ldq (factorisation in place);
 *   R : device double column-major n x n (ldr >= n), upper triangular
 *       (zeros below the diagonal); the signs of its diagonal are those of
 *       the Householder R0 of the sketch.
 * Other arguments as rcq_lstsq.  Synchronises `stream`.  Returns MSK_OK, -i,
 * or j+1 when R0[j][j] is zero or pivot j of chol(Q0^T Q0) is not positive. */
int rcq_qr(const void *A, int dtype, int64_t d, int64_t n, int64_t lda, int64_t k,
           int64_t p, uint64_t seed, int gemm_prec, double *Q, int64_t ldq,
           double *R, int64_t ldr, void *ws, size_t ws_bytes, void *stream);

/* ---- Batched solves (many uneven problems per launch) -------------------- */

/* One least-squares problem of a batch: FP32 A (device, column-major d x n,
 * lda >= d), FP64 b (device, d), the seed of its sketch, FP64 x (device, n,
 * output).  The batch uses the paper's sizes k = 2 n^2 (CountSketch) and
 * p = 4 n (Gaussian), Section 6.2; n must be 16, 32, 64, 128 or 256 and
 * d >= 4 n. */
typedef struct {
  const float *A;
  int64_t d, n, lda;
  const double *b;
  uint64_t seed;
  double *x;
} msk_batch_item;

/* Scratch bytes msk_batch_lstsq needs for these items. */
size_t msk_batch_workspace(const msk_batch_item *items, int nitems, int refine);

/* An upper bound of one item's part of msk_batch_workspace that adds up over
 * a batch: the sum over any batch's items is at least msk_batch_workspace of
 * that batch.  Host arithmetic only; the server admits requests by it in
 * time linear in the batch.  0 for a NULL item or an unsupported n.  The
 * paper has no counterpart. */
size_t msk_batch_item_bound(const msk_batch_item *item, int refine);

/* Solve every problem of the batch with the mixed-precision multisketch path:
 * FP32 CountSketch, split-BF16 tensor-core Gaussian stage with FP32
 * accumulators drained into double-single registers, FP64 Householder QR and
 * solve (Algorithm 1), and with refine = 1 the refinement of ms_lstsq (FP64
 * residual passes, double-single CG passes) with its convergence tests and
 * stops, per problem.  Each
 * stage is one launch over all problems, and the whole batch — the stages,
 * the outer refinement loop and the inner CG loop — is one CUDA-graph launch
 * whose loops are device-driven while nodes, so the host waits once, for the
 * results.  items: host array of nitems; infos: host array of nitems or
 * NULL.  Synchronises `stream`.  ws: 256-byte aligned, msk_batch_workspace
 * bytes.  Returns MSK_OK, MSK_ENOCONV if some problem stopped unconverged, or -1
 * (bad item), -2 (nitems < 1), -3 (bad refine), MSK_ENOMEM. */
int msk_batch_lstsq(const msk_batch_item *items, int nitems, int refine,
                    double tol, int32_t max_iter, msk_lstsq_info *infos,
                    void *ws, size_t ws_bytes, void *stream);

/* ---- Autotuner ----------------------------------------------------------- */

/* Scratch bytes msk_autotune needs for these items (the batch workspace at
 * its largest over the tuned split-K settings, plus a CountSketch output). */
size_t msk_autotune_workspace(const msk_batch_item *items, int nitems, int refine);

/* Time candidate values of the knobs "cs.fixed", "cs.l2_budget_bytes" (on
 * cs_sketch of the request with the most elements), "batch.kt_per",
 * "batch.round" and "pass.ctas_per_sm" (on msk_batch_lstsq of the whole
 * batch with refine, tol, max_iter), one knob at a time in that order, each
 * candidate as the median of `reps` runs (1..100) after a warm-up run, timed
 * with CUDA events on `stream`; leave the fastest value of each knob set in
 * the registry.  The paper has no counterpart (it tunes nothing).
 *   report: host buffer of report_bytes (may be NULL) receiving a JSON object
 *     {"knobs": {name: {"chosen": v, "timed_on": ..., "ms": {value: ms}}},
 *      "reps": r, "requests": nitems}, truncated to fit.
 *   ws: device scratch (256-byte aligned) of msk_autotune_workspace bytes.
 * Synchronous.  Errors: -1 items NULL, -2 nitems < 1, -3 refine not 0/1,
 * -6 reps out of range, MSK_ENOMEM scratch too small, MSK_ECUDA a timed run
 * failed (the knob being tuned is restored; earlier choices stay set). */
int msk_autotune(const msk_batch_item *items, int nitems, int refine, double tol,
                 int32_t max_iter, int reps, char *report, size_t report_bytes,
                 void *ws, size_t ws_bytes, void *stream);

/* ---- Request server (continuous batching) -------------------------------- */

/* A server for msk_batch_item requests.  mem_budget bytes of device memory are
 * reserved once here and split evenly over `workers` worker threads (each
 * with its own stream); nothing else is allocated while serving.  A free
 * worker admits waiting requests in arrival order while the sum of their
 * msk_batch_item_bound fits its share of the budget, at most max_batch per
 * batch, and solves them with msk_batch_lstsq(refine, tol, max_iter);
 * batches of different workers overlap on the GPU.  A request larger than a
 * share but not than the budget runs alone with the whole budget once the
 * other workers' batches are done (workers start nothing new meanwhile).
 * The paper serves single problems; this is the serving layer around its
 * solver.
 * Errors: -1 budget < 1 MiB, -2 workers outside 1..16, -3 max_batch < 1,
 * -4 bad refine, -7 srv NULL, MSK_ENOMEM when the pool cannot be reserved. */
int ms_server_create(size_t mem_budget, int workers, int max_batch, int refine,
                     double tol, int32_t max_iter, void **srv);

/* Queue one request (non-blocking).  The request's arrays must stay valid
 * until it is done; x is written in place.  *ticket identifies it.
 * MSK_ENOMEM when the request alone exceeds the whole budget, MSK_EBUSY when
 * the server is stopping or its queue is full. */
int ms_server_submit(void *srv, const msk_batch_item *req, uint64_t *ticket);

/* *done = 1 once the request is solved; then info (host, may be NULL) and
 * latency_s (seconds from submission to completion, may be NULL) are filled
 * and the return value is the request's status (MSK_OK, or the batch's
 * error).  -2 for an unknown ticket. */
int ms_server_poll(void *srv, uint64_t ticket, int *done, msk_lstsq_info *info,
                   double *latency_s);

/* Block until the queue is empty and no batch is in flight. */
int ms_server_wait_all(void *srv);

/* Requests solved, batches run, requests waiting (any pointer may be NULL). */
int ms_server_stats(void *srv, int64_t *solved, int64_t *batches,
                    int64_t *queued);

/* Text of the last failing batch of this server (empty when none). */
const char *ms_server_error(void *srv);

/* Finish the queued requests, stop the workers, release the pool. */
int ms_server_destroy(void *srv);

#ifdef __cplusplus
}
#endif
#endif /* MSKETCH_H */
