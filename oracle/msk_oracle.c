/*
 * msk_oracle.c — plain, slow CPU oracle for the CountSketch / multisketch /
 * least-squares hot path of "A High Performance GPU CountSketch
 * Implementation and Its Application to Multisketching and Least Squares
 * Problems" (Higgins, Boman, Yamazaki, arXiv 2508.14209).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline leg of bench.py may load this library.  It shares no code,
 * header, table or constant generator with the CUDA library: the counter
 * generator and the Gaussian sampler below are written here from their
 * published definitions, independently of the device code.
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math -shared -fPIC
 * (-ffp-contract=off matters: every float operation below is meant to be one
 * IEEE-754 round-to-nearest-even operation, on x86-64 and on aarch64 alike.)
 *
 * Conventions (all plain row/column loops, no blocking, no reordering):
 *   A  : d x n, column-major, leading dimension lda >= d, FP64 or FP32.
 *   b  : optional extra column of length d (FP64); when present the sketched
 *        matrix is [A b] with n+1 columns, as in Algorithm 1 (Y = SA, z = Sb).
 *   Y  : k x ncol, row-major (bucket-major), leading dimension ldy >= ncol —
 *        row m of Y is the sum of the rows of A that the sketch maps to m
 *        (the row form of Definition 3, Section 4).
 *   G  : p x k Gaussian, row-major.
 *   Z  : p x ncol, column-major, leading dimension ldz >= p.
 * All sums of more than two terms use Neumaier's compensated summation, so
 * the oracle's own rounding error stays far below the tolerances it checks.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Counter-based generator: splitmix64 (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014).  Output i of the generator
 * started from state `key` is mix(key + (i+1)*GAMMA) (mod 2^64).           */
#define OR_GAMMA 0x9E3779B97F4A7C15ULL
#define OR_STREAM_MUL 0xD1B54A32D192ED03ULL

static uint64_t or_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* Key of stream `tag` for a user seed (tag 0: CountSketch hash, tag 2:
 * Gaussian matrix).                                                         */
uint64_t or_stream_key(uint64_t seed, uint64_t tag) {
  return or_mix64(seed ^ (tag * OR_STREAM_MUL));
}

/* Output i (0-based) of splitmix64 started at state `key`.                  */
uint64_t or_draw(uint64_t key, uint64_t i) {
  return or_mix64(key + (i + 1) * OR_GAMMA);
}

/* CountSketch column data for rows i0..i0+count-1 (Definition 3, Section 4):
 * bucket h(i) in [0,k) from the top 32 bits of the draw by Lemire's
 * multiply-shift, sign s(i) = -1 when the lowest bit is set, else +1.       */
void or_hash(uint64_t seed, int64_t i0, int64_t count, int64_t k, uint32_t *h,
             int8_t *s) {
  uint64_t key = or_stream_key(seed, 0);
  for (int64_t t = 0; t < count; ++t) {
    uint64_t z = or_draw(key, (uint64_t)(i0 + t));
    h[t] = (uint32_t)(((z >> 32) * (uint64_t)k) >> 32);
    s[t] = (z & 1ULL) ? (int8_t)-1 : (int8_t)1;
  }
}

/* SRHT randomness (Section 5): the diagonal D, d_ii = -1 when the lowest bit
 * of draw i of stream tag 5 is set, else +1; the rows P samples, row l picks
 * j_l = ((z >> 32) * d) >> 32 for draw l of stream tag 6 (uniform in [0,d),
 * with replacement).                                                         */
void or_srht_signs(uint64_t seed, int64_t d, int8_t *s) {
  uint64_t key = or_stream_key(seed, 5);
  for (int64_t i = 0; i < d; ++i) s[i] = (or_draw(key, (uint64_t)i) & 1ULL) ? (int8_t)-1 : (int8_t)1;
}

void or_srht_rows(uint64_t seed, int64_t k, int64_t d, uint32_t *j) {
  uint64_t key = or_stream_key(seed, 6);
  for (int64_t l = 0; l < k; ++l) {
    uint64_t z = or_draw(key, (uint64_t)l);
    j[l] = (uint32_t)(((z >> 32) * (uint64_t)d) >> 32);
  }
}

/* ------------------------------------------------------------------------ */
/* Gaussian sampler in binary32 (the Gaussian sketch of Section 1, used as the
 * second stage of the multisketch).  Marsaglia & Bray's polar method:
 * draw (u, v) uniform in the open square (-1,1)^2 until s = u^2+v^2 < 1,
 * then u * sqrt(-2 ln(s) / s) is standard normal.  Every operation is one
 * rounded binary32 operation; ln is written out below so that the sampler is
 * reproducible bit for bit from its definition.                             */
static float or_f32_from_bits(uint32_t b) { float f; memcpy(&f, &b, 4); return f; }
static uint32_t or_bits_from_f32(float f) { uint32_t b; memcpy(&b, &f, 4); return b; }

/* ln(s) for normal positive s: s = m * 2^e with m in [sqrt(1/2), sqrt(2)),
 * ln(s) = e*ln2 + 2*atanh(t), t = (m-1)/(m+1), and
 * atanh(t) = t*(1 + t^2/3 + t^4/5 + t^6/7 + t^8/9 + ...)  (|t| <= 0.1716;
 * the first omitted term is below 2^-28 relative).                          */
float or_ln_f32(float s) {
  const float SQRT2 = or_f32_from_bits(0x3FB504F3u); /* 0x1.6a09e6p+0 */
  const float LN2 = or_f32_from_bits(0x3F317218u);   /* 0x1.62e430p-1 */
  const float C3 = or_f32_from_bits(0x3EAAAAABu);    /* 1/3 rounded */
  const float C5 = or_f32_from_bits(0x3E4CCCCDu);    /* 1/5 rounded */
  const float C7 = or_f32_from_bits(0x3E124925u);    /* 1/7 rounded */
  const float C9 = or_f32_from_bits(0x3DE38E39u);    /* 1/9 rounded */
  uint32_t bits = or_bits_from_f32(s);
  int e = (int)((bits >> 23) & 0xFFu) - 127;
  float m = or_f32_from_bits((bits & 0x007FFFFFu) | 0x3F800000u); /* [1,2) */
  if (m > SQRT2) { m = m * 0.5f; e = e + 1; }
  float num = m - 1.0f;
  float den = m + 1.0f;
  float t = num / den;
  float w = t * t;
  float p = C9;
  p = p * w; p = p + C7;
  p = p * w; p = p + C5;
  p = p * w; p = p + C3;
  p = p * w; p = p + 1.0f;
  float two_t = 2.0f * t;
  float lnm = two_t * p;
  float eln2 = (float)e * LN2;
  return eln2 + lnm;
}

/* Standard normal number `elem` of the stream with key `key`: attempt a uses
 * draw index elem*2^16 + a.  From draw z: U = bits 63..40, V = bits 39..16,
 * u = (2U + 1 - 2^24) * 2^-24 and likewise v, both odd multiples of 2^-24,
 * exactly representable and never zero.                                     */
float or_gauss_std(uint64_t key, uint64_t elem) {
  for (uint64_t a = 0; a < 65536u; ++a) {
    uint64_t z = or_draw(key, (elem << 16) | a);
    int32_t U = (int32_t)(z >> 40);
    int32_t V = (int32_t)((z >> 16) & 0xFFFFFFu);
    float u = (float)(2 * U + 1 - (1 << 24)) * 0x1p-24f;
    float v = (float)(2 * V + 1 - (1 << 24)) * 0x1p-24f;
    float uu = u * u;
    float vv = v * v;
    float s = uu + vv;
    if (s < 1.0f) {
      float L = or_ln_f32(s);
      float m2L = -2.0f * L;
      float q = m2L / s;
      float r = sqrtf(q);
      return u * r;
    }
  }
  return 0.0f; /* probability (1 - pi/4)^65536: never reached */
}

/* G (p x k, row-major, ldg >= k): G[r][c] = N(0,1) sample number r*k+c of
 * stream 2, divided by sqrt(p) so that the entries are N(0, 1/p).          */
void or_gaussian(uint64_t seed, int64_t p, int64_t k, float *G, int64_t ldg) {
  uint64_t key = or_stream_key(seed, 2);
  float sp = sqrtf((float)p);
  for (int64_t r = 0; r < p; ++r)
    for (int64_t c = 0; c < k; ++c)
      G[r * ldg + c] = or_gauss_std(key, (uint64_t)(r * k + c)) / sp;
}

/* ------------------------------------------------------------------------ */
/* Neumaier compensated accumulation: (s, c) with true sum ~ s + c.          */
static void or_neu_add(double *s, double *c, double x) {
  double t = *s + x;
  if (fabs(*s) >= fabs(x)) *c += (*s - t) + x;
  else *c += (x - t) + *s;
  *s = t;
}

static double or_getA(const void *A, int dtype, int64_t lda, int64_t i, int64_t j) {
  if (dtype == 0) return ((const double *)A)[i + j * lda];
  return (double)((const float *)A)[i + j * lda];
}

/* Element (i, j) of [A b]: column j < n from A, column n from b.            */
static double or_getAb(const void *A, int dtype, int64_t lda, int64_t n,
                       const double *b, int64_t i, int64_t j) {
  if (j < n) return or_getA(A, dtype, lda, i, j);
  return b[i];
}

/* CountSketch Y = S [A b] by its row form (Section 4):
 *   Y[m, :] = sum over rows i with h(i) = m of s(i) * [A b][i, :],
 * rows visited in increasing i.  dtype 0 = FP64 A, 1 = FP32 A (upcast
 * exactly).  b may be NULL.  Returns 0, or -1 when out of memory.           */
int or_countsketch(const void *A, int dtype, int64_t d, int64_t n, int64_t lda,
                   const double *b, int64_t k, uint64_t seed, double *Y,
                   int64_t ldy) {
  int64_t ncol = n + (b ? 1 : 0);
  double *comp = (double *)calloc((size_t)(k * ncol), sizeof(double));
  if (!comp) return -1;
  for (int64_t m = 0; m < k; ++m)
    for (int64_t j = 0; j < ncol; ++j) Y[m * ldy + j] = 0.0;
  uint64_t key = or_stream_key(seed, 0);
  for (int64_t i = 0; i < d; ++i) {
    uint64_t z = or_draw(key, (uint64_t)i);
    int64_t m = (int64_t)(((z >> 32) * (uint64_t)k) >> 32);
    double sg = (z & 1ULL) ? -1.0 : 1.0;
    for (int64_t j = 0; j < ncol; ++j)
      or_neu_add(&Y[m * ldy + j], &comp[m * ncol + j], sg * or_getAb(A, dtype, lda, n, b, i, j));
  }
  for (int64_t m = 0; m < k; ++m)
    for (int64_t j = 0; j < ncol; ++j) Y[m * ldy + j] += comp[m * ncol + j];
  free(comp);
  return 0;
}

/* The same sums for a chosen list of buckets only (nb buckets, output rows
 * Yb[q*ncol + j] for bucket list[q]); also returns the bucket absolute sums
 * sum |[A b][i, j]| in absb (same shape) and the row counts in cnt[q].  Used
 * to check sampled outputs of full-size problems.                           */
int or_countsketch_buckets(const void *A, int dtype, int64_t d, int64_t n,
                           int64_t lda, const double *b, int64_t k,
                           uint64_t seed, int64_t nb, const int64_t *list,
                           double *Yb, double *absb, int64_t *cnt) {
  int64_t ncol = n + (b ? 1 : 0);
  int64_t *slot = (int64_t *)malloc((size_t)k * sizeof(int64_t));
  double *comp = (double *)calloc((size_t)(nb * ncol), sizeof(double));
  if (!slot || !comp) { free(slot); free(comp); return -1; }
  for (int64_t m = 0; m < k; ++m) slot[m] = -1;
  for (int64_t q = 0; q < nb; ++q) slot[list[q]] = q;
  for (int64_t q = 0; q < nb * ncol; ++q) { Yb[q] = 0.0; absb[q] = 0.0; }
  for (int64_t q = 0; q < nb; ++q) cnt[q] = 0;
  uint64_t key = or_stream_key(seed, 0);
  for (int64_t i = 0; i < d; ++i) {
    uint64_t z = or_draw(key, (uint64_t)i);
    int64_t m = (int64_t)(((z >> 32) * (uint64_t)k) >> 32);
    int64_t q = slot[m];
    if (q < 0) continue;
    double sg = (z & 1ULL) ? -1.0 : 1.0;
    cnt[q] += 1;
    for (int64_t j = 0; j < ncol; ++j) {
      double a = or_getAb(A, dtype, lda, n, b, i, j);
      or_neu_add(&Yb[q * ncol + j], &comp[q * ncol + j], sg * a);
      absb[q * ncol + j] += fabs(a);
    }
  }
  for (int64_t q = 0; q < nb * ncol; ++q) Yb[q] += comp[q];
  free(slot);
  free(comp);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Gaussian stage of the multisketch, Z = G Y (Section 1, "Count-Gauss"):
 * Z[r, c] = sum_m G[r, m] * Y[m, c], each dot product compensated.  G is
 * given as FP64 values (the caller widens or pre-rounds them); Y row-major
 * (ldy), Z column-major (ldz).                                               */
void or_gemm(const double *G, int64_t ldg, const double *Y, int64_t ldy,
             int64_t p, int64_t k, int64_t ncol, double *Z, int64_t ldz) {
  for (int64_t r = 0; r < p; ++r)
    for (int64_t c = 0; c < ncol; ++c) {
      double s = 0.0, comp = 0.0;
      for (int64_t m = 0; m < k; ++m) or_neu_add(&s, &comp, G[r * ldg + m] * Y[m * ldy + c]);
      Z[r + c * ldz] = s + comp;
    }
}

/* Normal-equations operands (Section 6.3): Gm = A^T A (n x n, column-major)
 * and y = A^T b, each entry a compensated dot product over the d rows.      */
void or_gram(const void *A, int dtype, int64_t d, int64_t n, int64_t lda,
             const double *b, double *Gm, double *y) {
  for (int64_t a = 0; a < n; ++a) {
    for (int64_t c = 0; c < n; ++c) {
      double s = 0.0, comp = 0.0;
      for (int64_t i = 0; i < d; ++i)
        or_neu_add(&s, &comp, or_getA(A, dtype, lda, i, a) * or_getA(A, dtype, lda, i, c));
      Gm[a + c * n] = s + comp;
    }
    double s = 0.0, comp = 0.0;
    for (int64_t i = 0; i < d; ++i) or_neu_add(&s, &comp, or_getA(A, dtype, lda, i, a) * b[i]);
    y[a] = s + comp;
  }
}

/* Residual r = b - A x (each entry a compensated sum), its squared norm and
 * the squared norm of b (returned in out2[0], out2[1]); optionally r itself
 * and g = A^T r (compensated).  r and g may be NULL.                        */
void or_residual(const void *A, int dtype, int64_t d, int64_t n, int64_t lda,
                 const double *b, const double *x, double *r, double *g,
                 double *out2) {
  double rr = 0.0, rrc = 0.0, bb = 0.0, bbc = 0.0;
  double *gc = NULL;
  if (g) {
    gc = (double *)calloc((size_t)n, sizeof(double));
    for (int64_t j = 0; j < n; ++j) g[j] = 0.0;
  }
  for (int64_t i = 0; i < d; ++i) {
    double s = b[i], c = 0.0;
    for (int64_t j = 0; j < n; ++j) or_neu_add(&s, &c, -(or_getA(A, dtype, lda, i, j) * x[j]));
    double ri = s + c;
    if (r) r[i] = ri;
    or_neu_add(&rr, &rrc, ri * ri);
    or_neu_add(&bb, &bbc, b[i] * b[i]);
    if (g && gc)
      for (int64_t j = 0; j < n; ++j) or_neu_add(&g[j], &gc[j], or_getA(A, dtype, lda, i, j) * ri);
  }
  if (g && gc)
    for (int64_t j = 0; j < n; ++j) g[j] += gc[j];
  free(gc);
  out2[0] = rr + rrc;
  out2[1] = bb + bbc;
}
