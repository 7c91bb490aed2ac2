// msk_pass.cuh — refinement passes over an FP32 A (the operator applications
// of the sketch-and-precondition refinement: A preconditioned by the R of the
// sketched QR, as in the preconditioned normal equations of Section 6.3):
//   RESID = true : r_i = b_i - A_i x in FP64 (one DFMA per element);
//                  accumulates g = A^T r, ||r||^2, ||b||^2 and (specialised
//                  bodies) the column maxima of |A|.
//   RESID = false: w_i = A_i p and v = A^T w, both to about 44 bits.
// Two ways of summing products to about twice binary32's precision on the
// FP32 units (GB300's FP64 rate is about 1/64 of its FP32 rate):
//   Dot2 (Ogita, Rump and Oishi, SIAM J. Sci. Comput. 2005): a compensated
//     pair (s, c), TwoSum (Knuth) for the rounding error of s, one FMA
//     (Dekker) for the product's; 11 binary32 operations per term.  The
//     generic body (n > 256) uses it.
//   error-free extraction (xs_step; Rump, Ogita and Oishi 2008): each product
//     on an integer grid by one FMA against 1.5 2^k, the grid parts summed
//     exactly as integers, the part below the grid into a binary32 rest;
//     5 binary32 operations and one integer add per term.  The specialised
//     bodies' operator pass and both column phases use it.
//
// The generic body (pass32g_body) tiles R rows (a power of two, R n ~ 8192)
// column-major in shared memory by cp.async, two buffers deep; a thread (r, q)
// sums columns q, q + Q, ... of row r with the Q partials merged through
// shared memory, and a thread (g, j) accumulates column j over a rotated set
// of rows (32 lanes in 32 banks).  The specialised bodies (pass32n_body,
// n <= 256 as the next power of two) are described where they are defined.
// Output: part[cta][0..n) the CTA's vector partial, part[cta][n], [n+1] the
// scalars (RESID) or zeros; summed in fixed order by pass_reduce_body.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "msk_device.cuh"

namespace msk {

constexpr int kP32Threads = 256;
constexpr int kP32TileElems = 8192;  // R * n target (32 KiB per buffer)

// Width class of the specialised bodies: n <= 256 runs as NC = the next power
// of two >= max(n, 16) columns (the extra columns are zero-filled and
// contribute nothing); wider n runs the generic body (class 0).
__host__ __device__ __forceinline__ int pass32_class(int n) {
  if (n > 256) return 0;
  int c = 16;
  while (c < n) c *= 2;
  return c;
}
// Generic body: rows per tile, a power of two in [32, 1024] with R * n ~ 8192.
__host__ __device__ __forceinline__ int pass32g_rows(int n) {
  int R = 32;
  while (R < 1024 && 2 * R * n <= kP32TileElems) R *= 2;
  return R;
}
// Specialised bodies: elements per tile and pipeline depth by width class —
// 16 KiB tiles three deep up to 128 columns (two tiles of compute cover a
// tile's load latency), 32 KiB tiles two deep at 256 (a tile keeps >= 32 rows).
__host__ __device__ constexpr int pass32n_tile(int nc) { return nc <= 128 ? 4096 : 8192; }
__host__ __device__ constexpr int pass32n_stages(int nc) { return nc <= 128 ? 3 : 2; }
// Column pitch (floats) of a staged tile: R + 4, which is 4 mod 32, so that
// 16-byte reads of eight consecutive columns at one row fall in eight
// different quads of shared-memory banks.
__host__ __device__ constexpr int pass32n_pitch(int nc) { return pass32n_tile(nc) / nc + 4; }
// Length of a pass result (and of a residual pass's per-CTA partial in the
// specialised bodies): [A^T v (n), two scalars, column maxima of |A| (n)].
__host__ __device__ constexpr int64_t pass_out_len(int64_t n) { return 2 * n + 2; }
// Rows per tile of the body that runs for n.
__host__ __device__ __forceinline__ int pass32_rows(int n) {
  const int nc = pass32_class(n);
  return nc ? pass32n_tile(nc) / nc : pass32g_rows(n);
}
// Dynamic shared memory of a pass CTA for n columns (two tiles + vectors +
// merge space) of the body that runs for n.
__host__ __device__ __forceinline__ size_t pass32_smem(int n) {
  const int nc = pass32_class(n);
  if (nc) {
    const int R = pass32n_tile(nc) / nc;
    return sizeof(float) * (size_t)pass32n_stages(nc) * nc * pass32n_pitch(nc) + 8 * (size_t)nc +
           sizeof(double) * kP32Threads + sizeof(float2) * (size_t)R;
  }
  const int R = pass32g_rows(n);
  return sizeof(float) * 2 * (size_t)R * n + sizeof(double) * (size_t)n +
         sizeof(double) * kP32Threads + sizeof(float) * 2 * (size_t)R + sizeof(double) * kP32Threads;
}

struct D2 {
  float s, c;
};
// acc += a * (xh + xl) (Dot2 step: TwoProd by FMA, TwoSum, errors into c).
__device__ __forceinline__ void d2_fma(D2& acc, float a, float xh, float xl) {
  const float ph = __fmul_rn(a, xh);
  const float pe = __fmaf_rn(a, xh, -ph);
  const float s = __fadd_rn(acc.s, ph);
  const float v = __fsub_rn(s, acc.s);
  const float e = __fadd_rn(__fsub_rn(acc.s, __fsub_rn(s, v)), __fsub_rn(ph, v));
  acc.s = s;
  acc.c = __fadd_rn(acc.c, __fadd_rn(e, __fmaf_rn(a, xl, pe)));
}
// (s1, c1) + (s2, c2)
__device__ __forceinline__ D2 d2_merge(D2 a, D2 b) {
  const float s = __fadd_rn(a.s, b.s);
  const float v = __fsub_rn(s, a.s);
  const float e = __fadd_rn(__fsub_rn(a.s, __fsub_rn(s, v)), __fsub_rn(b.s, v));
  return D2{s, __fadd_rn(__fadd_rn(a.c, b.c), e)};
}

// Two binary32 lanes in one 64-bit register for the packed FP32x2
// instructions of sm_100+ (add/sub/mul/fma .rn.f32x2): each instruction does
// the same operation on both lanes, halving the instruction count of the
// extraction steps below.
typedef unsigned long long f2p;
__device__ __forceinline__ f2p f2p_make(float lo, float hi) {
  f2p r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ float2 f2p_split(f2p v) {
  float lo, hi;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
  return make_float2(lo, hi);
}
__device__ __forceinline__ f2p f2p_add(f2p a, f2p b) {
  f2p r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2p f2p_sub(f2p a, f2p b) {
  f2p r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2p f2p_mul(f2p a, f2p b) {
  f2p r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2p f2p_fma(f2p a, f2p b, f2p c) {
  f2p r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
// Extraction of a sum of products into an exact integer part and a small
// rest: the error-free transformation of Rump, Ogita and Oishi ("Accurate
// floating-point summation", SIAM J. Sci. Comput. 2008) with each product
// put on the grid by one FMA.  For terms x = a xh with |x| < 2^(k-1) and
// sigma = 1.5 2^k, t = fl(a xh + sigma) lies in [2^k, 2^(k+1)], so t - sigma is
// x rounded to a multiple of u = 2^(k-23), exactly (Sterbenz), and equals
// (bits(t) - bits(sigma)) u: the binary32 encodings of one binade and of its
// upper end are consecutive integers.  Those integers are summed exactly; the
// part below the grid, a xh - (t - sigma), is less than u/2 and comes from a
// second FMA, rounded once, and goes with a xl (xh + xl a double-single
// factor) into a binary32 rest.  Five binary32 operations per term, in packed
// f32x2 pairs, and one integer add, against eleven for a Dot2 step, at about
// the same accuracy (the rest carries the terms' bits below 2^(k-24)).
struct XSig {
  f2p s2;       // (sigma, sigma)
  unsigned sb;  // binary32 bits of sigma
  float u;      // the grid 2^(k-23)
  float u12;    // 2^(k-11)
};
// sigma for 2^(k-1) above every term, k clamped to [-100, 126] (the grid
// stays normal; terms of 2^125 and above are outside the method's range).
__device__ __forceinline__ XSig xsig_make(int k) {
  k = min(max(k, -100), 126);
  XSig x;
  x.sb = ((unsigned)(k + 127) << 23) | 0x00400000u;
  const float s = __uint_as_float(x.sb);
  x.s2 = f2p_make(s, s);
  x.u = __uint_as_float((unsigned)(k + 104) << 23);
  x.u12 = __uint_as_float((unsigned)(k + 116) << 23);
  return x;
}
// e with |v| < 2^(e+1), from the bits of |v| (zero and subnormals give -126;
// infinities and NaNs 128, which the clamp of xsig_make absorbs: the NaN then
// reaches the rest through the second FMA).
__device__ __forceinline__ int p32_exp_bound(unsigned abs_bits) {
  return (int)max(abs_bits >> 23, 1u) - 127;
}
// S += the grid parts of a xh (two lanes; S starts at -(terms) bits(sigma),
// modulo 2^32), lo += the parts below the grid and a xl.
__device__ __forceinline__ void xs_step(unsigned& S, f2p& lo, f2p a, f2p xh, f2p xl, f2p s2) {
  const f2p t = f2p_fma(a, xh, s2);
  const f2p nq = f2p_sub(s2, t);
  lo = f2p_add(lo, f2p_fma(a, xh, nq));
  lo = f2p_fma(a, xl, lo);
  const float2 tt = f2p_split(t);
  S += __float_as_uint(tt.x) + __float_as_uint(tt.y);
}
// u S + lo as a normalised double-single pair, for S a two's-complement
// integer below 2^31 in magnitude: S = H 2^12 + L (0 <= L < 2^12) gives two
// exactly representable parts, combined with lo by two TwoSums (Knuth).
__device__ __forceinline__ float2 xs_value(unsigned S, float lo, const XSig& x) {
  const int Si = (int)S;
  const float xh = __fmul_rn(__int2float_rn(Si >> 12), x.u12);
  const float xl = __fmul_rn(__int2float_rn(Si & 4095), x.u);
  const float s = __fadd_rn(xh, xl);
  float v = __fsub_rn(s, xh);
  const float e = __fadd_rn(__fsub_rn(xh, __fsub_rn(s, v)), __fsub_rn(xl, v));
  const float c = __fadd_rn(e, lo);
  const float h = __fadd_rn(s, c);
  v = __fsub_rn(h, s);
  return make_float2(h, __fadd_rn(__fsub_rn(s, __fsub_rn(h, v)), __fsub_rn(c, v)));
}
// acc += u S + lo for |S| <= 2^24 (one exact conversion, one TwoSum).
__device__ __forceinline__ void xs_flush(D2& acc, unsigned S, f2p lo, const XSig& x) {
  const float xv = __fmul_rn(__int2float_rn((int)S), x.u);
  const float2 l = f2p_split(lo);
  const float s = __fadd_rn(acc.s, xv);
  const float v = __fsub_rn(s, acc.s);
  const float e = __fadd_rn(__fsub_rn(acc.s, __fsub_rn(s, v)), __fsub_rn(xv, v));
  acc.s = s;
  acc.c = __fadd_rn(acc.c, __fadd_rn(e, __fadd_rn(l.x, l.y)));
}

__device__ __forceinline__ unsigned p32_smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
// 4-byte copy, zero-filled when !valid (the source is then not read).
__device__ __forceinline__ void p32_cp4(float* dst, const float* src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(p32_smem_addr(dst)), "l"(src),
               "r"(valid ? 4 : 0)
               : "memory");
}
// 16-byte copy of `bytes` (0..16) source bytes, the rest zero-filled.
__device__ __forceinline__ void p32_cp16(float* dst, const float* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(p32_smem_addr(dst)), "l"(src),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void p32_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void p32_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Stage rows [i0, i0 + R) of columns 0..ns-1 into buf (column-major, stride
// R); columns >= n and rows >= d are zero-filled without reading A.
// vec: A 16-byte aligned and lda a multiple of 4 (16-byte copies).
__device__ __forceinline__ void p32_issue(const float* __restrict__ A, int64_t lda, int64_t d, int n,
                                          int ns, int R, int lgR, bool vec, int64_t i0, float* buf) {
  const int t = threadIdx.x;
  if (vec) {
    const int lgR4 = lgR - 2, R4 = R >> 2;
    const int total = ns * R4;
    for (int e = t; e < total; e += kP32Threads) {
      const int j = e >> lgR4, r = (e & (R4 - 1)) << 2;
      const int64_t i = i0 + r;
      const int64_t left = j < n ? d - i : 0;
      const int bytes = left >= 4 ? 16 : (left > 0 ? (int)left * 4 : 0);
      p32_cp16(buf + (size_t)j * R + r, bytes > 0 ? A + i + (int64_t)j * lda : A, bytes);
    }
  } else {
    const int total = ns * R;
    for (int e = t; e < total; e += kP32Threads) {
      const int j = e >> lgR, r = e & (R - 1);
      const int64_t i = i0 + r;
      const bool ok = i < d && j < n;
      p32_cp4(buf + (size_t)j * R + r, ok ? A + i + (int64_t)j * lda : A, ok);
    }
  }
  p32_commit();
}

// Generic body (any n <= 512; used for n > 256).
// 8-byte copy of `bytes` (0, 4 or 8) source bytes, the rest zero-filled.
__device__ __forceinline__ void p32_cp8(float* dst, const float* src, int bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(p32_smem_addr(dst)), "l"(src),
               "r"(bytes)
               : "memory");
}

// Copy of W whole floats (no zero fill) to the shared address dst.
template <int W>
__device__ __forceinline__ void p32_cp_whole(unsigned dst, const float* src) {
  if constexpr (W == 4)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
  else if constexpr (W == 2)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}

// Copy width (floats per cp.async) usable for A: 4 when A is 16-byte aligned
// and lda a multiple of 4, 2 when 8-byte aligned with lda even, else 1.
__host__ __device__ __forceinline__ int pass32_copy_width(const float* A, int64_t lda) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(A);
  if ((a & 15) == 0 && (lda & 3) == 0) return 4;
  if ((a & 7) == 0 && (lda & 1) == 0) return 2;
  return 1;
}

// Staging of one tile for the specialised bodies: rows [i0, i0 + R) of the NC
// columns at pitch P, W floats per copy.  Chunk c = t + 256 k of the tile is column
// c / (R/W), rows (c mod (R/W)) * W ..; with R/W a power of two each thread's
// chunks advance by a fixed column step and (when R/W > 256) a fixed row
// step, so the unrolled loop needs one pointer add per copy.
template <int NC, int R, int W, int P>
__device__ __forceinline__ void p32n_issue(const float* __restrict__ A, int64_t lda, int64_t d, int n,
                                           int64_t i0, float* buf) {
  constexpr int CPC = R / W;               // chunks per column
  constexpr int KT = NC * CPC / kP32Threads;  // chunks per thread
  const int t = threadIdx.x;
  if constexpr (CPC <= kP32Threads) {
    constexpr int JS = kP32Threads / CPC;  // column step per chunk
    const int r = (t % CPC) * W, j0 = t / CPC;
    const int64_t i = i0 + r;
    const int64_t left = d - i;
    const int rbytes = left >= W ? 4 * W : (left > 0 ? (int)left * 4 : 0);
    const float* src = A + i + (int64_t)j0 * lda;
    const int64_t step = (int64_t)JS * lda;
    if (n == NC && i0 + R <= d) {
      // a whole tile: every copy full, shared offsets known at compile time
      const unsigned d0 = p32_smem_addr(buf + j0 * P + r);
#pragma unroll
      for (int k = 0; k < KT; ++k) p32_cp_whole<W>(d0 + 4u * (unsigned)(k * JS * P), src + k * step);
      p32_commit();
      return;
    }
    float* dst = buf + j0 * P + r;
    int j = j0;
#pragma unroll 8
    for (int k = 0; k < KT; ++k) {
      const int bytes = j < n ? rbytes : 0;
      if constexpr (W == 4) p32_cp16(dst, bytes > 0 ? src : A, bytes);
      else if constexpr (W == 2) p32_cp8(dst, bytes > 0 ? src : A, bytes);
      else p32_cp4(dst, bytes > 0 ? src : A, bytes > 0);
      src += step;
      dst += JS * P;
      j += JS;
    }
  } else {
    constexpr int RS = CPC / kP32Threads;  // chunks of one column per thread
#pragma unroll
    for (int k = 0; k < KT; ++k) {
      const int j = k / RS, r = (t + kP32Threads * (k % RS)) * W;
      const int64_t i = i0 + r;
      const int64_t left = j < n ? d - i : 0;
      const int bytes = left >= W ? 4 * W : (left > 0 ? (int)left * 4 : 0);
      const float* s = bytes > 0 ? A + i + (int64_t)j * lda : A;
      if constexpr (W == 4) p32_cp16(buf + j * P + r, s, bytes);
      else if constexpr (W == 2) p32_cp8(buf + j * P + r, s, bytes);
      else p32_cp4(buf + j * P + r, s, bytes > 0);
    }
  }
  p32_commit();
}

// Exact binary32 -> binary64 widening on the integer units (GB300's FP64 pipe,
// which a conversion instruction would occupy, is 1/64 of the FP32 rate):
// sign, exponent rebiased by 1023 - 127 (255 -> 2047 for infinities and
// NaNs), fraction shifted into place.  e == 0: zero keeps only its sign; a
// subnormal m 2^-149 is renormalised (leading one of m at bit 31 - clz(m),
// so the value is 1.f 2^(-118 - clz(m))).
__device__ __forceinline__ double f2d_exact(float a) {
  const unsigned u = __float_as_uint(a);
  const unsigned sign = u & 0x80000000u;
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned m = u & 0x007fffffu;
  const unsigned ex = e == 255u ? 2047u : e + 896u;
  unsigned hi = sign | (ex << 20) | (m >> 3);
  unsigned lo = m << 29;
  if (e == 0u) {
    if (m == 0u) {
      hi = sign;
      lo = 0u;
    } else {
      const unsigned lz = (unsigned)__clz((int)m);  // 9 .. 31
      const unsigned f = (m << (lz - 8u)) & 0x007fffffu;
      hi = sign | ((905u - lz) << 20) | (f >> 3);
      lo = f << 29;
    }
  }
  return __hiloint2double((int)hi, (int)lo);
}

template <bool RESID>
__device__ __forceinline__ void pass32g_body(const float* __restrict__ A, int64_t lda, int64_t d, int n,
                                             bool vec, const double* __restrict__ b,
                                             const double* __restrict__ vin,
                                             double* __restrict__ part, int cta, int nctas,
                                             unsigned char* smem) {
  constexpr int T = kP32Threads;
  const int t = threadIdx.x;
  const int R = pass32g_rows(n);
  int lgR = 5;
  while ((1 << lgR) < R) ++lgR;
  const int tile_elems = R * n;
  float* tiles = reinterpret_cast<float*>(smem);
  double* vd = reinterpret_cast<double*>(tiles + 2 * (size_t)tile_elems);  // n
  double* wp = vd + n;                                                     // T (dot partials)
  float* wh = reinterpret_cast<float*>(wp + T);                            // R
  float* wl = wh + R;                                                      // R
  double* red = reinterpret_cast<double*>(wl + R);                         // T
  float* ph = reinterpret_cast<float*>(vd);
  float* pl = ph + n;
  if (RESID) {
    for (int j = t; j < n; j += T) vd[j] = vin[j];
  } else {
    // p = ph + pl (n <= 2T)
    const double x0 = t < n ? vin[t] : 0.0, x1 = t + T < n ? vin[t + T] : 0.0;
    if (t < n) {
      const float h = __double2float_rn(x0);
      ph[t] = h;
      pl[t] = __double2float_rn(x0 - (double)h);
    }
    if (t + T < n) {
      const float h = __double2float_rn(x1);
      ph[t + T] = h;
      pl[t + T] = __double2float_rn(x1 - (double)h);
    }
  }
  // geometry
  const int Q = R >= T ? 1 : T / R;   // threads per row in the dot phase
  const int RT = R >= T ? R / T : 1;  // rows per thread in the dot phase
  const int rq = R >= T ? t : (t & (R - 1));
  const int q = R >= T ? 0 : t / R;
  int G = 1;
  while (2 * G * n <= T) G *= 2;  // column groups (G = 1 when n > T/2)
  const int RG = R / G;
  const int g = t & (G - 1);
  const int jc = t / G;  // column of this thread (n <= T: one column; else t and t + T)

  D2 acc0{0.f, 0.f}, acc1{0.f, 0.f};
  double s1 = 0.0, s2 = 0.0;
  const int64_t ntiles = (d + R - 1) / R;
  int64_t tile = cta;
  if (tile < ntiles) p32_issue(A, lda, d, n, n, R, lgR, vec, tile * R, tiles);
  int buf = 0;
  for (; tile < ntiles; tile += nctas, buf ^= 1) {
    const int64_t next = tile + nctas;
    __syncthreads();  // previous tile's readers are done with the other buffer and wh/wl
    if (next < ntiles) {
      p32_issue(A, lda, d, n, n, R, lgR, vec, next * R, tiles + (size_t)(buf ^ 1) * tile_elems);
      p32_wait<1>();
    } else {
      p32_wait<0>();
    }
    __syncthreads();
    const float* tl = tiles + (size_t)buf * tile_elems;
    const int64_t i0 = tile * R;
    // ---- dot phase
    for (int m = 0; m < RT; ++m) {
      const int r = rq + m * T;
      if (RESID) {
        double w = 0.0;
        for (int j = q; j < n; j += Q) w = fma((double)tl[(size_t)j * R + r], vd[j], w);
        if (Q == 1) {
          const int64_t i = i0 + r;
          float h = 0.f, l = 0.f;
          if (i < d) {
            const double bi = b[i];
            const double ri = bi - w;
            s1 = fma(ri, ri, s1);
            s2 = fma(bi, bi, s2);
            h = __double2float_rn(ri);
            l = __double2float_rn(ri - (double)h);
          }
          wh[r] = h;
          wl[r] = l;
        } else {
          wp[q * R + r] = w;
        }
      } else {
        D2 w{0.f, 0.f};
        for (int j = q; j < n; j += Q) d2_fma(w, tl[(size_t)j * R + r], ph[j], pl[j]);
        if (Q == 1) {
          const float h = __fadd_rn(w.s, w.c);
          wh[r] = h;
          wl[r] = __fsub_rn(w.c, __fsub_rn(h, w.s));
        } else {
          reinterpret_cast<float2*>(wp)[q * R + r] = make_float2(w.s, w.c);
        }
      }
    }
    if (Q > 1) {
      __syncthreads();
      if (t < R) {
        const int64_t i = i0 + t;
        if (RESID) {
          double w = 0.0;
          for (int qq = 0; qq < Q; ++qq) w += wp[qq * R + t];
          float h = 0.f, l = 0.f;
          if (i < d) {
            const double bi = b[i];
            const double ri = bi - w;
            s1 = fma(ri, ri, s1);
            s2 = fma(bi, bi, s2);
            h = __double2float_rn(ri);
            l = __double2float_rn(ri - (double)h);
          }
          wh[t] = h;
          wl[t] = l;
        } else {
          const float2* w2 = reinterpret_cast<const float2*>(wp);
          D2 w{w2[t].x, w2[t].y};
          for (int qq = 1; qq < Q; ++qq) w = d2_merge(w, D2{w2[qq * R + t].x, w2[qq * R + t].y});
          const float h = __fadd_rn(w.s, w.c);
          wh[t] = h;
          wl[t] = __fsub_rn(w.c, __fsub_rn(h, w.s));
        }
      }
    }
    __syncthreads();
    // ---- column phase
    if (jc < n) {
      const float* col = tl + (size_t)jc * R;
      for (int x = 0; x < RG; ++x) {
        const int r = g + G * ((x + jc) & (RG - 1));
        d2_fma(acc0, col[r], wh[r], wl[r]);
      }
    }
    if (G == 1 && t + T < n) {
      const int j = t + T;
      const float* col = tl + (size_t)j * R;
      for (int x = 0; x < R; ++x) {
        const int r = (x + j) & (R - 1);
        d2_fma(acc1, col[r], wh[r], wl[r]);
      }
    }
  }
  // ---- per-CTA partials
  double* out = part + (int64_t)cta * (n + 2);
  __syncthreads();
  if (G > 1) {
    red[t] = jc < n ? (double)acc0.s + (double)acc0.c : 0.0;
    __syncthreads();
    if (t < n) {
      double s = 0.0;
      for (int gg = 0; gg < G; ++gg) s += red[gg + G * t];
      out[t] = s;
    }
  } else {
    if (t < n) out[t] = (double)acc0.s + (double)acc0.c;
    if (t + T < n) out[t + T] = (double)acc1.s + (double)acc1.c;
  }
  if (RESID) {
    __shared__ double sred[2][T / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if ((t & 31) == 0) {
      sred[0][t >> 5] = s1;
      sred[1][t >> 5] = s2;
    }
    __syncthreads();
    if (t == 0) {
      double a = 0.0, c = 0.0;
      for (int w = 0; w < T / 32; ++w) {
        a += sred[0][w];
        c += sred[1][w];
      }
      out[n] = a;
      out[n + 1] = c;
    }
  } else if (t == 0) {
    out[n] = 0.0;
    out[n + 1] = 0.0;
  }
}

// Dot phase of the operator pass (not RESID): warp w takes rows w RW .. w RW
// + RW - 1 of the tile (RW = R / 8) with LR = 32 / RW lanes per row; lane
// (rs, cl) = (lane mod RW, lane / RW) sums the DCL = NC / LR columns
// dot_col(cl, k), k = 0 .. DCL - 1: runs of SB = RW / 4 consecutive columns,
// run cl of every LR runs.  At a column pitch of 4 mod 32 the 32 lanes of one
// load (fixed k) touch banks RW cl + rs + const, all distinct; a row's LR
// partial sums meet by shuffles, with no shared-memory merge and no barrier.
template <int NC>
struct DotMap {
  static constexpr int R = pass32n_tile(NC) / NC, RW = R / 8, LR = 32 / RW, SB = RW / 4, DCL = NC / LR;
  static_assert(RW >= 4 && RW <= 32 && DCL % 2 == 0, "dot map");
};
template <int NC>
__host__ __device__ constexpr int dot_col(int cl, int k) {
  return DotMap<NC>::SB * cl + k % DotMap<NC>::SB + (k / DotMap<NC>::SB) * DotMap<NC>::SB * DotMap<NC>::LR;
}

// Specialised body for NC = pass32_class(n) staged columns (n <= NC real).
// Tile: R = TE / NC rows (RB = R / 32 row blocks of 32 rows), columns at
// pitch P = pass32n_pitch(NC) in shared memory.
//   dot phase   : RESID: warp w takes row blocks rb0 .. rb0 + DR - 1 and
//                 the DC columns of column group cg (M = 8 / min(RB, 8) groups
//                 share a row block; their partials are merged through shared
//                 memory); lane = row; FP64, one DFMA per element.  Else the
//                 lanes of DotMap, by the extraction (xs_step) with one sigma
//                 for the pass, from the column maxima of |A| that the
//                 residual pass recorded (cmax) and the largest |ph_j|.
//   column phase: thread (jc, g) = (t mod NC, t / NC) takes column jc over
//                 the RPT rows g RPT .. of the tile (G = T / NC row groups),
//                 by the extraction with sigma from the column's maximum of
//                 |A| (cmax; the residual pass takes the tile's own and keeps
//                 the running maximum for its output) and the tile's largest
//                 |w_i|, and flushes the tile's sum into a compensated pair.
//                 A margin of 2^MG in sigma keeps that integer sum within 2^24
//                 (an exact conversion).  16-byte reads of the column, and
//                 of w_i (one address per row group: a broadcast).
// Output: part[cta][0..n) the CTA's vector partial, [n], [n+1] the scalars
// (RESID) or zeros, and for RESID [n+2, 2n+2) its column maxima of |A|
// (stride pass_out_len(n) for RESID, n + 2 otherwise).
template <int NC, bool RESID>
__device__ __forceinline__ void pass32n_body(const float* __restrict__ A, int64_t lda, int64_t d, int n,
                                             int cw, const double* __restrict__ b,
                                             const double* __restrict__ vin,
                                             const double* __restrict__ cmax,
                                             double* __restrict__ part, int cta, int nctas,
                                             unsigned char* smem) {
  constexpr int T = kP32Threads;
  constexpr int TE = pass32n_tile(NC), S = pass32n_stages(NC);
  constexpr int R = TE / NC, RB = R / 32, P = pass32n_pitch(NC), TP = NC * P;
  constexpr int DR = RB >= 8 ? RB / 8 : 1;   // dot rows per thread
  constexpr int M = RB >= 8 ? 1 : 8 / RB;    // dot column groups per row block
  constexpr int DC = NC / M;                 // dot columns per thread
  constexpr int WPB = 8 / M;                 // warps per column group
  constexpr int G = T / NC, RPT = R / G;     // column phase: row groups, rows per thread
  constexpr int MG = RPT <= 16 ? 2 : 3;      // RPT 2^(22 - MG) <= 2^24
  constexpr int DLR = DotMap<NC>::LR;        // operator pass: lanes per row
  static_assert(RPT % 4 == 0 && RPT <= 32 && G * NC == T, "column-phase shape");
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  float* tiles = reinterpret_cast<float*>(smem);
  unsigned char* vreg = reinterpret_cast<unsigned char*>(tiles + S * TP);  // 8 NC bytes
  double* vd = reinterpret_cast<double*>(vreg);   // RESID: x
  float4* pvx = reinterpret_cast<float4*>(vreg);  // else (ph0, ph1, pl0, pl1) per column pair
  double* wpd = reinterpret_cast<double*>(vreg + 8 * NC);  // T: merge space
  float* qhs = reinterpret_cast<float*>(wpd + T);  // R: w_i = qhs[i] + qls[i]
  float* qls = qhs + R;
  __shared__ unsigned s_wmax[2];  // by tile parity: bits of the largest |qh_i|
  __shared__ int s_e;             // dot phase: max_j of the exponent bounds of cmax_j |ph_j|
  auto issue = [&](int64_t i0, float* buf) {
    if (cw == 4) p32n_issue<NC, R, 4, P>(A, lda, d, n, i0, buf);
    else if (cw == 2) p32n_issue<NC, R, 2, P>(A, lda, d, n, i0, buf);
    else p32n_issue<NC, R, 1, P>(A, lda, d, n, i0, buf);
  };
  if (t == 0) {
    s_wmax[0] = 0u;
    s_wmax[1] = 0u;
    s_e = -1000;
  }
  __syncthreads();
  if (RESID) {
    for (int j = t; j < NC; j += T) vd[j] = j < n ? vin[j] : 0.0;
  } else {
    // entry h = (k2, cl) of the dot phase's table: columns dot_col(cl, 2 k2)
    // and dot_col(cl, 2 k2 + 1)
    for (int h = t; h < NC / 2; h += T) {
      const int cl = h % DLR, k = 2 * (h / DLR);
      const int c0 = dot_col<NC>(cl, k), c1 = dot_col<NC>(cl, k + 1);
      const double x0 = c0 < n ? vin[c0] : 0.0, x1 = c1 < n ? vin[c1] : 0.0;
      const float h0 = __double2float_rn(x0), h1 = __double2float_rn(x1);
      pvx[h] = make_float4(h0, h1, __double2float_rn(x0 - (double)h0), __double2float_rn(x1 - (double)h1));
      int e = -1000;
      if (c0 < n)
        e = p32_exp_bound(__float_as_uint(__double2float_ru(cmax[c0]))) +
            p32_exp_bound(__float_as_uint(fabsf(h0)));
      if (c1 < n)
        e = max(e, p32_exp_bound(__float_as_uint(__double2float_ru(cmax[c1]))) +
                       p32_exp_bound(__float_as_uint(fabsf(h1))));
      atomicMax(&s_e, e);
    }
  }
  // column phase: this thread's column, row group and (not RESID) the
  // exponent part of sigma from the column's maximum
  const int jc = t % NC, g = t / NC;
  int kc = -1000;
  if (!RESID && jc < n) kc = p32_exp_bound(__float_as_uint(__double2float_ru(cmax[jc]))) + 3 + MG;
  __syncthreads();
  // |a_ij ph_j| < 2^(s_e + 2) = 2^(k - 1)
  const XSig xd = xsig_make(RESID ? 0 : s_e + 3);
  const int rb0 = (w % WPB) * DR, cg = w / WPB;
  // operator pass at <= 16 columns per lane: this lane's (ph, pl) pairs in
  // registers for the whole pass (they are the same in every tile)
  float4 vreg_x[DotMap<NC>::DCL <= 16 ? DotMap<NC>::DCL / 2 : 1];
  if constexpr (!RESID && DotMap<NC>::DCL <= 16) {
#pragma unroll
    for (int k2 = 0; k2 < DotMap<NC>::DCL / 2; ++k2) vreg_x[k2] = pvx[k2 * DLR + (lane / DotMap<NC>::RW)];
  }
  D2 acc{0.f, 0.f};  // column jc over this thread's rows of every tile
  float cm = 0.f;    // RESID: running maximum of |A| in column jc
  double s1 = 0.0, s2 = 0.0;
  const int64_t ntiles = (d + R - 1) / R;
  // S-stage pipeline: tiles cta + m nctas, m = 0, 1, ...; stage m mod S
  for (int m = 0; m < S - 1; ++m) {
    const int64_t tm = cta + (int64_t)m * nctas;
    if (tm < ntiles) issue(tm * R, tiles + m * TP);
    else p32_commit();
  }
  for (int64_t m = 0;; ++m) {
    const int64_t tile = cta + m * nctas;
    if (tile >= ntiles) break;
    p32_wait<S - 2>();  // this thread's copies of tile m have landed
    // everyone's have, and tile m - 1 is consumed: its stage (refilled next),
    // qhs/qls and s_wmax[(m + 1) & 1] are free
    __syncthreads();
    if (t == 0) s_wmax[(m + 1) & 1] = 0u;
    const int64_t next = tile + (int64_t)(S - 1) * nctas;
    if (next < ntiles) issue(next * R, tiles + (int)((m + S - 1) % S) * TP);
    else p32_commit();
    const float* tl = tiles + (int)(m % S) * TP;
    const int64_t i0 = tile * R;
    unsigned* wmax = &s_wmax[m & 1];
    // ---- dot phase
    const float* tdot = tl + cg * DC * P + rb0 * 32 + lane;
    if (RESID) {
      // four independent DFMA chains per row (FP64 latency), summed in order
      constexpr int KS = DC >= 4 ? 4 : DC;
      double wd[DR], wk[DR][KS];
#pragma unroll
      for (int q = 0; q < DR; ++q)
#pragma unroll
        for (int kk = 0; kk < KS; ++kk) wk[q][kk] = 0.0;
#pragma unroll
      for (int jj = 0; jj < DC; ++jj) {
        const double xj = vd[cg * DC + jj];
#pragma unroll
        for (int q = 0; q < DR; ++q)
          wk[q][jj % KS] = fma(f2d_exact(tdot[jj * P + q * 32]), xj, wk[q][jj % KS]);
      }
#pragma unroll
      for (int q = 0; q < DR; ++q) {
        wd[q] = wk[q][0];
#pragma unroll
        for (int kk = 1; kk < KS; ++kk) wd[q] += wk[q][kk];
      }
      if (M == 1) {
        unsigned mx = 0u;
#pragma unroll
        for (int q = 0; q < DR; ++q) {
          const int r = (rb0 + q) * 32 + lane;
          const int64_t i = i0 + r;
          float h = 0.f, l = 0.f;
          if (i < d) {
            const double bi = b[i];
            const double ri = bi - wd[q];
            s1 = fma(ri, ri, s1);
            s2 = fma(bi, bi, s2);
            h = __double2float_rn(ri);
            l = __double2float_rn(ri - (double)h);
          }
          qhs[r] = h;
          qls[r] = l;
          mx = max(mx, __float_as_uint(fabsf(h)));
        }
        mx = __reduce_max_sync(0xffffffffu, mx);
        if (lane == 0) atomicMax(wmax, mx);
      } else {
        wpd[cg * R + rb0 * 32 + lane] = wd[0];
      }
    } else {
      // lane (rs, cl) of DotMap: column pairs (k, k + 1) as the two lanes
      constexpr int RW = DotMap<NC>::RW, DCL = DotMap<NC>::DCL;
      const int rs = lane % RW, cl = lane / RW, r = w * RW + rs;
      const float* ta = tl + (size_t)(DotMap<NC>::SB * cl) * P + r;
      unsigned sx = 0u - (unsigned)DCL * xd.sb;
      f2p lo[2] = {0ull, 0ull};
#pragma unroll
      for (int k = 0; k < DCL; k += 2) {
        float4 xv;
        if constexpr (DCL <= 16) xv = vreg_x[k / 2];
        else xv = pvx[(k / 2) * DLR + cl];
        xs_step(sx, lo[(k >> 1) & 1], f2p_make(ta[dot_col<NC>(0, k) * P], ta[dot_col<NC>(0, k + 1) * P]),
                f2p_make(xv.x, xv.y), f2p_make(xv.z, xv.w), xd.s2);
      }
      const float2 l2 = f2p_split(f2p_add(lo[0], lo[1]));
      float ls = __fadd_rn(l2.x, l2.y);
#pragma unroll
      for (int o = RW; o < 32; o <<= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        ls = __fadd_rn(ls, __shfl_xor_sync(0xffffffffu, ls, o));
      }
      unsigned mx = 0u;
      if (cl == 0) {
        const float2 v = xs_value(sx, ls, xd);
        qhs[r] = v.x;
        qls[r] = v.y;
        mx = __float_as_uint(fabsf(v.x));
      }
      mx = __reduce_max_sync(0xffffffffu, mx);
      if (lane == 0) atomicMax(wmax, mx);
    }
    if (RESID && M > 1) {
      __syncthreads();
      if (t < R) {  // whole warps (R is a multiple of 32)
        float h = 0.f, l = 0.f;
        double wsum = 0.0;
#pragma unroll
        for (int q = 0; q < M; ++q) wsum += wpd[q * R + t];
        const int64_t i = i0 + t;
        if (i < d) {
          const double bi = b[i];
          const double ri = bi - wsum;
          s1 = fma(ri, ri, s1);
          s2 = fma(bi, bi, s2);
          h = __double2float_rn(ri);
          l = __double2float_rn(ri - (double)h);
        }
        qhs[t] = h;
        qls[t] = l;
        const unsigned mx = __reduce_max_sync(0xffffffffu, __float_as_uint(fabsf(h)));
        if (lane == 0) atomicMax(wmax, mx);
      }
    }
    __syncthreads();
    // ---- column phase
    {
      const float* ca = tl + jc * P + g * RPT;
      const float* qa = qhs + g * RPT;
      const float* qb = qls + g * RPT;
      float4 av[RPT / 4];
#pragma unroll
      for (int v = 0; v < RPT / 4; ++v) av[v] = *reinterpret_cast<const float4*>(ca + 4 * v);
      int k = kc;
      if (RESID) {
        float ct = 0.f;
#pragma unroll
        for (int v = 0; v < RPT / 4; ++v)
          ct = fmaxf(ct, fmaxf(fmaxf(fabsf(av[v].x), fabsf(av[v].y)), fmaxf(fabsf(av[v].z), fabsf(av[v].w))));
        cm = fmaxf(cm, ct);
        k = p32_exp_bound(__float_as_uint(ct)) + 3 + MG;
      }
      // |a_ij qh_i| < 2^(ecol + eq + 2) = 2^(k - 1 - MG)
      const XSig xc = xsig_make(k + p32_exp_bound(*wmax));
      unsigned sx = 0u - (unsigned)RPT * xc.sb;
      f2p lo0 = 0ull, lo1 = 0ull;
#pragma unroll
      for (int v = 0; v < RPT / 4; ++v) {
        const float4 h4 = *reinterpret_cast<const float4*>(qa + 4 * v);
        const float4 l4 = *reinterpret_cast<const float4*>(qb + 4 * v);
        xs_step(sx, lo0, f2p_make(av[v].x, av[v].y), f2p_make(h4.x, h4.y), f2p_make(l4.x, l4.y), xc.s2);
        xs_step(sx, lo1, f2p_make(av[v].z, av[v].w), f2p_make(h4.z, h4.w), f2p_make(l4.z, l4.w), xc.s2);
      }
      xs_flush(acc, sx, f2p_add(lo0, lo1), xc);
    }
  }
  // ---- per-CTA partials: each column's G row groups summed in FP64
  double* out = part + (int64_t)cta * (RESID ? pass_out_len(n) : (int64_t)n + 2);
  __syncthreads();  // the last tile's reads of the merge space and the tiles are done
  wpd[t] = (double)acc.s + (double)acc.c;  // t = g NC + jc
  float* cmx = tiles;                       // T floats
  if (RESID) cmx[t] = cm;
  __syncthreads();
  if (t < n) {
    double s = 0.0;
    float mx = 0.f;
#pragma unroll
    for (int gg = 0; gg < G; ++gg) {
      s += wpd[gg * NC + t];
      if (RESID) mx = fmaxf(mx, cmx[gg * NC + t]);
    }
    out[t] = s;
    if (RESID) out[n + 2 + t] = (double)mx;
  }
  if (RESID) {
    __shared__ double sred[2][T / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if (lane == 0) {
      sred[0][w] = s1;
      sred[1][w] = s2;
    }
    __syncthreads();
    if (t == 0) {
      double a = 0.0, c = 0.0;
      for (int q = 0; q < T / 32; ++q) {
        a += sred[0][q];
        c += sred[1][q];
      }
      out[n] = a;
      out[n + 1] = c;
    }
  } else if (t == 0) {
    out[n] = 0.0;
    out[n + 1] = 0.0;
  }
}

// CTAs per SM of each body (the shared-memory pipeline allows three; the
// 256-wide body's 32 column accumulators per thread need 128 registers).
__host__ __device__ constexpr int pass32_ctas_per_sm(int nc) { return nc >= 256 ? 2 : 3; }

// Kernel wrappers (one per width class, each compiled for its own occupancy)
// live in the translation units that launch them.
}  // namespace msk
