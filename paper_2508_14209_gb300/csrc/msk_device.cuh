// msk_device.cuh — device-side helpers shared by the libmsketch kernels:
// the splitmix64 counter generator, the CountSketch bucket/sign map
// (Definition 3, Section 4) and the binary32 polar-method Gaussian sampler
// (the Gaussian sketch of Section 1).  Written from the published definitions
// (Steele, Lea, Flood, OOPSLA 2014 for splitmix64; Marsaglia & Bray 1964 for
// the polar method), every float step an explicit round-to-nearest
// intrinsic so that no contraction or approximation changes a bit.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace msk {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kStreamMul = 0xD1B54A32D192ED03ull;
constexpr uint64_t kTagHash = 0;
constexpr uint64_t kTagGauss = 2;
constexpr uint64_t kTagSrhtSign = 5;  // SRHT: the signs of D
constexpr uint64_t kTagSrhtRow = 6;   // SRHT: the rows P samples

__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Key of stream `tag` for a user seed.
__host__ __device__ __forceinline__ uint64_t stream_key(uint64_t seed, uint64_t tag) {
  return mix64(seed ^ (tag * kStreamMul));
}

// Output i of splitmix64 started from state `key`.
__host__ __device__ __forceinline__ uint64_t draw(uint64_t key, uint64_t i) {
  return mix64(key + (i + 1) * kGamma);
}

// Checked builds (compiled with MSK_CHECKED): a failed index check records
// its site in g_msk_check (the first one stays) and the guarded access is
// skipped; msk_check_status reports and clears it.  Other builds evaluate
// nothing.  Sites:
constexpr int kCheckBucket = 1;  // CountSketch bucket h(i) < k
constexpr int kCheckSlice = 2;   // sliced FP64 stage: |G| < 2^eG, |Y[:,c]| < 2^eY_c
constexpr int kCheckBatch = 3;   // batch tables: problem and chunk indices
#ifdef MSK_CHECKED
extern __device__ int g_msk_check;
__device__ __forceinline__ bool msk_index_ok(bool cond, int site) {
  if (!cond) atomicCAS(&g_msk_check, 0, site);
  return cond;
}
#define MSK_CHECK_OR(cond, site, action) \
  if (!::msk::msk_index_ok((cond), (site))) action
#else
#define MSK_CHECK_OR(cond, site, action)
#endif

// Bucket in [0,k) from the top 32 bits (multiply-shift), sign from bit 0.
__device__ __forceinline__ uint32_t bucket_of(uint64_t z, uint32_t k) {
  return (uint32_t)(((z >> 32) * (uint64_t)k) >> 32);
}
__device__ __forceinline__ bool negative_of(uint64_t z) { return (z & 1ull) != 0; }

// ln(s) for a normal positive binary32 s:
//   s = m 2^e, m in [sqrt(1/2), sqrt(2)),  ln s = e ln2 + 2 atanh(t),
//   t = (m-1)/(m+1),  atanh(t) ~ t (1 + t^2/3 + t^4/5 + t^6/7 + t^8/9).
__device__ __forceinline__ float ln_f32(float s) {
  const float kSqrt2 = __uint_as_float(0x3FB504F3u);
  const float kLn2 = __uint_as_float(0x3F317218u);
  const float c3 = __uint_as_float(0x3EAAAAABu);
  const float c5 = __uint_as_float(0x3E4CCCCDu);
  const float c7 = __uint_as_float(0x3E124925u);
  const float c9 = __uint_as_float(0x3DE38E39u);
  const uint32_t bits = __float_as_uint(s);
  int e = (int)((bits >> 23) & 0xFFu) - 127;
  float m = __uint_as_float((bits & 0x007FFFFFu) | 0x3F800000u);
  if (m > kSqrt2) {
    m = __fmul_rn(m, 0.5f);
    e += 1;
  }
  const float t = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
  const float w = __fmul_rn(t, t);
  float p = c9;
  p = __fadd_rn(__fmul_rn(p, w), c7);
  p = __fadd_rn(__fmul_rn(p, w), c5);
  p = __fadd_rn(__fmul_rn(p, w), c3);
  p = __fadd_rn(__fmul_rn(p, w), 1.0f);
  const float lnm = __fmul_rn(__fmul_rn(2.0f, t), p);
  return __fadd_rn(__fmul_rn((float)e, kLn2), lnm);
}

// Standard normal number `elem` of the stream `key` (polar method; attempt a
// uses draw index elem*2^16 + a; u, v are odd multiples of 2^-24 in (-1,1)).
// The rejection loop only draws; the logarithm, division and square root
// run once, after it, so that a warp whose lanes accept at different
// attempts does not repeat them.
__device__ __forceinline__ float gauss_std(uint64_t key, uint64_t elem) {
  float u = 0.0f, s = 1.0f;
  for (uint32_t a = 0; a < 65536u; ++a) {
    const uint64_t z = draw(key, (elem << 16) | a);
    const int32_t U = (int32_t)(z >> 40);
    const int32_t V = (int32_t)((z >> 16) & 0xFFFFFFu);
    u = __fmul_rn((float)(2 * U + 1 - (1 << 24)), 0x1p-24f);
    const float v = __fmul_rn((float)(2 * V + 1 - (1 << 24)), 0x1p-24f);
    s = __fadd_rn(__fmul_rn(u, u), __fmul_rn(v, v));
    if (s < 1.0f) break;
  }
  if (!(s < 1.0f)) return 0.0f;
  const float q = __fdiv_rn(__fmul_rn(-2.0f, ln_f32(s)), s);
  return __fmul_rn(u, __fsqrt_rn(q));
}

// L2 reductions (the atomic adds of Algorithm 2, issued without a return value).
__device__ __forceinline__ void red_add(double* p, double v) {
  asm volatile("red.relaxed.gpu.global.add.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}
__device__ __forceinline__ void red_add(float* p, float v) {
  asm volatile("red.relaxed.gpu.global.add.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}
__device__ __forceinline__ void red_add_v4(float* p, float a, float b, float c, float d) {
  asm volatile("red.relaxed.gpu.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a),
               "f"(b), "f"(c), "f"(d)
               : "memory");
}

// Sign of a CountSketch row applied by flipping the sign bit.
__device__ __forceinline__ double flip(double x, unsigned long long s) {
  return __longlong_as_double(__double_as_longlong(x) ^ s);
}
__device__ __forceinline__ float flip(float x, unsigned s) {
  return __uint_as_float(__float_as_uint(x) ^ s);
}


// Double-single arithmetic: a value carried as an unevaluated sum hi + lo of
// two binary32 numbers (Dekker 1971; Knuth's TwoSum; the exact product
// a*b = hi + lo from one FMA), about 48 significant bits.
struct DS {
  float hi, lo;
};
__device__ __forceinline__ DS ds_add(DS a, float bh, float bl) {
  const float s = a.hi + bh;
  const float v = s - a.hi;
  float e = (a.hi - (s - v)) + (bh - v);  // TwoSum error of a.hi + bh
  e += a.lo + bl;
  const float h = s + e;
  return DS{h, e - (h - s)};
}
// acc += a * (xh + xl), a exact binary32.
__device__ __forceinline__ DS ds_fma(DS acc, float a, float xh, float xl) {
  const float ph = a * xh;
  float pl = fmaf(a, xh, -ph);  // exact: a*xh = ph + pl
  pl = fmaf(a, xl, pl);
  return ds_add(acc, ph, pl);
}
__device__ __forceinline__ DS ds_shfl_xor(DS v, int m) {
  return DS{__shfl_xor_sync(0xffffffffu, v.hi, m), __shfl_xor_sync(0xffffffffu, v.lo, m)};
}

}  // namespace msk
