// gaussian.cu — the p x k Gaussian G of the multisketch's second stage
// (Gaussian sketch with N(0,1/p) entries, Section 1; Section 6.2 applies a
// 2n x 2n^2 one after the CountSketch).  Entry (r, c) is standard normal number
// r*k + c of the counter stream (tag 2), divided by sqrt(p) in binary32, then
// converted (exactly to FP64, or round-to-nearest-even to bf16 / fp16).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "msk_device.cuh"
#include "msk_internal.h"

namespace msk {

template <typename O>
__device__ __forceinline__ O convert_out(float x);
template <>
__device__ __forceinline__ double convert_out<double>(float x) { return (double)x; }
template <>
__device__ __forceinline__ float convert_out<float>(float x) { return x; }
template <>
__device__ __forceinline__ __nv_bfloat16 convert_out<__nv_bfloat16>(float x) {
  return __float2bfloat16_rn(x);
}
template <>
__device__ __forceinline__ __half convert_out<__half>(float x) { return __float2half_rn(x); }

template <typename O>
__global__ void gaussian_kernel(uint64_t key, int64_t p, int64_t k, float sqrt_p, O* __restrict__ G,
                                int64_t ldg) {
  const int64_t total = p * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / k, c = e - r * k;
    const float g = __fdiv_rn(gauss_std(key, (uint64_t)e), sqrt_p);
    G[r * ldg + c] = convert_out<O>(g);
  }
}

int launch_gaussian(uint64_t key, int64_t p, int64_t k, int out_prec, void* G, int64_t ldg,
                    cudaStream_t st) {
  const int64_t total = p * k;
  if (total == 0) return MSK_OK;
  // sqrt(p) rounded once in binary32 (p < 2^24 is exact in binary32)
  const float sqrt_p = __builtin_sqrtf((float)p);
  const unsigned grid = (unsigned)std::min<int64_t>((total + 255) / 256, (int64_t)num_sms() * 32);
  switch (out_prec) {
    case MSK_GEMM_F64:
      gaussian_kernel<double><<<grid, 256, 0, st>>>(key, p, k, sqrt_p, static_cast<double*>(G), ldg);
      break;
    case MSK_GEMM_F32:
      gaussian_kernel<float><<<grid, 256, 0, st>>>(key, p, k, sqrt_p, static_cast<float*>(G), ldg);
      break;
    case MSK_GEMM_BF16:
      gaussian_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>(key, p, k, sqrt_p,
                                                           static_cast<__nv_bfloat16*>(G), ldg);
      break;
    case MSK_GEMM_F16:
      gaussian_kernel<__half><<<grid, 256, 0, st>>>(key, p, k, sqrt_p, static_cast<__half*>(G), ldg);
      break;
    default:
      return -4;
  }
  MSK_CHECK_LAUNCH("gaussian_kernel");
  return MSK_OK;
}

}  // namespace msk
