// noalloc.cu — msk_gemm_noalloc: the Gaussian-stage GEMM (Z = G Y) with its
// scratch space in a fixed array that this library owns, for callers that must
// not allocate device memory themselves.
//
// Who needs this: some host programs are not allowed to call cudaMalloc at the
// point where they want a sketch — for example a plug-in living inside a larger
// application whose own allocator owns every byte of device memory, or a
// latency-critical loop that cannot afford the implicit device-wide
// synchronisation an allocation may cause.  Such callers still pass their own
// Y and Z; only the scratch (the Gaussian G or its slices, the slices of Y and
// the split-K partial products) comes from here.
//
// The scratch is the file-scope array below, kNoallocScratchBytes long.  Every
// GPU that loads this library reserves it for the life of the process.  All
// calls share it: a call overwrites what the previous call left there, and two
// calls whose GPU work overlaps in time (for example on two streams) race on it
// and produce garbage — order such calls on one stream or synchronise between
// them.  Nothing in the scratch has to start at zero: the Gaussian kernel
// writes every entry of G and the GEMM kernel writes every partial before the
// reduction reads it.
//
// Host code cannot use the array's name as a device address (in host code the
// name refers to a host-side stand-in).  The device address is therefore
// looked up with cudaGetSymbolAddress once per device, with that device
// current, on the first call made while that device is current; that first
// call should come before any stream capture begins on that device.  The
// address belongs to the device's current context: after cudaDeviceReset (or
// any other teardown of that context) the module is loaded again, possibly
// elsewhere, so the cached address is keyed by the context and looked up
// afresh, by the next call, once the context has changed (make that call
// before any capture too).
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "msk_internal.h"

namespace msk {

constexpr size_t kNoallocScratchBytes = MSK_NOALLOC_SCRATCH_BYTES;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

namespace {
// The driver API's cuCtxGetCurrent, looked up once through the runtime (no
// link against libcuda, so the library still loads where no driver is
// installed); null when unavailable.
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = [] {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &ptr, 4000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<CtxGetCurrentFn>(ptr);
    return static_cast<CtxGetCurrentFn>(nullptr);
  }();
  return fn;
}

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {nullptr};
CUcontext g_scratch_ctx[kMaxDevices] = {nullptr};
}  // namespace

// Device address of the scratch array on the current device (set up once per
// device and context).  Returns MSK_OK or MSK_ECUDA.
static int noalloc_scratch(void** out) {
  int dev = 0;
  MSK_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return MSK_ENOTSUP;
  // A thread on which the runtime has not yet made the device's context
  // current sees none here; the look-up below makes it current.
  CtxGetCurrentFn get_ctx = ctx_get_current();
  if (!get_ctx) {
    set_error_text("msk_gemm_noalloc: cuCtxGetCurrent entry point not available");
    return MSK_ECUDA;
  }
  CUcontext ctx = nullptr;
  if (get_ctx(&ctx) != CUDA_SUCCESS) ctx = nullptr;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev] || !ctx || g_scratch_ctx[dev] != ctx) {
    void* p = nullptr;
    MSK_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    if (get_ctx(&ctx) != CUDA_SUCCESS || !ctx) {
      set_error_text("msk_gemm_noalloc: no current CUDA context");
      return MSK_ECUDA;
    }
    g_scratch_ptr[dev] = p;
    g_scratch_ctx[dev] = ctx;
  }
  *out = g_scratch_ptr[dev];
  return MSK_OK;
}

}  // namespace msk

using namespace msk;

extern "C" int msk_gemm_noalloc(uint64_t seed, int64_t p, int64_t k, int64_t ncol, const void* Y,
                                int64_t ldy, int gemm_prec, double* Z, int64_t ldz, void* stream) {
  if (p < 1 || p >= (1LL << 24)) return -2;
  if (k < 1) return -3;
  if (ncol < 1) return -4;
  if (!Y) return -5;
  if (ldy < ncol) return -6;
  if (gemm_prec < MSK_GEMM_F64 || gemm_prec > MSK_GEMM_BF16X3) return -7;
  if (!Z) return -8;
  if (ldz < p) return -9;
  const size_t need = msk_gemm_workspace(p, k, ncol, gemm_prec);
  if (need > kNoallocScratchBytes) {
    set_error_text("msk_gemm_noalloc: problem needs more scratch than the fixed array holds");
    return MSK_ENOMEM;
  }
  void* ws = nullptr;
  int rc = noalloc_scratch(&ws);
  if (rc) return rc;
  const int y_dtype = gemm_prec == MSK_GEMM_F64 ? MSK_F64 : MSK_F32;
  return gemm_stage(seed, p, k, ncol, Y, y_dtype, ldy, gemm_prec, Z, ldz, ws,
                    kNoallocScratchBytes, as_stream(stream));
}
