// autotune.cu — the autotuner: picks the tile and chunk schedules of the
// batched path by timing candidate values of the registry knobs on the
// device, on a caller-supplied batch of requests, and leaves the fastest
// values set.
//
// Knobs (coordinate descent, in this order, each timed with CUDA events on
// the caller's stream, median of `reps` runs after one warm-up run):
//   cs.fixed           fixed-width CountSketch kernels on (1) or off (0);
//   cs.l2_budget_bytes column-chunk width of the CountSketch: the bytes of Y a
//                      chunk may keep resident in L2 (1/8 .. 3/5 of L2);
//       both timed on cs_sketch of the request with the most elements;
//   batch.kt_per       K tiles per CTA of the batched tensor-core GEMM;
//   batch.round        CG iterations per captured graph round;
//   pass.ctas_per_sm   refinement-pass CTAs per SM;
//       timed on msk_batch_lstsq of the whole batch.
// Knobs change speed only: results differ at most by rounding order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "msk_internal.h"

using namespace msk;

namespace {

struct Knob {
  const char* name;
  std::vector<long long> cands;
  bool batch;  // timed on the batch solve (else on the CountSketch)
};

std::vector<Knob> knobs_for_device() {
  int dev = 0, l2 = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess || l2 <= 0)
    l2 = 64 << 20;
  const long long L = l2;
  return {
      {"cs.fixed", {1, 0}, false},
      {"cs.l2_budget_bytes", {L / 8, L / 4, L * 2 / 5, L * 3 / 5}, false},
      {"batch.kt_per", {8, 16, 32}, true},
      {"batch.round", {2, 4, 8}, true},
      {"pass.ctas_per_sm", {1, 2, 3}, true},
  };
}

// The request with the most elements (the CountSketch timing case).
int largest(const msk_batch_item* items, int nitems) {
  int best = 0;
  for (int j = 1; j < nitems; ++j)
    if (items[j].d * items[j].n > items[best].d * items[best].n) best = j;
  return best;
}

// Row pitch of the timing sketch's Y: [A b] columns rounded up to a multiple
// of 4, as the batched path lays Y out (the fixed-width FP32 kernels need it).
int64_t cs_ldy(const msk_batch_item& it) { return (it.n + 1 + 3) / 4 * 4; }

size_t cs_scratch(const msk_batch_item& it) {
  const int64_t k = 2 * it.n * it.n;
  return (size_t)k * (size_t)cs_ldy(it) * sizeof(float);
}

}  // namespace

extern "C" {

size_t msk_autotune_workspace(const msk_batch_item* items, int nitems, int refine) {
  if (!items || nitems <= 0) return 0;
  // the batch workspace depends on batch.kt_per (split-K partials): take the
  // largest over the candidates
  const long long saved = msk_tune_get("batch.kt_per", -1);
  size_t need = 0;
  for (long long kt : {8LL, 16LL, 32LL}) {
    msk_tune_set("batch.kt_per", kt);
    need = std::max(need, msk_batch_workspace(items, nitems, refine));
  }
  if (saved < 0) msk_tune_clear("batch.kt_per");
  else msk_tune_set("batch.kt_per", saved);
  const size_t cs = cs_scratch(items[largest(items, nitems)]);
  return (need + 255) / 256 * 256 + (cs + 255) / 256 * 256;
}

int msk_autotune(const msk_batch_item* items, int nitems, int refine, double tol, int32_t max_iter,
                 int reps, char* report, size_t report_bytes, void* ws, size_t ws_bytes,
                 void* stream) {
  if (!items) return -1;
  if (nitems < 1) return -2;
  if (refine != 0 && refine != 1) return -3;
  if (reps < 1 || reps > 100) return -6;
  if (!ws || ws_bytes < msk_autotune_workspace(items, nitems, refine) ||
      (reinterpret_cast<uintptr_t>(ws) & 255) != 0)
    return MSK_ENOMEM;
  cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : cudaStreamLegacy;
  size_t batch_ws = 0;
  {
    const long long saved = msk_tune_get("batch.kt_per", -1);
    for (long long kt : {8LL, 16LL, 32LL}) {
      msk_tune_set("batch.kt_per", kt);
      batch_ws = std::max(batch_ws, msk_batch_workspace(items, nitems, refine));
    }
    if (saved < 0) msk_tune_clear("batch.kt_per");
    else msk_tune_set("batch.kt_per", saved);
  }
  batch_ws = (batch_ws + 255) / 256 * 256;
  char* base = static_cast<char*>(ws);
  void* Y = base + batch_ws;
  const msk_batch_item& big = items[largest(items, nitems)];
  std::vector<msk_lstsq_info> infos(nitems);
  cudaEvent_t e0, e1;
  MSK_CUDA(cudaEventCreate(&e0));
  MSK_CUDA(cudaEventCreate(&e1));
  // one timed run of the case a knob is tuned on; returns ms or < 0 on error
  auto run = [&](bool batch) -> double {
    int rc;
    if (batch) {
      rc = msk_batch_lstsq(items, nitems, refine, tol, max_iter, infos.data(), base, batch_ws, st);
      if (rc == MSK_ENOCONV) rc = MSK_OK;
    } else {
      const int64_t k = 2 * big.n * big.n;
      rc = cs_sketch(big.A, MSK_F32, big.d, big.n, big.lda, big.b, k, big.seed, Y, cs_ldy(big),
                     MSK_CS_ATOMIC, nullptr, 0, st);
    }
    return rc ? -1.0 - std::abs((double)rc) : 0.0;
  };
  auto timed = [&](bool batch) -> double {
    if (run(batch) < 0) return -1.0;  // warm-up
    std::vector<double> t;
    for (int r = 0; r < reps; ++r) {
      if (cudaEventRecord(e0, st) != cudaSuccess) return -1.0;
      if (run(batch) < 0) return -1.0;
      if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return -1.0;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      t.push_back(ms);
    }
    std::sort(t.begin(), t.end());
    return t[t.size() / 2];
  };
  std::string js = "{\"knobs\": {";
  int status = MSK_OK;
  bool first = true;
  for (const Knob& kb : knobs_for_device()) {
    const long long before = msk_tune_get(kb.name, -1);
    long long best_v = 0;
    double best_t = -1.0;
    std::string times;
    for (long long v : kb.cands) {
      msk_tune_set(kb.name, v);
      const double t = timed(kb.batch);
      if (t < 0.0) {
        status = MSK_ECUDA;
        break;
      }
      char buf[96];
      std::snprintf(buf, sizeof(buf), "%s\"%lld\": %.6f", times.empty() ? "" : ", ", v, t);
      times += buf;
      if (best_t < 0.0 || t < best_t) {
        best_t = t;
        best_v = v;
      }
    }
    if (status) {
      if (before < 0) msk_tune_clear(kb.name);
      else msk_tune_set(kb.name, before);
      break;
    }
    msk_tune_set(kb.name, best_v);
    char head[160];
    std::snprintf(head, sizeof(head), "%s\"%s\": {\"chosen\": %lld, \"timed_on\": \"%s\", \"ms\": {",
                  first ? "" : ", ", kb.name, best_v, kb.batch ? "batch" : "countsketch");
    js += head;
    js += times + "}}";
    first = false;
  }
  js += "}, \"reps\": " + std::to_string(reps) + ", \"requests\": " + std::to_string(nitems) + "}";
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (report && report_bytes > 0) {
    const size_t n = std::min(report_bytes - 1, js.size());
    js.copy(report, n);
    report[n] = '\0';
  }
  return status;
}

}  // extern "C"
