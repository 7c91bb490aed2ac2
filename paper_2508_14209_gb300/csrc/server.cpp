// server.cpp — request server for least-squares solves (continuous batching).
//
// A server owns a device memory pool reserved once at creation (the budget)
// and W worker threads, each with its own CUDA stream and an equal slice of the
// pool.  Submitted requests wait in a FIFO queue.  A free worker admits, in
// arrival order, the waiting requests whose additive workspace bounds
// (msk_batch_item_bound) still fit its slice — admission by device memory, in
// time linear in the batch — solves them with one msk_batch_lstsq call and
// records, per ticket, the result summary and the latency from submission to
// completion.  A request larger than a slice (but not than the pool; larger
// ones are refused at submission) runs alone with the whole pool once the
// other workers' batches are done; no worker starts a batch meanwhile.
// While one worker's batch is on the GPU, requests that arrive meanwhile are
// admitted by the next free worker, so batches overlap on the device.
// Nothing is allocated on the device after creation.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/msketch.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Ticket {
  msk_batch_item item;
  Clock::time_point submitted;
  Clock::time_point finished;
  msk_lstsq_info info{};
  int status = 0;
  bool done = false;
};

struct Server {
  int device = 0;
  int refine = 1;
  double tol = 1e-10;
  int max_iter = 10;
  int max_batch = 64;
  size_t slice = 0;
  size_t pool_bytes = 0;
  char* pool = nullptr;
  bool exclusive = false;  // a request larger than a slice holds (or awaits) the whole pool
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> streams;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, Ticket> tickets;
  uint64_t next_ticket = 1;
  size_t max_queue = 1 << 20;
  bool stopping = false;
  int in_flight = 0;
  std::atomic<int64_t> batches{0};
  std::atomic<int64_t> solved{0};
  char last_error[256] = {0};
};

void worker_loop(Server* S, int w) {
  cudaSetDevice(S->device);
  char* const own = S->pool + (size_t)w * S->slice;
  std::vector<uint64_t> ids;
  std::vector<msk_batch_item> items;
  std::vector<msk_lstsq_info> infos;
  for (;;) {
    ids.clear();
    items.clear();
    char* arena = own;
    size_t cap = S->slice;
    bool whole = false;
    {
      std::unique_lock<std::mutex> lock(S->mu);
      S->cv_work.wait(lock, [&] {
        return (S->stopping && S->queue.empty()) || (!S->queue.empty() && !S->exclusive);
      });
      if (S->queue.empty()) return;  // stopping, nothing left
      const uint64_t head = S->queue.front();
      if (msk_batch_item_bound(&S->tickets[head].item, S->refine) > S->slice) {
        // larger than a slice: alone, with the whole pool, once the other
        // workers' batches are done (no worker starts a batch meanwhile)
        S->exclusive = true;
        S->cv_done.wait(lock, [&] { return S->in_flight == 0; });
        items.push_back(S->tickets[head].item);
        ids.push_back(head);
        S->queue.pop_front();
        arena = S->pool;
        cap = S->pool_bytes;
        whole = true;
      } else {
        // admit in arrival order while the items' additive workspace bounds
        // fit this slice (linear in the batch)
        size_t used = 0;
        while (!S->queue.empty() && (int)items.size() < S->max_batch) {
          const uint64_t id = S->queue.front();
          const size_t need = msk_batch_item_bound(&S->tickets[id].item, S->refine);
          if (used + need > S->slice) break;
          used += need;
          items.push_back(S->tickets[id].item);
          ids.push_back(id);
          S->queue.pop_front();
        }
      }
      if (items.empty()) continue;  // cannot happen: submit refuses oversized requests
      ++S->in_flight;
    }
    infos.assign(items.size(), msk_lstsq_info{});
    const int rc = msk_batch_lstsq(items.data(), (int)items.size(), S->refine, S->tol, S->max_iter,
                                   infos.data(), arena, cap, S->streams[w]);
    const auto now = Clock::now();
    {
      std::lock_guard<std::mutex> lock(S->mu);
      for (size_t j = 0; j < ids.size(); ++j) {
        Ticket& t = S->tickets[ids[j]];
        t.info = infos[j];
        t.status = (rc == MSK_ENOCONV && infos[j].converged) ? MSK_OK : rc;
        t.finished = now;
        t.done = true;
      }
      if (rc != MSK_OK && rc != MSK_ENOCONV)
        std::snprintf(S->last_error, sizeof(S->last_error), "batch status %d: %s", rc,
                      msk_last_error());
      --S->in_flight;
      if (whole) S->exclusive = false;
      S->batches += 1;
      S->solved += (int64_t)ids.size();
    }
    S->cv_done.notify_all();
    S->cv_work.notify_all();
  }
}

}  // namespace

extern "C" {

int ms_server_create(size_t mem_budget, int workers, int max_batch, int refine, double tol,
                     int32_t max_iter, void** srv) {
  if (!srv) return -7;
  if (mem_budget < (1u << 20)) return -1;
  if (workers < 1 || workers > 16) return -2;
  if (max_batch < 1) return -3;
  if (refine != 0 && refine != 1) return -4;
  Server* S = new Server();
  S->refine = refine;
  S->tol = tol;
  S->max_iter = max_iter;
  S->max_batch = max_batch;
  S->slice = mem_budget / (size_t)workers / 256 * 256;
  S->pool_bytes = S->slice * (size_t)workers;
  if (cudaGetDevice(&S->device) != cudaSuccess || cudaMalloc(&S->pool, S->pool_bytes) != cudaSuccess) {
    delete S;
    return MSK_ENOMEM;
  }
  S->streams.resize(workers);
  for (int w = 0; w < workers; ++w) cudaStreamCreateWithFlags(&S->streams[w], cudaStreamNonBlocking);
  for (int w = 0; w < workers; ++w) S->workers.emplace_back(worker_loop, S, w);
  *srv = S;
  return MSK_OK;
}

int ms_server_submit(void* srv, const msk_batch_item* req, uint64_t* ticket) {
  Server* S = static_cast<Server*>(srv);
  if (!S) return -1;
  if (!req || !ticket) return -2;
  if (msk_batch_item_bound(req, S->refine) > S->pool_bytes) return MSK_ENOMEM;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    if (S->stopping) return MSK_EBUSY;
    if (S->queue.size() >= S->max_queue) return MSK_EBUSY;
    const uint64_t id = S->next_ticket++;
    Ticket t;
    t.item = *req;
    t.submitted = Clock::now();
    S->tickets.emplace(id, t);
    S->queue.push_back(id);
    *ticket = id;
  }
  S->cv_work.notify_one();
  return MSK_OK;
}

int ms_server_poll(void* srv, uint64_t ticket, int* done, msk_lstsq_info* info, double* latency_s) {
  Server* S = static_cast<Server*>(srv);
  if (!S) return -1;
  std::lock_guard<std::mutex> lock(S->mu);
  auto it = S->tickets.find(ticket);
  if (it == S->tickets.end()) return -2;
  const Ticket& t = it->second;
  if (done) *done = t.done ? 1 : 0;
  if (!t.done) return MSK_OK;
  if (info) *info = t.info;
  if (latency_s) *latency_s = std::chrono::duration<double>(t.finished - t.submitted).count();
  return t.status;
}

int ms_server_wait_all(void* srv) {
  Server* S = static_cast<Server*>(srv);
  if (!S) return -1;
  std::unique_lock<std::mutex> lock(S->mu);
  S->cv_done.wait(lock, [&] { return S->queue.empty() && S->in_flight == 0; });
  return MSK_OK;
}

int ms_server_stats(void* srv, int64_t* solved, int64_t* batches, int64_t* queued) {
  Server* S = static_cast<Server*>(srv);
  if (!S) return -1;
  std::lock_guard<std::mutex> lock(S->mu);
  if (solved) *solved = S->solved.load();
  if (batches) *batches = S->batches.load();
  if (queued) *queued = (int64_t)S->queue.size();
  return MSK_OK;
}

const char* ms_server_error(void* srv) {
  Server* S = static_cast<Server*>(srv);
  return S ? S->last_error : "";
}

int ms_server_destroy(void* srv) {
  Server* S = static_cast<Server*>(srv);
  if (!S) return -1;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    S->stopping = true;
  }
  S->cv_work.notify_all();
  for (auto& t : S->workers) t.join();
  for (auto st : S->streams) cudaStreamDestroy(st);
  cudaFree(S->pool);
  delete S;
  return MSK_OK;
}

}  // extern "C"
