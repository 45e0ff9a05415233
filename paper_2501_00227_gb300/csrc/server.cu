// server.cpp -- serving entry points of libtn (tn_server_create, tn_submit,
// tn_poll, tn_server_destroy): continuous batching of contraction requests.
//
// Requests of any size and semiring arrive at any time.  A worker thread
// admits a pending request as soon as (a) the predicted peak workspace of its
// plan (the space complexity of its order, Sec. 4.1 of arXiv:2501.00227,
// times the bytes per entry) fits in the unused part of the HBM budget and
// (b) fewer than max_inflight requests run.  Each admitted request gets a
// stream from a pool and a stream-ordered workspace allocation; its kernels
// overlap on the device with those of every other running request.  The
// worker retires finished requests in completion order, decodes their result
// on the host and frees their workspace, which admits more requests.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "kernels.h"
#include "tn_internal.h"

namespace tn {
int contract_enqueue(const tn_plan_s* p, tn_semiring_t s, const dev::ModTable& mods,
                     int32_t nprimes, void* ws, cudaStream_t st, void* d_raw,
                     cudaEvent_t* step_events);
int decode_raw(tn_semiring_t s, const dev::ModTable& mods, int32_t nprimes,
               const unsigned char* raw, tn_result_t* out);
size_t required_bytes(tn_plan_s* p, tn_semiring_t s, int32_t nprimes);
}  // namespace tn

namespace {

struct Request {
  uint64_t ticket;
  const tn_plan_s* plan;
  tn_semiring_t semiring;
  std::vector<uint32_t> primes;
  size_t bytes;
  // while running
  int slot = -1;
  void* ws = nullptr;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  unsigned char* h_raw = nullptr;  // pinned, TN_RAW_BYTES
  bool busy = false;
  Request req;
};

}  // namespace

struct tn_server_s {
  size_t budget = 0, used = 0;
  int32_t max_inflight = 1;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request> pending;
  std::unordered_map<uint64_t, tn_result_t> done;
  std::unordered_map<uint64_t, int> state;  // 0 pending, 1 running, 2 done
  std::vector<Slot> slots;
  uint64_t next_ticket = 1;
  std::atomic<bool> stop{false};
  std::thread worker;
  int fatal = TN_OK;
};

namespace {

int make_mod_table(tn_semiring_t s, const std::vector<uint32_t>& pr, tn::dev::ModTable* mt) {
  std::memset(mt, 0, sizeof(*mt));
  mt->q[0].p = 2;
  if (s != TN_COUNT_MODP) return TN_OK;
  for (size_t i = 0; i < pr.size(); ++i) {
    mt->q[i].p = pr[i];
    mt->q[i].r32 = static_cast<uint32_t>((uint64_t(1) << 32) % pr[i]);
    mt->q[i].mu = ~0ull / pr[i];
  }
  return TN_OK;
}

void worker_loop(tn_server_s* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  while (!S->stop.load()) {
    bool progressed = false;
    // admit: first-come first-served among requests that fit
    for (auto it = S->pending.begin(); it != S->pending.end();) {
      int free_slot = -1;
      for (size_t k = 0; k < S->slots.size(); ++k)
        if (!S->slots[k].busy) { free_slot = static_cast<int>(k); break; }
      if (free_slot < 0) break;
      if (S->used + it->bytes > S->budget) { ++it; continue; }
      Request r = *it;
      it = S->pending.erase(it);
      Slot& sl = S->slots[free_slot];
      void* ws = nullptr;
      tn::dev::ModTable mods;
      make_mod_table(r.semiring, r.primes, &mods);
      int rc = cudaMallocAsync(&ws, r.bytes, sl.stream) == cudaSuccess ? TN_OK : TN_ENOMEM;
      if (rc == TN_OK)
        rc = tn::contract_enqueue(r.plan, r.semiring, mods, static_cast<int32_t>(r.primes.size()),
                                  ws, sl.stream, static_cast<char*>(ws) + 64, nullptr);
      if (rc == TN_OK)
        rc = cudaMemcpyAsync(sl.h_raw, static_cast<char*>(ws) + 64, TN_RAW_BYTES,
                             cudaMemcpyDeviceToHost, sl.stream) == cudaSuccess ? TN_OK : TN_ECUDA;
      if (rc == TN_OK)
        rc = cudaEventRecord(sl.done, sl.stream) == cudaSuccess ? TN_OK : TN_ECUDA;
      if (rc != TN_OK) {
        if (ws) cudaFreeAsync(ws, sl.stream);
        tn_result_t res;
        std::memset(&res, 0, sizeof(res));
        res.status = rc;
        S->done[r.ticket] = res;
        S->state[r.ticket] = 2;
        continue;
      }
      r.slot = free_slot;
      r.ws = ws;
      sl.req = r;
      sl.busy = true;
      S->used += r.bytes;
      S->state[r.ticket] = 1;
      progressed = true;
    }
    // retire finished requests
    for (auto& sl : S->slots) {
      if (!sl.busy) continue;
      cudaError_t q = cudaEventQuery(sl.done);
      if (q == cudaErrorNotReady) continue;
      tn_result_t res;
      std::memset(&res, 0, sizeof(res));
      if (q != cudaSuccess) {
        res.status = TN_ECUDA;
      } else {
        tn::dev::ModTable mods;
        make_mod_table(sl.req.semiring, sl.req.primes, &mods);
        int rc = tn::decode_raw(sl.req.semiring, mods, static_cast<int32_t>(sl.req.primes.size()),
                                sl.h_raw, &res);
        if (rc != TN_OK) res.status = rc;
      }
      cudaFreeAsync(sl.req.ws, sl.stream);
      S->used -= sl.req.bytes;
      S->done[sl.req.ticket] = res;
      S->state[sl.req.ticket] = 2;
      sl.busy = false;
      progressed = true;
    }
    bool any_busy = false;
    for (auto& sl : S->slots) any_busy |= sl.busy;
    if (!progressed) {
      if (any_busy) {
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(20));
        lk.lock();
      } else {
        S->cv.wait_for(lk, std::chrono::milliseconds(50));
      }
    }
  }
}

}  // namespace

extern "C" {

int tn_server_create(size_t hbm_budget_bytes, int32_t max_inflight, tn_server_t* out) {
  if (!out || max_inflight < 1 || max_inflight > 1024 || hbm_budget_bytes == 0) return TN_EINVAL;
  *out = nullptr;
  tn_server_s* S = new (std::nothrow) tn_server_s();
  if (!S) return TN_ENOMEM;
  S->budget = hbm_budget_bytes;
  S->max_inflight = max_inflight;
  if (cudaGetDevice(&S->device) != cudaSuccess) {
    delete S;
    return TN_ECUDA;
  }
  S->slots.resize(static_cast<size_t>(max_inflight));
  for (auto& sl : S->slots) {
    if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
        cudaMallocHost(reinterpret_cast<void**>(&sl.h_raw), TN_RAW_BYTES) != cudaSuccess) {
      tn_server_destroy(S);
      return TN_ECUDA;
    }
  }
  S->worker = std::thread(worker_loop, S);
  *out = S;
  return TN_OK;
}

int tn_submit(tn_server_t S, tn_plan_t plan, tn_semiring_t semiring, const uint32_t* primes,
              int32_t nprimes, uint64_t* ticket) {
  if (!S || !plan || !ticket) return TN_EINVAL;
  if (semiring < TN_TROPICAL_F32 || semiring > TN_COUNT_MODP) return TN_EINVAL;
  Request r;
  r.plan = plan;
  r.semiring = semiring;
  if (semiring == TN_COUNT_MODP) {
    if (!primes || nprimes < 1 || nprimes > TN_MAX_PRIMES) return TN_EINVAL;
    tn_result_t scratch;
    // validates the moduli the same way tn_contract does
    unsigned char zero[TN_RAW_BYTES] = {0};
    int rc = tn_result_decode(semiring, primes, nprimes, zero, &scratch);
    if (rc != TN_OK) return rc;
    r.primes.assign(primes, primes + nprimes);
  }
  r.bytes = tn::required_bytes(plan, semiring, nprimes);
  if (r.bytes > S->budget) return TN_ENOMEM;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    r.ticket = S->next_ticket++;
    S->state[r.ticket] = 0;
    S->pending.push_back(r);
  }
  S->cv.notify_one();
  *ticket = r.ticket;
  return TN_OK;
}

int tn_poll(tn_server_t S, uint64_t ticket, tn_result_t* out) {
  if (!S || !out) return TN_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  auto st = S->state.find(ticket);
  if (st == S->state.end()) return TN_EINVAL;
  if (st->second != 2) return TN_EAGAIN;
  *out = S->done[ticket];
  S->done.erase(ticket);
  S->state.erase(st);
  return TN_OK;
}

void tn_server_destroy(tn_server_t S) {
  if (!S) return;
  S->stop.store(true);
  S->cv.notify_all();
  if (S->worker.joinable()) S->worker.join();
  for (auto& sl : S->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    if (sl.busy && sl.req.ws) cudaFree(sl.req.ws);
    if (sl.h_raw) cudaFreeHost(sl.h_raw);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.stream) cudaStreamDestroy(sl.stream);
  }
  delete S;
}

}  // extern "C"
