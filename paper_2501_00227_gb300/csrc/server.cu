// server.cu -- serving entry points of libtn (tn_server_create, tn_submit,
// tn_poll, tn_server_destroy): continuous batching of contraction requests.
//
// Requests of any size and semiring arrive at any time; tn_submit only
// queues them.  A worker thread keeps up to max_inflight grouped launches on
// the GPU, each on a stream of its own.  Whenever a launch slot is free it
// takes the oldest pending request and, in arrival order, every other
// pending request with the same semiring and primes, as long as the sum of
// their predicted workspaces (the executor layout of each plan: its space
// complexity, Sec. 4.1 of arXiv:2501.00227, times the bytes per entry, plus
// scratch) fits in the unused part of the HBM budget; these go out as ONE
// persistent executor launch (the batch machinery of batch.cu).  Requests
// that arrive while launches run join the next free slot, so their work
// overlaps on the device with the launches still running.  The worker
// retires launches as they complete, decodes every request's scalar on the
// host and frees the launch's memory, which admits more requests.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "exec.h"
#include "kernels.h"
#include "tn_internal.h"

namespace tn {
int decode_raw(tn_semiring_t s, const dev::ModTable& mods, int32_t nprimes, const unsigned char* raw,
               tn_result_t* out);
size_t required_bytes(tn_plan_s* p, tn_semiring_t s, int32_t nprimes);
int make_mod_table_checked(tn_semiring_t s, const uint32_t* primes, int32_t nprimes, void* mods);
}  // namespace tn

namespace {

constexpr int kMaxBatch = 512;  // requests per grouped launch

struct Request {
  uint64_t ticket;
  tn_plan_s* plan;
  tn_semiring_t semiring;
  std::vector<uint32_t> primes;
  size_t bytes;
};

struct Flight {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  unsigned char* h_raw = nullptr;  // pinned, kMaxBatch * TN_RAW_BYTES
  bool busy = false;
  std::vector<Request> reqs;
  std::unique_ptr<tn::ExecPlan> plan;
  tn::dev::ModTable mods;
  void* ws = nullptr;
  void* d_raw = nullptr;
  void* d_tables = nullptr;
  size_t bytes = 0;
};

bool same_key(const Request& a, const Request& b) {
  return a.semiring == b.semiring && a.primes == b.primes;
}

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
  std::deque<uint64_t> completed;            // finished tickets not yet reported by tn_server_completed
  std::vector<Flight> flights;
  uint64_t next_ticket = 1;
  int group_h = 4;  // height of the groups of tiny steps one CTA runs back to back
  std::atomic<bool> stop{false};
  std::thread worker;
};

namespace {

void finish_with_status(tn_server_s* S, const std::vector<Request>& reqs, int status) {
  for (const Request& r : reqs) {
    tn_result_t res;
    std::memset(&res, 0, sizeof(res));
    res.status = status;
    S->done[r.ticket] = res;
    S->state[r.ticket] = 2;
    S->completed.push_back(r.ticket);
  }
}

void release_flight(Flight& f) {
  if (f.ws) cudaFreeAsync(f.ws, f.stream);
  if (f.d_raw) cudaFreeAsync(f.d_raw, f.stream);
  if (f.d_tables) cudaFreeAsync(f.d_tables, f.stream);
  f.ws = f.d_raw = f.d_tables = nullptr;
  f.plan.reset();
  f.reqs.clear();
  f.busy = false;
}

// Launches `reqs` as one grouped executor launch on flight f.
int launch_flight(tn_server_s* S, Flight& f, std::vector<Request>&& reqs) {
  f.reqs = std::move(reqs);
  const Request& r0 = f.reqs.front();
  const int32_t np = static_cast<int32_t>(r0.primes.size());
  int rc = tn::make_mod_table_checked(r0.semiring, np ? r0.primes.data() : nullptr, np, &f.mods);
  if (rc) return rc;
  std::vector<tn_plan_s*> plans;
  for (const Request& r : f.reqs) plans.push_back(r.plan);
  f.plan.reset(new tn::ExecPlan());
  try {
    rc = tn::build_batch_plan(plans.data(), static_cast<int32_t>(plans.size()), r0.semiring, np < 1 ? 1 : np,
                              S->group_h, f.plan.get());
  } catch (const std::bad_alloc&) {
    rc = TN_ENOMEM;
  }
  if (rc) return rc;
  tn::ExecPlan& X = *f.plan;
  const size_t raw_bytes = f.reqs.size() * TN_RAW_BYTES;
  if (cudaMallocAsync(&f.ws, X.total_bytes, f.stream) != cudaSuccess ||
      cudaMallocAsync(&f.d_raw, raw_bytes, f.stream) != cudaSuccess ||
      cudaMallocAsync(&f.d_tables, X.table_bytes, f.stream) != cudaSuccess)
    return TN_ENOMEM;
  if (cudaMemcpyAsync(f.d_tables, X.table_image.data(), X.table_bytes, cudaMemcpyHostToDevice, f.stream) !=
      cudaSuccess)
    return TN_ECUDA;
  rc = tn::exec_launch_core(&X, r0.semiring, &f.mods, f.ws, f.stream, f.d_raw, nullptr, f.d_tables);
  if (rc) return rc;
  if (cudaMemcpyAsync(f.h_raw, f.d_raw, raw_bytes, cudaMemcpyDeviceToHost, f.stream) != cudaSuccess ||
      cudaEventRecord(f.done, f.stream) != cudaSuccess)
    return TN_ECUDA;
  f.bytes = X.total_bytes;
  f.busy = true;
  return TN_OK;
}

void worker_loop(tn_server_s* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  while (!S->stop.load()) {
    bool progressed = false;
    // retire finished launches
    for (Flight& f : S->flights) {
      if (!f.busy) continue;
      cudaError_t q = cudaEventQuery(f.done);
      if (q == cudaErrorNotReady) continue;
      for (size_t i = 0; i < f.reqs.size(); ++i) {
        tn_result_t res;
        std::memset(&res, 0, sizeof(res));
        if (q != cudaSuccess) {
          res.status = TN_ECUDA;
        } else {
          const int32_t np = static_cast<int32_t>(f.reqs[i].primes.size());
          int rc = tn::decode_raw(f.reqs[i].semiring, f.mods, np, f.h_raw + i * TN_RAW_BYTES, &res);
          if (rc != TN_OK) res.status = rc;
        }
        S->done[f.reqs[i].ticket] = res;
        S->state[f.reqs[i].ticket] = 2;
        S->completed.push_back(f.reqs[i].ticket);
      }
      S->used -= f.bytes;
      release_flight(f);
      progressed = true;
    }
    // fill free launch slots
    for (Flight& f : S->flights) {
      if (f.busy || S->pending.empty()) continue;
      std::vector<Request> take;
      size_t bytes = 0;
      const Request key = S->pending.front();
      for (auto it = S->pending.begin(); it != S->pending.end() && take.size() < kMaxBatch;) {
        if (same_key(*it, key) && S->used + bytes + it->bytes <= S->budget) {
          bytes += it->bytes;
          take.push_back(*it);
          it = S->pending.erase(it);
        } else {
          ++it;
        }
      }
      if (take.empty()) break;  // the oldest request waits for memory
      for (const Request& r : take) S->state[r.ticket] = 1;
      // merging the plans and enqueueing the launch touch only this flight
      // and the requests' plans: clients may submit and poll meanwhile
      lk.unlock();
      int rc = launch_flight(S, f, std::move(take));
      lk.lock();
      if (rc != TN_OK) {
        finish_with_status(S, f.reqs, rc);
        release_flight(f);
        continue;
      }
      S->used += f.bytes;
      progressed = true;
    }
    bool any_busy = false;
    for (const Flight& f : S->flights) any_busy |= f.busy;
    if (!progressed) {
      if (any_busy) {
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(20));
        lk.lock();
      } else {
        S->cv.wait_for(lk, std::chrono::milliseconds(20));
      }
    }
  }
}

}  // namespace

extern "C" {

int tn_server_create(size_t hbm_budget_bytes, int32_t max_inflight, tn_server_t* out) {
  if (!out || max_inflight < 1 || max_inflight > 64 || hbm_budget_bytes == 0) return TN_EINVAL;
  *out = nullptr;
  tn_server_s* S = new (std::nothrow) tn_server_s();
  if (!S) return TN_ENOMEM;
  S->budget = hbm_budget_bytes;
  S->max_inflight = max_inflight;
  if (const char* e = getenv("TN_SERVE_GROUP_HEIGHT")) S->group_h = atoi(e) > 0 ? atoi(e) : 1;
  if (cudaGetDevice(&S->device) != cudaSuccess) {
    delete S;
    return TN_ECUDA;
  }
  S->flights.resize(static_cast<size_t>(max_inflight));
  for (Flight& f : S->flights) {
    if (cudaStreamCreateWithFlags(&f.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&f.done, cudaEventDisableTiming) != cudaSuccess ||
        cudaMallocHost(reinterpret_cast<void**>(&f.h_raw), size_t(kMaxBatch) * TN_RAW_BYTES) != cudaSuccess) {
      tn_server_destroy(S);
      return TN_ECUDA;
    }
  }
  S->worker = std::thread(worker_loop, S);
  *out = S;
  return TN_OK;
}

int tn_submit(tn_server_t S, tn_plan_t plan, tn_semiring_t semiring, const uint32_t* primes, int32_t nprimes,
              uint64_t* ticket) {
  if (!S || !plan || !ticket) return TN_EINVAL;
  Request r;
  r.plan = plan;
  r.semiring = semiring;
  tn::dev::ModTable mods;
  int rc = tn::make_mod_table_checked(semiring, primes, nprimes, &mods);
  if (rc) return rc;
  if (semiring == TN_COUNT_MODP) r.primes.assign(primes, primes + nprimes);
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

int tn_server_completed(tn_server_t S, uint64_t* tickets, int32_t max_tickets, int32_t* count) {
  if (!S || !count || max_tickets < 0 || (max_tickets > 0 && !tickets)) return TN_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  int32_t k = 0;
  while (k < max_tickets && !S->completed.empty()) {
    tickets[k++] = S->completed.front();
    S->completed.pop_front();
  }
  *count = k;
  return TN_OK;
}

void tn_server_destroy(tn_server_t S) {
  if (!S) return;
  S->stop.store(true);
  S->cv.notify_all();
  if (S->worker.joinable()) S->worker.join();
  for (Flight& f : S->flights) {
    if (f.stream) cudaStreamSynchronize(f.stream);
    if (f.busy) release_flight(f);
    if (f.stream) cudaStreamSynchronize(f.stream);
    if (f.h_raw) cudaFreeHost(f.h_raw);
    if (f.done) cudaEventDestroy(f.done);
    if (f.stream) cudaStreamDestroy(f.stream);
  }
  delete S;
}

}  // extern "C"
