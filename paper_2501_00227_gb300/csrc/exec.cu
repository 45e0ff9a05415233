// exec.cu -- host side of the persistent plan executor (see exec.h and
// exec_device.cuh): launch set-up, table upload and the launches of the
// tropical, counting and mod-p instantiations of k_exec.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <type_traits>

#include "exec_device.cuh"

namespace tn {

namespace {
// Whether the int32 tropical or counting launches of X may use the packed
// 16-bit tiles (TN_PACKED=0 in the environment keeps the 32-bit tiles, for
// measurement and tests).
bool use_packed(const ExecPlan* X) {
  static const bool off = [] {
    const char* e = getenv("TN_PACKED");
    return e && e[0] == '0';
  }();
  return !off && X->value_bound <= (X->semiring == TN_COUNTING_TROPICAL ? dev::kPackedCntMax : dev::kPackedMax);
}
}  // namespace

int exec_prepare_launch(tn_semiring_t s, const void* mods_v) {
  const dev::ModTable& mods = *static_cast<const dev::ModTable*>(mods_v);
  size_t smem;
  int r = 0;
  switch (s) {
    case TN_TROPICAL_F32: r = dev::exec_resident<dev::SrF32, 1>(&smem); break;
    case TN_TROPICAL_I32:
      r = dev::exec_resident<dev::SrI32, 1>(&smem);
      if (r >= 0) r = dev::exec_resident<dev::SrI32, dev::kPackedI16>(&smem);
      break;
    case TN_COUNTING_TROPICAL:
      r = dev::exec_resident<dev::SrCnt, 1>(&smem);
      if (r >= 0) r = dev::exec_resident<dev::SrCnt, dev::kPackedI16>(&smem);
      break;
    case TN_COUNT_MODP: {
      bool fold4 = true;
      for (int i = 0; i < TN_MAX_PRIMES && mods.q[i].p; ++i)
        fold4 = fold4 && dev::mod_fold_interval(mods.q[i].p, mods.q[i].r32) == 4;
      r = fold4 ? dev::exec_resident<dev::SrMod, 4>(&smem) : dev::exec_resident<dev::SrMod, 1>(&smem);
      break;
    }
    default: return TN_EINVAL;
  }
  return r < 0 ? TN_ECUDA : TN_OK;
}

size_t exec_acc_bytes(tn_semiring_t s, int32_t kw) {
  switch (s) {
    case TN_TROPICAL_F32: return sizeof(float);
    case TN_TROPICAL_I32: return sizeof(int32_t);
    case TN_COUNTING_TROPICAL: return sizeof(dev::CntVal);
    case TN_COUNT_MODP: return sizeof(uint64_t);
    case TN_SIZE_MAX_K: return kw <= 2 ? sizeof(dev::KMaxVal<2>) : sizeof(dev::KMaxVal<4>);
    case TN_COUNTING_MAX_K: return kw <= 2 ? sizeof(dev::KPolyVal<2>) : sizeof(dev::KPolyVal<4>);
  }
  return 0;
}

int exec_enqueue(tn_plan_s* p, tn_semiring_t s, const void* mods_v, int32_t nprimes, void* ws,
                 size_t ws_bytes, void* stream, void* d_raw, void* d_trace, bool keep, bool stored_leaves) {
  int rc;
  ExecPlan* X = keep || stored_leaves ? exec_plan_get_h(p, s, nprimes, 1, false, &rc, keep, stored_leaves)
                                      : exec_plan_get(p, s, nprimes, &rc);
  if (!X) return rc;
  if (ws_bytes < X->total_bytes) return TN_ENOMEM;
  {
    // one-time upload of the step / dependency / task tables to this device
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    int dev;
    if (cudaGetDevice(&dev) != cudaSuccess) return TN_ECUDA;
    if (!X->d_tables || X->device != dev) {
      if (X->d_tables) cudaFree(X->d_tables);
      X->d_tables = nullptr;
      if (cudaMalloc(&X->d_tables, X->table_bytes) != cudaSuccess) return TN_ENOMEM;
      if (cudaMemcpy(X->d_tables, X->table_image.data(), X->table_bytes, cudaMemcpyHostToDevice) != cudaSuccess)
        return TN_ECUDA;
      X->device = dev;
      X->grid = 0;
    }
  }
  return exec_launch_core(X, s, mods_v, ws, stream, d_raw, d_trace, X->d_tables);
}

// Limit of every dependency wait of the launches that follow (ns); see
// tn_set_wait_timeout_ns.
constexpr unsigned long long kDefaultWaitNs = 2000000000ull;  // 2 s
std::atomic<unsigned long long> g_wait_timeout_ns{kDefaultWaitNs};

int exec_launch_core(ExecPlan* X, tn_semiring_t s, const void* mods_v, void* ws, void* stream, void* d_raw,
                     void* d_trace, const void* d_tables) {
  const dev::ModTable& mods = *static_cast<const dev::ModTable*>(mods_v);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(ws);
  dev::ExecArgs a;
  std::memset(&a, 0, sizeof(a));
  // clear the header and counters: in the kernel (launch gate) unless the
  // launch is being captured into a graph, whose replays would reuse the
  // epoch -- then with a memset node before it
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return TN_ECUDA;
  if (cap == cudaStreamCaptureStatusNone && X->ctr_off == kHeaderBytes) {
    static std::atomic<unsigned long long> epoch{0x9e3779b97f4a7c15ull ^ reinterpret_cast<uintptr_t>(&epoch)};
    unsigned long long e;
    do e = epoch.fetch_add(1, std::memory_order_relaxed) + 1; while (e == 0);
    a.epoch = e;
    a.ws = reinterpret_cast<uint32_t*>(w);
    a.ctr_words = static_cast<int32_t>(X->ctr_bytes / 4);
  } else if (cudaMemsetAsync(w, 0, X->ctr_off + X->ctr_bytes, st) != cudaSuccess) {
    return TN_ECUDA;
  }
  const int ns = static_cast<int>(X->steps.size());
  const char* tables = static_cast<const char*>(d_tables);
  a.steps = reinterpret_cast<const ExecStep*>(tables + X->off_steps);
  a.deps = reinterpret_cast<const int2*>(tables + X->off_deps);
  a.tasks = reinterpret_cast<const ExecTask*>(tables + X->off_tasks);
  a.group_begin = reinterpret_cast<const int32_t*>(tables + X->off_groups);
  a.group_members = reinterpret_cast<const int32_t*>(tables + X->off_members);
  a.ntasks_total = static_cast<int32_t>(X->tasks.size());
  a.nprimes = X->nprimes;
  int32_t* ctr = reinterpret_cast<int32_t*>(w + X->ctr_off);
  a.done = ctr;
  a.arrive = ctr + ns;
  a.task_ctr = ctr + ns + X->n_arrive;
  a.status = reinterpret_cast<uint32_t*>(w);
  const size_t e = static_cast<size_t>(X->arena_entries);
  const size_t b4 = (4 * e + 255) / 256 * 256;
  a.r0 = w + X->arena_base;
  a.r1 = s == TN_COUNTING_TROPICAL || s == TN_COUNTING_MAX_K ? a.r0 + b4 : nullptr;
  a.prime_stride = static_cast<int64_t>(b4 / 4);
  a.scratch = w + X->scratch_base;
  a.raw = static_cast<unsigned char*>(d_raw);
  a.mods = mods;
  a.semiring = s;
  a.timeout_ns = g_wait_timeout_ns.load(std::memory_order_relaxed);
  a.trace = static_cast<unsigned long long*>(d_trace);
  a.nraw = X->nraw;
  switch (s) {
    case TN_SIZE_MAX_K:
    case TN_COUNTING_MAX_K: return kbest_launch(X, s, &a, st);
    case TN_TROPICAL_F32: return dev::exec_launch_t<dev::SrF32, 1>(X, a, st);
    case TN_TROPICAL_I32:
      return use_packed(X) ? dev::exec_launch_t<dev::SrI32, dev::kPackedI16>(X, a, st)
                           : dev::exec_launch_t<dev::SrI32, 1>(X, a, st);
    case TN_COUNTING_TROPICAL:
      return use_packed(X) ? dev::exec_launch_t<dev::SrCnt, dev::kPackedI16>(X, a, st)
                           : dev::exec_launch_t<dev::SrCnt, 1>(X, a, st);
    case TN_COUNT_MODP: {
      bool fold4 = true;
      for (int i = 0; i < X->nprimes; ++i) fold4 = fold4 && dev::mod_fold_interval(mods.q[i].p, mods.q[i].r32) == 4;
      return fold4 ? dev::exec_launch_t<dev::SrMod, 4>(X, a, st) : dev::exec_launch_t<dev::SrMod, 1>(X, a, st);
    }
  }
  return TN_EINVAL;
}

}  // namespace tn

extern "C" int tn_set_wait_timeout_ns(uint64_t ns) {
  if (ns > 60000000000ull) return TN_EINVAL;
  tn::g_wait_timeout_ns.store(ns ? ns : tn::kDefaultWaitNs, std::memory_order_relaxed);
  return TN_OK;
}
