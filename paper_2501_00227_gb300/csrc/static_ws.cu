// static_ws.cu -- tn_contract_static: a contraction that allocates no device
// memory.  Its workspace (executor counters, split-K scratch, arena, and the
// step / task tables) lives in one file-scope __device__ array of
// TN_STATIC_WORKSPACE_BYTES, which every GPU that loads libtn holds until the
// process exits.
//
// Host code cannot use the array's name as a device address (it names a
// host-side shadow), so the first call on each device looks the address up
// with cudaGetSymbolAddress while that device is current and caches it.
// Every call reuses the same array: the counters and the result block are
// cleared at the start of each call, and calls that overlap on the GPU (from
// several threads or streams) race on it.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "exec.h"
#include "kernels.h"
#include "tn_internal.h"

namespace tn {
int make_mod_table_checked(tn_semiring_t s, const uint32_t* primes, int32_t nprimes, void* mods);
int decode_raw_any(tn_semiring_t s, const void* mods, int32_t nprimes, const unsigned char* raw,
                   tn_result_t* out);
size_t required_bytes(tn_plan_s* p, tn_semiring_t s, int32_t nprimes);
}  // namespace tn

namespace {

__device__ __align__(256) unsigned char g_static_workspace[TN_STATIC_WORKSPACE_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Device address of the array on the current device (set-up on first use).
int static_base(void** out) {
  int dev;
  if (cudaGetDevice(&dev) != cudaSuccess) return TN_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return TN_EINVAL;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_workspace) != cudaSuccess || !p) return TN_ECUDA;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return TN_OK;
}

}  // namespace

extern "C" int tn_contract_static(tn_plan_t plan, tn_semiring_t semiring, const uint32_t* primes,
                                  int32_t nprimes, void* cuda_stream, tn_result_t* out) {
  using namespace tn;
  if (!plan || !out) return TN_EINVAL;
  alignas(16) unsigned char mods[sizeof(dev::ModTable)];
  int rc = make_mod_table_checked(semiring, primes, nprimes, mods);
  if (rc) return rc;
  ExecPlan* X = exec_plan_get(plan, semiring, nprimes, &rc);
  if (!X) return rc;
  // layout inside the array: workspace | step / task tables.  The workspace
  // part is sized by the same rule as tn_contract's (tn_plan_info
  // peak_bytes), so a plan is accepted exactly when the header says it is.
  const size_t ws_bytes = align256(required_bytes(plan, semiring, nprimes));
  if (ws_bytes + align256(X->table_bytes) > static_cast<size_t>(TN_STATIC_WORKSPACE_BYTES)) return TN_ENOMEM;
  void* base;
  rc = static_base(&base);
  if (rc) return rc;
  char* ws = static_cast<char*>(base);
  char* tables = ws + ws_bytes;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  if (cudaMemcpyAsync(tables, X->table_image.data(), X->table_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return TN_ECUDA;
  void* d_raw = ws + 64;
  rc = exec_launch_core(X, semiring, mods, ws, st, d_raw, nullptr, tables);
  if (rc) return rc;
  unsigned char raw[TN_RAW_BYTES];
  if (cudaMemcpyAsync(raw, d_raw, TN_RAW_BYTES, cudaMemcpyDeviceToHost, st) != cudaSuccess) return TN_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return TN_ECUDA;
  rc = decode_raw_any(semiring, mods, nprimes, raw, out);
  // a dependency wait that ran out leaves an unspecified result: report it
  // as tn_contract does
  return rc ? rc : out->status == TN_ETIMEOUT ? TN_ETIMEOUT : TN_OK;
}
