// kbest.cu -- SizeMax(k) and CountingMax(k) (Sec. 5.3, Table 1 of
// arXiv:2501.00227) in one executor launch: the k-best element types of
// kbest.cuh contracted along the plan's pairwise order by the general step
// body (kbest.cuh explains the arithmetic and the tensor layout).
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "exec_device.cuh"

namespace tn {

int kbest_launch(ExecPlan* X, tn_semiring_t s, const void* args, void* stream) {
  const dev::ExecArgs& a = *static_cast<const dev::ExecArgs*>(args);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (s == TN_SIZE_MAX_K)
    return X->nprimes <= 2 ? dev::exec_launch_t<dev::SrKMax<2>, 1>(X, a, st)
                           : dev::exec_launch_t<dev::SrKMax<4>, 1>(X, a, st);
  if (s == TN_COUNTING_MAX_K)
    return X->nprimes <= 2 ? dev::exec_launch_t<dev::SrKPoly<2>, 1>(X, a, st)
                           : dev::exec_launch_t<dev::SrKPoly<4>, 1>(X, a, st);
  return TN_EINVAL;
}

namespace {

// element width instantiated for k (the k best are a prefix of the K best)
int kbest_width(int32_t k) { return k <= 2 ? 2 : 4; }

bool kbest_args_ok(tn_plan_t plan, tn_semiring_t s, int32_t k) {
  return plan && is_kbest(s) && k >= 1 && k <= TN_KBEST_MAX && plan->sliced.empty();
}

}  // namespace
}  // namespace tn

extern "C" int tn_kbest_workspace_bytes(tn_plan_t plan, tn_semiring_t semiring, int32_t k, uint64_t* bytes) {
  using namespace tn;
  if (!kbest_args_ok(plan, semiring, k) || !bytes) return TN_EINVAL;
  int rc;
  ExecPlan* X = exec_plan_get(plan, semiring, kbest_width(k), &rc);
  if (!X) return rc;
  *bytes = X->total_bytes;
  return TN_OK;
}

extern "C" int tn_contract_kbest(tn_plan_t plan, tn_semiring_t semiring, int32_t k, void* d_workspace,
                                 size_t ws_bytes, void* cuda_stream, int32_t* values, uint64_t* counts,
                                 int32_t* status) {
  using namespace tn;
  if (!kbest_args_ok(plan, semiring, k) || !d_workspace || !values || !status) return TN_EINVAL;
  if (semiring == TN_COUNTING_MAX_K && !counts) return TN_EINVAL;
  if (reinterpret_cast<uintptr_t>(d_workspace) % 256 != 0) return TN_EINVAL;
  dev::ModTable mods;
  std::memset(&mods, 0, sizeof(mods));
  void* d_raw = static_cast<char*>(d_workspace) + 64;
  int rc = exec_enqueue(plan, semiring, &mods, kbest_width(k), d_workspace, ws_bytes, cuda_stream, d_raw, nullptr);
  if (rc) return rc;
  unsigned char raw[TN_RAW_BYTES];
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  if (cudaMemcpyAsync(raw, d_raw, TN_RAW_BYTES, cudaMemcpyDeviceToHost, st) != cudaSuccess) return TN_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return TN_ECUDA;
  uint32_t flags;
  std::memcpy(&flags, raw + 96, 4);
  *status = flags ? TN_ETIMEOUT : TN_OK;
  auto value = [&](int t) {
    int32_t v;
    std::memcpy(&v, raw + 4 * t, 4);
    return v < TN_I32_NEG_INF / 2 ? INT32_MIN : v;
  };
  if (semiring == TN_SIZE_MAX_K) {
    for (int t = 0; t < k; ++t) values[t] = value(t);
  } else {
    values[0] = value(0);
    for (int t = 0; t < k; ++t) {
      std::memcpy(&counts[t], raw + 32 + 8 * t, 8);
      if (values[0] == INT32_MIN) counts[t] = 0;
      if (counts[t] == ~0ull && *status == TN_OK) *status = TN_EOVERFLOW;
    }
  }
  return *status == TN_ETIMEOUT ? TN_ETIMEOUT : TN_OK;
}
