// batch.cu -- grouped contraction of many independent networks in ONE
// persistent executor launch (tn_batch_*), optionally replayed from a CUDA
// graph.
//
// Each network keeps its own executor plan (steps, dependencies, tasks,
// workspace layout).  The batch concatenates them: every network gets its
// own slice of the counters, the split-K scratch and the arena, its step and
// dependency indices are shifted, and the tasks of all networks are merged in
// dependency-level order (level 0 of every network first, then level 1, ...),
// so independent networks advance side by side and the GPU stays full even
// when each network alone would be latency-bound.  Every network's final task
// writes its raw result into its own TN_RAW_BYTES slot.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <vector>

#include "exec.h"
#include "kernels.h"
#include "tn_internal.h"

namespace tn {
int make_mod_table_checked(tn_semiring_t s, const uint32_t* primes, int32_t nprimes, void* mods);
int exec_prepare_launch(tn_semiring_t s, const void* mods);
}  // namespace tn

struct tn_batch_s {
  tn_semiring_t semiring;
  int32_t nprimes = 1;
  int32_t count = 0;
  int32_t group_h = 64;  // networks of a batch run their tiny subtrees whole
  alignas(16) unsigned char mods[512];
  tn::ExecPlan X;  // the merged plan
  std::mutex mu;
  // captured graphs, keyed by (workspace, raw, stream)
  struct Graph {
    void* ws;
    void* raw;
    void* stream;
    cudaGraphExec_t exec;
  };
  std::vector<Graph> graphs;
};

namespace {

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

namespace tn {

// Merges the executor plans of `count` networks into one plan M (see the
// file comment).  nprimes: as given to the mod-p semiring (1 otherwise).
int build_batch_plan(tn_plan_s* const* plans, int32_t count, tn_semiring_t semiring, int32_t nprimes,
                     int group_h, ExecPlan* out, bool stored_leaves) {
  std::vector<ExecPlan*> xs(count);
  for (int i = 0; i < count; ++i) {
    int rc;
    xs[i] = exec_plan_get_h(plans[i], semiring, nprimes, group_h, true, &rc, false, stored_leaves);
    if (!xs[i]) return rc;
  }
  ExecPlan& M = *out;
  M.semiring = semiring;
  M.nprimes = xs.empty() ? 1 : xs[0]->nprimes;
  std::vector<int64_t> step_base(count), arena_base(count), group_base(count);
  std::vector<size_t> scratch_base(count);
  std::vector<int32_t> arrive_base(count);
  int64_t nsteps = 0, arena = 0, arrive = 0, ngroups = 0;
  size_t scratch = 0;
  int maxlev = 0;
  for (int i = 0; i < count; ++i) {
    step_base[i] = nsteps;
    group_base[i] = ngroups;
    ngroups += xs[i]->ngroups;
    arena_base[i] = arena;
    scratch_base[i] = scratch;
    arrive_base[i] = static_cast<int32_t>(arrive);
    nsteps += static_cast<int64_t>(xs[i]->steps.size());
    arena += static_cast<int64_t>(align_up(static_cast<size_t>(xs[i]->arena_entries), kArenaAlign));
    scratch += align_up(xs[i]->scratch_bytes, 256);
    arrive += xs[i]->n_arrive;
    maxlev = std::max(maxlev, xs[i]->nlevels);
  }
  if (nsteps > (int64_t(1) << 30) || arrive > (int64_t(1) << 30)) return TN_EINVAL;
  M.steps.clear();
  M.deps.clear();
  M.tasks.clear();
  M.step_level.clear();
  M.group_begin.clear();
  M.group_members.clear();
  for (int i = 0; i < count; ++i) {
    const ExecPlan& x = *xs[i];
    for (int gi = 0; gi < x.ngroups; ++gi) {
      M.group_begin.push_back(static_cast<int32_t>(M.group_members.size()));
      for (int32_t k = x.group_begin[gi]; k < x.group_begin[gi + 1]; ++k)
        M.group_members.push_back(x.group_members[k] + static_cast<int32_t>(step_base[i]));
    }
  }
  M.ngroups = static_cast<int32_t>(M.group_begin.size());
  M.group_begin.push_back(static_cast<int32_t>(M.group_members.size()));
  M.steps.reserve(static_cast<size_t>(nsteps));
  M.step_level.reserve(static_cast<size_t>(nsteps));
  for (int i = 0; i < count; ++i) {
    const ExecPlan& x = *xs[i];
    for (size_t s = 0; s < x.steps.size(); ++s) {
      ExecStep e = x.steps[s];
      e.final_slot = -1;  // final tasks write the results of a batch
      if (e.g.a_kind == kOpArena) e.a_off += arena_base[i];
      if (e.g.b_kind == kOpArena) e.b_off += arena_base[i];
      if (!e.c_shared) e.c_off += arena_base[i];
      e.scratch_off += static_cast<int64_t>(scratch_base[i]);
      e.arrive_off += arrive_base[i];
      const int32_t db = static_cast<int32_t>(M.deps.size());
      for (int d = 0; d < e.dep_count; ++d)
        M.deps.push_back(x.deps[e.dep_begin + d] + static_cast<int32_t>(step_base[i]));
      e.dep_begin = db;
      M.steps.push_back(e);
      M.step_level.push_back(x.step_level[s]);
    }
  }
  // tasks by (level, network); each network's final task after its last level
  std::vector<std::vector<ExecTask>> by_level(static_cast<size_t>(maxlev) + 1);
  for (int i = 0; i < count; ++i) {
    const ExecPlan& x = *xs[i];
    for (const ExecTask& t : x.tasks) {
      ExecTask u = t;
      u.step += static_cast<int32_t>(step_base[i]);
      int lev;
      if (t.kind == kTaskFinal) {
        u.local = i;  // raw-result slot of this network
        lev = maxlev;
      } else if (t.kind == kTaskGroup) {
        u.local += static_cast<int32_t>(group_base[i]);
        lev = x.step_level[t.step];
      } else {
        lev = x.step_level[t.step];
      }
      by_level[static_cast<size_t>(lev)].push_back(u);
    }
  }
  for (auto& v : by_level) M.tasks.insert(M.tasks.end(), v.begin(), v.end());
  if (M.tasks.size() > static_cast<size_t>(INT32_MAX)) return TN_EINVAL;
  M.arena_entries = std::max<int64_t>(arena, kArenaAlign);
  M.net_arena_base = arena_base;
  M.stored_leaves = stored_leaves;
  M.value_bound = 0;
  for (int i = 0; i < count; ++i) M.value_bound = std::max(M.value_bound, xs[i]->value_bound);
  M.leaf_base = count ? xs[0]->leaf_base : 0;
  M.scratch_bytes = scratch;
  M.n_arrive = static_cast<int32_t>(arrive);
  M.nlevels = maxlev;
  M.nraw = count;
  M.root_step = -1;
  // workspace: header | counters | scratch | arena regions
  M.ctr_off = kHeaderBytes;
  M.ctr_bytes = align_up(sizeof(int32_t) * (static_cast<size_t>(nsteps) + static_cast<size_t>(arrive) + 8), 256);
  M.scratch_base = M.ctr_off + M.ctr_bytes;
  M.arena_base = M.scratch_base + align_up(scratch, 256);
  const size_t e = static_cast<size_t>(M.arena_entries);
  size_t regions = 0;
  switch (semiring) {
    case TN_TROPICAL_F32:
    case TN_TROPICAL_I32: regions = align_up(4 * e, 256); break;
    case TN_COUNTING_TROPICAL: regions = align_up(4 * e, 256) + align_up(8 * e, 256); break;
    case TN_COUNT_MODP: regions = static_cast<size_t>(M.nprimes) * align_up(4 * e, 256); break;
  }
  M.total_bytes = M.arena_base + regions;
  exec_write_table_image(&M);
  return TN_OK;
}

int upload_tables(tn::ExecPlan* X) {
  int dev;
  if (cudaGetDevice(&dev) != cudaSuccess) return TN_ECUDA;
  if (X->d_tables && X->device == dev) return TN_OK;
  if (X->d_tables) cudaFree(X->d_tables);
  X->d_tables = nullptr;
  if (cudaMalloc(&X->d_tables, X->table_bytes) != cudaSuccess) return TN_ENOMEM;
  if (cudaMemcpy(X->d_tables, X->table_image.data(), X->table_bytes, cudaMemcpyHostToDevice) != cudaSuccess)
    return TN_ECUDA;
  X->device = dev;
  return TN_OK;
}

}  // namespace

extern "C" {

int tn_batch_create(const tn_plan_t* plans, int32_t count, tn_semiring_t semiring, const uint32_t* primes,
                    int32_t nprimes, tn_batch_t* out) {
  if (!out || !plans || count < 1) return TN_EINVAL;
  *out = nullptr;
  for (int i = 0; i < count; ++i)
    if (!plans[i]) return TN_EINVAL;
  std::unique_ptr<tn_batch_s> B(new (std::nothrow) tn_batch_s());
  if (!B) return TN_ENOMEM;
  B->semiring = semiring;
  B->nprimes = semiring == TN_COUNT_MODP ? nprimes : 1;
  B->count = count;
  {
    const char* e = getenv("TN_GROUP_HEIGHT");
    if (e && *e) B->group_h = atoi(e);
  }
  static_assert(sizeof(tn::dev::ModTable) <= sizeof(B->mods), "modulus table");
  int rc = tn::make_mod_table_checked(semiring, primes, nprimes, B->mods);
  if (rc) return rc;
  try {
    rc = tn::build_batch_plan(plans, count, semiring, B->nprimes, B->group_h, &B->X);
  } catch (const std::bad_alloc&) {
    rc = TN_ENOMEM;
  }
  if (rc) return rc;
  *out = B.release();
  return TN_OK;
}

int tn_batch_info(tn_batch_t b, uint64_t* workspace_bytes, int32_t* tasks, int32_t* levels,
                  uint64_t* table_bytes) {
  if (!b) return TN_EINVAL;
  if (workspace_bytes) *workspace_bytes = b->X.total_bytes;
  if (tasks) *tasks = static_cast<int32_t>(b->X.tasks.size());
  if (levels) *levels = b->X.nlevels;
  if (table_bytes) *table_bytes = b->X.table_bytes;
  return TN_OK;
}

int tn_batch_contract(tn_batch_t b, void* d_workspace, size_t ws_bytes, void* cuda_stream, void* d_raw) {
  if (!b || !d_workspace || !d_raw) return TN_EINVAL;
  if (reinterpret_cast<uintptr_t>(d_workspace) % 256 != 0) return TN_EINVAL;
  if (ws_bytes < b->X.total_bytes) return TN_ENOMEM;
  std::lock_guard<std::mutex> lk(b->mu);
  int rc = upload_tables(&b->X);
  if (rc) return rc;
  return tn::exec_launch_core(&b->X, b->semiring, b->mods, d_workspace, cuda_stream, d_raw, nullptr,
                              b->X.d_tables);
}

int tn_batch_contract_graph(tn_batch_t b, void* d_workspace, size_t ws_bytes, void* cuda_stream, void* d_raw) {
  if (!b || !d_workspace || !d_raw) return TN_EINVAL;
  if (reinterpret_cast<uintptr_t>(d_workspace) % 256 != 0) return TN_EINVAL;
  if (ws_bytes < b->X.total_bytes) return TN_ENOMEM;
  std::lock_guard<std::mutex> lk(b->mu);
  int rc = upload_tables(&b->X);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  for (auto& g : b->graphs)
    if (g.ws == d_workspace && g.raw == d_raw && g.stream == cuda_stream)
      return cudaGraphLaunch(g.exec, st) == cudaSuccess ? TN_OK : TN_ECUDA;
  // one-time kernel set-up (attributes, occupancy) outside the capture
  rc = tn::exec_prepare_launch(b->semiring, b->mods);
  if (rc) return rc;
  // a stream of our own is captured (the caller's may be the legacy stream)
  cudaStream_t cap;
  if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return TN_ECUDA;
  cudaGraph_t graph = nullptr;
  rc = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess ? TN_OK : TN_ECUDA;
  if (!rc) {
    int lrc = tn::exec_launch_core(&b->X, b->semiring, b->mods, d_workspace, cap, d_raw, nullptr, b->X.d_tables);
    rc = cudaStreamEndCapture(cap, &graph) == cudaSuccess ? lrc : TN_ECUDA;
  }
  cudaStreamDestroy(cap);
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  cudaGraphExec_t exec;
  rc = cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess ? TN_OK : TN_ECUDA;
  cudaGraphDestroy(graph);
  if (rc) return rc;
  b->graphs.push_back({d_workspace, d_raw, cuda_stream, exec});
  return cudaGraphLaunch(exec, st) == cudaSuccess ? TN_OK : TN_ECUDA;
}

void tn_batch_destroy(tn_batch_t b) {
  if (!b) return;
  for (auto& g : b->graphs) cudaGraphExecDestroy(g.exec);
  if (b->X.d_tables) cudaFree(b->X.d_tables);
  delete b;
}

}  // extern "C"
