// config.cu -- one optimal configuration (the SingleConfigMax property of
// Sec. 5.3, Table 1) by a backward pass over the tropical contraction.
//
// The forward pass is the (max,+) contraction of the network (unit-weight
// or weighted IS, or the spin glass maximising -H) with the executor plan
// that keeps every intermediate, and the leaves, in the arena.  The
// backward pass walks the pairwise steps from the root down.  When a step is reached, the labels of
// its output C are already fixed (by the step that consumed C), so its
// output entry c is known; the step's summed labels K are then set to the
// first assignment t (lowest index) with A[a(c, t)] + B[b(c, t)] = C[c],
// which exists because C[c] is that maximum.  Every label is summed by
// exactly one step (the network's output is a scalar), so the walk assigns
// every vertex once, and the configuration reaches the maximum: each fixed
// entry of each tensor lies on a maximising path.
//
// k_backtrack runs the walk in one CTA, level by level from the root (a
// step's depth is its consumer's plus one): the steps of one level fix
// disjoint labels and read only labels fixed at lower depths.  Steps with at
// most 8 summed labels go one per warp (t scanned in rounds of 32 lanes,
// stop at the first round with a match, a ballot gives the lowest t);
// longer scans take the whole CTA in rounds of 256 with an atomicMin; a
// barrier separates the levels.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstring>
#include <vector>

#include "exec.h"
#include "kernels.h"
#include "tn_internal.h"

namespace tn {
int contract_weighted_raw(tn_plan_s* p, tn_semiring_t s, int32_t problem, const int32_t* ew, const int32_t* vw,
                          const uint32_t* primes, const uint32_t* xs, int32_t nslots, void* d_ws, size_t ws_bytes,
                          cudaStream_t st, unsigned char* raw_out, bool keep, ExecPlan** Xout, uint64_t slice);
int weighted_checks(tn_plan_s* p, tn_semiring_t s, int32_t problem, const int32_t* ew, const int32_t* vw);
size_t weighted_workspace(tn_plan_s* p, tn_semiring_t s, int32_t nslots, bool keep);
}  // namespace tn

namespace tn {
namespace dev {
namespace {

// Step record of the backward walk (plan order); operand sources: 0 = an
// arena tensor (intermediate, or leaf of the stored-leaf plan), 2 = the
// rank-0 identity.  Source codes of an operand bit: j < 32 -> output bit j,
// 32 + j -> summed bit j.
struct BtStep {
  int32_t ra, rb, rc, nk;
  int32_t a_src, b_src;
  int32_t lab;   // first entry in the label pool: LC (rc), K (nk), codes of A (ra), codes of B (rb)
  int32_t pad_;
  int64_t a_off, b_off, c_off;  // arena entry offsets
};

struct BtArgs {
  const BtStep* steps;    // ordered by depth from the root
  const int32_t* level;   // steps of depth d: [level[d], level[d + 1])
  int32_t nlevels;
  int32_t pad_;
  const int32_t* pool;
  const int32_t* arena;   // int32 (max,+) values of the intermediates and leaves
  int8_t* asg;            // out: the value of every label (vertex)
  int32_t* status;        // out: 0, or 1 + the step where no maximiser was found
  int32_t nsteps;
  int32_t n;
};

__device__ __forceinline__ int32_t bt_value(const BtArgs& a, int32_t src, int64_t off, uint32_t e) {
  if (src == 2) return 0;
  return a.arena[off + e];
}

// the output entry c of step st and its value, from the labels fixed so far
__device__ __forceinline__ uint32_t bt_entry(const BtArgs& a, const BtStep& st) {
  const int32_t* lc = a.pool + st.lab;
  uint32_t c = 0;
  for (int j = 0; j < st.rc; ++j) c |= uint32_t(a.asg[lc[j]] > 0) << j;
  return c;
}

// does summed-label assignment t reach C[c]?
__device__ __forceinline__ bool bt_hit(const BtArgs& a, const BtStep& st, uint32_t c, int32_t target, uint32_t t) {
  const int32_t* ca = a.pool + st.lab + st.rc + st.nk;
  const int32_t* cb = ca + st.ra;
  uint32_t ea = 0, eb = 0;
  for (int j = 0; j < st.ra; ++j) ea |= ((ca[j] < 32 ? c >> ca[j] : t >> (ca[j] - 32)) & 1u) << j;
  for (int j = 0; j < st.rb; ++j) eb |= ((cb[j] < 32 ? c >> cb[j] : t >> (cb[j] - 32)) & 1u) << j;
  const int32_t va = bt_value(a, st.a_src, st.a_off, ea), vb = bt_value(a, st.b_src, st.b_off, eb);
  return va > TN_I32_NEG_INF / 2 && vb > TN_I32_NEG_INF / 2 && va + vb == target;
}

__device__ __forceinline__ void bt_fix(const BtArgs& a, const BtStep& st, int s, uint32_t best) {
  if (best == UINT_MAX) {
    atomicCAS(a.status, 0, 1 + s);
    return;
  }
  const int32_t* lk = a.pool + st.lab + st.rc;
  for (int j = 0; j < st.nk; ++j) a.asg[lk[j]] = static_cast<int8_t>((best >> j) & 1u);
}

constexpr int kBtWarpMaxK = 8;  // steps summing more labels are scanned by the whole CTA

__global__ void __launch_bounds__(256) k_backtrack(const __grid_constant__ BtArgs a) {
  __shared__ uint32_t s_best;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int v = threadIdx.x; v < a.n; v += blockDim.x) a.asg[v] = -1;
  __syncthreads();
  for (int d = 0; d < a.nlevels; ++d) {
    // short scans: one warp per step, rounds of 32 assignments
    for (int s = a.level[d] + warp; s < a.level[d + 1]; s += nwarps) {
      const BtStep st = a.steps[s];
      if (st.nk > kBtWarpMaxK) continue;
      const uint32_t c = bt_entry(a, st);
      const int32_t target = a.arena[st.c_off + c];
      const uint32_t nt = 1u << st.nk;
      uint32_t best = UINT_MAX;
      for (uint32_t t0 = 0; t0 < nt && best == UINT_MAX; t0 += 32) {
        const unsigned m = __ballot_sync(0xffffffffu, t0 + lane < nt && bt_hit(a, st, c, target, t0 + lane));
        if (m) best = t0 + (__ffs(m) - 1);
      }
      if (lane == 0) bt_fix(a, st, s, best);
      __syncwarp();
    }
    // long scans: the whole CTA per step, rounds of blockDim assignments
    for (int s = a.level[d]; s < a.level[d + 1]; ++s) {
      const BtStep st = a.steps[s];
      if (st.nk <= kBtWarpMaxK) continue;
      __syncthreads();
      const uint32_t c = bt_entry(a, st);
      const int32_t target = a.arena[st.c_off + c];
      if (threadIdx.x == 0) s_best = UINT_MAX;
      __syncthreads();
      const uint32_t nt = 1u << st.nk;
      for (uint32_t t0 = 0; t0 < nt; t0 += blockDim.x) {
        const uint32_t t = t0 + threadIdx.x;
        if (t < nt && bt_hit(a, st, c, target, t)) atomicMin(&s_best, t);
        __syncthreads();
        if (s_best != UINT_MAX) break;
      }
      if (threadIdx.x == 0) bt_fix(a, st, s, s_best);
    }
    __syncthreads();
  }
}

}  // namespace
}  // namespace dev

namespace {

size_t align256(size_t b) { return (b + 255) / 256 * 256; }
int cuda_rc(cudaError_t e) { return e == cudaSuccess ? TN_OK : TN_ECUDA; }

// Host image of the backward walk's tables (steps, then the label pool).
struct BtImage {
  std::vector<dev::BtStep> steps;  // by depth from the root
  std::vector<int32_t> level;      // nlevels + 1 offsets into steps
  std::vector<int32_t> pool;
  size_t bytes() const { return align256(sizeof(dev::BtStep) * steps.size()) + align256(4 * pool.size()); }
};

int build_bt(tn_plan_s* p, const ExecPlan* X, BtImage* B) {
  const int ns = static_cast<int>(p->steps.size());
  std::vector<int64_t> c_off(ns, -1);
  for (size_t x = 0; x < X->steps.size(); ++x) c_off[X->exec_to_plan[x]] = X->steps[x].c_off;
  auto source = [&](int32_t id, int32_t* src, int64_t* off) {
    const TensorInfo& t = p->tensors[id];
    if (t.kind == kOpArena) {
      *src = 0;
      *off = c_off[t.producer];
    } else if (t.kind == kOpEdge || t.kind == kOpVertex) {
      *src = 0;
      *off = X->leaf_base + p->leaf_off[id];
    } else {
      *src = 2;
      *off = 0;
    }
    return *src != 0 || *off >= 0;
  };
  // depth from the root: the root step is the last; a step's output is
  // consumed by a later step, one level nearer the root
  std::vector<int32_t> depth(ns, 0);
  int32_t maxd = 0;
  for (int s = ns - 2; s >= 0; --s) {
    const int32_t cons = p->tensors[p->steps[s].c_id].consumer;
    if (cons <= s || cons >= ns) return TN_EINVAL;
    depth[s] = depth[cons] + 1;
    maxd = std::max(maxd, depth[s]);
  }
  std::vector<int32_t> by_depth(ns);
  for (int s = 0; s < ns; ++s) by_depth[s] = s;
  std::stable_sort(by_depth.begin(), by_depth.end(), [&](int32_t x, int32_t y) { return depth[x] < depth[y]; });
  B->level.assign(maxd + 2, 0);
  for (int s = 0; s < ns; ++s) B->level[depth[s] + 1]++;
  for (int d = 0; d <= maxd; ++d) B->level[d + 1] += B->level[d];
  B->steps.resize(ns);
  for (int k = 0; k < ns; ++k) {
    const int s = by_depth[k];
    const Step& S = p->steps[s];
    const auto& la = p->tensors[S.a_id].labels;
    const auto& lb = p->tensors[S.b_id].labels;
    const auto& lc = p->tensors[S.c_id].labels;
    std::vector<int32_t> lk;
    for (const auto* L : {&la, &lb})
      for (int32_t l : *L)
        if (std::find(lc.begin(), lc.end(), l) == lc.end() && std::find(lk.begin(), lk.end(), l) == lk.end())
          lk.push_back(l);
    if (lk.size() > 30 || lc.size() > 30 || la.size() > 30 || lb.size() > 30) return TN_EINVAL;
    dev::BtStep& b = B->steps[k];
    std::memset(&b, 0, sizeof(b));
    b.ra = static_cast<int32_t>(la.size());
    b.rb = static_cast<int32_t>(lb.size());
    b.rc = static_cast<int32_t>(lc.size());
    b.nk = static_cast<int32_t>(lk.size());
    if (!source(S.a_id, &b.a_src, &b.a_off) || !source(S.b_id, &b.b_src, &b.b_off)) return TN_EINVAL;
    b.c_off = c_off[s];
    if (b.c_off < 0) return TN_EINVAL;
    b.lab = static_cast<int32_t>(B->pool.size());
    B->pool.insert(B->pool.end(), lc.begin(), lc.end());
    B->pool.insert(B->pool.end(), lk.begin(), lk.end());
    for (const auto* L : {&la, &lb})
      for (int32_t l : *L) {
        const auto ic = std::find(lc.begin(), lc.end(), l);
        B->pool.push_back(ic != lc.end() ? int32_t(ic - lc.begin()) : 32 + int32_t(std::find(lk.begin(), lk.end(), l) - lk.begin()));
      }
  }
  return TN_OK;
}

size_t config_workspace(tn_plan_s* p, size_t* bt_off) {
  const size_t w = align256(weighted_workspace(p, TN_TROPICAL_I32, 1, true));
  if (bt_off) *bt_off = w;
  // tables: one record per step and at most 4 * 30 pool entries per step;
  // then the label values and the status word
  const size_t ns = p->steps.size();
  return w + align256(sizeof(dev::BtStep) * ns) + align256(4 * 120 * ns) + align256(size_t(p->n)) + 256 +
         align256(4 * (ns + 2));
}

}  // namespace
}  // namespace tn

using namespace tn;

extern "C" {

int tn_single_config_workspace_bytes(tn_plan_t plan, uint64_t* out) {
  if (!plan || !out) return TN_EINVAL;
  try {
    *out = config_workspace(plan, nullptr);
  } catch (const std::bad_alloc&) {
    return TN_ENOMEM;
  }
  return TN_OK;
}

int tn_single_config_max(tn_plan_t plan, int32_t problem, const int32_t* edge_w, const int32_t* vertex_w,
                         void* d_workspace, size_t ws_bytes, void* cuda_stream, int32_t* value, uint8_t* config) {
  if (!plan || !d_workspace || !value || !config || !plan->sliced.empty()) return TN_EINVAL;
  if (reinterpret_cast<uintptr_t>(d_workspace) % 256 != 0) return TN_EINVAL;
  int rc = weighted_checks(plan, TN_TROPICAL_I32, problem, edge_w, vertex_w);
  if (rc) return rc;
  try {
    size_t bt_off;
    if (ws_bytes < config_workspace(plan, &bt_off)) return TN_ENOMEM;
    int rcx;
    ExecPlan* X = exec_plan_get_h(plan, TN_TROPICAL_I32, 1, 1, false, &rcx, true, true);
    if (!X) return rcx;
    BtImage B;
    rc = build_bt(plan, X, &B);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    unsigned char raw[TN_RAW_BYTES];
    ExecPlan* Xc = nullptr;
    rc = contract_weighted_raw(plan, TN_TROPICAL_I32, problem, edge_w, vertex_w, nullptr, nullptr, 0, d_workspace,
                               bt_off, st, raw, true, &Xc, 0);
    if (rc) return rc;
    if (Xc != X) return TN_EINVAL;  // the tables above describe the plan that ran
    uint32_t flags;
    std::memcpy(&flags, raw + 96, 4);
    if (flags) return TN_ETIMEOUT;
    int32_t vmax;
    std::memcpy(&vmax, raw, 4);
    if (vmax < TN_I32_NEG_INF / 2) return TN_EINVAL;  // no allowed configuration
    char* w = static_cast<char*>(d_workspace);
    char* d_steps = w + bt_off;
    char* d_pool = d_steps + align256(sizeof(dev::BtStep) * B.steps.size());
    char* d_asg = d_pool + align256(4 * 120 * B.steps.size());
    char* d_status = d_asg + align256(size_t(plan->n));
    char* d_level = d_status + 256;
    rc = cuda_rc(cudaMemcpyAsync(d_steps, B.steps.data(), sizeof(dev::BtStep) * B.steps.size(),
                                 cudaMemcpyHostToDevice, st));
    if (!rc) rc = cuda_rc(cudaMemcpyAsync(d_pool, B.pool.data(), 4 * B.pool.size(), cudaMemcpyHostToDevice, st));
    if (!rc) rc = cuda_rc(cudaMemcpyAsync(d_level, B.level.data(), 4 * B.level.size(), cudaMemcpyHostToDevice, st));
    if (!rc) rc = cuda_rc(cudaMemsetAsync(d_status, 0, 4, st));
    if (rc) return rc;
    dev::BtArgs a;
    a.steps = reinterpret_cast<const dev::BtStep*>(d_steps);
    a.level = reinterpret_cast<const int32_t*>(d_level);
    a.nlevels = static_cast<int32_t>(B.level.size()) - 1;
    a.pad_ = 0;
    a.pool = reinterpret_cast<const int32_t*>(d_pool);
    a.arena = reinterpret_cast<const int32_t*>(w + X->arena_base);
    a.asg = reinterpret_cast<int8_t*>(d_asg);
    a.status = reinterpret_cast<int32_t*>(d_status);
    a.nsteps = static_cast<int32_t>(B.steps.size());
    a.n = plan->n;
    dev::k_backtrack<<<1, 256, 0, st>>>(a);
    rc = cuda_rc(cudaGetLastError());
    if (rc) return rc;
    std::vector<int8_t> asg(plan->n);
    int32_t status = 0;
    rc = cuda_rc(cudaMemcpyAsync(asg.data(), d_asg, size_t(plan->n), cudaMemcpyDeviceToHost, st));
    if (!rc) rc = cuda_rc(cudaMemcpyAsync(&status, d_status, 4, cudaMemcpyDeviceToHost, st));
    if (!rc) rc = cuda_rc(cudaStreamSynchronize(st));
    if (rc) return rc;
    if (status) return TN_EINVAL;
    for (int v = 0; v < plan->n; ++v) {
      if (asg[v] < 0) return TN_EINVAL;
      config[v] = static_cast<uint8_t>(asg[v]);
    }
    *value = vmax;
    return TN_OK;
  } catch (const std::bad_alloc&) {
    return TN_ENOMEM;
  }
}

}  // extern "C"
