// tune.cu -- the process-wide table of measured launch shapes (tn_tune_set)
// and the per-step launch report (tn_plan_step_info).
//
// The host heuristic pick_launch estimates a tiled step's time from a cost
// model; an autotuner (paper_2501_00227_gb300/tune.py) measures candidate
// tile shapes and split-K factors for the step shapes of real plans and
// installs the winners here.  pick_launch consults the table first.  Each
// change of the table bumps a generation number; executor plans built
// under an older generation are rebuilt on their next use.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>
#include <vector>

#include "exec.h"
#include "kernels.h"
#include "tn_internal.h"

namespace tn {

namespace {

using Key = std::tuple<int32_t, int32_t, int32_t, int32_t, int32_t>;  // semiring, nb, nm, nn, nk
struct Entry {
  int32_t tile, split;
};

std::mutex g_mu;
std::shared_ptr<const std::map<Key, Entry>> g_table;
std::atomic<int32_t> g_generation{0};

}  // namespace

int32_t tune_generation() { return g_generation.load(); }

bool tune_lookup(tn_semiring_t s, const StepGeom& g, int* tile, int* split) {
  std::shared_ptr<const std::map<Key, Entry>> t;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    t = g_table;
  }
  if (!t) return false;
  auto it = t->find(Key{static_cast<int32_t>(s), g.nb, g.nm, g.nn, g.nk});
  if (it == t->end()) return false;
  *tile = it->second.tile;
  *split = it->second.split;
  return true;
}

}  // namespace tn

extern "C" {

int tn_tune_set(const int32_t* entries, int32_t count) {
  using namespace tn;
  if (count < 0 || (count > 0 && !entries)) return TN_EINVAL;
  auto t = std::make_shared<std::map<Key, Entry>>();
  for (int32_t i = 0; i < count; ++i) {
    const int32_t* e = entries + 7 * i;
    const int32_t s = e[0], tile = e[5], split = e[6];
    if (s < TN_TROPICAL_F32 || s > TN_COUNT_MODP) return TN_EINVAL;
    if (e[1] < 0 || e[2] < 0 || e[3] < 0 || e[4] < 0 || e[1] + e[2] + e[3] + e[4] > kMaxStepBits) return TN_EINVAL;
    if (tile < -1 || tile > 5 || split < 1 || split > 16) return TN_EINVAL;  // shapes 0..5
    if (tile == 0 && s != TN_TROPICAL_F32 && s != TN_TROPICAL_I32) return TN_EINVAL;
    (*t)[Key{s, e[1], e[2], e[3], e[4]}] = Entry{tile, split};
  }
  {
    std::lock_guard<std::mutex> lk(g_mu);
    g_table = count ? std::shared_ptr<const std::map<Key, Entry>>(t) : nullptr;
  }
  g_generation.fetch_add(1);
  return TN_OK;
}

int tn_plan_step_info(tn_plan_t plan, tn_semiring_t semiring, int32_t nprimes, int32_t* out, int32_t nsteps) {
  using namespace tn;
  if (!plan || !out || semiring < TN_TROPICAL_F32 || semiring > TN_COUNT_MODP) return TN_EINVAL;
  if (nsteps != static_cast<int32_t>(plan->steps.size())) return TN_EINVAL;
  int rc;
  ExecPlan* X = exec_plan_get(plan, semiring, nprimes < 1 ? 1 : nprimes, &rc);
  if (!X) return rc;
  for (int32_t x = 0; x < nsteps; ++x) {
    const ExecStep& E = X->steps[x];
    const int32_t st = X->exec_to_plan[x];
    int32_t* o = out + 10 * st;
    o[0] = x;
    o[1] = X->step_level[x];
    o[2] = E.kernel;
    o[3] = E.kernel == kKernTiled ? E.tile : -1;
    o[4] = E.kernel == kKernTiled ? E.split : E.ks;
    o[5] = E.ntasks;
    o[6] = E.g.nb;
    o[7] = E.g.nm;
    o[8] = E.g.nn;
    o[9] = E.g.nk;
  }
  return TN_OK;
}

}  // extern "C"
