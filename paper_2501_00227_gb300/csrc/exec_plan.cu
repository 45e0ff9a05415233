// exec_plan.cu -- host side of the persistent executor: turns a plan's
// pairwise steps into a level-ordered task list with dependencies, lays out
// the workspace (counters, split-K scratch, arena) and caches the result per
// (semiring, number of primes) inside the plan.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <utility>

#include "exec.h"
#include "kernels.h"
#include "step_device.cuh"
#include "tile_device.cuh"

namespace tn {

namespace {

struct Cache {
  std::mutex mu;
  std::vector<std::unique_ptr<ExecPlan>> plans;
};

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

// Largest height of a group of tiny steps run by one CTA for a single
// contraction (TN_GROUP_HEIGHT, default 1 = no grouping: a lone contraction
// is latency-bound and the dependency levels already run in parallel;
// batches and the server group whole tiny subtrees, see batch.cu).
int group_height() {
  const char* e = getenv("TN_GROUP_HEIGHT");
  if (!e || !*e) return 1;
  return atoi(e);
}

namespace {

// First-fit arena whose free blocks remember which steps released them: a
// step that takes memory another step released must run after that step
// (write-after-read), so the releasers become dependencies.
class LevelArena {
 public:
  explicit LevelArena(int64_t align = kArenaAlign) : align_(align) {}
  int64_t alloc(int64_t size, std::vector<int32_t>* war) {
    size = static_cast<int64_t>(align_up(static_cast<size_t>(size), static_cast<size_t>(align_)));
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second.len >= size) {
        const int64_t off = it->first;
        Block blk = std::move(it->second);
        free_.erase(it);
        war->insert(war->end(), blk.rel.begin(), blk.rel.end());
        if (blk.len > size) free_.emplace(off + size, Block{blk.len - size, std::move(blk.rel)});
        return off;
      }
    }
    int64_t off = top_;
    top_ += size;
    return off;
  }
  void release(int64_t off, int64_t size, int32_t releaser) {
    size = static_cast<int64_t>(align_up(static_cast<size_t>(size), static_cast<size_t>(align_)));
    auto it = free_.emplace(off, Block{size, {releaser}}).first;
    auto next = std::next(it);
    if (next != free_.end() && it->first + it->second.len == next->first) {
      merge(&it->second, next->second);
      free_.erase(next);
    }
    if (it != free_.begin()) {
      auto prev = std::prev(it);
      if (prev->first + prev->second.len == it->first) {
        merge(&prev->second, it->second);
        free_.erase(it);
      }
    }
  }
  int64_t top() const { return top_; }

 private:
  struct Block {
    int64_t len;
    std::vector<int32_t> rel;
  };
  static void merge(Block* a, const Block& b) {
    // both releaser lists are sorted and duplicate-free: merged in place
    a->len += b.len;
    const size_t mid = a->rel.size();
    a->rel.insert(a->rel.end(), b.rel.begin(), b.rel.end());
    std::inplace_merge(a->rel.begin(), a->rel.begin() + mid, a->rel.end());
    a->rel.erase(std::unique(a->rel.begin(), a->rel.end()), a->rel.end());
  }
  std::map<int64_t, Block> free_;
  int64_t top_ = 0;
  int64_t align_;
};

int build_exec(const tn_plan_s* p, tn_semiring_t s, int32_t nprimes, ExecPlan* X) {
  const int ns = static_cast<int>(p->steps.size());
  const int H = X->group_h;
  // np: prime slots of mod p (one task set each) or the width of a k-best
  // element type (one task set, np blocks per tensor)
  const int np = s == TN_COUNT_MODP || is_kbest(s) ? nprimes : 1;
  X->semiring = s;
  X->nprimes = np;
  const int kw = is_kbest(s) ? np : 1;
  const int npt = s == TN_COUNT_MODP ? np : 1;  // task sets (one per prime slot)

  // dependency levels (leaves at -1)
  std::vector<int32_t> level(ns);
  auto prod = [&](int32_t id) { return p->tensors[id].producer; };
  for (int i = 0; i < ns; ++i) {
    int la = prod(p->steps[i].a_id), lb = prod(p->steps[i].b_id);
    level[i] = 1 + std::max(la >= 0 ? level[la] : -1, lb >= 0 ? level[lb] : -1);
  }
  std::vector<int32_t> order(ns);
  for (int i = 0; i < ns; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return level[a] < level[b]; });
  std::vector<int32_t> pos(ns);
  for (int i = 0; i < ns; ++i) pos[order[i]] = i;
  X->nlevels = ns ? level[order[ns - 1]] + 1 : 0;
  X->step_level.resize(ns);
  for (int i = 0; i < ns; ++i) X->step_level[i] = level[order[i]];
  X->exec_to_plan = order;

  // ---- groups: trees of tiny steps (one output chunk, little work) of
  // height <= H run back to back inside one CTA (one task, barriers between
  // the steps) instead of one task per step.  Only a group's root output
  // leaves the group; the other members' outputs ("internal" tensors) live in
  // a region of their own that is never reused.
  std::vector<int32_t> groot(ns, -1), gh(ns, 0);
  std::vector<std::vector<int32_t>> gmem(ns);
  auto tiny = [&](int st) {
    const StepGeom& g = p->steps[st].g;
    int kernel, tile, split;
    dev::pick_launch(g, s, np, &kernel, &tile, &split, X->batched);
    return kernel == kKernNaive && g.rc <= 10 && g.rc + g.nk <= 13;
  };
  if (H > 1) {
    for (int st = 0; st < ns; ++st) {  // plan order is topological
      if (!tiny(st)) continue;
      groot[st] = st;
      gh[st] = 1;
      gmem[st] = {st};
      for (int32_t id : {p->steps[st].a_id, p->steps[st].b_id}) {
        const int pr = prod(id);
        if (pr < 0 || groot[pr] != pr || gh[pr] + 1 > H ||
            gmem[st].size() + gmem[pr].size() > static_cast<size_t>(kGroupMaxMembers))
          continue;
        for (int32_t m : gmem[pr]) groot[m] = st;
        gmem[st].insert(gmem[st].end(), gmem[pr].begin(), gmem[pr].end());
        gmem[pr].clear();
        gh[st] = std::max(gh[st], gh[pr] + 1);
      }
    }
  }
  // a group of one step is an ordinary step
  for (int st = 0; st < ns; ++st)
    if (groot[st] == st && gmem[st].size() < 2) groot[st] = -1;
  auto internal = [&](int st) { return groot[st] >= 0 && groot[st] != st; };
  auto owner = [&](int st) { return internal(st) ? groot[st] : st; };  // step that runs st

  // memory: a level's outputs may only reuse memory released by earlier
  // levels; the releasing steps become (write-after-read) dependencies.
  // Inputs consumed inside a group are released when the group's root level
  // is reached, by the root.
  // launch shape of every step, and the split-K scratch it needs (bytes)
  const size_t acc_bytes = exec_acc_bytes(s, kw);
  struct Launch {
    int kernel, tile, split;
    dev::NaiveShape sh;
    size_t scratch;
  };
  std::vector<Launch> ln(ns);
  for (int st = 0; st < ns; ++st) {
    Launch& L = ln[st];
    const StepGeom& g = p->steps[st].g;
    dev::pick_launch(g, s, np, &L.kernel, &L.tile, &L.split, X->batched);
    L.scratch = 0;
    if (groot[st] >= 0) {
      L.kernel = kKernNaive;
      L.sh = dev::naive_shape(g.rc, g.nk, false);
    } else if (L.kernel == kKernTiled) {
      const int64_t bm = dev::tiled_tile_bm(L.tile), bn = dev::tiled_tile_bn(L.tile);
      const int64_t ntiles = ((int64_t(1) << g.nm) + bm - 1) / bm * (((int64_t(1) << g.nn) + bn - 1) / bn) << g.nb;
      if (L.split > 1) L.scratch = static_cast<size_t>(ntiles * npt * L.split * bm * bn) * acc_bytes;
    } else {
      L.kernel = kKernNaive;
      L.sh = dev::naive_shape(g.rc, g.nk, !is_kbest(s), npt);
      if (L.sh.ks > 1) L.scratch = static_cast<size_t>(L.sh.nchunks * npt * L.sh.ks * L.sh.chunk) * acc_bytes;
    }
  }

  std::vector<std::vector<int32_t>> dep(ns);  // in plan-step indices
  std::vector<int64_t> c_off(ns, 0);
  LevelArena arena;
  // split-K scratch, in 256-byte blocks: a step's scratch is free again once
  // the step has completed, so later steps may reuse it (with a dependency)
  LevelArena sarena(1);
  std::vector<int64_t> s_off(ns, 0);
  for (int i = 0; i < ns;) {
    int j = i;
    while (j < ns && level[order[j]] == level[order[i]]) ++j;
    for (int x = i; x < j; ++x) {
      const int st = order[x];
      if (internal(st)) continue;
      const Step& S = p->steps[st];
      std::vector<int32_t> war;
      c_off[st] = arena.alloc(int64_t(1) << S.g.rc, &war);
      dep[st].swap(war);
      if (ln[st].scratch) {
        war.clear();
        s_off[st] = sarena.alloc(static_cast<int64_t>((ln[st].scratch + 255) / 256), &war);
        dep[st].insert(dep[st].end(), war.begin(), war.end());
      }
    }
    for (int x = i; x < j; ++x) {
      const int st = order[x];
      if (internal(st)) continue;
      const std::vector<int32_t> runs = groot[st] == st ? gmem[st] : std::vector<int32_t>{st};
      for (int32_t m : runs) {
        const Step& S = p->steps[m];
        for (int32_t id : {S.a_id, S.b_id}) {
          const int pr = prod(id);
          if (pr < 0 || owner(pr) == st) continue;  // a leaf, or internal to this group
          dep[st].push_back(owner(pr));
          if (!X->keep) arena.release(c_off[pr], int64_t(1) << p->steps[pr].g.rc, st);
        }
      }
    }
    for (int x = i; x < j; ++x) {
      const int st = order[x];
      if (!internal(st) && ln[st].scratch)
        sarena.release(s_off[st], static_cast<int64_t>((ln[st].scratch + 255) / 256), st);
    }
    i = j;
  }
  // internal tensors: in the group CTA's shared memory where they fit
  // (first fit over the members in execution order; a tensor is live from
  // its producer to its consumer), else in the global region below
  std::vector<int64_t> sh_off(ns, -1);
  for (int st = 0; st < ns; ++st) {
    if (groot[st] != st) continue;
    std::vector<int32_t> mem = gmem[st];
    std::sort(mem.begin(), mem.end(), [&](int a, int b) { return pos[a] < pos[b]; });
    std::map<int64_t, int64_t> free_blocks{{0, kGroupSmem}};  // offset -> length
    auto take = [&](int64_t size) -> int64_t {
      for (auto it = free_blocks.begin(); it != free_blocks.end(); ++it)
        if (it->second >= size) {
          const int64_t off = it->first, len = it->second;
          free_blocks.erase(it);
          if (len > size) free_blocks[off + size] = len - size;
          return off;
        }
      return -1;
    };
    auto give = [&](int64_t off, int64_t size) {
      auto it = free_blocks.emplace(off, size).first;
      auto nx = std::next(it);
      if (nx != free_blocks.end() && it->first + it->second == nx->first) {
        it->second += nx->second;
        free_blocks.erase(nx);
      }
      if (it != free_blocks.begin()) {
        auto pv = std::prev(it);
        if (pv->first + pv->second == it->first) {
          pv->second += it->second;
          free_blocks.erase(it);
        }
      }
    };
    for (int32_t m : mem) {
      if (internal(m)) sh_off[m] = take(shared_tensor_bytes(s, np, p->steps[m].g.rc));
      for (int32_t id : {p->steps[m].a_id, p->steps[m].b_id}) {
        const int pr = prod(id);
        if (pr >= 0 && internal(pr) && groot[pr] == st && sh_off[pr] >= 0)
          give(sh_off[pr], shared_tensor_bytes(s, np, p->steps[pr].g.rc));
      }
    }
  }
  // the remaining internal tensors after the shared arena
  int64_t top = arena.top();
  for (int st = 0; st < ns; ++st)
    if (internal(st) && sh_off[st] < 0) {
      c_off[st] = top;
      top += static_cast<int64_t>(align_up(size_t(1) << p->steps[st].g.rc, kArenaAlign));
    }
  X->arena_entries = std::max<int64_t>(top, kArenaAlign);
  if (X->stored_leaves) {
    // the leaf tensors of a weighted network, after the intermediates
    X->leaf_base = static_cast<int64_t>(align_up(static_cast<size_t>(X->arena_entries), kArenaAlign));
    X->arena_entries = X->leaf_base + static_cast<int64_t>(align_up(static_cast<size_t>(p->leaf_entries), kArenaAlign));
  }

  // transitive reduction of the dependencies (ancestor bitsets, exec order)
  const int words = (ns + 63) / 64;
  std::vector<uint64_t> anc(static_cast<size_t>(ns) * words, 0);
  std::vector<std::vector<int32_t>> red(ns);
  for (int x = 0; x < ns; ++x) {
    const int st = order[x];
    auto& d = dep[st];
    std::sort(d.begin(), d.end());
    d.erase(std::unique(d.begin(), d.end()), d.end());
    // a: the union of the dependencies' (strict) ancestors; a dependency in
    // it is implied by another one.  Then the dependencies themselves join a.
    uint64_t* a = &anc[static_cast<size_t>(x) * words];
    for (int32_t u : d) {
      const uint64_t* au = &anc[static_cast<size_t>(pos[u]) * words];
      for (int w = 0; w < words; ++w) a[w] |= au[w];
    }
    for (int32_t u : d) {
      const int pu = pos[u];
      if (!((a[pu / 64] >> (pu % 64)) & 1)) red[st].push_back(pu);
    }
    for (int32_t u : d) a[pos[u] / 64] |= 1ull << (pos[u] % 64);
  }

  // steps, tasks, split-K scratch and arrival counters
  X->steps.assign(ns, ExecStep());
  X->deps.clear();
  X->tasks.clear();
  X->group_begin.clear();
  X->group_members.clear();
  const size_t scratch = static_cast<size_t>(sarena.top()) * 256;
  int32_t arrive = 0;
  for (int x = 0; x < ns; ++x) {
    const int st = order[x];
    const Step& S = p->steps[st];
    ExecStep& E = X->steps[x];
    std::memset(&E, 0, sizeof(E));
    E.final_slot = -1;
    E.g = S.g;
    // a stored leaf (edges first, then vertices, 2^rank entries each) is an
    // arena tensor at leaf_base; a generated leaf needs no offset
    auto stored = [&](int32_t id) {
      return X->stored_leaves && (p->tensors[id].kind == kOpEdge || p->tensors[id].kind == kOpVertex);
    };
    auto off = [&](int32_t id) -> int64_t {
      const int pr = prod(id);
      if (pr < 0) return stored(id) ? X->leaf_base + p->leaf_off[id] : 0;
      return sh_off[pr] >= 0 ? sh_off[pr] : c_off[pr];
    };
    E.a_off = off(S.a_id);
    E.b_off = off(S.b_id);
    if (stored(S.a_id)) E.g.a_kind = kOpArena;
    if (stored(S.b_id)) E.g.b_kind = kOpArena;
    if (prod(S.a_id) >= 0 && sh_off[prod(S.a_id)] >= 0) E.g.a_kind = kOpShared;
    if (prod(S.b_id) >= 0 && sh_off[prod(S.b_id)] >= 0) E.g.b_kind = kOpShared;
    E.c_shared = sh_off[st] >= 0 ? 1 : 0;
    E.c_off = E.c_shared ? sh_off[st] : c_off[st];
    E.dep_begin = static_cast<int32_t>(X->deps.size());
    E.dep_count = static_cast<int32_t>(red[st].size());
    X->deps.insert(X->deps.end(), red[st].begin(), red[st].end());
    // the launch shape chosen above (one cost-model call per step)
    const int kernel = ln[st].kernel, tile = ln[st].tile, split = ln[st].split;
    if (internal(st) || groot[st] == st) {
      // group member: one whole-output chunk, no k split
      const dev::NaiveShape sh = dev::naive_shape(S.g.rc, S.g.nk, false);
      E.kernel = kKernNaive;
      E.R = sh.R;
      E.chunk = int64_t(1) << S.g.rc;
      E.ks = 1;
      E.nchunks = 1;
      E.ntasks = internal(st) ? 0 : 1;
      if (groot[st] == st) {
        // members in execution order (level, then plan order)
        std::vector<int32_t> mem = gmem[st];
        std::sort(mem.begin(), mem.end(), [&](int a, int b) { return pos[a] < pos[b]; });
        const int32_t gid = static_cast<int32_t>(X->group_begin.size());
        X->group_begin.push_back(static_cast<int32_t>(X->group_members.size()));
        for (int32_t m : mem) X->group_members.push_back(pos[m]);
        X->tasks.push_back(ExecTask{x, gid, npt > 1 ? -1 : 0, kTaskGroup});  // all primes in one task
        E.done_target = 1;
      }
    } else if (kernel == kKernTiled) {
      const int64_t bm = dev::tiled_tile_bm(tile), bn = dev::tiled_tile_bn(tile);
      E.kernel = kKernTiled;
      E.tile = tile;
      E.split = split;
      E.tiles_m = static_cast<int32_t>(((int64_t(1) << S.g.nm) + bm - 1) / bm);
      E.tiles_n = static_cast<int32_t>(((int64_t(1) << S.g.nn) + bn - 1) / bn);
      const int64_t ntiles = int64_t(E.tiles_m) * E.tiles_n << S.g.nb;
      E.ntasks = static_cast<int32_t>(ntiles * split);
      // 16-byte staging where an operand's two lowest stored bits are the
      // step's m (n) bits 0 and 1 (the planner stores intermediates for that)
      const StepGeom& G = S.g;
      if (E.g.a_kind == kOpArena && G.nm >= 2 && G.a_pos[G.nb] == 0 && G.a_pos[G.nb + 1] == 1 && E.a_off % 4 == 0)
        E.vec |= dev::kVecA;
      if (E.g.b_kind == kOpArena && G.nn >= 2 && G.b_pos[G.nb + G.nk] == 0 && G.b_pos[G.nb + G.nk + 1] == 1 &&
          E.b_off % 4 == 0)
        E.vec |= dev::kVecB;
      if (split > 1) {
        E.arrive_off = arrive;
        arrive += static_cast<int32_t>(ntiles * npt);
        E.scratch_off = s_off[st] * 256;
      }
    } else {
      const dev::NaiveShape& sh = ln[st].sh;
      E.kernel = kKernNaive;
      E.R = sh.R;
      E.chunk = sh.chunk;
      E.ks = sh.ks;
      E.nchunks = static_cast<int32_t>(sh.nchunks);
      E.ntasks = static_cast<int32_t>(sh.ntasks);
      if (sh.ks > 1) {
        E.arrive_off = arrive;
        arrive += static_cast<int32_t>(sh.nchunks * npt);
        E.scratch_off = s_off[st] * 256;
      }
    }
    if ((E.split > 1 || E.ks > 1) != (ln[st].scratch > 0)) return TN_EINVAL;  // launch shapes disagree
    if (groot[st] < 0) {
      if (E.kernel == kKernNaive && E.ks == 1 && npt > 1) {
        // a general step without k split does every prime inside each task
        for (int t = 0; t < E.ntasks; ++t) X->tasks.push_back(ExecTask{x, t, -1, kTaskNaive});
        E.done_target = E.ntasks;
      } else {
        for (int q = 0; q < npt; ++q)
          for (int t = 0; t < E.ntasks; ++t)
            X->tasks.push_back(ExecTask{x, t, q, E.kernel == kKernTiled ? kTaskTile : kTaskNaive});
        E.done_target = E.ntasks * npt;
      }
    }
  }
  X->ngroups = static_cast<int32_t>(X->group_begin.size());
  X->group_begin.push_back(static_cast<int32_t>(X->group_members.size()));
  X->root_step = pos[ns - 1];
  X->root_off = c_off[ns - 1];

  // Self-check (TN_EXEC_CHECK=1): the schedule is safe if (1) every step
  // depends only on steps earlier in the execution order and (2) whenever
  // the output of a step y overlaps the memory of an earlier tensor x, every
  // reader of x (its consumer) is an ancestor of y, so y cannot overwrite x
  // while it is still being read; (3) stored leaves overlap no intermediate
  // and (4) the plan that keeps its intermediates has no two overlapping.
  const char* chk = getenv("TN_EXEC_CHECK");
  if (chk && chk[0] == '1') {
    for (int x = 0; x < ns; ++x)
      for (int d = 0; d < X->steps[x].dep_count; ++d)
        if (X->deps[X->steps[x].dep_begin + d] >= x) return TN_EINVAL;
    auto is_anc = [&](int a_pos, int of_pos) {
      const uint64_t* av = &anc[static_cast<size_t>(of_pos) * words];
      return ((av[a_pos / 64] >> (a_pos % 64)) & 1) != 0;
    };
    for (int y = 0; y < ns; ++y) {
      const int sy = order[y];
      if (sh_off[sy] >= 0) continue;  // in a group's shared memory
      const int64_t y0 = c_off[sy], y1 = y0 + (int64_t(1) << p->steps[sy].g.rc);
      for (int x = 0; x < y; ++x) {
        const int sx = order[x];
        if (sh_off[sx] >= 0) continue;
        const int64_t x0 = c_off[sx], x1 = x0 + (int64_t(1) << p->steps[sx].g.rc);
        if (x1 <= y0 || y1 <= x0) continue;
        if (internal(sx) || internal(sy)) return TN_EINVAL;  // internal tensors are never shared
        const int cons = p->tensors[p->steps[sx].c_id].consumer;
        if (cons < 0 || !is_anc(pos[owner(cons)], y)) return TN_EINVAL;
      }
    }
    // stored leaves lie after every intermediate; a kept plan reuses no block
    for (int y = 0; y < ns; ++y) {
      const int sy = order[y];
      if (sh_off[sy] >= 0) continue;
      const int64_t y0 = c_off[sy], y1 = y0 + (int64_t(1) << p->steps[sy].g.rc);
      if (X->stored_leaves && y1 > X->leaf_base) return TN_EINVAL;
      if (X->keep)
        for (int x = 0; x < y; ++x) {
          const int sx = order[x];
          const int64_t x0 = c_off[sx], x1 = x0 + (int64_t(1) << p->steps[sx].g.rc);
          if (sh_off[sx] < 0 && x0 < y1 && y0 < x1) return TN_EINVAL;
        }
    }
    // split-K scratch: a later step may only overlap the scratch of a step it
    // (transitively) depends on
    for (int y = 0; y < ns; ++y) {
      const int sy = order[y];
      if (!ln[sy].scratch || internal(sy)) continue;
      const int64_t y0 = s_off[sy] * 256, y1 = y0 + static_cast<int64_t>(ln[sy].scratch);
      for (int x = 0; x < y; ++x) {
        const int sx = order[x];
        if (!ln[sx].scratch || internal(sx)) continue;
        const int64_t x0 = s_off[sx] * 256, x1 = x0 + static_cast<int64_t>(ln[sx].scratch);
        if (x1 <= y0 || y1 <= x0) continue;
        if (!is_anc(x, y)) return TN_EINVAL;
      }
    }
  }
  // the result: written by the CTA that completes the last step (one
  // dependency hop less), or by a final task after it when that step runs
  // inside a group task or the plan is merged into a batch (whose final
  // tasks carry each network's result slot)
  bool fold = !X->batched;
  for (const ExecTask& t : X->tasks)
    if (t.step == X->root_step && t.kind == kTaskGroup) fold = false;
  if (fold) X->steps[X->root_step].final_slot = 0;
  else X->tasks.push_back(ExecTask{X->root_step, 0, 0, kTaskFinal});
  X->n_arrive = arrive;
  X->scratch_bytes = scratch;

  // workspace layout: header | counters | scratch | arena regions
  X->ctr_off = kHeaderBytes;
  X->ctr_bytes = align_up(sizeof(int32_t) * (static_cast<size_t>(ns) + arrive + 8), 256);
  X->scratch_base = X->ctr_off + X->ctr_bytes;
  X->arena_base = X->scratch_base + align_up(scratch, 256);
  const size_t e = static_cast<size_t>(X->arena_entries);
  size_t regions = 0;
  switch (s) {
    case TN_TROPICAL_F32:
    case TN_TROPICAL_I32: regions = align_up(4 * e, 256); break;
    case TN_COUNTING_TROPICAL: regions = align_up(4 * e, 256) + align_up(8 * e, 256); break;
    case TN_COUNT_MODP: regions = static_cast<size_t>(np) * align_up(4 * e, 256); break;
    // k-best: K int32 blocks; or one int32 block and K uint64 blocks of twice
    // its size (so that one entry stride serves both)
    case TN_SIZE_MAX_K: regions = static_cast<size_t>(np) * align_up(4 * e, 256); break;
    case TN_COUNTING_MAX_K: regions = static_cast<size_t>(2 * np + 1) * align_up(4 * e, 256); break;
  }
  X->total_bytes = X->arena_base + regions;

  exec_write_table_image(X);
  return TN_OK;
}

}  // namespace

void exec_write_table_image(ExecPlan* X) {
  X->off_steps = 0;
  X->off_deps = align_up(sizeof(ExecStep) * X->steps.size(), 256);
  X->off_tasks = X->off_deps + align_up(2 * sizeof(int32_t) * (X->deps.size() + 1), 256);
  X->off_groups = X->off_tasks + align_up(sizeof(ExecTask) * X->tasks.size(), 256);
  X->off_members = X->off_groups + align_up(sizeof(int32_t) * X->group_begin.size(), 256);
  X->table_bytes = X->off_members + sizeof(int32_t) * (X->group_members.size() + 1);
  X->table_image.assign(X->table_bytes, 0);
  std::memcpy(X->table_image.data() + X->off_groups, X->group_begin.data(), sizeof(int32_t) * X->group_begin.size());
  std::memcpy(X->table_image.data() + X->off_members, X->group_members.data(),
              sizeof(int32_t) * X->group_members.size());
  std::memcpy(X->table_image.data() + X->off_steps, X->steps.data(), sizeof(ExecStep) * X->steps.size());
  int32_t* dp = reinterpret_cast<int32_t*>(X->table_image.data() + X->off_deps);
  for (size_t i = 0; i < X->deps.size(); ++i) {
    dp[2 * i] = X->deps[i];
    dp[2 * i + 1] = X->steps[X->deps[i]].done_target;
  }
  std::memcpy(X->table_image.data() + X->off_tasks, X->tasks.data(), sizeof(ExecTask) * X->tasks.size());
}

ExecPlan* exec_plan_get(tn_plan_s* p, tn_semiring_t s, int32_t nprimes, int* rc) {
  return exec_plan_get_h(p, s, nprimes, group_height(), false, rc);
}

ExecPlan* exec_plan_get_h(tn_plan_s* p, tn_semiring_t s, int32_t nprimes, int H, bool batched, int* rc, bool keep,
                          bool stored_leaves) {
  if (!stored_leaves && !p->sliced.empty()) {
    // the leaves of a sliced network depend on the slice: stored leaves only
    *rc = TN_EINVAL;
    return nullptr;
  }
  if (keep || stored_leaves || is_kbest(s)) H = 1;
  if (!p->exec_cache) {
    static std::mutex init_mu;
    std::lock_guard<std::mutex> lk(init_mu);
    if (!p->exec_cache) p->exec_cache = new Cache();
  }
  Cache* c = static_cast<Cache*>(p->exec_cache);
  const int np = s == TN_COUNT_MODP || is_kbest(s) ? nprimes : 1;
  std::lock_guard<std::mutex> lk(c->mu);
  for (auto& x : c->plans)
    if (x->semiring == s && x->nprimes == np && x->group_h == H && x->batched == batched && x->keep == keep &&
        x->stored_leaves == stored_leaves && x->tune_gen == tune_generation()) {
      *rc = TN_OK;
      return x.get();
    }
  // plans built under an older launch table stay alive (a caller may still
  // hold them); the current one is appended
  std::unique_ptr<ExecPlan> X(new ExecPlan());
  X->group_h = H;
  X->batched = batched;
  X->keep = keep;
  X->stored_leaves = stored_leaves;
  X->value_bound = stored_leaves ? INT64_MAX : p->n;
  X->tune_gen = tune_generation();
  *rc = build_exec(p, s, nprimes, X.get());
  if (*rc != TN_OK) return nullptr;
  c->plans.push_back(std::move(X));
  return c->plans.back().get();
}

void exec_plans_free(tn_plan_s* p) {
  Cache* c = static_cast<Cache*>(p->exec_cache);
  if (!c) return;
  for (auto& x : c->plans)
    if (x->d_tables) cudaFree(x->d_tables);
  delete c;
  p->exec_cache = nullptr;
}

}  // namespace tn
