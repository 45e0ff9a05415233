// plan.cpp -- host side of libtn: validation, the greedy contraction order,
// per-step label classes, workspace layout and complexity (tc / sc / rwc).
//
// Paper references (arXiv:2501.00227): the IS network and its leaves are
// Sec. 3.2 (Eqs. 4-8); binary contraction orders and the tc / sc / rwc
// measures are Sec. 4.1; the greedy method is Sec. 4.2.1 (Eq. 9).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <unordered_map>
#include <utility>

#include "tn_internal.h"

namespace tn {

namespace {

bool graph_ok(int32_t n, const int32_t* edges, int32_t m) {
  if (n < 1 || m < 0 || (m > 0 && edges == nullptr)) return false;
  std::vector<std::pair<int32_t, int32_t>> seen;
  seen.reserve(static_cast<size_t>(m));
  for (int32_t e = 0; e < m; ++e) {
    int32_t u = edges[2 * e], v = edges[2 * e + 1];
    if (u < 0 || v < 0 || u >= n || v >= n || u == v) return false;
    seen.emplace_back(std::min(u, v), std::max(u, v));
  }
  std::sort(seen.begin(), seen.end());
  return std::adjacent_find(seen.begin(), seen.end()) == seen.end();
}

int position(const std::vector<int32_t>& v, int32_t x) {
  for (size_t i = 0; i < v.size(); ++i)
    if (v[i] == x) return static_cast<int>(i);
  return -1;
}

// First-fit allocator over [0, inf) in units of entries.
class Arena {
 public:
  int64_t alloc(int64_t size) {
    size = (size + kArenaAlign - 1) / kArenaAlign * kArenaAlign;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= size) {
        int64_t off = it->first, len = it->second;
        free_.erase(it);
        if (len > size) free_[off + size] = len - size;
        return off;
      }
    }
    int64_t off = top_;
    top_ += size;
    return off;
  }
  void release(int64_t off, int64_t size) {
    size = (size + kArenaAlign - 1) / kArenaAlign * kArenaAlign;
    auto it = free_.emplace(off, size).first;
    auto next = std::next(it);
    if (next != free_.end() && it->first + it->second == next->first) {
      it->second += next->second;
      free_.erase(next);
    }
    if (it != free_.begin()) {
      auto prev = std::prev(it);
      if (prev->first + prev->second == it->first) {
        prev->second += it->second;
        free_.erase(it);
      }
    }
  }
  int64_t top() const { return top_; }

 private:
  std::map<int64_t, int64_t> free_;  // offset -> length
  int64_t top_ = 0;
};

}  // namespace

int classify_step(const std::vector<int32_t>& la, const std::vector<int32_t>& lb,
                  const std::vector<int32_t>& lc_set, StepGeom* g,
                  std::vector<int32_t>* lc_order, const std::vector<int32_t>* n_first) {
  if (la.size() > static_cast<size_t>(kMaxRank) || lb.size() > static_cast<size_t>(kMaxRank) ||
      lc_set.size() > static_cast<size_t>(kMaxRank))
    return TN_EINVAL;
  for (int32_t l : lc_set)
    if (position(la, l) < 0 && position(lb, l) < 0) return TN_EINVAL;
  std::vector<int32_t> bt, M, N, K;
  for (int32_t l : la) {
    bool in_b = position(lb, l) >= 0, in_c = position(lc_set, l) >= 0;
    if (in_c && in_b) bt.push_back(l);
    else if (in_c) M.push_back(l);
    else K.push_back(l);
  }
  for (int32_t l : lb) {
    bool in_a = position(la, l) >= 0, in_c = position(lc_set, l) >= 0;
    if (in_a) continue;
    if (in_c) N.push_back(l);
    else K.push_back(l);
  }
  if (n_first) {
    std::stable_partition(N.begin(), N.end(), [&](int32_t l) { return position(*n_first, l) >= 0; });
  }
  int total = static_cast<int>(bt.size() + M.size() + N.size() + K.size());
  if (total > kMaxStepBits) return TN_EINVAL;
  std::memset(g, 0, sizeof(*g));
  std::memset(g->a_pos, -1, sizeof(g->a_pos));
  std::memset(g->b_pos, -1, sizeof(g->b_pos));
  g->nb = static_cast<int32_t>(bt.size());
  g->nm = static_cast<int32_t>(M.size());
  g->nn = static_cast<int32_t>(N.size());
  g->nk = static_cast<int32_t>(K.size());
  g->ra = static_cast<int32_t>(la.size());
  g->rb = static_cast<int32_t>(lb.size());
  g->rc = g->nb + g->nm + g->nn;
  g->c_identity = 1;
  for (int j = 0; j < g->rc; ++j) g->c_pos[j] = static_cast<int8_t>(j);
  int i = 0;
  for (int32_t l : bt) g->a_pos[i++] = static_cast<int8_t>(position(la, l));
  for (int32_t l : M) g->a_pos[i++] = static_cast<int8_t>(position(la, l));
  for (int32_t l : K) g->a_pos[i++] = static_cast<int8_t>(position(la, l));
  i = 0;
  for (int32_t l : bt) g->b_pos[i++] = static_cast<int8_t>(position(lb, l));
  for (int32_t l : K) g->b_pos[i++] = static_cast<int8_t>(position(lb, l));
  for (int32_t l : N) g->b_pos[i++] = static_cast<int8_t>(position(lb, l));
  if (lc_order) {
    lc_order->clear();
    lc_order->insert(lc_order->end(), N.begin(), N.end());
    lc_order->insert(lc_order->end(), M.begin(), M.end());
    lc_order->insert(lc_order->end(), bt.begin(), bt.end());
  }
  return TN_OK;
}

size_t bytes_per_entry(tn_semiring_t s, int32_t nprimes) {
  switch (s) {
    case TN_TROPICAL_F32:
    case TN_TROPICAL_I32: return 4;
    case TN_COUNTING_TROPICAL: return 12;
    case TN_COUNT_MODP: return 4 * static_cast<size_t>(nprimes < 1 ? 1 : nprimes);
  }
  return 0;
}

static size_t align256(size_t x) { return (x + 255) / 256 * 256; }

size_t workspace_bytes(const tn_plan_s* p, tn_semiring_t s, int32_t nprimes) {
  size_t e = static_cast<size_t>(p->arena_entries);
  switch (s) {
    case TN_TROPICAL_F32:
    case TN_TROPICAL_I32: return kHeaderBytes + align256(4 * e);
    case TN_COUNTING_TROPICAL: return kHeaderBytes + align256(4 * e) + align256(8 * e);
    case TN_COUNT_MODP:
      return kHeaderBytes + static_cast<size_t>(nprimes < 1 ? 1 : nprimes) * align256(4 * e);
  }
  return 0;
}

// Storage order of the intermediates.  A step's kernels stage operand A
// along its M labels and operand B along its N labels (consecutive threads
// take consecutive m, resp. n, and the M / N labels are numbered in the
// operand's storage order).  The first pass stores every output as (N, M,
// batch) of its own step; this pass re-stores each intermediate with the
// labels its consumer stages along (the consumer's M labels if it is the
// consumer's A, its N labels if B) as the lowest bits, the others after them
// in the first pass's order, so that neighbouring staging threads read
// neighbouring entries.  The producing step then writes through c_pos (its
// output index bits scattered to the chosen positions).  Only orders change:
// labels, sizes, arena offsets and the step's classes stay the same.
int consumer_layouts(tn_plan_s* p) {
  const int32_t ns = static_cast<int32_t>(p->steps.size());
  std::vector<std::vector<int32_t>> natural(static_cast<size_t>(ns));  // (N, M, bt) of each step
  for (int32_t s = 0; s < ns; ++s) natural[s] = p->tensors[p->steps[s].c_id].labels;
  for (int32_t s = 0; s < ns; ++s) {
    Step& st = p->steps[s];
    const auto& la = p->tensors[st.a_id].labels;
    const auto& lb = p->tensors[st.b_id].labels;
    TensorInfo& c = p->tensors[st.c_id];
    // only for consumers that run as GEMM tiles with real work (the same
    // shape test as the launch choice; their class sizes are order-free)
    auto big_tiled = [&](const StepGeom& qg) {
      const int bits = qg.nb + qg.nm + qg.nn + qg.nk;
      return bits >= 20 && qg.nk >= 3 && qg.nm + qg.nn >= 10 && qg.nm >= 2 && qg.nn >= 2;
    };
    // the consumer's staging labels (in c, not in the consumer's other
    // operand, kept by the consumer)
    std::vector<int32_t> staged;
    if (c.consumer >= 0 && big_tiled(p->steps[c.consumer].g)) {
      const Step& q = p->steps[c.consumer];
      const auto& other = p->tensors[q.a_id == st.c_id ? q.b_id : q.a_id].labels;
      for (int32_t l : natural[s])
        if (position(other, l) < 0 && position(natural[c.consumer], l) >= 0) staged.push_back(l);
    }
    // classes and the output order of this step from the operands' final
    // storage orders, numbering the staged N labels first: when two or more
    // of them exist the output keeps index order (16-byte stores) and is
    // still staged along its lowest two labels by the consumer
    std::vector<int32_t> nat;
    int rc = classify_step(la, lb, natural[s], &st.g, &nat, staged.empty() ? nullptr : &staged);
    if (rc != TN_OK) return rc;
    st.g.a_kind = p->tensors[st.a_id].kind;
    st.g.b_kind = p->tensors[st.b_id].kind;
    std::vector<int32_t> chosen = nat;
    if (!staged.empty()) {
      std::vector<int32_t> first, rest;
      for (int32_t l : nat) (position(staged, l) >= 0 ? first : rest).push_back(l);
      // already staged along its lowest two labels: keep the step's order;
      // else the staged labels first (the producer then scatters its stores)
      const bool natural_ok = first.size() >= 2 && position(first, nat[0]) >= 0 && position(first, nat[1]) >= 0;
      if (!natural_ok) {
        chosen = first;
        chosen.insert(chosen.end(), rest.begin(), rest.end());
      }
    }
    c.labels = chosen;
    st.g.c_identity = chosen == nat ? 1 : 0;
    for (int j = 0; j < st.g.rc; ++j) st.g.c_pos[j] = static_cast<int8_t>(position(chosen, nat[j]));
  }
  return TN_OK;
}

int build_plan(int32_t n, const int32_t* edges, int32_t m, const int32_t* order, int32_t nsteps,
               tn_plan_s* p, const int32_t* sliced, int32_t nsliced) {
  if (!graph_ok(n, edges, m)) return TN_EINVAL;
  const int32_t T = n + m;
  if (nsteps != T - 1 || (nsteps > 0 && order == nullptr)) return TN_EINVAL;
  if (nsliced < 0 || nsliced > 62 || (nsliced > 0 && sliced == nullptr)) return TN_EINVAL;
  std::vector<char> is_sliced(static_cast<size_t>(n), 0);
  for (int32_t j = 0; j < nsliced; ++j) {
    if (sliced[j] < 0 || sliced[j] >= n || is_sliced[sliced[j]]) return TN_EINVAL;
    is_sliced[sliced[j]] = 1;
  }
  p->n = n;
  p->m = m;
  p->T = T;
  p->edges.assign(edges, edges + 2 * static_cast<size_t>(m));
  p->order.assign(order, order + 2 * static_cast<size_t>(nsteps));
  p->sliced.assign(sliced, sliced + nsliced);

  // Leaves: edges first, then vertices (the flattened einsum of Sec. 3.2);
  // a sliced label is fixed per slice, so it is dropped from every leaf.
  p->tensors.assign(static_cast<size_t>(T), TensorInfo());
  for (int32_t e = 0; e < m; ++e) {
    for (int k = 0; k < 2; ++k)
      if (!is_sliced[edges[2 * e + k]]) p->tensors[e].labels.push_back(edges[2 * e + k]);
    p->tensors[e].kind = kOpEdge;
  }
  for (int32_t v = 0; v < n; ++v) {
    if (!is_sliced[v]) p->tensors[m + v].labels = {v};
    p->tensors[m + v].kind = kOpVertex;
  }
  p->leaf_off.assign(static_cast<size_t>(T), 0);
  p->leaf_entries = 0;
  for (int32_t t = 0; t < T; ++t) {
    p->leaf_off[t] = p->leaf_entries;
    p->leaf_entries += int64_t(1) << p->tensors[t].labels.size();
  }
  // Internal step list.  A network with a single leaf (one vertex, no edge)
  // has no pairwise step; it is reduced by contracting it with the rank-0
  // identity, so that every network runs through the same kernels.
  std::vector<std::pair<int32_t, int32_t>> pairs;
  if (T == 1) {
    TensorInfo one;
    one.kind = kOpOne;
    p->tensors.push_back(one);
    pairs.emplace_back(0, 1);
  } else {
    std::vector<char> used(static_cast<size_t>(2 * T), 0);
    for (int32_t s = 0; s < nsteps; ++s) {
      int32_t i = order[2 * s], j = order[2 * s + 1];
      if (i < 0 || j < 0 || i >= T + s || j >= T + s || i == j || used[i] || used[j]) return TN_EINVAL;
      used[i] = used[j] = 1;
      pairs.emplace_back(i, j);
    }
  }
  const int32_t first_new = static_cast<int32_t>(p->tensors.size());
  p->tensors.reserve(p->tensors.size() + pairs.size());

  std::vector<int32_t> users(static_cast<size_t>(n), 0);
  for (const auto& t : p->tensors)
    for (int32_t l : t.labels) users[l]++;

  Arena arena;
  p->steps.clear();
  p->tc = p->rwc = p->sc = 0;
  for (size_t s = 0; s < pairs.size(); ++s) {
    Step st;
    st.a_id = pairs[s].first;
    st.b_id = pairs[s].second;
    st.c_id = first_new + static_cast<int32_t>(s);
    const auto& la = p->tensors[st.a_id].labels;
    const auto& lb = p->tensors[st.b_id].labels;
    // Output labels: labels of the pair that another live tensor still uses.
    std::vector<int32_t> lc_set;
    for (int32_t l : la) {
      int others = users[l] - 1 - (position(lb, l) >= 0 ? 1 : 0);
      if (others > 0) lc_set.push_back(l);
    }
    for (int32_t l : lb)
      if (position(la, l) < 0 && users[l] - 1 > 0) lc_set.push_back(l);
    TensorInfo c;
    int rc = classify_step(la, lb, lc_set, &st.g, &c.labels);
    if (rc != TN_OK) return rc;
    st.g.a_kind = p->tensors[st.a_id].kind;
    st.g.b_kind = p->tensors[st.b_id].kind;
    int uni = st.g.nb + st.g.nm + st.g.nn + st.g.nk;
    st.ops = uni >= 64 ? ~0ull : (1ull << uni);
    p->tc += st.ops;
    uint64_t csz = 1ull << c.labels.size();
    p->rwc += (1ull << la.size()) + (1ull << lb.size()) + csz;
    p->sc = std::max(p->sc, csz);
    c.producer = static_cast<int32_t>(s);
    c.kind = kOpArena;
    c.offset = arena.alloc(static_cast<int64_t>(csz));
    for (int32_t l : la) users[l]--;
    for (int32_t l : lb) users[l]--;
    for (int32_t l : c.labels) users[l]++;
    p->tensors[st.a_id].consumer = static_cast<int32_t>(s);
    p->tensors[st.b_id].consumer = static_cast<int32_t>(s);
    // Inputs die after this step (their memory is reused by later outputs;
    // steps run in order on one stream, so there is no overlap hazard).
    for (int32_t id : {st.a_id, st.b_id}) {
      const TensorInfo& t = p->tensors[id];
      if (t.kind == kOpArena) arena.release(t.offset, static_cast<int64_t>(1ull << t.labels.size()));
    }
    p->tensors.push_back(c);
    p->steps.push_back(st);
  }
  p->root = static_cast<int32_t>(p->tensors.size()) - 1;
  if (!p->tensors[p->root].labels.empty()) return TN_EINVAL;  // cannot happen for a full order
  p->arena_entries = std::max<int64_t>(arena.top(), kArenaAlign);
  return consumer_layouts(p);
}

// ---------------------------------------------------------------------------
// Greedy order (Sec. 4.2.1).
// ---------------------------------------------------------------------------
namespace {

// PCG32 (O'Neill 2014): small, seedable, statistically sound.
struct Pcg32 {
  uint64_t state, inc;
  Pcg32(uint64_t seed, uint64_t stream) : state(0), inc((stream << 1u) | 1u) {
    next();
    state += seed;
    next();
  }
  uint32_t next() {
    uint64_t old = state;
    state = old * 6364136223846793005ull + inc;
    uint32_t xorshifted = static_cast<uint32_t>(((old >> 18u) ^ old) >> 27u);
    uint32_t rot = static_cast<uint32_t>(old >> 59u);
    return (xorshifted >> rot) | (xorshifted << ((-rot) & 31));
  }
  uint32_t below(uint32_t bound) {  // unbiased, Lemire-style rejection
    uint32_t threshold = (-bound) % bound;
    for (;;) {
      uint32_t r = next();
      if (r >= threshold) return r % bound;
    }
  }
};

struct Greedy {
  int32_t n;
  double alpha;
  std::vector<std::vector<int32_t>> lab;      // sorted labels per tensor id
  std::vector<char> live;
  std::vector<int32_t> users;                 // live holders per label
  std::vector<std::vector<int32_t>> holders;  // label -> live tensor ids
  std::unordered_map<uint64_t, double> cost;  // label-sharing pair -> Eq. (9) cost
  std::unordered_map<uint64_t, int> out_rank; // pair -> |LC|

  static uint64_t key(int32_t i, int32_t j) {
    if (i > j) std::swap(i, j);
    return (static_cast<uint64_t>(static_cast<uint32_t>(i)) << 32) | static_cast<uint32_t>(j);
  }

  // |LC| and |LA u LB| for contracting i and j now.
  void sizes(int32_t i, int32_t j, int* rc, int* ru) const {
    const auto& a = lab[i];
    const auto& b = lab[j];
    size_t x = 0, y = 0;
    int r = 0, u = 0;
    while (x < a.size() || y < b.size()) {
      int32_t l;
      int holders_here;
      if (y == b.size() || (x < a.size() && a[x] < b[y])) { l = a[x++]; holders_here = 1; }
      else if (x == a.size() || b[y] < a[x]) { l = b[y++]; holders_here = 1; }
      else { l = a[x]; ++x; ++y; holders_here = 2; }
      ++u;
      if (users[l] - holders_here > 0) ++r;
    }
    *rc = r;
    *ru = u;
  }

  void refresh_pairs_of(int32_t x) {
    for (int32_t l : lab[x])
      for (int32_t y : holders[l]) {
        if (y == x) continue;
        int rc, ru;
        sizes(x, y, &rc, &ru);
        double c = std::ldexp(1.0, rc) -
                   alpha * (std::ldexp(1.0, static_cast<int>(lab[x].size())) +
                            std::ldexp(1.0, static_cast<int>(lab[y].size())));
        cost[key(x, y)] = c;
        out_rank[key(x, y)] = rc;
      }
  }

  void drop_pairs_of(int32_t x) {
    for (int32_t l : lab[x])
      for (int32_t y : holders[l]) {
        if (y == x) continue;
        cost.erase(key(x, y));
        out_rank.erase(key(x, y));
      }
  }
};

int greedy_once(int32_t n, const int32_t* edges, int32_t m, double alpha, Pcg32* rng,
                int32_t* order, int* sc_out, double* tc_out) {
  const int32_t T = n + m;
  Greedy G;
  G.n = n;
  G.alpha = alpha;
  G.lab.resize(static_cast<size_t>(2 * T));
  G.live.assign(static_cast<size_t>(2 * T), 0);
  G.users.assign(static_cast<size_t>(n), 0);
  G.holders.assign(static_cast<size_t>(n), {});
  for (int32_t e = 0; e < m; ++e) {
    int32_t u = edges[2 * e], v = edges[2 * e + 1];
    G.lab[e] = {std::min(u, v), std::max(u, v)};
  }
  for (int32_t v = 0; v < n; ++v) G.lab[m + v] = {v};
  for (int32_t t = 0; t < T; ++t) {
    G.live[t] = 1;
    for (int32_t l : G.lab[t]) {
      G.users[l]++;
      G.holders[l].push_back(t);
    }
  }
  for (int32_t t = 0; t < T; ++t) G.refresh_pairs_of(t);

  int sc = 0;
  double tc = 0.0;
  std::vector<uint64_t> best;
  for (int32_t s = 0; s < T - 1; ++s) {
    int32_t pi = -1, pj = -1;
    if (!G.cost.empty()) {
      double bc = 0;
      best.clear();
      for (const auto& kv : G.cost) {
        if (best.empty() || kv.second < bc) {
          bc = kv.second;
          best.clear();
          best.push_back(kv.first);
        } else if (kv.second == bc) {
          best.push_back(kv.first);
        }
      }
      // unordered_map iteration order is unspecified: sort for determinism
      std::sort(best.begin(), best.end());
      uint64_t k = best[best.size() == 1 ? 0 : rng->below(static_cast<uint32_t>(best.size()))];
      pi = static_cast<int32_t>(k >> 32);
      pj = static_cast<int32_t>(k & 0xffffffffu);
    } else {
      // No label-sharing pair: outer product of the two lowest-rank tensors.
      for (int32_t t = 0; t < T + s; ++t) {
        if (!G.live[t]) continue;
        if (pi < 0 || G.lab[t].size() < G.lab[pi].size()) { pj = pi; pi = t; }
        else if (pj < 0 || G.lab[t].size() < G.lab[pj].size()) pj = t;
      }
    }
    const int32_t c = T + s;
    int rc, ru;
    G.sizes(pi, pj, &rc, &ru);
    // labels of c (sorted): those of the pair still used elsewhere
    std::vector<int32_t> lc;
    {
      const auto& a = G.lab[pi];
      const auto& b = G.lab[pj];
      std::vector<int32_t> uni;
      std::set_union(a.begin(), a.end(), b.begin(), b.end(), std::back_inserter(uni));
      for (int32_t l : uni) {
        int held = (std::binary_search(a.begin(), a.end(), l) ? 1 : 0) +
                   (std::binary_search(b.begin(), b.end(), l) ? 1 : 0);
        if (G.users[l] - held > 0) lc.push_back(l);
      }
    }
    if (static_cast<int>(lc.size()) > 62) return TN_EINVAL;
    sc = std::max(sc, static_cast<int>(lc.size()));
    tc += std::ldexp(1.0, ru);
    order[2 * s] = pi;
    order[2 * s + 1] = pj;

    // the labels whose holder counts change
    std::vector<int32_t> changed;
    std::set_union(G.lab[pi].begin(), G.lab[pi].end(), G.lab[pj].begin(), G.lab[pj].end(),
                   std::back_inserter(changed));
    G.drop_pairs_of(pi);
    G.drop_pairs_of(pj);
    for (int32_t id : {pi, pj}) {
      G.live[id] = 0;
      for (int32_t l : G.lab[id]) {
        G.users[l]--;
        auto& h = G.holders[l];
        h.erase(std::find(h.begin(), h.end(), id));
      }
    }
    G.lab[c] = lc;
    G.live[c] = 1;
    for (int32_t l : lc) {
      G.users[l]++;
      G.holders[l].push_back(c);
    }
    // every pair whose cost depends on a changed holder count
    std::vector<int32_t> touched;
    for (int32_t l : changed)
      for (int32_t t : G.holders[l]) touched.push_back(t);
    std::sort(touched.begin(), touched.end());
    touched.erase(std::unique(touched.begin(), touched.end()), touched.end());
    for (int32_t t : touched) G.refresh_pairs_of(t);
  }
  *sc_out = sc;
  *tc_out = tc;
  return TN_OK;
}

}  // namespace

int greedy_order(int32_t n, const int32_t* edges, int32_t m, double alpha, int32_t nrepeat,
                 uint64_t seed, int32_t* order_out) {
  if (!graph_ok(n, edges, m) || order_out == nullptr || !(alpha >= 0.0)) return TN_EINVAL;
  const int32_t T = n + m;
  if (T < 2) return TN_OK;
  if (nrepeat < 1) nrepeat = 1;
  std::vector<int32_t> tmp(static_cast<size_t>(2 * (T - 1)));
  int best_sc = -1;
  double best_tc = 0;
  for (int32_t r = 0; r < nrepeat; ++r) {
    Pcg32 rng(seed, static_cast<uint64_t>(r) + 1);
    int sc;
    double tc;
    int rc = greedy_once(n, edges, m, alpha, &rng, tmp.data(), &sc, &tc);
    if (rc != TN_OK) return rc;
    if (best_sc < 0 || sc < best_sc || (sc == best_sc && tc < best_tc)) {
      best_sc = sc;
      best_tc = tc;
      std::copy(tmp.begin(), tmp.end(), order_out);
    }
  }
  return TN_OK;
}

// ---------------------------------------------------------------------------
// Chinese remainder theorem, Garner's mixed-radix form (Knuth, TAOCP vol. 2,
// Sec. 4.3.2): x = v0 + v1 p0 + v2 p0 p1 + ...,  with
// v_k = (r_k - (v0 + v1 p0 + ...)) * (p0 ... p_{k-1})^{-1}  mod p_k.
// ---------------------------------------------------------------------------
namespace {

uint32_t big_mod(const std::vector<uint32_t>& a, uint32_t p) {
  uint64_t r = 0;
  for (size_t i = a.size(); i-- > 0;) r = ((r << 32) | a[i]) % p;
  return static_cast<uint32_t>(r);
}

void big_mul_add(std::vector<uint32_t>* a, uint32_t mul, uint32_t add) {
  uint64_t carry = add;
  for (auto& limb : *a) {
    uint64_t t = static_cast<uint64_t>(limb) * mul + carry;
    limb = static_cast<uint32_t>(t);
    carry = t >> 32;
  }
  if (carry) a->push_back(static_cast<uint32_t>(carry));
}

// a += b * c (b big, c small)
void big_addmul(std::vector<uint32_t>* a, const std::vector<uint32_t>& b, uint32_t c) {
  if (a->size() < b.size() + 1) a->resize(b.size() + 1, 0);
  uint64_t carry = 0;
  size_t i = 0;
  for (; i < b.size(); ++i) {
    uint64_t t = static_cast<uint64_t>(b[i]) * c + (*a)[i] + carry;
    (*a)[i] = static_cast<uint32_t>(t);
    carry = t >> 32;
  }
  for (; carry && i < a->size(); ++i) {
    uint64_t t = static_cast<uint64_t>((*a)[i]) + carry;
    (*a)[i] = static_cast<uint32_t>(t);
    carry = t >> 32;
  }
  if (carry) a->push_back(static_cast<uint32_t>(carry));
  while (!a->empty() && a->back() == 0) a->pop_back();
}

// modular inverse by the extended Euclidean algorithm; 0 if none
uint32_t inv_mod(uint32_t a, uint32_t p) {
  int64_t t = 0, newt = 1, r = p, newr = a % p;
  while (newr != 0) {
    int64_t q = r / newr;
    int64_t tmp = t - q * newt; t = newt; newt = tmp;
    tmp = r - q * newr; r = newr; newr = tmp;
  }
  if (r != 1) return 0;
  if (t < 0) t += p;
  return static_cast<uint32_t>(t);
}

}  // namespace

int crt_garner(const uint32_t* residues, const uint32_t* primes, int nprimes, uint32_t* limbs,
               int max_limbs) {
  std::vector<uint32_t> x;            // running value
  std::vector<uint32_t> M = {1};      // product of the moduli so far
  for (int k = 0; k < nprimes; ++k) {
    uint32_t p = primes[k];
    uint32_t xm = big_mod(x, p), Mm = big_mod(M, p);
    uint32_t inv = inv_mod(Mm, p);
    if (inv == 0) return -1;
    uint64_t diff = (static_cast<uint64_t>(residues[k] % p) + p - xm) % p;
    uint32_t v = static_cast<uint32_t>((diff * inv) % p);
    big_addmul(&x, M, v);
    big_mul_add(&M, p, 0);
  }
  if (static_cast<int>(x.size()) > max_limbs) return -1;
  for (size_t i = 0; i < x.size(); ++i) limbs[i] = x[i];
  return static_cast<int>(x.size());
}

}  // namespace tn
