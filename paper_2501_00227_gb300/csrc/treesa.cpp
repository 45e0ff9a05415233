// treesa.cpp -- the local-search (simulated annealing) contraction-order
// optimiser of Sec. 4.2.2 ("TreeSA").
//
// A contraction order is a binary tree over the network's leaves (edge
// tensors, then vertex tensors).  A node's labels are those of its subtree
// that some leaf outside it still carries (Sec. 4.1); a leaf keeps all of its
// labels.  With lab(x) those labels, a node x = (a, b) costs
//   tc(x) = 2^{|lab(a) u lab(b)|},  rw(x) = 2^|lab(a)| + 2^|lab(b)| + 2^|lab(x)|,
// and the tree costs (Eq. 10, on log2 scales as the paper's sc_target is)
//   L = log2(sum tc) + w_s * max(0, log2 sc - sc_target) + w_rw * log2(sum rw),
// sc = the largest 2^|lab(x)|.
//
// Moves: at an internal node N whose child I = (X, Y) is internal and whose
// other child is Z, swap Z with X or with Y -- the four rewrites
// (A*B)*C = (A*C)*B = (C*B)*A and A*(B*C) = B*(A*C) = C*(B*A).  Only I
// changes its labels:
//   lab(I') = (lab(Z) u lab(keep)) n (lab(N) u lab(out)),
// (a label of I's new subtree is still needed iff it appears outside N or in
// the child swapped out), so a move is evaluated from two nodes.  A move is
// taken with the Metropolis probability min(1, e^{-beta dL}) (Eq. 11), beta
// rising through the schedule, where dL is the change of the cost of the
// two rewritten contractions alone (with the whole tree's dL, a change to a
// small contraction moves log2 of the sum by almost nothing and is taken
// blindly, and the schedule never settles them); the tree's own cost keeps
// the best tree seen.  Every sweep visits all internal nodes in a random
// order, niters sweeps per beta.  Trials start from greedy orders
// (Sec. 4.2.1, one run each, own seed) or random trees, run on host threads,
// and the best tree seen over all trials is returned as an SSA order.
//
// Slicing (the optimiser's nslices / fixed_slices): a sliced label leaves
// every tensor, so it is cut from every node's label set and the sums are
// recounted; costs are then those of one slice.  Fixed labels are cut from
// the start, the others picked while annealing (struct Slicer).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <random>
#include <thread>
#include <vector>

#include "tn_internal.h"

namespace tn {
namespace {

struct Rng {
  std::mt19937_64 g;
  explicit Rng(uint64_t seed) : g(seed) {}
  double uniform() { return static_cast<double>(g() >> 11) * (1.0 / 9007199254740992.0); }
  uint32_t below(uint32_t k) { return static_cast<uint32_t>(g() % k); }
};

// A sum of powers of two kept exactly as a count per exponent (a running
// double would lose the small terms after a large one comes and goes);
// log2 of the sum reads the 63 exponents below the largest.
struct ExpSum {
  std::vector<int64_t> cnt;
  int top = 0;
  void reset(int kmax) {
    cnt.assign(kmax + 1, 0);
    top = 0;
  }
  void add(int k, int64_t d) {
    cnt[k] += d;
    if (d > 0 && k > top) top = k;
    while (top > 0 && cnt[top] == 0) --top;
  }
  double log2sum() const {
    double s = 0;
    for (int k = top; k >= 0 && k >= top - 62; --k) s += std::ldexp(static_cast<double>(cnt[k]), k - top);
    return top + std::log2(s);
  }
};

struct Tree {
  int T = 0, W = 0;                 // leaves, 64-bit words per label set
  std::vector<int32_t> left, right, parent;
  std::vector<uint64_t> lab;        // W words per node
  std::vector<int32_t> rank;        // |lab|
  std::vector<int32_t> tce;         // per internal node: log2 tc = |lab(a) u lab(b)|
  std::vector<int32_t> rank_hist;   // internal nodes per rank (for sc)
  ExpSum TC, RW;                    // sum of tc; sum of rw (three terms per internal node)
  int root = -1;

  uint64_t* L(int x) { return &lab[size_t(x) * W]; }
  const uint64_t* L(int x) const { return &lab[size_t(x) * W]; }
  int popc(const uint64_t* a) const {
    int c = 0;
    for (int w = 0; w < W; ++w) c += __builtin_popcountll(a[w]);
    return c;
  }
  int popc_or(const uint64_t* a, const uint64_t* b) const {
    int c = 0;
    for (int w = 0; w < W; ++w) c += __builtin_popcountll(a[w] | b[w]);
    return c;
  }
  int sc() const {
    for (int r = static_cast<int>(rank_hist.size()) - 1; r >= 0; --r)
      if (rank_hist[r]) return r;
    return 0;
  }
};

// Cost of Eq. 10 from the running sums.
double cost(const Tree& t, double sc_target, double ws, double wrw) {
  return t.TC.log2sum() + ws * std::max(0.0, t.sc() - sc_target) + wrw * t.RW.log2sum();
}

void recount(Tree* t);

// Tree from an SSA order; leaf labels: edge e = {u, v}, vertex v = {v}.
void build_tree(int32_t n, const int32_t* edges, int32_t m, const int32_t* order, Tree* t) {
  const int T = n + m, N = 2 * T - 1;
  t->T = T;
  t->W = (n + 63) / 64;
  t->left.assign(N, -1);
  t->right.assign(N, -1);
  t->parent.assign(N, -1);
  t->lab.assign(size_t(N) * t->W, 0);
  t->rank.assign(N, 0);
  t->tce.assign(N, 0);
  std::vector<int32_t> total(n, 0);  // leaves carrying each label
  for (int e = 0; e < m; ++e)
    for (int k = 0; k < 2; ++k) {
      const int v = edges[2 * e + k];
      t->L(e)[v / 64] |= 1ull << (v % 64);
      total[v]++;
    }
  for (int v = 0; v < n; ++v) {
    t->L(m + v)[v / 64] |= 1ull << (v % 64);
    total[v]++;
  }
  // internal nodes: labels of the union still carried by some leaf outside;
  // cs[x] = (label, leaves of x's subtree carrying it), sorted by label
  std::vector<std::vector<std::pair<int32_t, int32_t>>> cs(N);
  for (int x = 0; x < T; ++x)
    for (int v = 0; v < n; ++v)
      if ((t->L(x)[v / 64] >> (v % 64)) & 1) cs[x].push_back({v, 1});
  for (int s = 0; s < T - 1; ++s) {
    const int a = order[2 * s], b = order[2 * s + 1], c = T + s;
    t->left[c] = a;
    t->right[c] = b;
    t->parent[a] = c;
    t->parent[b] = c;
    std::vector<std::pair<int32_t, int32_t>> merged;
    auto &A = cs[a], &B = cs[b];
    size_t i = 0, j = 0;
    while (i < A.size() || j < B.size()) {
      if (j == B.size() || (i < A.size() && A[i].first < B[j].first)) merged.push_back(A[i++]);
      else if (i == A.size() || B[j].first < A[i].first) merged.push_back(B[j++]);
      else {
        merged.push_back({A[i].first, A[i].second + B[j].second});
        ++i;
        ++j;
      }
    }
    for (auto& kv : merged)
      if (kv.second < total[kv.first]) t->L(c)[kv.first / 64] |= 1ull << (kv.first % 64);
    cs[c] = std::move(merged);
    std::vector<std::pair<int32_t, int32_t>>().swap(cs[a]);
    std::vector<std::pair<int32_t, int32_t>>().swap(cs[b]);
  }
  t->root = N - 1;
  recount(t);
}

// Ranks of all nodes and the running sums, from the label sets.
void recount(Tree* t) {
  const int T = t->T, N = static_cast<int>(t->left.size()), nl = t->W * 64;
  t->rank_hist.assign(nl + 2, 0);
  t->TC.reset(nl + 2);
  t->RW.reset(nl + 2);
  for (int x = 0; x < T; ++x) t->rank[x] = t->popc(t->L(x));
  for (int c = T; c < N; ++c) {
    t->rank[c] = t->popc(t->L(c));
    const int a = t->left[c], b = t->right[c];
    t->tce[c] = t->popc_or(t->L(a), t->L(b));
    t->TC.add(t->tce[c], 1);
    t->RW.add(t->rank[a], 1);
    t->RW.add(t->rank[b], 1);
    t->RW.add(t->rank[c], 1);
    t->rank_hist[t->rank[c]]++;
  }
}

// Slice label v: it leaves every tensor (a sliced network's leaves do not
// carry it), so it leaves every node's label set.
void slice_label(Tree* t, int v) {
  const int N = static_cast<int>(t->left.size());
  for (int x = 0; x < N; ++x) t->L(x)[v / 64] &= ~(1ull << (v % 64));
  recount(t);
}

// The label whose slicing leaves the smallest largest intermediate, ties by
// the smallest total work (the rule of tn_slice_labels, on the tree's
// current label sets); -1 when every label is sliced already.
int pick_slice(const Tree& t, int n, const std::vector<char>& cut) {
  const int T = t.T, N = static_cast<int>(t.left.size());
  int best = -1, bsc = 0;
  double btc = 0;
  for (int v = 0; v < n; ++v) {
    if (cut[v]) continue;
    const int w = v / 64;
    const uint64_t bit = 1ull << (v % 64);
    int sc = 0;
    double tc = 0;
    for (int c = T; c < N; ++c) {
      sc = std::max(sc, t.rank[c] - ((t.L(c)[w] & bit) ? 1 : 0));
      const bool in = ((t.L(t.left[c])[w] | t.L(t.right[c])[w]) & bit) != 0;
      tc += std::ldexp(1.0, t.tce[c] - (in ? 1 : 0));
    }
    if (best < 0 || sc < bsc || (sc == bsc && tc < btc)) {
      best = v;
      bsc = sc;
      btc = tc;
    }
  }
  return best;
}

// SSA order of the tree (children before parents, post-order).
void tree_order(const Tree& t, int32_t* order) {
  std::vector<int32_t> id(t.left.size(), -1);
  for (int x = 0; x < t.T; ++x) id[x] = x;
  int next = t.T, s = 0;
  std::vector<std::pair<int32_t, bool>> stack{{t.root, false}};
  while (!stack.empty()) {
    auto [x, done] = stack.back();
    stack.pop_back();
    if (x < t.T) continue;
    if (!done) {
      stack.push_back({x, true});
      stack.push_back({t.right[x], false});
      stack.push_back({t.left[x], false});
    } else {
      order[2 * s] = id[t.left[x]];
      order[2 * s + 1] = id[t.right[x]];
      ++s;
      id[x] = next++;
    }
  }
}

struct Params {
  double sc_target, b0, db, b1, ws, wrw;
  int niters;
};

// Slicing inside the annealing: `want` more labels are sliced, one at a time
// (pick_slice) after a beta step, whenever the tree is above sc_target and
// in any case once the schedule is half done, so that the tree keeps
// adapting to the slices; any still missing at the end are picked then.
struct Slicer {
  int n = 0, m = 0, want = 0;
  const int32_t* edges = nullptr;
  std::vector<int32_t> fixed;
  std::vector<char> cut;          // sliced labels (fixed ones included)
  std::vector<int32_t> picked;    // in the order picked
  std::vector<int32_t> best_picked;  // those of the best tree
};

void slice_one(Tree* t, Slicer* sl) {
  const int v = pick_slice(*t, sl->n, sl->cut);
  if (v < 0) {  // every label sliced already: nothing more to take
    sl->want = static_cast<int>(sl->picked.size());
    return;
  }
  sl->cut[v] = 1;
  sl->picked.push_back(v);
  slice_label(t, v);
}

// Once all slices are in: pick them again, from scratch, on the current
// tree (rebuilt from its order with the fixed labels cut), and keep the new
// set if the tree's cost drops -- labels picked on an early tree would
// otherwise stay whatever the annealing made of it.
bool reslice(Tree* t, Slicer* sl, const Params& P) {
  std::vector<int32_t> ord(2 * size_t(t->T - 1));
  tree_order(*t, ord.data());
  Tree u;
  build_tree(sl->n, sl->edges, sl->m, ord.data(), &u);
  std::vector<char> cut(static_cast<size_t>(sl->n), 0);
  for (int32_t f : sl->fixed) {
    cut[f] = 1;
    slice_label(&u, f);
  }
  std::vector<int32_t> picked;
  for (int j = 0; j < sl->want; ++j) {
    const int v = pick_slice(u, sl->n, cut);
    if (v < 0) return false;
    cut[v] = 1;
    picked.push_back(v);
    slice_label(&u, v);
  }
  if (!(cost(u, P.sc_target, P.ws, P.wrw) < cost(*t, P.sc_target, P.ws, P.wrw) - 1e-12)) return false;
  *t = std::move(u);
  sl->cut = std::move(cut);
  sl->picked = std::move(picked);
  return true;
}

// One annealing run on t; returns the best cost seen and leaves the best
// tree's SSA order in best_order.  With a slicer, the best tree is taken
// among those carrying all of its slices.
double anneal(Tree* t, const Params& P, Rng* rng, std::vector<int32_t>* best_order, Slicer* sl = nullptr) {
  const int N = static_cast<int>(t->left.size());
  const int W = t->W;
  std::vector<int32_t> internal;
  for (int x = t->T; x < N; ++x) internal.push_back(x);
  std::vector<uint64_t> nl(W);
  double cur = cost(*t, P.sc_target, P.ws, P.wrw);
  double best = cur;
  best_order->assign(2 * size_t(t->T - 1), 0);
  auto keep_best = [&]() {
    best = cur;
    tree_order(*t, best_order->data());
    if (sl) sl->best_picked = sl->picked;
  };
  keep_best();
  const int nbeta = static_cast<int>(std::floor((P.b1 - P.b0) / P.db + 1e-9)) + 1;
  for (int bi = 0; bi < nbeta; ++bi) {
    const double beta = P.b0 + bi * P.db;
    for (int it = 0; it < P.niters; ++it) {
      for (size_t i = internal.size(); i > 1; --i) std::swap(internal[i - 1], internal[rng->below(uint32_t(i))]);
      for (int Nn : internal) {
        const int l = t->left[Nn], r = t->right[Nn];
        const bool li = l >= t->T, ri = r >= t->T;
        if (!li && !ri) continue;
        // inner node I, its sibling Z; pick which of I's children leaves
        const bool use_left = li && (!ri || (rng->below(2) == 0));
        const int I = use_left ? l : r, Z = use_left ? r : l;
        const bool swap_x = rng->below(2) == 0;
        const int out = swap_x ? t->left[I] : t->right[I];
        const int keep = swap_x ? t->right[I] : t->left[I];
        // new labels of I = (Z, keep)
        const uint64_t *lz = t->L(Z), *lk = t->L(keep), *ln = t->L(Nn), *lo = t->L(out);
        for (int w = 0; w < W; ++w) nl[w] = (lz[w] | lk[w]) & (ln[w] | lo[w]);
        int nrank = 0, tcI = 0, tcN = 0;
        for (int w = 0; w < W; ++w) {
          nrank += __builtin_popcountll(nl[w]);
          tcI += __builtin_popcountll(lz[w] | lk[w]);
          tcN += __builtin_popcountll(nl[w] | lo[w]);
        }
        // replace I's and N's terms: tc, rw = (children, self) ranks, and I's rank
        const int rX = t->rank[t->left[I]], rY = t->rank[t->right[I]], rI = t->rank[I];
        const int rZ = t->rank[Z], rK = t->rank[keep], rO = t->rank[out], rN = t->rank[Nn];
        auto apply_terms = [&](int64_t d, int tcI_, int tcN_, int a1, int a2, int a3, int b1, int b2) {
          t->TC.add(tcI_, d);
          t->TC.add(tcN_, d);
          t->RW.add(a1, d);
          t->RW.add(a2, d);
          t->RW.add(a3, d);  // I's rw
          t->RW.add(a3, d);  // I's rank inside N's rw
          t->RW.add(b1, d);
          t->RW.add(b2, d);
        };
        // the move is scored by the cost of the two rewritten contractions
        // (their log2 tc sum, rank penalty and log2 rw sum); the tree's cost
        // of Eq. 10 picks the best tree seen
        auto local = [&](int tc1, int tc2, int r1, int a1, int a2, int b1, int b2) {
          const double tcs = std::log2(std::ldexp(1.0, tc1) + std::ldexp(1.0, tc2));
          const double rws = std::log2(std::ldexp(1.0, a1) + std::ldexp(1.0, a2) + 2 * std::ldexp(1.0, r1) +
                                       std::ldexp(1.0, b1) + std::ldexp(1.0, b2));
          return tcs + P.ws * std::max(0.0, r1 - P.sc_target) + P.wrw * rws;
        };
        const double d = local(tcI, tcN, nrank, rZ, rK, rO, rN) - local(t->tce[I], t->tce[Nn], rI, rX, rY, rZ, rN);
        if (d <= 0 || rng->uniform() < std::exp(-beta * d)) {
          apply_terms(-1, t->tce[I], t->tce[Nn], rX, rY, rI, rZ, rN);
          apply_terms(+1, tcI, tcN, rZ, rK, nrank, rO, rN);
          t->rank_hist[rI]--;
          t->rank_hist[nrank]++;
          const double c2 = cost(*t, P.sc_target, P.ws, P.wrw);
          // apply: I = (Z, keep), N = (I, out) keeping I on the same side
          t->left[I] = Z;
          t->right[I] = keep;
          t->parent[Z] = I;
          t->parent[keep] = I;
          if (use_left) t->right[Nn] = out;
          else t->left[Nn] = out;
          t->parent[out] = Nn;
          std::memcpy(t->L(I), nl.data(), sizeof(uint64_t) * W);
          t->rank[I] = nrank;
          t->tce[I] = tcI;
          t->tce[Nn] = tcN;
          cur = c2;
          if (cur < best - 1e-12) keep_best();
        }
      }
    }
    if (!sl) continue;
    if (static_cast<int>(sl->picked.size()) < sl->want) {
      if (t->sc() > P.sc_target || 2 * (bi + 1) >= nbeta || bi + 1 == nbeta) {
        do slice_one(t, sl);
        while (bi + 1 == nbeta && static_cast<int>(sl->picked.size()) < sl->want);
        // the trees seen so far carry fewer slices: start the best over
        cur = cost(*t, P.sc_target, P.ws, P.wrw);
        keep_best();
      }
    } else if (sl->want > 0 && reslice(t, sl, P)) {
      cur = cost(*t, P.sc_target, P.ws, P.wrw);
      if (cur < best - 1e-12) keep_best();
    }
  }
  return best;
}

// A random binary tree: repeatedly join two random live subtrees.
void random_order(int T, Rng* rng, int32_t* order) {
  std::vector<int32_t> live(T);
  for (int x = 0; x < T; ++x) live[x] = x;
  for (int s = 0; s < T - 1; ++s) {
    const uint32_t i = rng->below(uint32_t(live.size()));
    std::swap(live[i], live.back());
    const int a = live.back();
    live.pop_back();
    const uint32_t j = rng->below(uint32_t(live.size()));
    order[2 * s] = a;
    order[2 * s + 1] = live[j];
    live[j] = T + s;
  }
}

}  // namespace
}  // namespace tn

namespace tn {
namespace {

// Both entry points: anneal ntrials trees (the fixed slices cut from the
// start, nslices more picked while annealing) and return the best.
int treesa_run(int32_t n, const int32_t* edges, int32_t m, const tn_treesa_params_t* prm, const int32_t* fixed,
               int32_t nfixed, int32_t nslices, int32_t* order_out, int32_t* sliced_out, double* log2_out) {
  if (!prm || !order_out || n < 1 || m < 0 || (m > 0 && !edges)) return TN_EINVAL;
  if (!(prm->beta_step > 0) || !(prm->beta_stop >= prm->beta_start) || prm->niters < 0 || prm->ntrials < 1 ||
      !(prm->sc_weight >= 0) || !(prm->rw_weight >= 0) || (prm->beta_stop - prm->beta_start) / prm->beta_step > 1e6)
    return TN_EINVAL;
  if (nfixed < 0 || nslices < 0 || nfixed + nslices > std::min(n, 62) || (nfixed > 0 && !fixed) ||
      (nfixed + nslices > 0 && !sliced_out))
    return TN_EINVAL;
  std::vector<char> cut0(static_cast<size_t>(n), 0);
  for (int j = 0; j < nfixed; ++j) {
    if (fixed[j] < 0 || fixed[j] >= n || cut0[fixed[j]]) return TN_EINVAL;
    cut0[fixed[j]] = 1;
  }
  const int32_t T = n + m;
  if (T < 2) {  // one vertex tensor, no contraction: label 0 is the only one
    for (int j = 0; j < nfixed + nslices; ++j) sliced_out[j] = 0;
    if (log2_out) log2_out[0] = log2_out[1] = log2_out[2] = 0;
    return TN_OK;
  }
  try {
    // validate the graph (and get a greedy order) through the greedy optimiser
    std::vector<int32_t> init(2 * size_t(T - 1));
    int rc = greedy_order(n, edges, m, 0.0, 1, prm->seed, init.data());
    if (rc) return rc;
    Params P{prm->sc_target, prm->beta_start, prm->beta_step, prm->beta_stop, prm->sc_weight, prm->rw_weight,
             prm->niters};
    const int trials = prm->ntrials;
    std::vector<double> best(trials, INFINITY);
    std::vector<std::vector<int32_t>> orders(trials), picks(trials);
    std::vector<int> rcs(trials, TN_OK);
    auto run = [&](int k) {
      try {
        Rng rng(prm->seed * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull * uint64_t(k + 1));
        std::vector<int32_t> start(2 * size_t(T - 1));
        if (prm->random_init) {
          random_order(T, &rng, start.data());
        } else {
          const int r = greedy_order(n, edges, m, 0.0, 1, prm->seed + 7919ull * uint64_t(k), start.data());
          if (r) {
            rcs[k] = r;
            return;
          }
        }
        Tree t;
        build_tree(n, edges, m, start.data(), &t);
        for (int j = 0; j < nfixed; ++j) slice_label(&t, fixed[j]);
        Slicer sl;
        sl.n = n;
        sl.m = m;
        sl.edges = edges;
        sl.fixed.assign(fixed, fixed + nfixed);
        sl.want = nslices;
        sl.cut = cut0;
        best[k] = anneal(&t, P, &rng, &orders[k], nslices > 0 ? &sl : nullptr);
        picks[k] = sl.best_picked;
      } catch (const std::bad_alloc&) {
        rcs[k] = TN_ENOMEM;
      }
    };
    int nth = prm->nthreads > 0 ? prm->nthreads : static_cast<int>(std::thread::hardware_concurrency());
    nth = std::max(1, std::min(nth, trials));
    for (int k0 = 0; k0 < trials; k0 += nth) {
      std::vector<std::thread> pool;
      for (int k = k0; k < std::min(trials, k0 + nth); ++k) pool.emplace_back(run, k);
      for (auto& th : pool) th.join();
    }
    int kb = -1;
    for (int k = 0; k < trials; ++k) {
      if (rcs[k]) return rcs[k];
      if (kb < 0 || best[k] < best[kb]) kb = k;
    }
    if (static_cast<int>(picks[kb].size()) != nslices) return TN_EINVAL;
    std::copy(orders[kb].begin(), orders[kb].end(), order_out);
    for (int j = 0; j < nfixed; ++j) sliced_out[j] = fixed[j];
    for (int j = 0; j < nslices; ++j) sliced_out[nfixed + j] = picks[kb][j];
    if (log2_out) {
      // per slice: work, largest intermediate, reads and writes; the work
      // and traffic of all 2^s slices are 2^s times one slice's
      Tree t;
      build_tree(n, edges, m, order_out, &t);
      for (int j = 0; j < nfixed + nslices; ++j) slice_label(&t, sliced_out[j]);
      log2_out[0] = t.TC.log2sum() + nfixed + nslices;
      log2_out[1] = t.sc();
      log2_out[2] = t.RW.log2sum() + nfixed + nslices;
    }
    return TN_OK;
  } catch (const std::bad_alloc&) {
    return TN_ENOMEM;
  }
}

}  // namespace
}  // namespace tn

extern "C" int tn_order_treesa(int32_t n, const int32_t* edges, int32_t m, const tn_treesa_params_t* prm,
                               int32_t* order_out, double* log2_out) {
  return tn::treesa_run(n, edges, m, prm, nullptr, 0, 0, order_out, nullptr, log2_out);
}

extern "C" int tn_order_treesa_sliced(int32_t n, const int32_t* edges, int32_t m, const tn_treesa_params_t* prm,
                                      int32_t nslices, const int32_t* fixed_slices, int32_t nfixed,
                                      int32_t* order_out, int32_t* sliced_out, double* log2_out) {
  return tn::treesa_run(n, edges, m, prm, fixed_slices, nfixed, nslices, order_out, sliced_out, log2_out);
}
