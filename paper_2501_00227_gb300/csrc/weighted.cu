// weighted.cu -- networks with integer weights on the same executor:
// vertex-weighted independent sets (Eqs. 5-7 with weights w_v) and the spin
// glass of Eq. 1 (couplings J_ij, fields h_i, spin s = 2n - 1).
//
// The unit-weight IS network generates its leaves inside the contraction
// kernels from the entry index.  A weighted network's leaves depend on
// per-edge / per-vertex data, so it runs with the executor plan whose leaf
// operands are arena tensors (4 entries per edge, then 2 per vertex, at the
// plan's leaf_base, in every prime block and in the count region alike):
// k_leaves writes them there before each launch, and the contraction
// kernels read them exactly like intermediates (no extra test on the hot
// path).
//
// Leaf values (entry x of an edge tensor: n_u = x & 1, n_v = x >> 1):
//   IS          B = [one, one, one, zero]; W = [one, w_v]  (tropical w_v,
//               counting (w_v, 1), mod p x^{w_v} for the slot's point x)
//   spin glass  tropical / counting maximise -H: B = -J s_u s_v,
//               W = -h s_v (count 1); mod p with the slot's point y:
//               B = y^{J s_u s_v + |J|}, W = y^{h s_v + |h|}, so the network
//               is sum_sigma y^{H(sigma) + sum|J| + sum|h|}.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "exec.h"
#include "kernels.h"
#include "tn_internal.h"

using tn::dev::ModTable;

namespace tn {
int make_mod_table_slots(const uint32_t* primes, const uint32_t* xs, int32_t nslots, void* mods);
int make_mod_table_checked(tn_semiring_t s, const uint32_t* primes, int32_t nprimes, void* mods);
int decode_raw_any(tn_semiring_t s, const void* mods, int32_t nprimes, const unsigned char* raw, tn_result_t* out);
}  // namespace tn

namespace tn {
namespace dev {
namespace {

struct LeafArgs {
  int32_t m, n, T, problem, semiring;
  int32_t nslots;
  int64_t stride;         // entries between prime-slot blocks (mod p)
  const int32_t* edges;   // 2m endpoints
  const int64_t* loff;    // entry offset of each leaf (edges, then vertices)
  const int8_t* fixed;    // per vertex: -1, or the value of a sliced label in this slice
  const int32_t* ew;      // J per edge (spin glass), or NULL
  const int32_t* vw;      // w_v (IS) or h_v (spin glass), or NULL
  char* l0;               // values of leaf entry 0 (prime block 0)
  char* l1;               // counts of leaf entry 0 (counting)
  int64_t net_stride;     // several networks (blockIdx.y): arena entries between their leaves
  uint32_t p[TN_MAX_PRIMES];
  uint32_t x[TN_MAX_PRIMES];
};

__device__ uint32_t pow_mod(uint32_t b, int64_t e, uint32_t p) {
  uint64_t r = 1u % p, base = b % p;
  while (e > 0) {
    if (e & 1) r = r * base % p;
    base = base * base % p;
    e >>= 1;
  }
  return static_cast<uint32_t>(r);
}

// (value, exponent, allowed) of an edge / vertex tensor entry for the 0/1
// labels n_u, n_v (vertex: n_v only): value for max-plus, exponent of the
// slot's point for mod p
__device__ void edge_entry(const LeafArgs& a, int64_t k, int nu, int nv, int64_t* val, int64_t* mexp, bool* ok) {
  *ok = true;
  if (a.problem == TN_PROBLEM_INDEPENDENT_SET) {
    *ok = !(nu && nv);
    *val = 0;
    *mexp = 0;
  } else {
    const int64_t J = a.ew ? a.ew[k] : 1;
    const int64_t ss = nu == nv ? 1 : -1;  // s_u s_v
    *val = -J * ss;
    *mexp = J * ss + (J < 0 ? -J : J);
  }
}
__device__ void vertex_entry(const LeafArgs& a, int64_t v, int nv, int64_t* val, int64_t* mexp, bool* ok) {
  *ok = true;
  if (a.problem == TN_PROBLEM_INDEPENDENT_SET) {
    const int64_t w = a.vw ? a.vw[v] : 1;
    *val = nv ? w : 0;
    *mexp = *val;
  } else {
    const int64_t h = a.vw ? a.vw[v] : 0;
    const int64_t s = nv ? 1 : -1;
    *val = -h * s;
    *mexp = h * s + (h < 0 ? -h : h);
  }
}

// One thread per (prime slot, leaf): every entry of the leaf.  A leaf keeps
// its unsliced labels in order (u, then v); entry bit j is the j-th of them,
// and a sliced label takes its value in this slice.
__global__ void k_leaves(const __grid_constant__ LeafArgs a) {
  const int nq = a.semiring == TN_COUNT_MODP ? a.nslots : 1;
  const int64_t total = int64_t(a.T) * nq;
  // network blockIdx.y (a slice of a batch): its own label values and leaves
  const int8_t* fixed = a.fixed + int64_t(blockIdx.y) * a.n;
  const int64_t base = int64_t(blockIdx.y) * a.net_stride;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total; t += int64_t(gridDim.x) * blockDim.x) {
    const int32_t leaf = static_cast<int32_t>(t % a.T);
    const int q = static_cast<int>(t / a.T);
    const bool edge = leaf < a.m;
    const int32_t u = edge ? a.edges[2 * leaf] : leaf - a.m;
    const int32_t v = edge ? a.edges[2 * leaf + 1] : -1;
    const int fu = fixed[u], fv = edge ? fixed[v] : 0;
    const int rank = (fu < 0 ? 1 : 0) + (edge && fv < 0 ? 1 : 0);
    for (int x = 0; x < (1 << rank); ++x) {
      int bit = 0;
      const int nu = fu < 0 ? (x >> bit++) & 1 : fu;
      const int nv = edge ? (fv < 0 ? (x >> bit) & 1 : fv) : 0;
      int64_t val, mexp;
      bool ok;
      if (edge) edge_entry(a, leaf, nu, nv, &val, &mexp, &ok);
      else vertex_entry(a, u, nu, &val, &mexp, &ok);
      const int64_t i = base + a.loff[leaf] + x;
      switch (a.semiring) {
        case TN_TROPICAL_F32:
          reinterpret_cast<float*>(a.l0)[i] = ok ? static_cast<float>(val) : -INFINITY;
          break;
        case TN_TROPICAL_I32:
          reinterpret_cast<int32_t*>(a.l0)[i] = ok ? static_cast<int32_t>(val) : TN_I32_NEG_INF;
          break;
        case TN_COUNTING_TROPICAL:
          reinterpret_cast<int32_t*>(a.l0)[i] = ok ? static_cast<int32_t>(val) : TN_I32_NEG_INF;
          reinterpret_cast<uint64_t*>(a.l1)[i] = ok ? 1ull : 0ull;
          break;
        default:
          reinterpret_cast<uint32_t*>(a.l0)[q * a.stride + i] = ok ? pow_mod(a.x[q], mexp, a.p[q]) : 0u;
          break;
      }
    }
  }
}

}  // namespace
}  // namespace dev

namespace {

size_t align256(size_t b) { return (b + 255) / 256 * 256; }
int cuda_rc(cudaError_t e) { return e == cudaSuccess ? TN_OK : TN_ECUDA; }

// Workspace of a weighted contraction: the executor's (stored-leaf plan),
// then the weights (n + m int32), the edge list, the leaf offsets and the
// sliced-label values.
struct WeightedLayout {
  size_t exec_bytes, ew_off, vw_off, edges_off, loff_off, fixed_off, total;
};

ExecPlan* weighted_plan(tn_plan_s* p, tn_semiring_t s, int32_t nslots, bool keep, int* rc) {
  return exec_plan_get_h(p, s, nslots, 1, false, rc, keep, true);
}

WeightedLayout weighted_layout(tn_plan_s* p, tn_semiring_t s, int32_t nslots, bool keep, int* rc) {
  WeightedLayout L{};
  ExecPlan* X = weighted_plan(p, s, nslots, keep, rc);
  if (!X) return L;
  L.exec_bytes = align256(X->total_bytes);
  L.ew_off = L.exec_bytes;
  L.vw_off = L.ew_off + align256(4 * size_t(std::max(p->m, 1)));
  L.edges_off = L.vw_off + align256(4 * size_t(std::max(p->n, 1)));
  L.loff_off = L.edges_off + align256(8 * size_t(std::max(p->m, 1)));
  L.fixed_off = L.loff_off + align256(8 * size_t(p->T));
  L.total = L.fixed_off + align256(size_t(std::max(p->n, 1)));
  return L;
}

// Host-side checks of the weights: int32 sums of the max-plus values stay far
// from TN_I32_NEG_INF (and exact in float32); mod p needs exponents >= 0.
int check_weights(tn_plan_s* p, tn_semiring_t s, int32_t problem, const int32_t* ew, const int32_t* vw) {
  if (problem != TN_PROBLEM_INDEPENDENT_SET && problem != TN_PROBLEM_SPIN_GLASS) return TN_EINVAL;
  double total = 0;
  if (problem == TN_PROBLEM_SPIN_GLASS && ew)
    for (int k = 0; k < p->m; ++k) total += std::fabs(double(ew[k]));
  else if (problem == TN_PROBLEM_SPIN_GLASS)
    total += p->m;
  if (vw)
    for (int v = 0; v < p->n; ++v) {
      total += std::fabs(double(vw[v]));
      if (problem == TN_PROBLEM_INDEPENDENT_SET && s == TN_COUNT_MODP && vw[v] < 0) return TN_EINVAL;
    }
  else if (problem == TN_PROBLEM_INDEPENDENT_SET)
    total += p->n;
  const double cap = s == TN_TROPICAL_F32 ? double(1 << 24) : double(1 << 28);
  if (s != TN_COUNT_MODP && total > cap) return TN_EINVAL;
  return TN_OK;
}

}  // namespace

// Weighted contraction of slots (primes[q], xs[q]) (mod p) or of one
// max-plus / counting network; the raw result block is copied to raw_out.
// keep: contract with the plan that keeps every intermediate; *Xout is the
// executor plan used (its arena holds the leaves at leaf_base).
int contract_weighted_raw(tn_plan_s* p, tn_semiring_t s, int32_t problem, const int32_t* ew, const int32_t* vw,
                          const uint32_t* primes, const uint32_t* xs, int32_t nslots, void* d_ws, size_t ws_bytes,
                          cudaStream_t st, unsigned char* raw_out, bool keep, ExecPlan** Xout, uint64_t slice) {
  ModTable mods;
  int rc = s == TN_COUNT_MODP ? make_mod_table_slots(primes, xs, nslots, &mods)
                              : make_mod_table_checked(s, nullptr, 0, &mods);
  if (rc) return rc;
  const int32_t np = s == TN_COUNT_MODP ? nslots : 1;
  const WeightedLayout L = weighted_layout(p, s, np, keep, &rc);
  if (rc) return rc;
  ExecPlan* X = weighted_plan(p, s, np, keep, &rc);
  if (!X) return rc;
  if (Xout) *Xout = X;
  if (ws_bytes < L.total) return TN_ENOMEM;
  char* w = static_cast<char*>(d_ws);
  // the weights, edges, leaf offsets and this slice's label values (a few KB)
  // are copied every call; the copies finish before this call returns
  std::vector<int8_t> fixed(static_cast<size_t>(p->n), -1);
  for (size_t j = 0; j < p->sliced.size(); ++j) fixed[p->sliced[j]] = static_cast<int8_t>((slice >> j) & 1);
  if (ew && p->m) rc = cuda_rc(cudaMemcpyAsync(w + L.ew_off, ew, 4 * size_t(p->m), cudaMemcpyHostToDevice, st));
  if (!rc && vw && p->n) rc = cuda_rc(cudaMemcpyAsync(w + L.vw_off, vw, 4 * size_t(p->n), cudaMemcpyHostToDevice, st));
  if (!rc && p->m)
    rc = cuda_rc(cudaMemcpyAsync(w + L.edges_off, p->edges.data(), 8 * size_t(p->m), cudaMemcpyHostToDevice, st));
  if (!rc)
    rc = cuda_rc(cudaMemcpyAsync(w + L.loff_off, p->leaf_off.data(), 8 * size_t(p->T), cudaMemcpyHostToDevice, st));
  if (!rc) rc = cuda_rc(cudaMemcpyAsync(w + L.fixed_off, fixed.data(), size_t(p->n), cudaMemcpyHostToDevice, st));
  if (rc) return rc;
  // arena regions as the executor lays them out (exec_launch_core)
  const size_t e = static_cast<size_t>(X->arena_entries);
  const size_t b4 = align256(4 * e);
  char* r0 = w + X->arena_base;
  dev::LeafArgs la;
  std::memset(&la, 0, sizeof(la));
  la.m = p->m;
  la.n = p->n;
  la.T = p->T;
  la.problem = problem;
  la.semiring = s;
  la.nslots = np;
  la.stride = static_cast<int64_t>(b4 / 4);
  la.edges = reinterpret_cast<const int32_t*>(w + L.edges_off);
  la.loff = reinterpret_cast<const int64_t*>(w + L.loff_off);
  la.fixed = reinterpret_cast<const int8_t*>(w + L.fixed_off);
  la.ew = ew ? reinterpret_cast<const int32_t*>(w + L.ew_off) : nullptr;
  la.vw = vw ? reinterpret_cast<const int32_t*>(w + L.vw_off) : nullptr;
  la.l0 = r0 + 4 * X->leaf_base;
  la.l1 = s == TN_COUNTING_TROPICAL ? r0 + b4 + 8 * X->leaf_base : nullptr;
  for (int q = 0; q < np && s == TN_COUNT_MODP; ++q) {
    la.p[q] = primes[q];
    la.x[q] = xs[q] % primes[q];
  }
  const int64_t total = int64_t(p->T) * np;
  const int blocks = static_cast<int>(std::min<int64_t>((total + 255) / 256, 1024));
  if (total > 0) {
    dev::k_leaves<<<blocks, 256, 0, st>>>(la);
    rc = cuda_rc(cudaGetLastError());
    if (rc) return rc;
  }
  void* d_raw = w + 64;
  rc = exec_enqueue(p, s, &mods, np, d_ws, L.exec_bytes, st, d_raw, nullptr, keep, true);
  if (rc) return rc;
  rc = cuda_rc(cudaMemcpyAsync(raw_out, d_raw, TN_RAW_BYTES, cudaMemcpyDeviceToHost, st));
  if (!rc) rc = cuda_rc(cudaStreamSynchronize(st));
  return rc;
}

// Leaves of `count` copies of plan p in one merged executor plan (slices of
// a sliced network): copy k's leaves at arena entry net_base0 + k *
// net_stride + leaf_base, label values fixed[k * n ..].  The device buffers
// (weights, edges, leaf offsets, fixed values) are already in place.
int enqueue_leaves_batch(tn_plan_s* p, tn_semiring_t s, int32_t problem, const int32_t* d_ew, const int32_t* d_vw,
                         const int32_t* d_edges, const int64_t* d_loff, const int8_t* d_fixed, int32_t count,
                         char* r0, char* r1, int64_t prime_stride, int64_t first_leaf, int64_t net_stride,
                         const uint32_t* primes, const uint32_t* xs, int32_t np, cudaStream_t st) {
  dev::LeafArgs la;
  std::memset(&la, 0, sizeof(la));
  la.m = p->m;
  la.n = p->n;
  la.T = p->T;
  la.problem = problem;
  la.semiring = s;
  la.nslots = np;
  la.stride = prime_stride;
  la.edges = d_edges;
  la.loff = d_loff;
  la.fixed = d_fixed;
  la.ew = d_ew;
  la.vw = d_vw;
  la.l0 = r0 + 4 * first_leaf;
  la.l1 = r1 ? r1 + 8 * first_leaf : nullptr;
  la.net_stride = net_stride;
  for (int q = 0; q < np && s == TN_COUNT_MODP; ++q) {
    la.p[q] = primes[q];
    la.x[q] = xs[q] % primes[q];
  }
  const int64_t total = int64_t(p->T) * np;
  if (total <= 0 || count < 1 || count > 65535) return total <= 0 ? TN_OK : TN_EINVAL;
  const dim3 grid(static_cast<unsigned>(std::min<int64_t>((total + 255) / 256, 1024)), static_cast<unsigned>(count));
  dev::k_leaves<<<grid, 256, 0, st>>>(la);
  return cuda_rc(cudaGetLastError());
}

int weighted_checks(tn_plan_s* p, tn_semiring_t s, int32_t problem, const int32_t* ew, const int32_t* vw) {
  return check_weights(p, s, problem, ew, vw);
}

size_t weighted_workspace(tn_plan_s* p, tn_semiring_t s, int32_t nslots, bool keep) {
  int rc = TN_OK;
  const WeightedLayout L = weighted_layout(p, s, s == TN_COUNT_MODP ? nslots : 1, keep, &rc);
  return rc ? ~size_t(0) : L.total;
}

}  // namespace tn

using namespace tn;

extern "C" {

int tn_weighted_workspace_bytes(tn_plan_t plan, tn_semiring_t semiring, int32_t nslots, uint64_t* out) {
  if (!plan || !out || semiring < TN_TROPICAL_F32 || semiring > TN_COUNT_MODP) return TN_EINVAL;
  if (semiring == TN_COUNT_MODP && (nslots < 1 || nslots > TN_MAX_PRIMES)) return TN_EINVAL;
  try {
    *out = weighted_workspace(plan, semiring, nslots, false);
  } catch (const std::bad_alloc&) {
    return TN_ENOMEM;
  }
  return *out == ~size_t(0) ? TN_ENOMEM : TN_OK;
}

int tn_contract_weighted(tn_plan_t plan, tn_semiring_t semiring, int32_t problem, const int32_t* edge_w,
                         const int32_t* vertex_w, const uint32_t* primes, const uint32_t* xs, int32_t nslots,
                         void* d_workspace, size_t ws_bytes, void* cuda_stream, tn_result_t* out) {
  if (!plan || !out || !d_workspace || semiring < TN_TROPICAL_F32 || semiring > TN_COUNT_MODP) return TN_EINVAL;
  if (reinterpret_cast<uintptr_t>(d_workspace) % 256 != 0) return TN_EINVAL;
  if (semiring == TN_COUNT_MODP && (!primes || !xs || nslots < 1 || nslots > TN_MAX_PRIMES)) return TN_EINVAL;
  int rc = check_weights(plan, semiring, problem, edge_w, vertex_w);
  if (rc) return rc;
  try {
    unsigned char raw[TN_RAW_BYTES];
    rc = contract_weighted_raw(plan, semiring, problem, edge_w, vertex_w, primes, xs, nslots, d_workspace, ws_bytes,
                               static_cast<cudaStream_t>(cuda_stream), raw, false, nullptr, 0);
    if (rc) return rc;
    if (semiring != TN_COUNT_MODP) {
      ModTable mods;
      make_mod_table_checked(semiring, nullptr, 0, &mods);
      return decode_raw_any(semiring, &mods, 0, raw, out);
    }
    // slots may repeat a prime: residues only, no CRT
    std::memset(out, 0, sizeof(*out));
    uint32_t flags;
    std::memcpy(&flags, raw + 96, 4);
    out->status = flags ? TN_ETIMEOUT : TN_OK;
    out->nprimes = nslots;
    for (int q = 0; q < nslots; ++q) {
      out->primes[q] = primes[q];
      std::memcpy(&out->residues[q], raw + 16 + 4 * q, 4);
    }
    return flags ? TN_ETIMEOUT : TN_OK;
  } catch (const std::bad_alloc&) {
    return TN_ENOMEM;
  }
}

}  // extern "C"
