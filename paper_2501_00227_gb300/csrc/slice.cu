// slice.cu -- slicing (Sec. 4.2.2): s vertex labels are fixed, the network is
// contracted once per assignment of them (2^s slices, each with the same
// smaller plan), and the slice results are combined with the element type's
// addition.  Slicing lowers the space complexity by up to 2^s (each sliced
// label leaves every tensor that held it) at the price of up to 2^s times the
// work, and the slices are independent units for several GPUs.
//
//   tn_slice_labels     picks labels for a given order: each pick is the label
//                       whose removal gives the smallest largest intermediate,
//                       ties by the smallest total work of all slices
//   tn_plan_sliced      a plan whose leaves drop the sliced labels
//   tn_contract_sliced  contracts slices [begin, end) on the GPU (stored leaves
//                       written per slice) and combines them
//   tn_result_combine   the element type's addition of two results (also for
//                       combining the slice ranges of several ranks)
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <vector>

#include "exec.h"
#include "kernels.h"
#include "tn_internal.h"

namespace tn {
int contract_weighted_raw(tn_plan_s* p, tn_semiring_t s, int32_t problem, const int32_t* ew, const int32_t* vw,
                          const uint32_t* primes, const uint32_t* xs, int32_t nslots, void* d_ws, size_t ws_bytes,
                          cudaStream_t st, unsigned char* raw_out, bool keep, ExecPlan** Xout, uint64_t slice);
int weighted_checks(tn_plan_s* p, tn_semiring_t s, int32_t problem, const int32_t* ew, const int32_t* vw);
int make_mod_table_checked(tn_semiring_t s, const uint32_t* primes, int32_t nprimes, void* mods);
int decode_raw_any(tn_semiring_t s, const void* mods, int32_t nprimes, const unsigned char* raw, tn_result_t* out);
int make_mod_table_slots(const uint32_t* primes, const uint32_t* xs, int32_t nslots, void* mods);
int enqueue_leaves_batch(tn_plan_s* p, tn_semiring_t s, int32_t problem, const int32_t* d_ew, const int32_t* d_vw,
                         const int32_t* d_edges, const int64_t* d_loff, const int8_t* d_fixed, int32_t count,
                         char* r0, char* r1, int64_t prime_stride, int64_t first_leaf, int64_t net_stride,
                         const uint32_t* primes, const uint32_t* xs, int32_t np, cudaStream_t st);
}  // namespace tn

using namespace tn;

namespace {

// a (+) b in the element type; counts saturate at 2^64 - 1
int combine(tn_semiring_t s, const tn_result_t& a, const tn_result_t& b, tn_result_t* out) {
  tn_result_t r = a;
  r.status = a.status ? a.status : b.status;
  if (s == TN_TROPICAL_F32 || s == TN_TROPICAL_I32) {
    if (b.max_i32 > a.max_i32) {
      r.max_i32 = b.max_i32;
      r.max_f32 = b.max_f32;
    }
  } else if (s == TN_COUNTING_TROPICAL) {
    if (b.max_i32 > a.max_i32) {
      r.max_i32 = b.max_i32;
      r.max_f32 = b.max_f32;
      r.count = b.count;
    } else if (b.max_i32 == a.max_i32 && a.max_i32 != INT32_MIN) {
      r.count = a.count + b.count < a.count ? ~0ull : a.count + b.count;
    }
    if (r.count == ~0ull && r.status == TN_OK) r.status = TN_EOVERFLOW;
  } else {
    if (a.nprimes != b.nprimes) return TN_EINVAL;
    for (int q = 0; q < a.nprimes; ++q) {
      if (a.primes[q] != b.primes[q] || a.primes[q] < 2) return TN_EINVAL;
      r.residues[q] = static_cast<uint32_t>((uint64_t(a.residues[q]) + b.residues[q]) % a.primes[q]);
    }
    r.crt_nlimbs = 0;
  }
  *out = r;
  return TN_OK;
}

// the additive zero of the element type, as a result
void zero_result(tn_semiring_t s, const uint32_t* primes, int32_t nslots, tn_result_t* r) {
  std::memset(r, 0, sizeof(*r));
  r->max_i32 = INT32_MIN;
  r->max_f32 = -INFINITY;
  if (s == TN_COUNT_MODP) {
    r->nprimes = nslots;
    for (int q = 0; q < nslots; ++q) r->primes[q] = primes[q];
  }
}

size_t align256(size_t b) { return (b + 255) / 256 * 256; }
int cuda_rc(cudaError_t e) { return e == cudaSuccess ? TN_OK : TN_ECUDA; }

// Merged executor plans of `count` slices of one plan (stored leaves), kept
// with the plan and uploaded once per device.
struct SliceBatch {
  tn_semiring_t s;
  int32_t np, count;
  ExecPlan X;
  int device = -1;
};
struct SliceCache {
  std::vector<std::unique_ptr<SliceBatch>> v;
};
// Plans may be shared across threads: the slice-batch caches (creation,
// lookup, the one-time table upload) are guarded by one lock.
std::mutex g_slice_mu;

constexpr int32_t kMaxSliceBatch = 256;

// workspace of one batched launch: the merged plan's, then the weights,
// edges, leaf offsets, count x n label values and count raw results
struct SliceLayout {
  size_t ew, vw, edges, loff, fixed, raw, total;
};
SliceLayout slice_layout(const tn_plan_s* p, const ExecPlan& X, int32_t count) {
  SliceLayout L;
  L.ew = align256(X.total_bytes);
  L.vw = L.ew + align256(4 * size_t(std::max(p->m, 1)));
  L.edges = L.vw + align256(4 * size_t(std::max(p->n, 1)));
  L.loff = L.edges + align256(8 * size_t(std::max(p->m, 1)));
  L.fixed = L.loff + align256(8 * size_t(p->T));
  L.raw = L.fixed + align256(size_t(count) * size_t(std::max(p->n, 1)));
  L.total = L.raw + size_t(count) * TN_RAW_BYTES;
  return L;
}

SliceBatch* slice_batch(tn_plan_s* p, tn_semiring_t s, int32_t np, int32_t count, int* rc) {
  std::lock_guard<std::mutex> lk(g_slice_mu);
  if (!p->slice_cache) p->slice_cache = new SliceCache();
  auto* C = static_cast<SliceCache*>(p->slice_cache);
  for (auto& b : C->v)
    if (b->s == s && b->np == np && b->count == count) return b.get();
  std::unique_ptr<SliceBatch> B(new SliceBatch());
  B->s = s;
  B->np = np;
  B->count = count;
  std::vector<tn_plan_s*> plans(static_cast<size_t>(count), p);
  *rc = build_batch_plan(plans.data(), count, s, np, 1, &B->X, true);
  if (*rc) return nullptr;
  C->v.push_back(std::move(B));
  return C->v.back().get();
}

int upload(SliceBatch* B) {
  std::lock_guard<std::mutex> lk(g_slice_mu);
  int dev;
  if (cudaGetDevice(&dev) != cudaSuccess) return TN_ECUDA;
  if (B->X.d_tables && B->device == dev) return TN_OK;
  if (B->X.d_tables) cudaFree(B->X.d_tables);
  B->X.d_tables = nullptr;
  if (cudaMalloc(&B->X.d_tables, B->X.table_bytes) != cudaSuccess) return TN_ENOMEM;
  if (cudaMemcpy(B->X.d_tables, B->X.table_image.data(), B->X.table_bytes, cudaMemcpyHostToDevice) != cudaSuccess)
    return TN_ECUDA;
  B->device = dev;
  return TN_OK;
}

// Slices [b, b + count) in one executor launch; their results are added
// into *acc.
int contract_slice_batch(tn_plan_s* p, SliceBatch* B, tn_semiring_t s, int32_t problem, const int32_t* ew,
                         const int32_t* vw, const uint32_t* primes, const uint32_t* xs, int32_t nslots, uint64_t b,
                         void* d_ws, cudaStream_t st, tn_result_t* acc) {
  const int32_t count = B->count;
  const SliceLayout L = slice_layout(p, B->X, count);
  alignas(16) unsigned char mods[512];
  int rc = s == TN_COUNT_MODP ? make_mod_table_slots(primes, xs, nslots, mods)
                              : make_mod_table_checked(s, nullptr, 0, mods);
  if (rc) return rc;
  rc = upload(B);
  if (rc) return rc;
  char* w = static_cast<char*>(d_ws);
  std::vector<int8_t> fixed(size_t(count) * size_t(p->n), -1);
  for (int32_t k = 0; k < count; ++k)
    for (size_t j = 0; j < p->sliced.size(); ++j)
      fixed[size_t(k) * p->n + p->sliced[j]] = static_cast<int8_t>(((b + k) >> j) & 1);
  if (ew && p->m) rc = cuda_rc(cudaMemcpyAsync(w + L.ew, ew, 4 * size_t(p->m), cudaMemcpyHostToDevice, st));
  if (!rc && vw && p->n) rc = cuda_rc(cudaMemcpyAsync(w + L.vw, vw, 4 * size_t(p->n), cudaMemcpyHostToDevice, st));
  if (!rc && p->m)
    rc = cuda_rc(cudaMemcpyAsync(w + L.edges, p->edges.data(), 8 * size_t(p->m), cudaMemcpyHostToDevice, st));
  if (!rc)
    rc = cuda_rc(cudaMemcpyAsync(w + L.loff, p->leaf_off.data(), 8 * size_t(p->T), cudaMemcpyHostToDevice, st));
  if (!rc && p->n) rc = cuda_rc(cudaMemcpyAsync(w + L.fixed, fixed.data(), fixed.size(), cudaMemcpyHostToDevice, st));
  if (rc) return rc;
  // the merged plan's arena regions (as exec_launch_core lays them out)
  const ExecPlan& X = B->X;
  const size_t b4 = align256(4 * static_cast<size_t>(X.arena_entries));
  char* r0 = w + X.arena_base;
  char* r1 = s == TN_COUNTING_TROPICAL ? r0 + b4 : nullptr;
  const int64_t net_stride = count > 1 ? X.net_arena_base[1] - X.net_arena_base[0] : 0;
  rc = enqueue_leaves_batch(p, s, problem, ew ? reinterpret_cast<const int32_t*>(w + L.ew) : nullptr,
                            vw ? reinterpret_cast<const int32_t*>(w + L.vw) : nullptr,
                            reinterpret_cast<const int32_t*>(w + L.edges), reinterpret_cast<const int64_t*>(w + L.loff),
                            reinterpret_cast<const int8_t*>(w + L.fixed), count, r0, r1,
                            static_cast<int64_t>(b4 / 4), X.net_arena_base[0] + X.leaf_base, net_stride, primes, xs,
                            s == TN_COUNT_MODP ? nslots : 1, st);
  if (rc) return rc;
  rc = exec_launch_core(&B->X, s, mods, d_ws, st, w + L.raw, nullptr, B->X.d_tables);
  if (rc) return rc;
  std::vector<unsigned char> raw(size_t(count) * TN_RAW_BYTES);
  rc = cuda_rc(cudaMemcpyAsync(raw.data(), w + L.raw, raw.size(), cudaMemcpyDeviceToHost, st));
  if (!rc) rc = cuda_rc(cudaStreamSynchronize(st));
  if (rc) return rc;
  for (int32_t k = 0; k < count; ++k) {
    const unsigned char* rk = raw.data() + size_t(k) * TN_RAW_BYTES;
    tn_result_t r;
    if (s != TN_COUNT_MODP) {
      rc = decode_raw_any(s, mods, 0, rk, &r);
      if (rc) return rc;
    } else {
      zero_result(s, primes, nslots, &r);
      uint32_t flags;
      std::memcpy(&flags, rk + 96, 4);
      r.status = flags ? TN_ETIMEOUT : TN_OK;
      for (int q = 0; q < nslots; ++q) std::memcpy(&r.residues[q], rk + 16 + 4 * q, 4);
    }
    if (r.status == TN_ETIMEOUT) return TN_ETIMEOUT;
    rc = combine(s, *acc, r, acc);
    if (rc) return rc;
  }
  return TN_OK;
}

}  // namespace

namespace tn {
void slice_cache_free(tn_plan_s* p) {
  std::lock_guard<std::mutex> lk(g_slice_mu);
  auto* C = static_cast<SliceCache*>(p->slice_cache);
  if (!C) return;
  for (auto& b : C->v)
    if (b->X.d_tables) cudaFree(b->X.d_tables);
  delete C;
  p->slice_cache = nullptr;
}
}  // namespace tn

extern "C" {

int tn_sliced_workspace_bytes(tn_plan_t plan, tn_semiring_t semiring, int32_t nslots, int32_t batch,
                              uint64_t* out) {
  if (!plan || !out || semiring < TN_TROPICAL_F32 || semiring > TN_COUNT_MODP || batch < 1 ||
      batch > kMaxSliceBatch)
    return TN_EINVAL;
  if (semiring == TN_COUNT_MODP && (nslots < 1 || nslots > TN_MAX_PRIMES)) return TN_EINVAL;
  const int32_t np = semiring == TN_COUNT_MODP ? nslots : 1;
  try {
    uint64_t single;
    int rc = tn_weighted_workspace_bytes(plan, semiring, np, &single);
    if (rc) return rc;
    if (batch == 1) {
      *out = single;
      return TN_OK;
    }
    SliceBatch* B = slice_batch(plan, semiring, np, batch, &rc);
    if (!B) return rc;
    *out = std::max<uint64_t>(single, slice_layout(plan, B->X, batch).total);
    return TN_OK;
  } catch (const std::bad_alloc&) {
    return TN_ENOMEM;
  }
}

int tn_result_combine(tn_semiring_t semiring, const tn_result_t* a, const tn_result_t* b, tn_result_t* out) {
  if (!a || !b || !out || semiring < TN_TROPICAL_F32 || semiring > TN_COUNT_MODP) return TN_EINVAL;
  return combine(semiring, *a, *b, out);
}

int tn_plan_sliced(int32_t n_vertices, const int32_t* edges, int32_t m, const int32_t* order, int32_t order_len,
                   const int32_t* sliced, int32_t nsliced, tn_plan_t* out) {
  if (!out) return TN_EINVAL;
  *out = nullptr;
  tn_plan_s* p = new (std::nothrow) tn_plan_s();
  if (!p) return TN_ENOMEM;
  int rc;
  try {
    rc = build_plan(n_vertices, edges, m, order, order_len, p, sliced, nsliced);
  } catch (const std::bad_alloc&) {
    rc = TN_ENOMEM;
  }
  if (rc != TN_OK) {
    delete p;
    return rc;
  }
  *out = p;
  return TN_OK;
}

int tn_slice_labels(int32_t n, const int32_t* edges, int32_t m, const int32_t* order, int32_t order_len,
                    int32_t nslices, int32_t* sliced_out, double* log2_out) {
  if (!sliced_out || nslices < 0 || nslices > 62 || nslices > n) return TN_EINVAL;
  try {
    tn_plan_s p;
    int rc = build_plan(n, edges, m, order, order_len, &p);
    if (rc) return rc;
    // label sets of every step's operands and output
    const size_t ns = p.steps.size();
    std::vector<std::vector<int32_t>> in(ns), outl(ns);
    for (size_t s = 0; s < ns; ++s) {
      const Step& S = p.steps[s];
      in[s] = p.tensors[S.a_id].labels;
      for (int32_t l : p.tensors[S.b_id].labels)
        if (std::find(in[s].begin(), in[s].end(), l) == in[s].end()) in[s].push_back(l);
      outl[s] = p.tensors[S.c_id].labels;
    }
    std::vector<char> cut(static_cast<size_t>(n), 0);
    auto measure = [&](int32_t extra, int32_t* sc, double* tc) {
      *sc = 0;
      *tc = 0;
      for (size_t s = 0; s < ns; ++s) {
        int ri = 0, ro = 0;
        for (int32_t l : in[s]) ri += !(cut[l] || l == extra);
        for (int32_t l : outl[s]) ro += !(cut[l] || l == extra);
        *sc = std::max(*sc, ro);
        *tc += std::ldexp(1.0, ri);
      }
    };
    for (int32_t j = 0; j < nslices; ++j) {
      int32_t best = -1, bsc = 0;
      double btc = 0;
      for (int32_t v = 0; v < n; ++v) {
        if (cut[v]) continue;
        int32_t sc;
        double tc;
        measure(v, &sc, &tc);
        if (best < 0 || sc < bsc || (sc == bsc && tc < btc)) {
          best = v;
          bsc = sc;
          btc = tc;
        }
      }
      if (best < 0) return TN_EINVAL;
      cut[best] = 1;
      sliced_out[j] = best;
    }
    if (log2_out) {
      int32_t sc;
      double tc;
      measure(-1, &sc, &tc);
      log2_out[0] = std::log2(tc) + nslices;  // all slices
      log2_out[1] = sc;
    }
    return TN_OK;
  } catch (const std::bad_alloc&) {
    return TN_ENOMEM;
  }
}

int tn_contract_sliced(tn_plan_t plan, tn_semiring_t semiring, int32_t problem, const int32_t* edge_w,
                       const int32_t* vertex_w, const uint32_t* primes, const uint32_t* xs, int32_t nslots,
                       uint64_t slice_begin, uint64_t slice_end, void* d_workspace, size_t ws_bytes,
                       void* cuda_stream, tn_result_t* out) {
  if (!plan || !out || !d_workspace || semiring < TN_TROPICAL_F32 || semiring > TN_COUNT_MODP) return TN_EINVAL;
  if (reinterpret_cast<uintptr_t>(d_workspace) % 256 != 0) return TN_EINVAL;
  if (semiring == TN_COUNT_MODP && (!primes || !xs || nslots < 1 || nslots > TN_MAX_PRIMES)) return TN_EINVAL;
  const uint64_t nsl = uint64_t(1) << plan->sliced.size();
  if (slice_begin > slice_end || slice_end > nsl) return TN_EINVAL;
  int rc = weighted_checks(plan, semiring, problem, edge_w, vertex_w);
  if (rc) return rc;
  try {
    tn_result_t acc;
    zero_result(semiring, primes, nslots, &acc);
    alignas(16) unsigned char mods[512];
    rc = make_mod_table_checked(semiring, nullptr, 0, mods);
    if (rc && semiring != TN_COUNT_MODP) return rc;
    const int32_t np = semiring == TN_COUNT_MODP ? nslots : 1;
    for (uint64_t sl = slice_begin; sl < slice_end;) {
      // as many slices per launch as the workspace holds (up to kMaxSliceBatch)
      int32_t count = static_cast<int32_t>(std::min<uint64_t>(slice_end - sl, kMaxSliceBatch));
      SliceBatch* B = nullptr;
      while (count > 1) {
        int brc = TN_OK;
        B = slice_batch(plan, semiring, np, count, &brc);
        if (!B) return brc;
        if (slice_layout(plan, B->X, count).total <= ws_bytes) break;
        B = nullptr;
        count /= 2;
      }
      if (B) {
        rc = contract_slice_batch(plan, B, semiring, problem, edge_w, vertex_w, primes, xs, nslots, sl, d_workspace,
                                  static_cast<cudaStream_t>(cuda_stream), &acc);
        if (rc) return rc;
        sl += static_cast<uint64_t>(count);
        continue;
      }
      unsigned char raw[TN_RAW_BYTES];
      rc = contract_weighted_raw(plan, semiring, problem, edge_w, vertex_w, primes, xs, nslots, d_workspace, ws_bytes,
                                 static_cast<cudaStream_t>(cuda_stream), raw, false, nullptr, sl);
      if (rc) return rc;
      tn_result_t r;
      if (semiring != TN_COUNT_MODP) {
        rc = decode_raw_any(semiring, mods, 0, raw, &r);
        if (rc) return rc;
      } else {
        zero_result(semiring, primes, nslots, &r);
        uint32_t flags;
        std::memcpy(&flags, raw + 96, 4);
        r.status = flags ? TN_ETIMEOUT : TN_OK;
        for (int q = 0; q < nslots; ++q) std::memcpy(&r.residues[q], raw + 16 + 4 * q, 4);
      }
      if (r.status == TN_ETIMEOUT) return TN_ETIMEOUT;
      rc = combine(semiring, acc, r, &acc);
      if (rc) return rc;
      ++sl;
    }
    *out = acc;
    return TN_OK;
  } catch (const std::bad_alloc&) {
    return TN_ENOMEM;
  }
}

}  // extern "C"
