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

}  // namespace

extern "C" {

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
    for (uint64_t sl = slice_begin; sl < slice_end; ++sl) {
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
    }
    *out = acc;
    return TN_OK;
  } catch (const std::bad_alloc&) {
    return TN_ENOMEM;
  }
}

}  // extern "C"
