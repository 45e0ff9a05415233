// kbest.cuh -- the k-best element types of Table 1 (Sec. 5.3 of
// arXiv:2501.00227) on the device, for the general ("naive") step body:
//
//   SrKMax<K>   SizeMax(k), the ExtendedTropical{k} element: the K largest
//               total weights of the configurations an entry sums over,
//               counted with multiplicity, in decreasing order.
//                 a (x) b = the K largest of all sums a_i + b_j
//                 a (+) b = the K largest of the union
//               "-inf" padding is kNegInf; stored values are kNegInf or real
//               values (> kNegInf / 2), so a sum of two stored values stays
//               >= -2^31.
//   SrKPoly<K>  CountingMax(k), the TruncatedPoly{k} element: the K
//               highest-order terms of the polynomial sum_S x^{w(S)}: the
//               highest order d (kNegInf: the zero polynomial) and the
//               coefficients c[t] of x^{d - t}, t < K (uint64, saturating).
//                 a (x) b = the product, truncated to its K highest orders
//                 a (+) b = the sum, truncated to the K highest orders of the
//                           larger leading order
//
// Tensor layout in the arena (prime_stride S entries between blocks):
//   SrKMax<K>   K int32 blocks: value t of entry e at p0[t S + e]
//   SrKPoly<K>  int32 d[e] at p0[e]; uint64 c[t] of entry e at p1[t S + e]
#pragma once

#include <cstdint>

#include "semiring.cuh"

namespace tn {
namespace dev {

template <int K>
struct KMaxVal {
  int32_t v[K];
};

template <int K>
struct SrKMax {
  using Val = KMaxVal<K>;
  using Acc = KMaxVal<K>;
  static constexpr int kK = K;
  static __device__ __forceinline__ Acc zero(const ModParams&) {
    Acc r;
#pragma unroll
    for (int t = 0; t < K; ++t) r.v[t] = kNegInf;
    return r;
  }
  static __device__ __forceinline__ Val single(int32_t x) {
    Val r;
#pragma unroll
    for (int t = 0; t < K; ++t) r.v[t] = kNegInf;
    r.v[0] = x;
    return r;
  }
  // edge leaf B = [[one, one], [one, zero]]; vertex leaf W = [one, x^1]
  static __device__ __forceinline__ Val leaf(int32_t kind, uint32_t e) {
    if (kind == kOpEdge) return single(e == 3 ? kNegInf : 0);
    if (kind == kOpVertex) return single(e == 1 ? 1 : 0);
    return single(0);
  }
  template <bool CG = false>
  static __device__ __forceinline__ Val load(const Operand& o, uint32_t e) {
    if (o.kind != kOpArena) return leaf(o.kind, e);
    Val r;
    const int32_t* p = static_cast<const int32_t*>(o.p0) + e;
#pragma unroll
    for (int t = 0; t < K; ++t) r.v[t] = ldg_t<CG>(p + t * o.prime_stride);
    return r;
  }
  // inserts x into the decreasing list, dropping the smallest value
  static __device__ __forceinline__ void insert(Acc& acc, int32_t x) {
    if (x <= acc.v[K - 1]) return;
#pragma unroll
    for (int t = K - 1; t > 0; --t) {
      const int32_t up = acc.v[t - 1];
      if (up >= x) {
        acc.v[t] = x;
        return;
      }
      acc.v[t] = up;
    }
    acc.v[0] = x;
  }
  static __device__ __forceinline__ void mac(Acc& acc, const Val& a, const Val& b, const ModParams&) {
#pragma unroll
    for (int i = 0; i < K; ++i)
#pragma unroll
      for (int j = 0; j < K; ++j)
        if (a.v[i] > kNegInf / 2 && b.v[j] > kNegInf / 2) insert(acc, a.v[i] + b.v[j]);
  }
  static __device__ __forceinline__ void merge(Acc& acc, const Acc& o, const ModParams&) {
#pragma unroll
    for (int j = 0; j < K; ++j) insert(acc, o.v[j]);
  }
  static __device__ __forceinline__ void store(const Output& o, uint32_t e, const Acc& acc, const ModParams&) {
    int32_t* p = static_cast<int32_t*>(o.p0) + e;
#pragma unroll
    for (int t = 0; t < K; ++t) p[t * o.prime_stride] = acc.v[t];
  }
};

template <int K>
struct KPolyVal {
  int32_t d;
  uint64_t c[K];
};

template <int K>
struct SrKPoly {
  using Val = KPolyVal<K>;
  using Acc = KPolyVal<K>;
  static constexpr int kK = K;
  static __device__ __forceinline__ Acc zero(const ModParams&) {
    Acc r;
    r.d = kNegInf;
#pragma unroll
    for (int t = 0; t < K; ++t) r.c[t] = 0ull;
    return r;
  }
  // x^d with coefficient 1 (kNegInf: the zero polynomial)
  static __device__ __forceinline__ Val monomial(int32_t d) {
    Val r;
    r.d = d;
#pragma unroll
    for (int t = 0; t < K; ++t) r.c[t] = 0ull;
    r.c[0] = d == kNegInf ? 0ull : 1ull;
    return r;
  }
  static __device__ __forceinline__ Val leaf(int32_t kind, uint32_t e) {
    if (kind == kOpEdge) return monomial(e == 3 ? kNegInf : 0);
    if (kind == kOpVertex) return monomial(e == 1 ? 1 : 0);
    return monomial(0);
  }
  template <bool CG = false>
  static __device__ __forceinline__ Val load(const Operand& o, uint32_t e) {
    if (o.kind != kOpArena) return leaf(o.kind, e);
    Val r;
    r.d = ldg_t<CG>(static_cast<const int32_t*>(o.p0) + e);
    const uint64_t* p = static_cast<const uint64_t*>(o.p1) + e;
#pragma unroll
    for (int t = 0; t < K; ++t) r.c[t] = ldg_t<CG>(p + t * o.prime_stride);
    return r;
  }
  // acc += x^sh * o  with sh >= 0 orders below acc's leading order
  static __device__ __forceinline__ void add_shifted(Acc& acc, const Val& o, int32_t sh) {
#pragma unroll
    for (int t = K - 1; t >= 0; --t)
      if (t >= sh) acc.c[t] = sat_add_u64(acc.c[t], o.c[t - sh]);
  }
  static __device__ __forceinline__ void merge(Acc& acc, const Acc& o, const ModParams&) {
    if (o.d <= kNegInf / 2) return;
    if (acc.d <= kNegInf / 2) {
      acc = o;
      return;
    }
    if (o.d > acc.d) {
      Acc r = o;
      add_shifted(r, acc, o.d - acc.d);
      acc = r;
    } else {
      add_shifted(acc, o, acc.d - o.d);
    }
  }
  static __device__ __forceinline__ void mac(Acc& acc, const Val& a, const Val& b, const ModParams& mp) {
    if (a.d <= kNegInf / 2 || b.d <= kNegInf / 2) return;
    Acc p;
    p.d = a.d + b.d;
#pragma unroll
    for (int t = 0; t < K; ++t) {
      uint64_t s = 0ull;
#pragma unroll
      for (int i = 0; i <= t; ++i) s = sat_add_u64(s, sat_mul_u64(a.c[i], b.c[t - i]));
      p.c[t] = s;
    }
    merge(acc, p, mp);
  }
  static __device__ __forceinline__ void store(const Output& o, uint32_t e, const Acc& acc, const ModParams&) {
    static_cast<int32_t*>(o.p0)[e] = acc.d;
    uint64_t* p = static_cast<uint64_t*>(o.p1) + e;
#pragma unroll
    for (int t = 0; t < K; ++t) p[t * o.prime_stride] = acc.c[t];
  }
};

template <int K>
__device__ __forceinline__ KMaxVal<K> shfl_xor_val(KMaxVal<K> v, int off) {
  KMaxVal<K> r;
#pragma unroll
  for (int t = 0; t < K; ++t) r.v[t] = __shfl_xor_sync(0xffffffffu, v.v[t], off);
  return r;
}
template <int K>
__device__ __forceinline__ KPolyVal<K> shfl_xor_val(KPolyVal<K> v, int off) {
  KPolyVal<K> r;
  r.d = __shfl_xor_sync(0xffffffffu, v.d, off);
#pragma unroll
  for (int t = 0; t < K; ++t) r.c[t] = __shfl_xor_sync(0xffffffffu, v.c[t], off);
  return r;
}

// Element types that run only through the general step body (no GEMM tiles,
// no groups of tiny steps, no split reductions).
template <class SR>
struct IsKBest {
  static constexpr bool value = false;
};
template <int K>
struct IsKBest<SrKMax<K>> {
  static constexpr bool value = true;
};
template <int K>
struct IsKBest<SrKPoly<K>> {
  static constexpr bool value = true;
};

}  // namespace dev
}  // namespace tn
