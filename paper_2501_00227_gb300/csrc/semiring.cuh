// semiring.cuh -- device element types of libtn (Table 1, Secs. 5.2-5.3 of
// arXiv:2501.00227) and operand access for the step kernels.
//
//   SrF32  tropical (max,+) in float; zero = -inf, one = 0 (Sec. 5.2)
//   SrI32  tropical (max,+) in int32; "-inf" is kNegInf = -2^30 and every
//          accumulation starts there, so sums of two stored values stay
//          >= -2^31 and never wrap
//   SrCnt  counting tropical (CountingMax, Sec. 5.3): (max in int32, count in
//          uint64); (a,c)(x)(b,d) = (a+b, c*d); (+) keeps the larger max and
//          adds counts on a tie; counts saturate at 2^64-1
//   SrMod  ordinary (+,*) modulo a prime p < 2^31 (the count of all
//          independent sets, Z at beta = 0, one residue per prime)
#pragma once

#include <cstdint>

#include "tn_internal.h"

namespace tn {
namespace dev {

constexpr int32_t kNegInf = TN_I32_NEG_INF;

// One operand of a step: an array in device memory or a leaf generated on
// the fly (its entry index is the only input).  Entry indices are 32-bit
// (tensor ranks are at most 30).
struct Operand {
  int32_t kind;          // OperandKind
  uint32_t vx;           // mod p: a vertex leaf is W = [1, vx] (the prime slot's weight x)
  const void* p0;        // float / int32 values, or residues of prime 0
  const void* p1;        // uint64 counts (counting semiring)
  int64_t prime_stride;  // entries between consecutive prime blocks
};

struct Output {
  void* p0;
  void* p1;
  int64_t prime_stride;
};

// Constants of one prime slot (2 <= p < 2^31):
//   r32 = 2^32 mod p   (folds the high word of a 64-bit accumulator)
//   mu  = floor((2^64 - 1) / p)   (Barrett 1986 reciprocal)
//   x   = the vertex weight of the slot, reduced mod p: vertex leaves are
//         W = [1, x] (Eq. 7 with x = e^{beta w}), so the slot's result is the
//         independence polynomial evaluated at x; counting all sets is x = 1
struct ModParams {
  uint32_t p, r32;
  uint64_t mu;
  uint32_t x, pad_;
};

// Products a mod-p tile may add to its 64-bit accumulator between two folds
// (acc <- hi * r32 + lo): 4 when the largest folded accumulator,
// (r32 + 1)(2^32 - 1), plus four products of residues below p stays below
// 2^64 -- true for every p = 2^31 - c with c < 2^29, e.g. the primes next
// to 2^31 -- else 1 (exact for every p < 2^31).
inline int mod_fold_interval(uint32_t p, uint32_t r32) {
  const unsigned __int128 folded = static_cast<unsigned __int128>(r32 + 1ull) * 0xffffffffull;
  const unsigned __int128 terms = static_cast<unsigned __int128>(p - 1ull) * (p - 1ull) * 4u;
  return folded + terms < (static_cast<unsigned __int128>(1) << 64) ? 4 : 1;
}

// The same operand / output seen at the block of prime slot q (mod p keeps
// one residue array per slot; the element accessors below read p0 only).
__device__ __forceinline__ Operand at_prime(Operand o, int q, const ModParams& mp) {
  if ((o.kind == kOpArena || o.kind == kOpShared) && q) o.p0 = static_cast<const uint32_t*>(o.p0) + q * o.prime_stride;
  o.vx = mp.x;
  return o;
}
__device__ __forceinline__ Output at_prime(Output o, int q) {
  if (q) o.p0 = static_cast<uint32_t*>(o.p0) + q * o.prime_stride;
  return o;
}

struct ModTable {
  ModParams q[TN_MAX_PRIMES];
};

// Asynchronous global -> shared copies (cp.async, 4 or 8 bytes).
__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gmem_src) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gmem_src) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Global loads; CG = true reads through L2 only (ld.global.cg), which the
// persistent executor uses for tensors other CTAs wrote during the launch.
template <bool CG, class T>
__device__ __forceinline__ T ldg_t(const T* p) {
  if constexpr (CG) return __ldcg(p);
  else return *p;
}

// ---------------------------------------------------------------- float
struct SrF32 {
  using Val = float;
  using Acc = float;
  static __device__ __forceinline__ Acc zero(const ModParams&) { return -__int_as_float(0x7f800000); }
  static __device__ __forceinline__ Val leaf(int32_t kind, uint32_t e) {
    if (kind == kOpEdge) return e == 3 ? -__int_as_float(0x7f800000) : 0.0f;
    if (kind == kOpVertex) return e == 1 ? 1.0f : 0.0f;
    return 0.0f;
  }
  template <bool CG = false>
  static __device__ __forceinline__ Val load(const Operand& o, uint32_t e) {
    if (o.kind == kOpShared) return static_cast<const float*>(o.p0)[e];
    if (o.kind != kOpArena) return leaf(o.kind, e);
    return ldg_t<CG>(static_cast<const float*>(o.p0) + e);
  }
  static __device__ __forceinline__ void copy_async(Val* dst, const Operand& o, uint32_t e) {
    cp_async4(dst, static_cast<const float*>(o.p0) + e);
  }
  static __device__ __forceinline__ void mac(Acc& acc, Val a, Val b, const ModParams&) {
    acc = fmaxf(acc, a + b);
  }
  static __device__ __forceinline__ void merge(Acc& acc, const Acc& o, const ModParams&) {
    acc = fmaxf(acc, o);
  }
  static __device__ __forceinline__ void store(const Output& o, uint32_t e, const Acc& acc, const ModParams&) {
    static_cast<float*>(o.p0)[e] = acc;
  }
  // four consecutive entries e .. e+3 (e a multiple of 4, 16-byte aligned)
  static __device__ __forceinline__ void store4(const Output& o, uint32_t e, const Acc (&v)[4], const ModParams&) {
    *reinterpret_cast<float4*>(static_cast<float*>(o.p0) + e) = make_float4(v[0], v[1], v[2], v[3]);
  }
  static __device__ __forceinline__ void st4(Acc* p, const Acc (&v)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
  static __device__ __forceinline__ void ldcg4(const Acc* p, Acc (&v)[4]) {
    const float4 w = __ldcg(reinterpret_cast<const float4*>(p));
    v[0] = w.x;
    v[1] = w.y;
    v[2] = w.z;
    v[3] = w.w;
  }
};

// ---------------------------------------------------------------- int32
struct SrI32 {
  using Val = int32_t;
  using Acc = int32_t;
  static __device__ __forceinline__ Acc zero(const ModParams&) { return kNegInf; }
  static __device__ __forceinline__ Val leaf(int32_t kind, uint32_t e) {
    if (kind == kOpEdge) return e == 3 ? kNegInf : 0;
    if (kind == kOpVertex) return e == 1 ? 1 : 0;
    return 0;
  }
  template <bool CG = false>
  static __device__ __forceinline__ Val load(const Operand& o, uint32_t e) {
    if (o.kind == kOpShared) return static_cast<const int32_t*>(o.p0)[e];
    if (o.kind != kOpArena) return leaf(o.kind, e);
    return ldg_t<CG>(static_cast<const int32_t*>(o.p0) + e);
  }
  static __device__ __forceinline__ void copy_async(Val* dst, const Operand& o, uint32_t e) {
    cp_async4(dst, static_cast<const int32_t*>(o.p0) + e);
  }
  static __device__ __forceinline__ void mac(Acc& acc, Val a, Val b, const ModParams&) {
    acc = __viaddmax_s32(a, b, acc);  // max(a + b, acc)
  }
  static __device__ __forceinline__ void merge(Acc& acc, const Acc& o, const ModParams&) {
    acc = max(acc, o);
  }
  static __device__ __forceinline__ void store(const Output& o, uint32_t e, const Acc& acc, const ModParams&) {
    static_cast<int32_t*>(o.p0)[e] = acc;
  }
  static __device__ __forceinline__ void store4(const Output& o, uint32_t e, const Acc (&v)[4], const ModParams&) {
    *reinterpret_cast<int4*>(static_cast<int32_t*>(o.p0) + e) = make_int4(v[0], v[1], v[2], v[3]);
  }
  static __device__ __forceinline__ void st4(Acc* p, const Acc (&v)[4]) {
    *reinterpret_cast<int4*>(p) = make_int4(v[0], v[1], v[2], v[3]);
  }
  static __device__ __forceinline__ void ldcg4(const Acc* p, Acc (&v)[4]) {
    const int4 w = __ldcg(reinterpret_cast<const int4*>(p));
    v[0] = w.x;
    v[1] = w.y;
    v[2] = w.z;
    v[3] = w.w;
  }
};

// ---------------------------------------------------------------- counting
__device__ __forceinline__ uint64_t sat_mul_u64(uint64_t a, uint64_t b) {
  return __umul64hi(a, b) ? ~0ull : a * b;
}
__device__ __forceinline__ uint64_t sat_add_u64(uint64_t a, uint64_t b) {
  uint64_t s = a + b;
  return s < a ? ~0ull : s;
}

struct __align__(16) CntVal {
  int32_t v;
  uint64_t c;
};

struct SrCnt {
  using Val = CntVal;
  using Acc = CntVal;
  static __device__ __forceinline__ Acc zero(const ModParams&) { return CntVal{kNegInf, 0ull}; }
  static __device__ __forceinline__ Val leaf(int32_t kind, uint32_t e) {
    if (kind == kOpEdge) return e == 3 ? CntVal{kNegInf, 0ull} : CntVal{0, 1ull};
    if (kind == kOpVertex) return e == 1 ? CntVal{1, 1ull} : CntVal{0, 1ull};
    return CntVal{0, 1ull};
  }
  template <bool CG = false>
  static __device__ __forceinline__ Val load(const Operand& o, uint32_t e) {
    if (o.kind == kOpShared)
      return CntVal{static_cast<const int32_t*>(o.p0)[e], static_cast<const uint64_t*>(o.p1)[e]};
    if (o.kind != kOpArena) return leaf(o.kind, e);
    return CntVal{ldg_t<CG>(static_cast<const int32_t*>(o.p0) + e),
                  ldg_t<CG>(static_cast<const uint64_t*>(o.p1) + e)};
  }
  static __device__ __forceinline__ void copy_async(Val* dst, const Operand& o, uint32_t e) {
    cp_async4(&dst->v, static_cast<const int32_t*>(o.p0) + e);
    cp_async8(&dst->c, static_cast<const uint64_t*>(o.p1) + e);
  }
  static __device__ __forceinline__ void mac(Acc& acc, const Val& a, const Val& b, const ModParams&) {
    int32_t s = a.v + b.v;
    if (s > acc.v) {
      acc.v = s;
      acc.c = sat_mul_u64(a.c, b.c);
    } else if (s == acc.v) {
      acc.c = sat_add_u64(acc.c, sat_mul_u64(a.c, b.c));
    }
  }
  static __device__ __forceinline__ void merge(Acc& acc, const Acc& o, const ModParams&) {
    if (o.v > acc.v) acc = o;
    else if (o.v == acc.v) acc.c = sat_add_u64(acc.c, o.c);
  }
  static __device__ __forceinline__ void store(const Output& o, uint32_t e, const Acc& acc, const ModParams&) {
    static_cast<int32_t*>(o.p0)[e] = acc.v;
    static_cast<uint64_t*>(o.p1)[e] = acc.c;
  }
  static __device__ __forceinline__ void store4(const Output& o, uint32_t e, const Acc (&v)[4], const ModParams&) {
    *reinterpret_cast<int4*>(static_cast<int32_t*>(o.p0) + e) = make_int4(v[0].v, v[1].v, v[2].v, v[3].v);
    ulonglong2* c = reinterpret_cast<ulonglong2*>(static_cast<uint64_t*>(o.p1) + e);
    c[0] = make_ulonglong2(v[0].c, v[1].c);
    c[1] = make_ulonglong2(v[2].c, v[3].c);
  }
  static __device__ __forceinline__ void st4(Acc* p, const Acc (&v)[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
      *reinterpret_cast<int4*>(p + i) = make_int4(v[i].v, 0, static_cast<int32_t>(static_cast<uint32_t>(v[i].c)),
                                                  static_cast<int32_t>(static_cast<uint32_t>(v[i].c >> 32)));
  }
  static __device__ __forceinline__ void ldcg4(const Acc* p, Acc (&v)[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int4 w = __ldcg(reinterpret_cast<const int4*>(p + i));
      v[i].v = w.x;
      v[i].c = static_cast<uint64_t>(static_cast<uint32_t>(w.z)) | (static_cast<uint64_t>(static_cast<uint32_t>(w.w)) << 32);
    }
  }
};

// ---------------------------------------------------------------- mod p
// Accumulation: acc (64-bit) += a*b with a, b < p < 2^31, so a*b < 2^62.
// After every product the high word is folded back, acc <- hi * r32 + lo
// (2^32 = r32 mod p); this keeps acc < 2^63 + 2^32 and the sum below 2^64.
// The final residue is a Barrett reduction (Barrett 1986) of the 64-bit acc.
__device__ __forceinline__ uint64_t fold32(uint64_t x, uint32_t r32) {
  return static_cast<uint64_t>(static_cast<uint32_t>(x >> 32)) * r32 + static_cast<uint32_t>(x);
}
__device__ __forceinline__ uint32_t barrett64(uint64_t x, const ModParams& mp) {
  // q = floor(x * mu / 2^64) is floor(x / p) or one less.
  uint64_t q = __umul64hi(x, mp.mu);
  uint64_t r = x - q * mp.p;
  return static_cast<uint32_t>(r >= mp.p ? r - mp.p : r);
}

struct SrMod {
  using Val = uint32_t;
  using Acc = uint64_t;
  static __device__ __forceinline__ Acc zero(const ModParams&) { return 0ull; }
  // Leaves with vertex weight x (already reduced mod p): a forbidden edge
  // configuration weighs 0, an allowed one 1; W = [1, x].
  static __device__ __forceinline__ Val leaf(int32_t kind, uint32_t e, uint32_t x) {
    if (kind == kOpEdge) return e == 3 ? 0u : 1u;
    if (kind == kOpVertex) return e == 1 ? x : 1u;
    return 1u;
  }
  // x = 1 (counting all sets); leaf(kOpEdge, 3) is the additive zero
  static __device__ __forceinline__ Val leaf(int32_t kind, uint32_t e) { return leaf(kind, e, 1u); }
  template <bool CG = false>
  static __device__ __forceinline__ Val load(const Operand& o, uint32_t e) {
    if (o.kind == kOpShared) return static_cast<const uint32_t*>(o.p0)[e];
    if (o.kind != kOpArena) return leaf(o.kind, e, o.vx);
    return ldg_t<CG>(static_cast<const uint32_t*>(o.p0) + e);
  }
  static __device__ __forceinline__ void copy_async(Val* dst, const Operand& o, uint32_t e) {
    cp_async4(dst, static_cast<const uint32_t*>(o.p0) + e);
  }
  static __device__ __forceinline__ void mac(Acc& acc, Val a, Val b, const ModParams& mp) {
    acc = fold32(acc + static_cast<uint64_t>(a) * b, mp.r32);
  }
  static __device__ __forceinline__ void merge(Acc& acc, const Acc& o, const ModParams& mp) {
    acc = static_cast<uint64_t>(barrett64(acc, mp)) + barrett64(o, mp);  // < 2p
  }
  static __device__ __forceinline__ void store(const Output& o, uint32_t e, const Acc& acc, const ModParams& mp) {
    static_cast<uint32_t*>(o.p0)[e] = barrett64(acc, mp);
  }
  static __device__ __forceinline__ void store4(const Output& o, uint32_t e, const Acc (&v)[4],
                                                const ModParams& mp) {
    *reinterpret_cast<uint4*>(static_cast<uint32_t*>(o.p0) + e) =
        make_uint4(barrett64(v[0], mp), barrett64(v[1], mp), barrett64(v[2], mp), barrett64(v[3], mp));
  }
  static __device__ __forceinline__ void st4(Acc* p, const Acc (&v)[4]) {
    reinterpret_cast<ulonglong2*>(p)[0] = make_ulonglong2(v[0], v[1]);
    reinterpret_cast<ulonglong2*>(p)[1] = make_ulonglong2(v[2], v[3]);
  }
  static __device__ __forceinline__ void ldcg4(const Acc* p, Acc (&v)[4]) {
    const ulonglong2 w0 = __ldcg(reinterpret_cast<const ulonglong2*>(p));
    const ulonglong2 w1 = __ldcg(reinterpret_cast<const ulonglong2*>(p) + 1);
    v[0] = w0.x;
    v[1] = w0.y;
    v[2] = w1.x;
    v[3] = w1.y;
  }
};

}  // namespace dev
}  // namespace tn
