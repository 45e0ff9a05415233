// step_device.cuh -- device building blocks shared by the per-step kernels
// and the persistent plan executor: gather tables (operand offsets of an
// output or reduction index) and the general ("naive chunk") step body with
// K-parallel reduction.
//
// A step (Sec. 4.1 of arXiv:2501.00227) computes
//   C[b, m, n] = (+)_k A[b, m, k] (x) B[b, k, n],
// C stored contiguously as c = n | m << nn | b << (nn + nm) (or scattered
// through c_pos when the caller fixes the output label order).  Operands are
// read in place: the entry of A holding (b, m, k) has its label bits at the
// positions a_pos of A's own layout (likewise b_pos for B), so no permuted
// copy of an operand is ever made.
#pragma once

#include <cstdint>

#include "semiring.cuh"

namespace tn {
namespace dev {

// Scatter the bits of x into the positions pos[first .. first+count) (used
// for outputs whose label order the caller fixed).
__device__ __forceinline__ uint32_t deposit(uint32_t x, const int8_t* pos, int first, int count) {
  uint32_t r = 0;
  for (int j = 0; j < count; ++j)
    if ((x >> j) & 1u) {
      const int p = pos[first + j];
      if (p >= 0) r |= 1u << p;
    }
  return r;
}

constexpr int kBlock = 256;         // threads per CTA of every libtn kernel
constexpr int kNib = 8;             // 4-bit nibbles of a 32-bit index
constexpr int kNaiveKLoBits = 9;    // k offsets of the low 9 bits come from a table
constexpr int kNaiveKHi = 256;      // high-k blocks per task whose offsets are tabulated
constexpr int kNaiveWideU = 2;      // entries per thread in naive_chunk_wide (2: measured faster than 4)

__device__ __forceinline__ int nibbles(int bits) { return (bits + 3) >> 2; }

// Gather tables of one step.  The output index c (rc bits) and the
// reduction index k (nk bits) are cut into 4-bit nibbles; entry [i][v] is
// the pair (offset in A, offset in B) contributed by the value v of nibble i.
// Different bits of an index land on different operand positions, so the
// offsets of an index are the sums of one entry per nibble: the bit
// permutation between the step's index space and each operand's layout is
// resolved by table lookups instead of bit-by-bit scatters.
// o[i][v]: the offset in the stored output of the value v of output nibble
// i (the output index bits scattered through c_pos; only built for steps
// whose output is not stored in index order).
struct GatherTabs {
  uint2 c[kNib][16];
  uint2 k[kNib][16];
  uint32_t o[kNib][16];
};

// Fills the gather tables of step g: threads first, first + stride, ... of
// the CTA compute one entry each (no barrier).
__device__ __forceinline__ void gather_build(const StepGeom& g, GatherTabs& t, int first = threadIdx.x,
                                             int stride = kBlock) {
  // read once: the table stores below may alias the step record for the compiler
  const bool ident = g.c_identity != 0;
  for (int e = first; e < 2 * kNib * 16; e += stride) {
    const int field = e >> 7, i = (e >> 4) & (kNib - 1), v = e & 15;
    uint32_t oa = 0, ob = 0;
#pragma unroll
    uint32_t oc = 0;
    for (int bit = 0; bit < 4; ++bit) {
      if (!((v >> bit) & 1)) continue;
      const int j = 4 * i + bit;
      int pa = -1, pb = -1;
      if (field == 0) {  // output index bit j: n bits, then m bits, then batch bits
        if (!ident && j < g.rc) oc |= 1u << g.c_pos[j];
        if (j < g.nn) {
          pb = g.b_pos[g.nb + g.nk + j];
        } else if (j < g.nn + g.nm) {
          pa = g.a_pos[g.nb + j - g.nn];
        } else if (j < g.rc) {
          pa = g.a_pos[j - g.nn - g.nm];
          pb = g.b_pos[j - g.nn - g.nm];
        }
      } else if (j < g.nk) {  // reduction index bit j
        pa = g.a_pos[g.nb + g.nm + j];
        pb = g.b_pos[g.nb + j];
      }
      if (pa >= 0) oa |= 1u << pa;
      if (pb >= 0) ob |= 1u << pb;
    }
    (field ? t.k : t.c)[i][v] = make_uint2(oa, ob);
    if (field == 0 && !ident) t.o[i][v] = oc;
  }
}

// Offset of output index c in the stored output of step g (the gather
// tables' o part, or c itself for an output stored in index order).
__device__ __forceinline__ uint32_t out_offset(const StepGeom& g, const GatherTabs& t, uint32_t c) {
  if (g.c_identity) return c;
  uint32_t r = 0;
  const int nn = nibbles(g.rc);
#pragma unroll 1
  for (int i = 0; i < nn; ++i) r += t.o[i][(c >> (4 * i)) & 15u];
  return r;
}

// (offset in A, offset in B) of index x from nnib nibble tables.  This and
// out_offset keep their loops rolled: they run once per output or table
// entry, and unrolled copies at every inlined call site made the executor's
// code large enough that small tasks stalled on instruction fetch (rolled:
// -5 % on the headline step, -11 % for tropical).
__device__ __forceinline__ uint2 gather(const uint2 (*tab)[16], int nnib, uint32_t x) {
  uint2 r = make_uint2(0u, 0u);
#pragma unroll 1
  for (int i = 0; i < nnib; ++i) {
    const uint2 e = tab[i][(x >> (4 * i)) & 15u];
    r.x += e.x;
    r.y += e.y;
  }
  return r;
}

// Shared-memory scratch of one naive chunk: the gather tables, offsets of
// the low kNaiveKLoBits reduction bits (klo) and of the high-k blocks
// [kh_begin, kh_begin + kNaiveKHi) of the task (khi).
template <class SR>
struct NaiveSmem {
  GatherTabs gt;
  uint2 klo[1 << kNaiveKLoBits];
  uint2 khi[kNaiveKHi];
  typename SR::Acc red[kBlock / 32];
};

// Loads in flight per thread in the reduction loop of naive_chunk.
template <class SR>
struct NaiveUnroll {
  // 4: measured against 8 for 4-byte values, 2 % faster on the tropical
  // contractions (the general steps are latency-bound; fewer loads in flight
  // means a smaller loop)
  static constexpr int v = 4;
};

template <class T>
__device__ __forceinline__ T shfl_xor_val(T v, int off) {
  return __shfl_xor_sync(0xffffffffu, v, off);
}
__device__ __forceinline__ CntVal shfl_xor_val(CntVal v, int off) {
  CntVal r;
  r.v = __shfl_xor_sync(0xffffffffu, v.v, off);
  r.c = __shfl_xor_sync(0xffffffffu, v.c, off);
  return r;
}

// Several primes at once: the (+,*) ring modulo NP primes as one element
// type, so that a general step reads the residues of every prime of a term
// together (one round of loads instead of one per prime).
template <int NP>
struct ModParamsN {
  ModParams q[NP];
};

template <int NP>
struct ModValN {
  uint32_t v[NP];
};
template <int NP>
struct ModAccN {
  uint64_t a[NP];
};

template <int NP>
struct SrModN {
  using Val = ModValN<NP>;
  using Acc = ModAccN<NP>;
  static __device__ __forceinline__ Acc zero(const ModParamsN<NP>&) {
    Acc r;
#pragma unroll
    for (int q = 0; q < NP; ++q) r.a[q] = 0ull;
    return r;
  }
  static __device__ __forceinline__ Val leaf(int32_t kind, uint32_t e, const ModParamsN<NP>& mp) {
    Val r;
#pragma unroll
    for (int q = 0; q < NP; ++q) r.v[q] = SrMod::leaf(kind, e, mp.q[q].x);
    return r;
  }
  // the additive zero (the padding of short reduction batches)
  static __device__ __forceinline__ Val leaf(int32_t kind, uint32_t e) {
    Val r;
#pragma unroll
    for (int q = 0; q < NP; ++q) r.v[q] = SrMod::leaf(kind, e);
    return r;
  }
  static __device__ __forceinline__ void mac(Acc& acc, const Val& a, const Val& b, const ModParamsN<NP>& mp) {
#pragma unroll
    for (int q = 0; q < NP; ++q) SrMod::mac(acc.a[q], a.v[q], b.v[q], mp.q[q]);
  }
  static __device__ __forceinline__ void merge(Acc& acc, const Acc& o, const ModParamsN<NP>& mp) {
#pragma unroll
    for (int q = 0; q < NP; ++q) SrMod::merge(acc.a[q], o.a[q], mp.q[q]);
  }
};

template <int NP>
__device__ __forceinline__ ModAccN<NP> shfl_xor_val(ModAccN<NP> v, int off) {
  ModAccN<NP> r;
#pragma unroll
  for (int q = 0; q < NP; ++q) r.a[q] = __shfl_xor_sync(0xffffffffu, v.a[q], off);
  return r;
}

// Fills the tables of a step for the high-k blocks [kh_begin, kh_end) with
// threads first, first + stride, ...; sync() is a barrier over exactly those
// threads.  The tables are complete for the CTA after the next CTA-wide
// barrier.  Steps with at most 4 summed labels use the first k nibble table
// directly (no low / high k tables).
// have_low: the gather tables and the low-k table of this step are already
// in sm (an earlier task of the same step built them); only the high-k
// table of the task's block range is rebuilt.
template <class SR, class Sync>
__device__ __forceinline__ void naive_prepare(const StepGeom& g, NaiveSmem<SR>& sm, int32_t kh_begin,
                                              int32_t kh_end, int first, int stride, Sync sync,
                                              bool have_low = false) {
  if (!have_low) gather_build(g, sm.gt, first, stride);
  if (g.nk <= 4) return;  // the first k nibble table covers every term
  const int kl = g.nk < kNaiveKLoBits ? g.nk : kNaiveKLoBits;
  const int nkn = nibbles(g.nk);
  if (!have_low) {
    sync();
    for (int i = first; i < (1 << kl); i += stride) sm.klo[i] = gather(sm.gt.k, nkn, static_cast<uint32_t>(i));
  }
  if (kh_end - kh_begin <= kNaiveKHi)
    for (int i = first; i < kh_end - kh_begin; i += stride)
      sm.khi[i] = gather(sm.gt.k, nkn, static_cast<uint32_t>(kh_begin + i) << kl);
}

// The same with every thread of the CTA (ends with a barrier).
template <class SR>
__device__ __forceinline__ void naive_tables(const StepGeom& g, NaiveSmem<SR>& sm, int32_t kh_begin,
                                             int32_t kh_end) {
  naive_prepare<SR>(g, sm, kh_begin, kh_end, threadIdx.x, kBlock, [] { __syncthreads(); });
  __syncthreads();
}

// Computes output entries [c_begin, c_end) of a step over the high-k blocks
// [kh_begin, kh_end) (each block is 2^min(nk, 9) k's; naive_tables must
// have been called with the same block range).  R threads (a power of two,
// 1..256, R <= 2^nk) share each output entry: lane l takes the terms l,
// l + R, l + 2R, ... of the entry's flattened (block, low k) range,
// NaiveUnroll loads per operand in flight (the last, shorter batches are
// padded with the edge tensor's forbidden entry, the semiring zero: (max,+)
// -inf, (max, count) (-inf, 0), mod p 0), then the R partial results are
// merged with the semiring (+) by warp shuffles (R <= 32) or through shared
// memory.  The merged value of entry c goes to sink(c, acc) (called by one
// thread).  Every thread of the CTA must call this (it uses barriers when
// R > 32).
template <class SR, class LoadA, class LoadB, class Sink, class MP>
__device__ __forceinline__ void naive_chunk(const StepGeom& g, LoadA loadA, LoadB loadB, Sink sink,
                                            const MP& mp, int32_t c_begin, int32_t c_end,
                                            int32_t kh_begin, int32_t kh_end, int R, NaiveSmem<SR>& sm) {
  using Acc = typename SR::Acc;
  using Val = typename SR::Val;
  constexpr int U = NaiveUnroll<SR>::v;
  const int tid = threadIdx.x;
  const int slot = tid / R, lane = tid % R;
  const int per_pass = kBlock / R;
  const int kl = g.nk < kNaiveKLoBits ? g.nk : kNaiveKLoBits;
  const uint32_t mlo = (1u << kl) - 1u;
  const int ncn = nibbles(g.rc), nkn = nibbles(g.nk);
  const int32_t nterm = (kh_end - kh_begin) << kl;
  const bool tab = kh_end - kh_begin <= kNaiveKHi;
  // offsets (in A, in B) of term j of the task's k range
  auto koff = [&](int32_t j) -> uint2 {
    if (g.nk <= 4) return sm.gt.k[0][j];  // one nibble: a single k block
    const int32_t h = j >> kl;
    const uint2 hi = tab ? sm.khi[h] : gather(sm.gt.k, nkn, static_cast<uint32_t>(kh_begin + h) << kl);
    const uint2 lo = sm.klo[static_cast<uint32_t>(j) & mlo];
    return make_uint2(hi.x + lo.x, hi.y + lo.y);
  };
  for (int32_t cb = c_begin; cb < c_end; cb += per_pass) {
    const int32_t c = cb + slot;
    const bool valid = c < c_end;
    Acc acc = SR::zero(mp);
    if (valid) {
      const uint2 base = gather(sm.gt.c, ncn, static_cast<uint32_t>(c));
      // full batches of U terms, then the rest in batches of TU padded with
      // the semiring zero, so the loads of every batch are in flight together
      constexpr int TU = U > 4 ? 4 : 2;
      int32_t j = lane;
      for (; j + (U - 1) * R < nterm; j += U * R) {
        Val va[U], vb[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const uint2 o = koff(j + u * R);
          va[u] = loadA(base.x + o.x);
          vb[u] = loadB(base.y + o.y);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) SR::mac(acc, va[u], vb[u], mp);
      }
      for (; j < nterm; j += TU * R) {
        Val va[TU], vb[TU];
#pragma unroll
        for (int u = 0; u < TU; ++u) {
          const int32_t jj = j + u * R;
          const bool in = jj < nterm;
          const uint2 o = koff(in ? jj : j);
          va[u] = in ? loadA(base.x + o.x) : SR::leaf(kOpEdge, 3);
          vb[u] = in ? loadB(base.y + o.y) : SR::leaf(kOpEdge, 3);
        }
#pragma unroll
        for (int u = 0; u < TU; ++u) SR::mac(acc, va[u], vb[u], mp);
      }
    }
    // merge the R partial accumulators of each output entry
    const int rw = R < 32 ? R : 32;
    for (int off = rw / 2; off >= 1; off >>= 1) {
      Acc o = shfl_xor_val(acc, off);
      SR::merge(acc, o, mp);
    }
    if (R > 32) {
      if ((tid & 31) == 0) sm.red[tid >> 5] = acc;
      __syncthreads();
      if (lane == 0) {
        for (int w = 1; w < R / 32; ++w) SR::merge(acc, sm.red[(tid >> 5) + w], mp);
      }
      __syncthreads();
    }
    if (valid && lane == 0) sink(static_cast<uint32_t>(c), acc);
  }
}

// R = 1 variant of naive_chunk: each thread computes U output entries at
// once (entries cb + tid + 256 u), so U independent loads per operand are in
// flight (2U with the unrolled k loop).  Used for wide steps with short
// reductions; covers the whole k range (naive_tables over all high-k blocks).
template <class SR, int U, class LoadA, class LoadB, class Sink, class MP>
__device__ __forceinline__ void naive_chunk_wide(const StepGeom& g, LoadA loadA, LoadB loadB, Sink sink,
                                                 const MP& mp, int32_t c_begin, int32_t c_end,
                                                 NaiveSmem<SR>& sm) {
  using Acc = typename SR::Acc;
  const int kl = g.nk < kNaiveKLoBits ? g.nk : kNaiveKLoBits;
  const uint32_t mlo = (1u << kl) - 1u;
  const int32_t nterm = 1 << g.nk;
  const int ncn = nibbles(g.rc), nkn = nibbles(g.nk);
  const bool tab = (nterm >> kl) <= kNaiveKHi;
  for (int32_t cb = c_begin; cb < c_end; cb += U * kBlock) {
    uint2 base[U];
    Acc acc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int32_t c = cb + static_cast<int32_t>(threadIdx.x) + u * kBlock;
      const int32_t cc = c < c_end ? c : c_begin;  // out-of-range lanes recompute a valid entry
      base[u] = gather(sm.gt.c, ncn, static_cast<uint32_t>(cc));
      acc[u] = SR::zero(mp);
    }
#pragma unroll 2
    for (int32_t j = 0; j < nterm; ++j) {
      uint32_t ka, kb;
      if (g.nk <= 4) {
        ka = sm.gt.k[0][j].x;
        kb = sm.gt.k[0][j].y;
      } else {
        const int32_t h = j >> kl;
        const uint2 hi = tab ? sm.khi[h] : gather(sm.gt.k, nkn, static_cast<uint32_t>(h) << kl);
        const uint2 lo = sm.klo[static_cast<uint32_t>(j) & mlo];
        ka = hi.x + lo.x;
        kb = hi.y + lo.y;
      }
      typename SR::Val va[U], vb[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        va[u] = loadA(base[u].x + ka);
        vb[u] = loadB(base[u].y + kb);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) SR::mac(acc[u], va[u], vb[u], mp);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int32_t c = cb + static_cast<int32_t>(threadIdx.x) + u * kBlock;
      if (c < c_end) sink(static_cast<uint32_t>(c), acc[u]);
    }
  }
}

// Host-side shape of a general ("naive") step with E = 2^rc outputs and
// K = 2^nk terms: R threads per output entry, `chunk` outputs per task,
// `ks` tasks sharing each chunk along k (their partial results are merged by
// the last one to finish; ks > 1 only in the executor).
struct NaiveShape {
  int R;
  int64_t chunk;    // output entries per task (multiple of 256 / R)
  int64_t nchunks;  // output chunks
  int ks;           // k splits per chunk
  int64_t ntasks;   // nchunks * ks
};

inline NaiveShape naive_shape(int rc, int nk, bool allow_ksplit, int sets = 1) {
  NaiveShape s;
  const int64_t E = int64_t(1) << rc, K = int64_t(1) << nk;
  int R = 1;
  // give each thread at least ~8 terms (measured: 0.8 % faster on the
  // headline step than 16), but keep at least ~2^17 threads busy
  while (R < 256 && R * 2 <= K && K / (R * 2) >= 8 && E * R < (int64_t(1) << 17)) R *= 2;
  s.R = R;
  const int64_t per_pass = kBlock / R;
  int64_t chunk = per_pass;
  if (R == 1 && E >= int64_t(kNaiveWideU) * kBlock * 152) {
    // wide and shallow: U entries per thread, about one wave of ~2 tasks per SM
    chunk = int64_t(kNaiveWideU) * kBlock;
    while ((E + chunk - 1) / chunk > 608) chunk *= 2;
  } else {
    // at most ~8 passes per task and at most 4096 chunks
    while (chunk * 2 <= per_pass * 8 && (E + chunk - 1) / chunk > 4096) chunk *= 2;
    while ((E + chunk - 1) / chunk > 4096) chunk *= 2;
  }
  s.chunk = chunk;
  s.nchunks = (E + chunk - 1) / chunk;
  // split long reductions over several CTAs (whole high-k blocks each)
  const int kl = nk < kNaiveKLoBits ? nk : kNaiveKLoBits;
  const int64_t nkhi = int64_t(1) << (nk - kl);
  int ks = 1;
  while (allow_ksplit && s.nchunks * ks < 304 && ks * 2 <= nkhi && K / (int64_t(R) * ks * 2) >= 8 && ks < 256)
    ks *= 2;
  // a scalar output (the last step of a network): every task set (one per
  // prime slot) in one wave of the 304 resident CTAs
  if (rc == 0)
    while (ks > 1 && int64_t(ks) * sets > 304) ks /= 2;
  s.ks = ks;
  s.ntasks = s.nchunks * ks;
  return s;
}

}  // namespace dev
}  // namespace tn
