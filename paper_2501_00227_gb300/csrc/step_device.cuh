// step_device.cuh -- device building blocks shared by the per-step kernels
// and the persistent plan executor: bit-position maps and the general
// ("naive chunk") step body with K-parallel reduction.
//
// A step (Sec. 4.1 of arXiv:2501.00227) computes
//   C[b, m, n] = (+)_k A[b, m, k] (x) B[b, k, n],
// C stored contiguously as c = n | m << nn | b << (nn + nm) (or scattered
// through c_pos when the caller fixes the output label order).
#pragma once

#include <cstdint>

#include "semiring.cuh"

namespace tn {
namespace dev {

// Scatter the bits of x into the positions pos[first .. first+count).
__device__ __forceinline__ int64_t deposit(int64_t x, const int8_t* pos, int first, int count) {
  int64_t r = 0;
  for (int j = 0; j < count; ++j)
    if ((x >> j) & 1) {
      int p = pos[first + j];
      if (p >= 0) r |= int64_t(1) << p;
    }
  return r;
}

constexpr int kNaiveKLoBits = 9;    // k offsets of the low 9 bits come from a table
constexpr int kNaiveKHi = 256;      // high-k blocks per task whose offsets are tabulated
constexpr int kBlock = 256;         // threads per CTA of every libtn kernel
constexpr int kNaiveWideU = 4;      // entries per thread in naive_chunk_wide

// Shared-memory scratch of one naive chunk: offsets of the low k bits
// (ka / kb) and of the high-k blocks [kh_begin, kh_begin + kNaiveKHi) of
// the task (kha / khb).
template <class SR>
struct NaiveSmem {
  int64_t ka[1 << kNaiveKLoBits];
  int64_t kb[1 << kNaiveKLoBits];
  int64_t kha[kNaiveKHi];
  int64_t khb[kNaiveKHi];
  typename SR::Acc red[kBlock / 32];
};

// Loads in flight per thread in the reduction loop of naive_chunk.
template <class SR>
struct NaiveUnroll {
  static constexpr int v = sizeof(typename SR::Val) <= 4 ? 8 : 4;
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

// Fills the k-offset tables of a step for the high-k blocks
// [kh_begin, kh_end) (all threads of the CTA; ends with a barrier).
template <class SR>
__device__ __forceinline__ void naive_tables(const StepGeom& g, NaiveSmem<SR>& sm, int64_t kh_begin,
                                             int64_t kh_end) {
  const int kl = g.nk < kNaiveKLoBits ? g.nk : kNaiveKLoBits;
  const int a_k0 = g.nb + g.nm, b_k0 = g.nb;
  for (int i = threadIdx.x; i < (1 << kl); i += kBlock) {
    sm.ka[i] = deposit(i, g.a_pos, a_k0, kl);
    sm.kb[i] = deposit(i, g.b_pos, b_k0, kl);
  }
  if (kh_end - kh_begin <= kNaiveKHi)
    for (int i = threadIdx.x; i < kh_end - kh_begin; i += kBlock) {
      sm.kha[i] = deposit(kh_begin + i, g.a_pos, a_k0 + kl, g.nk - kl);
      sm.khb[i] = deposit(kh_begin + i, g.b_pos, b_k0 + kl, g.nk - kl);
    }
  __syncthreads();
}

// Computes output entries [c_begin, c_end) of a step for prime index q,
// over the high-k blocks [kh_begin, kh_end) (each block is 2^min(nk, 9) k's;
// naive_tables must have been called with the same block range).
// R threads (a power of two, 1..256, R <= 2^nk) share each output entry:
// lane l takes the terms l, l + R, l + 2R, ... of the entry's flattened
// (block, low k) range, NaiveUnroll loads per operand in flight (a batch
// beyond the range is padded with the edge tensor's forbidden entry, the
// semiring zero: (max,+) -inf, (max, count) (-inf, 0), mod p 0), then the R
// partial results are merged with the semiring (+) by warp shuffles
// (R <= 32) or through shared memory.  The merged value of entry c goes to
// sink(c, acc) (called by one thread).  Every thread of the CTA must call
// this (it uses barriers when R > 32).
template <class SR, class LoadA, class LoadB, class Sink>
__device__ __forceinline__ void naive_chunk(const StepGeom& g, LoadA loadA, LoadB loadB, Sink sink,
                                            const ModParams& mp, int64_t c_begin, int64_t c_end,
                                            int64_t kh_begin, int64_t kh_end, int R, NaiveSmem<SR>& sm) {
  using Acc = typename SR::Acc;
  using Val = typename SR::Val;
  constexpr int U = NaiveUnroll<SR>::v;
  const int tid = threadIdx.x;
  const int slot = tid / R, lane = tid % R;
  const int per_pass = kBlock / R;
  const int kl = g.nk < kNaiveKLoBits ? g.nk : kNaiveKLoBits;
  const int64_t mlo = (int64_t(1) << kl) - 1;
  const int a_k0 = g.nb + g.nm, b_k0 = g.nb;
  const int64_t mask_n = (int64_t(1) << g.nn) - 1, mask_m = (int64_t(1) << g.nm) - 1;
  const int64_t nterm = (kh_end - kh_begin) << kl;
  const bool tab = kh_end - kh_begin <= kNaiveKHi;
  // offsets of term j inside A and B (high block from the table or computed)
  auto koffA = [&](int64_t j) -> int64_t {
    const int64_t h = j >> kl;
    return (tab ? sm.kha[h] : deposit(kh_begin + h, g.a_pos, a_k0 + kl, g.nk - kl)) | sm.ka[j & mlo];
  };
  auto koffB = [&](int64_t j) -> int64_t {
    const int64_t h = j >> kl;
    return (tab ? sm.khb[h] : deposit(kh_begin + h, g.b_pos, b_k0 + kl, g.nk - kl)) | sm.kb[j & mlo];
  };
  for (int64_t cb = c_begin; cb < c_end; cb += per_pass) {
    const int64_t c = cb + slot;
    const bool valid = c < c_end;
    Acc acc = SR::zero(mp);
    if (valid) {
      const int64_t n = c & mask_n, m = (c >> g.nn) & mask_m, b = c >> (g.nn + g.nm);
      const int64_t base_a = deposit(b, g.a_pos, 0, g.nb) | deposit(m, g.a_pos, g.nb, g.nm);
      const int64_t base_b = deposit(b, g.b_pos, 0, g.nb) | deposit(n, g.b_pos, g.nb + g.nk, g.nn);
      // U terms per batch; the last batch pads with the semiring zero, so
      // its loads are in flight together as well
      for (int64_t j = lane; j < nterm; j += U * R) {
        Val va[U], vb[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int64_t jj = j + u * R;
          const bool in = jj < nterm;
          va[u] = in ? loadA(base_a | koffA(jj)) : SR::leaf(kOpEdge, 3);
          vb[u] = in ? loadB(base_b | koffB(jj)) : SR::leaf(kOpEdge, 3);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) SR::mac(acc, va[u], vb[u], mp);
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
    if (valid && lane == 0) sink(c, acc);
  }
}

// R = 1 variant of naive_chunk: each thread computes U output entries at
// once (entries cb + tid + 256 u), so U independent loads per operand are in
// flight (2U with the unrolled k loop).  Used for wide steps with short
// reductions; covers the whole k range (naive_tables over all high-k blocks).
template <class SR, int U, class LoadA, class LoadB, class Sink>
__device__ __forceinline__ void naive_chunk_wide(const StepGeom& g, LoadA loadA, LoadB loadB, Sink sink,
                                                 const ModParams& mp, int64_t c_begin, int64_t c_end,
                                                 NaiveSmem<SR>& sm) {
  using Acc = typename SR::Acc;
  const int kl = g.nk < kNaiveKLoBits ? g.nk : kNaiveKLoBits;
  const int64_t mlo = (int64_t(1) << kl) - 1, nterm = int64_t(1) << g.nk;
  const int a_k0 = g.nb + g.nm, b_k0 = g.nb;
  const bool tab = (nterm >> kl) <= kNaiveKHi;
  const int64_t mask_n = (int64_t(1) << g.nn) - 1, mask_m = (int64_t(1) << g.nm) - 1;
  for (int64_t cb = c_begin; cb < c_end; cb += int64_t(U) * kBlock) {
    int64_t base_a[U], base_b[U];
    Acc acc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t c = cb + threadIdx.x + int64_t(u) * kBlock;
      const int64_t cc = c < c_end ? c : c_begin;  // out-of-range lanes recompute a valid entry
      const int64_t n = cc & mask_n, m = (cc >> g.nn) & mask_m, b = cc >> (g.nn + g.nm);
      base_a[u] = deposit(b, g.a_pos, 0, g.nb) | deposit(m, g.a_pos, g.nb, g.nm);
      base_b[u] = deposit(b, g.b_pos, 0, g.nb) | deposit(n, g.b_pos, g.nb + g.nk, g.nn);
      acc[u] = SR::zero(mp);
    }
#pragma unroll 2
    for (int64_t j = 0; j < nterm; ++j) {
      const int64_t h = j >> kl;
      const int64_t ka = (tab ? sm.kha[h] : deposit(h, g.a_pos, a_k0 + kl, g.nk - kl)) | sm.ka[j & mlo];
      const int64_t kb = (tab ? sm.khb[h] : deposit(h, g.b_pos, b_k0 + kl, g.nk - kl)) | sm.kb[j & mlo];
      typename SR::Val va[U], vb[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        va[u] = loadA(base_a[u] | ka);
        vb[u] = loadB(base_b[u] | kb);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) SR::mac(acc[u], va[u], vb[u], mp);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t c = cb + threadIdx.x + int64_t(u) * kBlock;
      if (c < c_end) sink(c, acc[u]);
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

inline NaiveShape naive_shape(int rc, int nk, bool allow_ksplit) {
  NaiveShape s;
  const int64_t E = int64_t(1) << rc, K = int64_t(1) << nk;
  int R = 1;
  // give each thread at least ~16 terms, but keep at least ~2^17 threads busy
  while (R < 256 && R * 2 <= K && K / (R * 2) >= 16 && E * R < (int64_t(1) << 17)) R *= 2;
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
  s.ks = ks;
  s.ntasks = s.nchunks * ks;
  return s;
}

}  // namespace dev
}  // namespace tn
