// tile_device.cuh -- the register-blocked semiring GEMM tile shared by the
// per-step tiled kernel and the persistent executor.
//
//   C[b, m, n] = (+)_k A[b, m, k] (x) B[b, k, n]   (Sec. 4.1 of arXiv:2501.00227)
//
// A CTA (256 threads) computes a BM x BN output tile of one batch index.  The
// threads form KG groups of WM x WN threads; each thread owns a TM x TN
// micro-tile in registers (BM = WM TM, BN = WN TN).  k advances in chunks of
// BK = BKG KG staged in shared memory (A as [k][m], B as [k][n]) through a
// three-stage cp.async pipeline; group g consumes the k rows [BKG g, BKG g +
// BKG) of every chunk ("sliced K"), and the KG partial tiles are merged with
// the semiring (+) at the end.  KG > 1 lets small M x N tiles (32 x 32) keep
// 4 x 4 register blocking.
//
// Operands are read in place through the step's gather tables (see
// step_device.cuh): the offset of A[b, m, k] is the sum of the offset of the
// output index (b, m, n = 0) and of the reduction index k.  A tile covers the
// low bits of m, n and k, so each thread's staging offsets are fixed for the
// whole tile and only a per-chunk base (the high k bits) changes.
#pragma once

#include <cuda_fp16.h>

#include <type_traits>

#include "semiring.cuh"
#include "step_device.cuh"

namespace tn {
namespace dev {

// Per-semiring hooks of the tiled kernels on top of semiring.cuh.
template <class SR>
struct Tiled {
  static __device__ __forceinline__ void mac(typename SR::Acc& acc, const typename SR::Val& a,
                                             const typename SR::Val& b, const ModParams& mp) {
    SR::mac(acc, a, b, mp);
  }
  static __device__ __forceinline__ void fold(typename SR::Acc&, const ModParams&) {}
  static __device__ __forceinline__ typename SR::Val zero_val() { return SR::leaf(kOpEdge, 3); }
};

// mod p: plain 64-bit accumulation, folded every FOLD products (see SrMod)
template <>
struct Tiled<SrMod> {
  static __device__ __forceinline__ void mac(uint64_t& acc, uint32_t a, uint32_t b, const ModParams&) {
    acc += static_cast<uint64_t>(a) * b;
  }
  static __device__ __forceinline__ void fold(uint64_t& acc, const ModParams& mp) {
    acc = fold32(acc, mp.r32);
  }
  static __device__ __forceinline__ uint32_t zero_val() { return 0u; }
};

template <int TM_, int TN_, int WM_, int WN_, int KG_, int BKG_>
struct TileCfg {
  static constexpr int TM = TM_, TN = TN_, WM = WM_, WN = WN_, KG = KG_;
  static constexpr int BM = WM * TM, BN = WN * TN;
  static constexpr int GT = WM * WN;  // threads per k group
  static constexpr int BKG = BKG_;    // k rows per group per chunk
  static constexpr int BK = BKG * KG; // k rows per staged chunk
  static constexpr int EA = BK * BM / kBlock, EB = BK * BN / kBlock;  // staged elements per thread
  static_assert(GT * KG == kBlock, "a tile uses all 256 threads");
  static_assert(EA >= 1 && EB >= 1 && (BK * BM) % kBlock == 0 && (BK * BN) % kBlock == 0, "staging");
};

// Tile shapes (index = ExecStep.tile / the tile argument of the launchers).
// Shapes 0-4 stage 4 A and 4 B elements per thread and chunk; shape 5 (for
// short reductions over few rows and many columns) 2 and 8.
using TileC0 = TileCfg<8, 8, 16, 16, 1, 8>;   // 128 x 128, BK 8, tropical only
using TileC1 = TileCfg<4, 4, 16, 16, 1, 16>;  // 64 x 64, BK 16
using TileC2 = TileCfg<4, 4, 8, 8, 4, 8>;     // 32 x 32, sliced K 4 x 8
using TileC3 = TileCfg<4, 4, 4, 16, 4, 8>;    // 16 x 64, sliced K 4 x 8
using TileC4 = TileCfg<4, 4, 16, 4, 4, 8>;    // 64 x 16, sliced K 4 x 8
using TileC5 = TileCfg<4, 4, 8, 32, 1, 16>;   // 32 x 128, BK 16
constexpr int kNumTiles = 6;

// cp.async pipeline depth of the tile main loop: three stages for 4-byte
// elements, two for the 16-byte (max, count) pairs
template <class SR>
struct Stages {
  static constexpr int v = sizeof(typename SR::Val) <= 4 ? 3 : 2;
};

// Index part of a tile's shared memory (same place for every element type).
// offCm / offCn: stored-output offsets of the tile's rows (with the batch)
// and columns, for outputs not stored in index order.
template <class C>
struct TileIdx {
  GatherTabs gt;
  uint32_t offAm[C::BM];
  uint32_t offBn[C::BN];
  uint32_t offAk[C::BK];
  uint32_t offBk[C::BK];
  uint32_t offCm[C::BM];
  uint32_t offCn[C::BN];
};

template <class SR, class C>
struct TileSmem {
  TileIdx<C> idx;
  alignas(16) typename SR::Val As[Stages<SR>::v][C::BK * C::BM];
  alignas(16) typename SR::Val Bs[Stages<SR>::v][C::BK * C::BN];
};

// Index tables of tile (tm, tn_) of batch b: gather tables and the offsets
// of the tile's rows, columns and chunk rows, computed by threads first,
// first + stride, ...; sync() is a barrier over exactly those threads.  The
// tables are complete for the CTA after the next CTA-wide barrier.
// have_gather: the gather tables of this step are already in ix.gt (an
// earlier tile of the same step built them).
template <class C, class Sync>
__device__ __forceinline__ void tile_tables(const StepGeom& g, TileIdx<C>& ix, int64_t b, int64_t tm, int64_t tn_,
                                            int first, int stride, Sync sync, bool have_gather = false) {
  constexpr int BM = C::BM, BN = C::BN, BK = C::BK;
  const uint32_t M = 1u << g.nm, N = 1u << g.nn, K = 1u << g.nk;
  const uint32_t m0 = static_cast<uint32_t>(tm) * BM, n0 = static_cast<uint32_t>(tn_) * BN;
  const int ncn = nibbles(g.rc), nkn = nibbles(g.nk);
  if (!have_gather) {
    gather_build(g, ix.gt, first, stride);
    sync();
  }
  const uint32_t cb = static_cast<uint32_t>(b) << (g.nn + g.nm);
  // rolled loops: set-up code, kept small for the instruction cache
#pragma unroll 1
  for (int i = first; i < BM; i += stride)
    ix.offAm[i] = m0 + i < M ? gather(ix.gt.c, ncn, cb | ((m0 + i) << g.nn)).x : 0u;
#pragma unroll 1
  for (int i = first; i < BN; i += stride) ix.offBn[i] = n0 + i < N ? gather(ix.gt.c, ncn, cb | (n0 + i)).y : 0u;
  if (!g.c_identity) {
#pragma unroll 1
    for (int i = first; i < BM; i += stride)
      ix.offCm[i] = m0 + i < M ? out_offset(g, ix.gt, cb | ((m0 + i) << g.nn)) : 0u;
#pragma unroll 1
    for (int i = first; i < BN; i += stride) ix.offCn[i] = n0 + i < N ? out_offset(g, ix.gt, n0 + i) : 0u;
  }
#pragma unroll 1
  for (int i = first; i < BK; i += stride) {
    const uint2 o = gather(ix.gt.k, nkn, static_cast<uint32_t>(i) < K ? static_cast<uint32_t>(i) : 0u);
    ix.offAk[i] = o.x;
    ix.offBk[i] = o.y;
  }
}

// This thread's staging offsets (element e = tid + 256 j of a chunk: A as
// [k][m], B as [k][n]) from complete index tables, -1 for padding outside M,
// N or K.
template <class C>
__device__ __forceinline__ void tile_slots(const StepGeom& g, const TileIdx<C>& ix, int64_t tm, int64_t tn_,
                                           int32_t (&offA)[C::EA], int32_t (&offB)[C::EB]) {
  constexpr int BM = C::BM, BN = C::BN, BK = C::BK;
  const int tid = threadIdx.x;
  const uint32_t M = 1u << g.nm, N = 1u << g.nn, K = 1u << g.nk;
  const uint32_t m0 = static_cast<uint32_t>(tm) * BM, n0 = static_cast<uint32_t>(tn_) * BN;
  const uint32_t kvalid = K < BK ? K : BK;  // k rows that exist inside a chunk
#pragma unroll
  for (int j = 0; j < C::EA; ++j) {
    const int e = tid + kBlock * j, kk = e / BM, mm = e % BM;
    const bool ok = (m0 + mm < M) && (static_cast<uint32_t>(kk) < kvalid);
    offA[j] = ok ? static_cast<int32_t>(ix.offAm[mm] + ix.offAk[kk]) : -1;
  }
#pragma unroll
  for (int j = 0; j < C::EB; ++j) {
    const int e = tid + kBlock * j, kk = e / BN, nn = e % BN;
    const bool ok = (n0 + nn < N) && (static_cast<uint32_t>(kk) < kvalid);
    offB[j] = ok ? static_cast<int32_t>(ix.offBn[nn] + ix.offBk[kk]) : -1;
  }
}

// Staging offsets of tile (tm, tn_) of batch b for this thread; builds the
// index tables first unless `ready`.  All threads must call it (it has
// barriers).
template <class C>
__device__ __forceinline__ void tile_offsets(const StepGeom& g, TileIdx<C>& ix, int64_t b, int64_t tm,
                                             int64_t tn_, int32_t (&offA)[C::EA], int32_t (&offB)[C::EB],
                                             bool ready = false) {
  if (!ready) {
    tile_tables<C>(g, ix, b, tm, tn_, threadIdx.x, kBlock, [] { __syncthreads(); });
    __syncthreads();
  }
  tile_slots<C>(g, ix, tm, tn_, offA, offB);
}

// Vector staging.  kVecA / kVecB: the operand's two lowest stored bits are
// the step's m (resp. n) bits 0 and 1, it is an arena tensor and its entry
// offset is a multiple of 4 -- then every group of 4 consecutive m (n) of a
// staged row is one aligned 16-byte run in memory, and a thread stages it
// with one 16-byte cp.async instead of four 4-byte ones.  Slot s of a chunk
// is the 4-element group starting at element 4 s of the [k][m] ([k][n])
// staging array.
constexpr int kVecA = 1, kVecB = 2;

template <int ROW, int ELEMS>
struct VecSlots {
  static constexpr int total = ELEMS / 4;                       // 4-element groups per chunk
  static constexpr int per_thread = (total + kBlock - 1) / kBlock;
};

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem_src) : "memory");
}

// This thread's 16-byte staging slots of one operand (ROW = BM or BN): the
// offset of each slot's first element, -1 for slots outside the operand
// (M / N or K padding) or beyond the chunk.
template <int ROW, int BK, int NS>
__device__ __forceinline__ void tile_slots4(const uint32_t* off_row, const uint32_t* off_k, uint32_t row0,
                                            uint32_t rows, uint32_t kvalid, int32_t* off4) {
  constexpr int total = BK * ROW / 4;
#pragma unroll
  for (int j = 0; j < NS; ++j) {
    const int s = threadIdx.x + kBlock * j;
    const int e = 4 * s, kk = e / ROW, rr = e % ROW;
    const bool ok = s < total && (row0 + rr < rows) && (static_cast<uint32_t>(kk) < kvalid);
    off4[j] = ok ? static_cast<int32_t>(off_row[rr] + off_k[kk]) : -1;
  }
}

// Offsets (in A, in B) of the chunk of k rows starting at k0 (a multiple of
// BK: its bits are disjoint from those of the rows inside the chunk).
template <class C>
__device__ __forceinline__ uint2 tile_chunk_base(const StepGeom& g, const TileIdx<C>& ix, int64_t k0) {
  return gather(ix.gt.k, nibbles(g.nk), static_cast<uint32_t>(k0));
}

// Fragment of T consecutive 4-byte values from shared memory (16-byte
// vector loads when T is a multiple of 4, the address then 16-byte aligned;
// one 8-byte load when T = 2, the address 8-byte aligned).
template <int T, class V>
__device__ __forceinline__ void load_frag(const V* p, V (&out)[T]) {
  if constexpr (sizeof(V) == 4 && T == 2) {
    const uint2 w = *reinterpret_cast<const uint2*>(p);
    out[0] = __builtin_bit_cast(V, w.x);
    out[1] = __builtin_bit_cast(V, w.y);
  } else if constexpr (sizeof(V) == 4 && T % 4 == 0) {
#pragma unroll
    for (int i = 0; i < T; i += 4) {
      const uint4 w = *reinterpret_cast<const uint4*>(p + i);
      out[i] = __builtin_bit_cast(V, w.x);
      out[i + 1] = __builtin_bit_cast(V, w.y);
      out[i + 2] = __builtin_bit_cast(V, w.z);
      out[i + 3] = __builtin_bit_cast(V, w.w);
    }
  } else {
#pragma unroll
    for (int i = 0; i < T; ++i) out[i] = p[i];
  }
}

template <int X>
struct Log2 {
  static constexpr int v = X <= 1 ? 0 : 1 + Log2<X / 2>::v;
};
template <>
struct Log2<1> {
  static constexpr int v = 0;
};

// Stages the chunk of k rows starting at k0 into as / bs ([BK][BM] and
// [BK][BN]): cp.async for stored operands (16-byte runs where the layout
// allows, see tile_slots4), plain loads for leaves generated on the fly.
// offA / offB are this thread's element offsets (or its 16-byte slot
// offsets when va / vb); negative ones are padding and are not written.
template <class SR, class C, bool CG, int NSA, int NSB>
__device__ __forceinline__ void tile_stage(const StepGeom& g, const TileIdx<C>& ix, const Operand& A,
                                           const Operand& B, const int32_t (&offA)[C::EA],
                                           const int32_t (&offB)[C::EB], bool va, bool vb, typename SR::Val* as,
                                           typename SR::Val* bs, int64_t k0) {
  using Val = typename SR::Val;
  const int tid = threadIdx.x;
  const uint2 kb = tile_chunk_base<C>(g, ix, k0);
  if (va) {
#pragma unroll
    for (int j = 0; j < NSA; ++j)
      if (offA[j] >= 0)
        cp_async16(&as[4 * (tid + kBlock * j)], static_cast<const Val*>(A.p0) + (static_cast<uint32_t>(offA[j]) + kb.x));
  } else {
    const bool a_async = A.kind == kOpArena;
#pragma unroll
    for (int j = 0; j < C::EA; ++j)
      if (offA[j] >= 0) {
        const uint32_t e = static_cast<uint32_t>(offA[j]) + kb.x;
        if (a_async) SR::copy_async(&as[tid + kBlock * j], A, e);
        else as[tid + kBlock * j] = SR::template load<CG>(A, e);
      }
  }
  if (vb) {
#pragma unroll
    for (int j = 0; j < NSB; ++j)
      if (offB[j] >= 0)
        cp_async16(&bs[4 * (tid + kBlock * j)], static_cast<const Val*>(B.p0) + (static_cast<uint32_t>(offB[j]) + kb.y));
  } else {
    const bool b_async = B.kind == kOpArena;
#pragma unroll
    for (int j = 0; j < C::EB; ++j)
      if (offB[j] >= 0) {
        const uint32_t e = static_cast<uint32_t>(offB[j]) + kb.y;
        if (b_async) SR::copy_async(&bs[tid + kBlock * j], B, e);
        else bs[tid + kBlock * j] = SR::template load<CG>(B, e);
      }
  }
}

// Accumulates tile (tm, tn) of batch b over k in [kbeg, kend) into acc (of
// the calling thread's group; the partial tiles of the KG groups are NOT yet
// merged -- see tile_merge_groups).  FOLD: mod-p products accumulated between
// two folds (1 is safe for every p < 2^31; 4 where mod_fold_interval allows it).  All
// threads of the CTA must call it.
template <class SR, class C, int FOLD, bool CG>
__device__ __forceinline__ void tile_mainloop(const StepGeom& g, const Operand& A, const Operand& B,
                                              const ModParams& mp, int64_t b, int64_t tm, int64_t tn_,
                                              int64_t kbeg, int64_t kend, TileSmem<SR, C>& sm,
                                              typename SR::Acc (&acc)[C::TM][C::TN], bool ready = false,
                                              int vec = 0) {
  using Val = typename SR::Val;
  using T = Tiled<SR>;
  constexpr int kStages = Stages<SR>::v;
  constexpr int BM = C::BM, BN = C::BN, BK = C::BK, TM = C::TM, TN = C::TN;
  const int tid = threadIdx.x;
  const int grp = tid / C::GT, gt = tid % C::GT;
  const int tx = gt % C::WN, ty = gt / C::WN;

  int32_t offA[C::EA], offB[C::EB];
  tile_offsets<C>(g, sm.idx, b, tm, tn_, offA, offB, ready);
  // 16-byte slots (only for 4-byte elements of arena operands); their
  // offsets replace the first per-element offsets once the padding is set
  constexpr int NSA = VecSlots<BM, BK * BM>::per_thread, NSB = VecSlots<BN, BK * BN>::per_thread;
  static_assert(NSA <= C::EA && NSB <= C::EB, "a 16-byte slot covers four staged elements");
  const bool va = sizeof(Val) == 4 && (vec & kVecA) && A.kind == kOpArena;
  const bool vb = sizeof(Val) == 4 && (vec & kVecB) && B.kind == kOpArena;

#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = SR::zero(mp);

  // padding slots (outside M / N / K) hold the semiring zero in every stage;
  // the copies below never write them
#pragma unroll
  for (int j = 0; j < C::EA; ++j)
    if (offA[j] < 0)
      for (int st = 0; st < kStages; ++st) sm.As[st][tid + kBlock * j] = T::zero_val();
#pragma unroll
  for (int j = 0; j < C::EB; ++j)
    if (offB[j] < 0)
      for (int st = 0; st < kStages; ++st) sm.Bs[st][tid + kBlock * j] = T::zero_val();
  {
    const uint32_t K = 1u << g.nk, kvalid = K < BK ? K : BK;
    if (va) tile_slots4<BM, BK, NSA>(sm.idx.offAm, sm.idx.offAk, static_cast<uint32_t>(tm) * BM, 1u << g.nm, kvalid, offA);
    if (vb) tile_slots4<BN, BK, NSB>(sm.idx.offBn, sm.idx.offBk, static_cast<uint32_t>(tn_) * BN, 1u << g.nn, kvalid, offB);
  }

  auto issue = [&](int st, int64_t k0) {
    tile_stage<SR, C, CG, NSA, NSB>(g, sm.idx, A, B, offA, offB, va, vb, sm.As[st], sm.Bs[st], k0);
  };
#pragma unroll
  for (int st = 0; st < kStages - 1; ++st) {
    if (kbeg + st * BK < kend) issue(st, kbeg + st * BK);
    cp_async_commit();
  }
  int cur = 0;
  for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
    cp_async_wait<kStages - 2>();
    __syncthreads();
    {
      // refill the buffer computed on in the previous iteration
      const int64_t kn = k0 + (kStages - 1) * BK;
      const int nxt = (cur + kStages - 1) % kStages;
      if (kn < kend) issue(nxt, kn);
      cp_async_commit();
    }
    const Val* Ag = sm.As[cur] + grp * C::BKG * BM;
    const Val* Bg = sm.Bs[cur] + grp * C::BKG * BN;
    // the k rows of a chunk in groups of FOLD (mod p folds after each group);
    // the group loop stays rolled (measured: mod p 1.3 % faster than unrolled
    // twice -- smaller code)
#pragma unroll 1
    for (int k1 = 0; k1 < C::BKG; k1 += FOLD) {
#pragma unroll
      for (int k2 = 0; k2 < FOLD; ++k2) {
        const int kk = k1 + k2;
        if (FOLD > 1 && kk >= C::BKG) break;
        Val a[TM], bv[TN];
        load_frag<TM>(Ag + kk * BM + ty * TM, a);
        load_frag<TN>(Bg + kk * BN + tx * TN, bv);
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) T::mac(acc[i][j], a[i], bv[j], mp);
      }
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) T::fold(acc[i][j], mp);
    }
    cur = (cur + 1) % kStages;
  }
  cp_async_wait<0>();
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Packed (max,+) tile for int32 tropical networks with small values.
// Every finite value of an independent-set network with unit vertex weights
// is the size of an independent set of a subgraph, an integer in [0, n].
// When the host proves |finite value| <= kPackedMax for the whole network,
// two terms run in one __viaddmax_s16x2 (max(a + b, c) on each 16-bit half)
// and the result is exact:
//   - a staged value v becomes max(v, kPackedNegInf): finite values are
//     unchanged, every "-inf" (any int32 below TN_I32_NEG_INF / 2) becomes
//     -16384;
//   - finite + finite lies in [-8190, 8190]; a sum with a -inf term lies in
//     [-32768, -12289], and the accumulator starts at -16384, so no half
//     ever leaves the int16 range and every accumulated "-inf" stays below
//     -8192 while every finite maximum stays at or above -8190;
//   - the epilogue maps halves below -8192 back to TN_I32_NEG_INF.
// A's staged value a is stored as the pair (a, a) and B's values as pairs
// (b[n], b[n + 1]), so one instruction updates the two outputs (m, n) and
// (m, n + 1).  The chunk is staged as int32 by the same cp.async path as the
// int32 tile; each thread converts the entries it copied itself (its own
// copies are complete after its cp.async wait), so the chunk still needs a
// single barrier.  Two packed buffers alternate: the one converted at
// iteration t + 2 was last read before the barrier of iteration t + 1.
// ---------------------------------------------------------------------------
constexpr int32_t kPackedMax = 4095;        // largest |finite value| the packed tile accepts
constexpr int32_t kPackedNegInf = -16384;   // "-inf" in a 16-bit half
constexpr int32_t kPackedInfBelow = -8192;  // halves below this are "-inf"
constexpr int kPackedI16 = 16;              // FOLD argument selecting the packed tile of SrI32

__device__ __forceinline__ uint32_t pk_bcast(int32_t v) {
  return __byte_perm(static_cast<uint32_t>(max(v, kPackedNegInf)), 0u, 0x1010);
}
__device__ __forceinline__ uint32_t pk_pair(int32_t lo, int32_t hi) {
  return __byte_perm(static_cast<uint32_t>(max(lo, kPackedNegInf)), static_cast<uint32_t>(max(hi, kPackedNegInf)),
                     0x5410);
}
__device__ __forceinline__ int32_t pk_unpack(int32_t h) { return h < kPackedInfBelow ? kNegInf : h; }

template <class C>
struct TileSmemP {
  static constexpr int kSt = 3;
  TileIdx<C> idx;
  alignas(16) int32_t As[kSt][C::BK * C::BM];        // int32 staging
  alignas(16) int32_t Bs[kSt][C::BK * C::BN];
  alignas(16) uint32_t Ap[2][C::BK * C::BM];         // (a, a) pairs
  alignas(16) uint32_t Bp[2][C::BK * C::BN / 2];     // (b[n], b[n + 1]) pairs
};

// Converts this thread's staged entries of one chunk (those it copied or
// generated itself) into the packed buffers ap / bp.
template <class C, int NSA, int NSB>
__device__ __forceinline__ void tile_pack(const int32_t* as, const int32_t* bs, uint32_t* ap, uint32_t* bp,
                                          const int32_t (&offA)[C::EA], const int32_t (&offB)[C::EB], bool va,
                                          bool vb) {
  const int tid = threadIdx.x;
  if (va) {
#pragma unroll
    for (int j = 0; j < NSA; ++j)
      if (offA[j] >= 0) {
        const int e = 4 * (tid + kBlock * j);
        const int4 v = *reinterpret_cast<const int4*>(as + e);
        *reinterpret_cast<uint4*>(ap + e) = make_uint4(pk_bcast(v.x), pk_bcast(v.y), pk_bcast(v.z), pk_bcast(v.w));
      }
  } else {
#pragma unroll
    for (int j = 0; j < C::EA; ++j)
      if (offA[j] >= 0) ap[tid + kBlock * j] = pk_bcast(as[tid + kBlock * j]);
  }
  if (vb) {
#pragma unroll
    for (int j = 0; j < NSB; ++j)
      if (offB[j] >= 0) {
        const int e = 4 * (tid + kBlock * j);
        const int4 v = *reinterpret_cast<const int4*>(bs + e);
        *reinterpret_cast<uint2*>(bp + e / 2) = make_uint2(pk_pair(v.x, v.y), pk_pair(v.z, v.w));
      }
  } else {
    int16_t* bh = reinterpret_cast<int16_t*>(bp);
#pragma unroll
    for (int j = 0; j < C::EB; ++j)
      if (offB[j] >= 0) bh[tid + kBlock * j] = static_cast<int16_t>(max(bs[tid + kBlock * j], kPackedNegInf));
  }
}

// The packed counterpart of tile_mainloop for SrI32 (see above); acc
// receives int32 values (-inf as TN_I32_NEG_INF) of the calling thread's
// group, like tile_mainloop's.  All threads of the CTA must call it.
template <class C, bool CG>
__device__ __forceinline__ void tile_mainloop_packed(const StepGeom& g, const Operand& A, const Operand& B, int64_t b,
                                                     int64_t tm, int64_t tn_, int64_t kbeg, int64_t kend,
                                                     TileSmemP<C>& sm, int32_t (&acc)[C::TM][C::TN],
                                                     bool ready = false, int vec = 0) {
  constexpr int kStages = TileSmemP<C>::kSt;
  constexpr int BM = C::BM, BN = C::BN, BK = C::BK, TM = C::TM, TN = C::TN, TN2 = C::TN / 2;
  static_assert(TN % 2 == 0 && BN % 2 == 0, "pairs of columns");
  const int tid = threadIdx.x;
  const int grp = tid / C::GT, gt = tid % C::GT;
  const int tx = gt % C::WN, ty = gt / C::WN;

  int32_t offA[C::EA], offB[C::EB];
  tile_offsets<C>(g, sm.idx, b, tm, tn_, offA, offB, ready);
  constexpr int NSA = VecSlots<BM, BK * BM>::per_thread, NSB = VecSlots<BN, BK * BN>::per_thread;
  static_assert(NSA <= C::EA && NSB <= C::EB, "a 16-byte slot covers four staged elements");
  const bool va = (vec & kVecA) && A.kind == kOpArena;
  const bool vb = (vec & kVecB) && B.kind == kOpArena;

  // padding entries (outside M / N / K) are -inf in every staging and
  // packed buffer; nothing writes them afterwards
#pragma unroll
  for (int j = 0; j < C::EA; ++j)
    if (offA[j] < 0) {
      const int e = tid + kBlock * j;
      for (int st = 0; st < kStages; ++st) sm.As[st][e] = kNegInf;
      sm.Ap[0][e] = sm.Ap[1][e] = pk_bcast(kNegInf);
    }
#pragma unroll
  for (int j = 0; j < C::EB; ++j)
    if (offB[j] < 0) {
      const int e = tid + kBlock * j;
      for (int st = 0; st < kStages; ++st) sm.Bs[st][e] = kNegInf;
      reinterpret_cast<int16_t*>(sm.Bp[0])[e] = static_cast<int16_t>(kPackedNegInf);
      reinterpret_cast<int16_t*>(sm.Bp[1])[e] = static_cast<int16_t>(kPackedNegInf);
    }
  {
    const uint32_t K = 1u << g.nk, kvalid = K < BK ? K : BK;
    if (va) tile_slots4<BM, BK, NSA>(sm.idx.offAm, sm.idx.offAk, static_cast<uint32_t>(tm) * BM, 1u << g.nm, kvalid, offA);
    if (vb) tile_slots4<BN, BK, NSB>(sm.idx.offBn, sm.idx.offBk, static_cast<uint32_t>(tn_) * BN, 1u << g.nn, kvalid, offB);
  }

  uint32_t acc2[TM][TN2];
  const uint32_t ninf2 = pk_bcast(kNegInf);
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN2; ++j) acc2[i][j] = ninf2;

  auto issue = [&](int st, int64_t k0) {
    tile_stage<SrI32, C, CG, NSA, NSB>(g, sm.idx, A, B, offA, offB, va, vb, sm.As[st], sm.Bs[st], k0);
  };
#pragma unroll
  for (int st = 0; st < kStages - 1; ++st) {
    if (kbeg + st * BK < kend) issue(st, kbeg + st * BK);
    cp_async_commit();
  }
  int cur = 0, pb = 0;
  for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
    cp_async_wait<kStages - 2>();
    tile_pack<C, NSA, NSB>(sm.As[cur], sm.Bs[cur], sm.Ap[pb], sm.Bp[pb], offA, offB, va, vb);
    __syncthreads();
    {
      // refill the staging buffer this thread converted in the previous
      // iteration (only its own entries: no other thread reads them)
      const int64_t kn = k0 + (kStages - 1) * BK;
      const int nxt = (cur + kStages - 1) % kStages;
      if (kn < kend) issue(nxt, kn);
      cp_async_commit();
    }
    const uint32_t* Ag = sm.Ap[pb] + grp * C::BKG * BM;
    const uint32_t* Bg = sm.Bp[pb] + grp * C::BKG * (BN / 2);
#pragma unroll 2
    for (int kk = 0; kk < C::BKG; ++kk) {
      uint32_t a[TM], bv[TN2];
      load_frag<TM>(Ag + kk * BM + ty * TM, a);
      load_frag<TN2>(Bg + kk * (BN / 2) + tx * TN2, bv);
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN2; ++j) acc2[i][j] = __viaddmax_s16x2(a[i], bv[j], acc2[i][j]);
    }
    cur = (cur + 1) % kStages;
    pb ^= 1;
  }
  cp_async_wait<0>();
  __syncthreads();
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN2; ++j) {
      acc[i][2 * j] = pk_unpack(static_cast<int32_t>(acc2[i][j] << 16) >> 16);
      acc[i][2 * j + 1] = pk_unpack(static_cast<int32_t>(acc2[i][j]) >> 16);
    }
}

// Merges the KG partial tiles into group 0 (through shared memory `red`,
// KG-1 tiles of BM x BN accumulators).  Afterwards the threads of group 0
// hold the CTA's tile.  All threads must call it.
template <class SR, class C>
__device__ __forceinline__ void tile_merge_groups(typename SR::Acc (&acc)[C::TM][C::TN],
                                                  typename SR::Acc* red, const ModParams& mp) {
  if constexpr (C::KG > 1) {
    const int tid = threadIdx.x;
    const int grp = tid / C::GT, gt = tid % C::GT;
    const int tx = gt % C::WN, ty = gt / C::WN;
    if (grp > 0) {
#pragma unroll
      for (int i = 0; i < C::TM; ++i)
#pragma unroll
        for (int j = 0; j < C::TN; ++j)
          red[(grp - 1) * C::BM * C::BN + (ty * C::TM + i) * C::BN + tx * C::TN + j] = acc[i][j];
    }
    __syncthreads();
    if (grp == 0) {
      for (int r = 0; r < C::KG - 1; ++r)
#pragma unroll
        for (int i = 0; i < C::TM; ++i)
#pragma unroll
          for (int j = 0; j < C::TN; ++j)
            SR::merge(acc[i][j], red[r * C::BM * C::BN + (ty * C::TM + i) * C::BN + tx * C::TN + j], mp);
    }
    __syncthreads();
  }
}

template <class C>
struct TileSmemCnt;

// Byte offset of the group-merge buffer of tile_merge_groups: after the
// index tables, which therefore survive a tile (the next tile of the same
// step reuses its gather tables).
template <class C>
constexpr size_t tile_merge_off() {
  return (sizeof(TileIdx<C>) + 15) / 16 * 16;
}

// Shared memory a tile needs: index tables and staging, or index tables
// and the group-merge buffer.
template <class SR, class C>
constexpr size_t tile_smem_bytes() {
  size_t stage = sizeof(TileSmem<SR, C>);
  if constexpr (std::is_same<SR, SrCnt>::value)
    stage = sizeof(TileSmemCnt<C>) > sizeof(TileSmem<SrI32, C>) ? sizeof(TileSmemCnt<C>) : sizeof(TileSmem<SrI32, C>);
  const size_t merge = tile_merge_off<C>() + sizeof(typename SR::Acc) * (C::KG - 1) * C::BM * C::BN;
  return stage > merge ? stage : merge;
}

// The same for the packed (max,+) tile.
template <class C>
constexpr size_t tile_smem_bytes_packed() {
  const size_t merge = tile_merge_off<C>() + sizeof(int32_t) * (C::KG - 1) * C::BM * C::BN;
  return sizeof(TileSmemP<C>) > merge ? sizeof(TileSmemP<C>) : merge;
}

}  // namespace dev
}  // namespace tn

namespace tn {
namespace dev {

// ---------------------------------------------------------------------------
// Counting tropical (CountingMax of Sec. 5.3) over a tile, chunk by chunk.
// Every staged chunk of k rows (values and counts, staged once) is read
// twice from shared memory:
//   1. the chunk's (max,+) tile of the values alone, m_c = max_k a.v + b.v;
//      where m_c exceeds the running maximum the entry takes it and its count
//      restarts from 0;
//   2. count += a.c * b.c over the chunk's terms whose a.v + b.v equals the
//      running maximum (only chunks whose maximum reached it have any).
// The result equals the single pass with SrCnt::mac: counts are exact sums
// of products over the maximising terms, saturated at 2^64 - 1.  A chunk
// whose staged counts are all < 2^16 and whose accumulators are < 2^62 takes
// one predicated 64-bit multiply-add per term (no carry can leave 64 bits);
// other chunks use exact 64-bit products where counts are < 2^32 and
// saturating 64 x 64 products otherwise, with saturating additions.
// ---------------------------------------------------------------------------

// c += a * b when s == vmax (64-bit multiply-add; the caller guarantees that
// the sum stays below 2^64)
__device__ __forceinline__ void cnt_fma_wide(uint64_t& c, int32_t s, int32_t vmax, uint32_t a, uint32_t b) {
  asm("{\n\t.reg .pred p;\n\t"
      "setp.eq.s32 p, %1, %2;\n\t"
      "@p mad.wide.u32 %0, %3, %4, %0;\n\t}"
      : "+l"(c)
      : "r"(s), "r"(vmax), "r"(a), "r"(b));
}

// Low 32 bits of T consecutive uint64 counts in shared memory (16-byte loads).
template <int T>
__device__ __forceinline__ void load_lo_frag(const uint64_t* p, uint32_t (&out)[T]) {
  static_assert(T % 2 == 0, "pairs of counts");
#pragma unroll
  for (int i = 0; i < T; i += 2) {
    const uint4 w = *reinterpret_cast<const uint4*>(p + i);
    out[i] = w.x;
    out[i + 1] = w.z;
  }
}

// Shared memory of the counting tile: values and counts of each staged
// chunk in separate arrays.
template <class C>
struct TileSmemCnt {
  static constexpr int kSt = Stages<SrCnt>::v;
  TileIdx<C> idx;
  alignas(16) int32_t Av[kSt][C::BK * C::BM];
  alignas(16) int32_t Bv[kSt][C::BK * C::BN];
  alignas(16) uint64_t Ac[kSt][C::BK * C::BM];
  alignas(16) uint64_t Bc[kSt][C::BK * C::BN];
};

// ---------------------------------------------------------------------------
// Packed counting tile: the (max, count) tile of tile_mainloop_counting with
// the values of two terms in one register, as IEEE half precision.  Integers
// up to 2048 in magnitude are exact in binary16, so when the host proves
// |finite value| <= kPackedCntMax for the network (unit-weight networks with
// n <= 1024), every sum a + b of two finite values is exact and "-inf" is
// the half -inf (-inf + x = -inf; the counts of -inf entries are 0, so a
// -inf term that compares equal adds a zero product).  Per pair of terms:
//   first pass   add.f16x2 and max.f16x2 (the chunk's maxima);
//   second pass  add.f16x2, one setp.eq.f16x2 that sets a predicate per
//                half, and a predicated 64-bit multiply-add per term
// -- 2 instructions per counted term instead of 3, and half the value
// registers.  Values are staged as int32 exactly as in the unpacked tile;
// each thread converts the entries it copied itself into (a, a) and
// (b[n], b[n + 1]) half pairs (two buffers alternate, as in the packed
// (max,+) tile).  Counts, the slow path and the results are unchanged.
// ---------------------------------------------------------------------------
constexpr int32_t kPackedCntMax = 1024;  // largest |finite value| of the packed counting tile

__device__ __forceinline__ uint32_t h16_of(int32_t v) {
  return v < kNegInf / 2 ? 0xFC00u : static_cast<uint32_t>(__half_as_ushort(__int2half_rn(v)));
}
__device__ __forceinline__ int32_t i32_of_h16(uint32_t h) {
  return (h & 0xFFFFu) == 0xFC00u ? kNegInf : __half2int_rn(__ushort_as_half(static_cast<unsigned short>(h)));
}

template <class C>
struct TileSmemCntP {
  static constexpr int kSt = Stages<SrCnt>::v;
  TileIdx<C> idx;
  alignas(16) int32_t Av[kSt][C::BK * C::BM];
  alignas(16) int32_t Bv[kSt][C::BK * C::BN];
  alignas(16) uint64_t Ac[kSt][C::BK * C::BM];
  alignas(16) uint64_t Bc[kSt][C::BK * C::BN];
  alignas(16) uint32_t Ah[2][C::BK * C::BM];      // (a, a) half pairs
  alignas(16) uint32_t Bh[2][C::BK * C::BN / 2];  // (b[n], b[n + 1]) half pairs
};

template <class C>
constexpr size_t tile_smem_bytes_cnt_packed() {
  const size_t merge = tile_merge_off<C>() + sizeof(CntVal) * (C::KG - 1) * C::BM * C::BN;
  return sizeof(TileSmemCntP<C>) > merge ? sizeof(TileSmemCntP<C>) : merge;
}

// This thread's staged values of one chunk (those it copied or generated) as
// half pairs.
template <class C, int NSA, int NSB>
__device__ __forceinline__ void tile_pack_h16(const int32_t* as, const int32_t* bs, uint32_t* ah, uint32_t* bh,
                                              const int32_t (&offA)[C::EA], const int32_t (&offB)[C::EB], bool va,
                                              bool vb) {
  const int tid = threadIdx.x;
  if (va) {
#pragma unroll
    for (int j = 0; j < NSA; ++j)
      if (offA[j] >= 0) {
        const int e = 4 * (tid + kBlock * j);
        const int4 v = *reinterpret_cast<const int4*>(as + e);
        *reinterpret_cast<uint4*>(ah + e) =
            make_uint4(h16_of(v.x) * 0x10001u, h16_of(v.y) * 0x10001u, h16_of(v.z) * 0x10001u, h16_of(v.w) * 0x10001u);
      }
  } else {
#pragma unroll
    for (int j = 0; j < C::EA; ++j)
      if (offA[j] >= 0) ah[tid + kBlock * j] = h16_of(as[tid + kBlock * j]) * 0x10001u;
  }
  if (vb) {
#pragma unroll
    for (int j = 0; j < NSB; ++j)
      if (offB[j] >= 0) {
        const int e = 4 * (tid + kBlock * j);
        const int4 v = *reinterpret_cast<const int4*>(bs + e);
        *reinterpret_cast<uint2*>(bh + e / 2) =
            make_uint2(h16_of(v.x) | (h16_of(v.y) << 16), h16_of(v.z) | (h16_of(v.w) << 16));
      }
  } else {
    unsigned short* b16 = reinterpret_cast<unsigned short*>(bh);
#pragma unroll
    for (int j = 0; j < C::EB; ++j)
      if (offB[j] >= 0) b16[tid + kBlock * j] = static_cast<unsigned short>(h16_of(bs[tid + kBlock * j]));
  }
}

// mc = max(a + b, mc) on both halves
__device__ __forceinline__ void h2_addmax(uint32_t& mc, uint32_t a, uint32_t b) {
  asm("{\n\t.reg .b32 s;\n\tadd.rn.f16x2 s, %1, %2;\n\tmax.f16x2 %0, %0, s;\n\t}" : "+r"(mc) : "r"(a), "r"(b));
}
// a larger chunk maximum restarts the entry's count; vmax = max(vmax, mc)
__device__ __forceinline__ void h2_raise(uint32_t& vmax, uint32_t mc, uint64_t& c0, uint64_t& c1) {
  asm("{\n\t.reg .pred p, q;\n\tsetp.gt.f16x2 p|q, %3, %2;\n\t@p mov.b64 %0, 0;\n\t@q mov.b64 %1, 0;\n\t}"
      : "+l"(c0), "+l"(c1)
      : "r"(vmax), "r"(mc));
  asm("max.f16x2 %0, %0, %1;" : "+r"(vmax) : "r"(mc));
}
// c0 += ac * bc0 where a + b reaches vmax in the low half, c1 += ac * bc1 in
// the high half (64-bit multiply-adds; the caller guarantees no overflow)
__device__ __forceinline__ void h2_count(uint64_t& c0, uint64_t& c1, uint32_t a, uint32_t b, uint32_t vmax,
                                         uint32_t ac, uint32_t bc0, uint32_t bc1) {
  asm("{\n\t.reg .pred p, q;\n\t.reg .b32 s;\n\tadd.rn.f16x2 s, %2, %3;\n\tsetp.eq.f16x2 p|q, s, %4;\n\t"
      "@p mad.wide.u32 %0, %5, %6, %0;\n\t@q mad.wide.u32 %1, %5, %7, %1;\n\t}"
      : "+l"(c0), "+l"(c1)
      : "r"(a), "r"(b), "r"(vmax), "r"(ac), "r"(bc0), "r"(bc1));
}

template <class C, bool CG, bool Packed = false>
__device__ __forceinline__ void tile_mainloop_counting(const StepGeom& g, const Operand& A, const Operand& B,
                                                       const ModParams& mp, int64_t b, int64_t tm, int64_t tn_,
                                                       int64_t kbeg, int64_t kend, unsigned char* smem_raw,
                                                       CntVal (&acc)[C::TM][C::TN], bool ready = false,
                                                       int vec = 0) {
  constexpr int BM = C::BM, BN = C::BN, BK = C::BK, TM = C::TM, TN = C::TN;
  constexpr int kSt = Stages<SrCnt>::v;
  constexpr int NSA = VecSlots<BM, BK * BM>::per_thread, NSB = VecSlots<BN, BK * BN>::per_thread;
  static_assert(NSA <= C::EA && NSB <= C::EB, "a 16-byte slot covers four staged elements");
  const bool va = (vec & kVecA) && A.kind == kOpArena, vb = (vec & kVecB) && B.kind == kOpArena;
  // the packed layout extends the unpacked one (same leading members)
  auto& sm = *reinterpret_cast<TileSmemCntP<C>*>(smem_raw);
  const int tid = threadIdx.x;
  const int grp = tid / C::GT, gt = tid % C::GT;
  const int tx = gt % C::WN, ty = gt / C::WN;
  int32_t offA[C::EA], offB[C::EB];
  tile_offsets<C>(g, sm.idx, b, tm, tn_, offA, offB, ready);
  // padding slots (outside M / N / K) hold the semiring zero (-inf, 0)
#pragma unroll
  for (int j = 0; j < C::EA; ++j)
    if (offA[j] < 0)
      for (int st = 0; st < kSt; ++st) {
        sm.Av[st][tid + kBlock * j] = kNegInf;
        sm.Ac[st][tid + kBlock * j] = 0ull;
      }
#pragma unroll
  for (int j = 0; j < C::EA; ++j)
    if (Packed && offA[j] < 0) sm.Ah[0][tid + kBlock * j] = sm.Ah[1][tid + kBlock * j] = 0xFC00FC00u;
#pragma unroll
  for (int j = 0; j < C::EB; ++j)
    if (offB[j] < 0)
      for (int st = 0; st < kSt; ++st) {
        sm.Bv[st][tid + kBlock * j] = kNegInf;
        sm.Bc[st][tid + kBlock * j] = 0ull;
      }
#pragma unroll
  for (int j = 0; j < C::EB; ++j)
    if (Packed && offB[j] < 0) {
      reinterpret_cast<unsigned short*>(sm.Bh[0])[tid + kBlock * j] = 0xFC00u;
      reinterpret_cast<unsigned short*>(sm.Bh[1])[tid + kBlock * j] = 0xFC00u;
    }
  {
    // 16-byte slots (see tile_mainloop): four values, and four counts in two
    // 16-byte halves
    const uint32_t K = 1u << g.nk, kvalid = K < BK ? K : BK;
    if (va) tile_slots4<BM, BK, NSA>(sm.idx.offAm, sm.idx.offAk, static_cast<uint32_t>(tm) * BM, 1u << g.nm, kvalid, offA);
    if (vb) tile_slots4<BN, BK, NSB>(sm.idx.offBn, sm.idx.offBk, static_cast<uint32_t>(tn_) * BN, 1u << g.nn, kvalid, offB);
  }

  int32_t vmax[TM][TN];           // running maxima (unpacked)
  uint32_t vmax2[TM][TN / 2];     // running maxima as half pairs (packed)
  uint64_t cnt[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      vmax[i][j] = kNegInf;
      if (j % 2 == 0) vmax2[i][j / 2] = 0xFC00FC00u;
      cnt[i][j] = 0ull;
    }
  int pb = 0;  // packed buffer of the current chunk

  const bool a_async = A.kind == kOpArena, b_async = B.kind == kOpArena;
  auto issue = [&](int st, int64_t k0) {
    const uint2 kb = tile_chunk_base<C>(g, sm.idx, k0);
    if (va) {
#pragma unroll
      for (int j = 0; j < NSA; ++j)
        if (offA[j] >= 0) {
          const uint32_t e = static_cast<uint32_t>(offA[j]) + kb.x;
          const int d = 4 * (tid + kBlock * j);
          cp_async16(&sm.Av[st][d], static_cast<const int32_t*>(A.p0) + e);
          cp_async16(&sm.Ac[st][d], static_cast<const uint64_t*>(A.p1) + e);
          cp_async16(&sm.Ac[st][d + 2], static_cast<const uint64_t*>(A.p1) + e + 2);
        }
    }
#pragma unroll
    for (int j = 0; j < C::EA; ++j)
      if (!va && offA[j] >= 0) {
        const uint32_t e = static_cast<uint32_t>(offA[j]) + kb.x;
        if (a_async) {
          cp_async4(&sm.Av[st][tid + kBlock * j], static_cast<const int32_t*>(A.p0) + e);
          cp_async8(&sm.Ac[st][tid + kBlock * j], static_cast<const uint64_t*>(A.p1) + e);
        } else {
          const CntVal v = SrCnt::template load<CG>(A, e);
          sm.Av[st][tid + kBlock * j] = v.v;
          sm.Ac[st][tid + kBlock * j] = v.c;
        }
      }
    if (vb) {
#pragma unroll
      for (int j = 0; j < NSB; ++j)
        if (offB[j] >= 0) {
          const uint32_t e = static_cast<uint32_t>(offB[j]) + kb.y;
          const int d = 4 * (tid + kBlock * j);
          cp_async16(&sm.Bv[st][d], static_cast<const int32_t*>(B.p0) + e);
          cp_async16(&sm.Bc[st][d], static_cast<const uint64_t*>(B.p1) + e);
          cp_async16(&sm.Bc[st][d + 2], static_cast<const uint64_t*>(B.p1) + e + 2);
        }
    }
#pragma unroll
    for (int j = 0; j < C::EB; ++j)
      if (!vb && offB[j] >= 0) {
        const uint32_t e = static_cast<uint32_t>(offB[j]) + kb.y;
        if (b_async) {
          cp_async4(&sm.Bv[st][tid + kBlock * j], static_cast<const int32_t*>(B.p0) + e);
          cp_async8(&sm.Bc[st][tid + kBlock * j], static_cast<const uint64_t*>(B.p1) + e);
        } else {
          const CntVal v = SrCnt::template load<CG>(B, e);
          sm.Bv[st][tid + kBlock * j] = v.v;
          sm.Bc[st][tid + kBlock * j] = v.c;
        }
      }
  };
#pragma unroll
  for (int st = 0; st < kSt - 1; ++st) {
    if (kbeg + st * BK < kend) issue(st, kbeg + st * BK);
    cp_async_commit();
  }
  int cur = 0;
  for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
    cp_async_wait<kSt - 2>();
    if constexpr (Packed) tile_pack_h16<C, NSA, NSB>(sm.Av[cur], sm.Bv[cur], sm.Ah[pb], sm.Bh[pb], offA, offB, va, vb);
    // this thread's own copies of the chunk are complete: the chunk is fast
    // when every staged count is < 2^16 and every accumulator < 2^62 (16
    // products < 2^32 cannot carry out of 64 bits); the barrier publishes the
    // chunk to the CTA
    uint64_t hi = 0;
#pragma unroll
    for (int j = 0; j < C::EA; ++j) hi |= sm.Ac[cur][tid + kBlock * j];
#pragma unroll
    for (int j = 0; j < C::EB; ++j) hi |= sm.Bc[cur][tid + kBlock * j];
    uint64_t big = 0;
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) big |= cnt[i][j] >> 62;
    const bool slow = __syncthreads_or((hi >> 16) != 0 || big != 0) != 0;
    {
      const int64_t kn = k0 + (kSt - 1) * BK;
      const int nxt = (cur + kSt - 1) % kSt;
      if (kn < kend) issue(nxt, kn);
      cp_async_commit();
    }
    const int32_t* Agv = sm.Av[cur] + grp * C::BKG * BM;
    const int32_t* Bgv = sm.Bv[cur] + grp * C::BKG * BN;
    const uint64_t* Agc = sm.Ac[cur] + grp * C::BKG * BM;
    const uint64_t* Bgc = sm.Bc[cur] + grp * C::BKG * BN;
    const uint32_t* Agh = sm.Ah[pb] + grp * C::BKG * BM;
    const uint32_t* Bgh = sm.Bh[pb] + grp * C::BKG * (BN / 2);
    if constexpr (Packed) {
      // 1: the chunk's maxima on half pairs; a larger maximum restarts the
      // entry's count
      uint32_t mc2[TM][TN / 2];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN / 2; ++j) mc2[i][j] = 0xFC00FC00u;
#pragma unroll 8
      for (int kk = 0; kk < C::BKG; ++kk) {
        uint32_t ah[TM], bh[TN / 2];
        load_frag<TM>(Agh + kk * BM + ty * TM, ah);
        load_frag<TN / 2>(Bgh + kk * (BN / 2) + tx * (TN / 2), bh);
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN / 2; ++j) h2_addmax(mc2[i][j], ah[i], bh[j]);
      }
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN / 2; ++j) h2_raise(vmax2[i][j], mc2[i][j], cnt[i][2 * j], cnt[i][2 * j + 1]);
    } else {
      // 1: the chunk's maxima; a larger maximum restarts the entry's count
      int32_t mc[TM][TN];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) mc[i][j] = kNegInf;
#pragma unroll 4
      for (int kk = 0; kk < C::BKG; ++kk) {
        int32_t av[TM], bv[TN];
        load_frag<TM>(Agv + kk * BM + ty * TM, av);
        load_frag<TN>(Bgv + kk * BN + tx * TN, bv);
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) mc[i][j] = __viaddmax_s32(av[i], bv[j], mc[i][j]);
      }
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j)
          if (mc[i][j] > vmax[i][j]) {
            vmax[i][j] = mc[i][j];
            cnt[i][j] = 0ull;
          }
    }
    // 2: counts of the chunk's terms that reach the running maximum
    if (Packed && !slow) {
#pragma unroll 2
      for (int kk = 0; kk < C::BKG; ++kk) {
        uint32_t ah[TM], bh[TN / 2], ac[TM], bc[TN];
        load_frag<TM>(Agh + kk * BM + ty * TM, ah);
        load_frag<TN / 2>(Bgh + kk * (BN / 2) + tx * (TN / 2), bh);
        load_lo_frag<TM>(Agc + kk * BM + ty * TM, ac);
        load_lo_frag<TN>(Bgc + kk * BN + tx * TN, bc);
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN / 2; ++j)
            h2_count(cnt[i][2 * j], cnt[i][2 * j + 1], ah[i], bh[j], vmax2[i][j], ac[i], bc[2 * j], bc[2 * j + 1]);
      }
    } else if (!slow) {
#pragma unroll 2
      for (int kk = 0; kk < C::BKG; ++kk) {
        int32_t av[TM], bv[TN];
        uint32_t ac[TM], bc[TN];
        load_frag<TM>(Agv + kk * BM + ty * TM, av);
        load_frag<TN>(Bgv + kk * BN + tx * TN, bv);
        load_lo_frag<TM>(Agc + kk * BM + ty * TM, ac);
        load_lo_frag<TN>(Bgc + kk * BN + tx * TN, bc);
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) cnt_fma_wide(cnt[i][j], av[i] + bv[j], vmax[i][j], ac[i], bc[j]);
      }
    } else {
      for (int kk = 0; kk < C::BKG; ++kk) {
#pragma unroll
        for (int i = 0; i < TM; ++i) {
          const int32_t av = Agv[kk * BM + ty * TM + i];
          const uint64_t ac = Agc[kk * BM + ty * TM + i];
#pragma unroll
          for (int j = 0; j < TN; ++j)
            if (av + Bgv[kk * BN + tx * TN + j] ==
                (Packed ? i32_of_h16(vmax2[i][j / 2] >> (16 * (j % 2))) : vmax[i][j]))
              cnt[i][j] = sat_add_u64(cnt[i][j], sat_mul_u64(ac, Bgc[kk * BN + tx * TN + j]));
        }
      }
    }
    cur = (cur + 1) % kSt;
    pb ^= 1;
  }
  cp_async_wait<0>();
  __syncthreads();
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      acc[i][j].v = Packed ? i32_of_h16(vmax2[i][j / 2] >> (16 * (j % 2))) : vmax[i][j];
      acc[i][j].c = cnt[i][j];
    }
}

}  // namespace dev
}  // namespace tn
