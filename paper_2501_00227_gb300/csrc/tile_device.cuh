// tile_device.cuh -- the register-blocked semiring GEMM tile shared by the
// per-step tiled kernel and the persistent executor.
//
//   C[b, m, n] = (+)_k A[b, m, k] (x) B[b, k, n]   (Sec. 4.1 of arXiv:2501.00227)
//
// A CTA computes a BM x BN output tile (BM = 16 TM, BN = 16 TN) for one batch
// index; each of its 256 threads owns a TM x TN micro-tile in registers; k
// advances in chunks of BK staged in shared memory (A as [k][m], B as
// [k][n]).  Operands are read in place through bit-position maps: the offset
// of A[b, m, k] is dep_b(b) + dep_m(m) + dep_k(k); the tile covers the low
// bits of m, n and k, so in-tile offsets come from small shared tables and
// each tile adds one base.
#pragma once

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

template <class SR, int TM, int TN, int BK>
struct TileSmem {
  static constexpr int BM = 16 * TM, BN = 16 * TN;
  typename SR::Val As[BK * BM];
  typename SR::Val Bs[BK * BN];
  int64_t offAm[BM];
  int64_t offBn[BN];
  int64_t offAk[BK];
  int64_t offBk[BK];
};

// Accumulates the tile (tm, tn) of batch b over k in [kbeg, kend) into acc.
// FOLD: products accumulated between two folds of a mod-p accumulator
// (1 is safe for every p < 2^31; 3 needs 2^32 mod p < 2^20).  All threads of
// the CTA must call it.
template <class SR, int TM, int TN, int BK, int FOLD, bool CG>
__device__ __forceinline__ void tile_mainloop(const StepGeom& g, const Operand& A, const Operand& B,
                                              const ModParams& mp, int q, int64_t b, int64_t tm,
                                              int64_t tn_, int64_t kbeg, int64_t kend,
                                              TileSmem<SR, TM, TN, BK>& sm,
                                              typename SR::Acc (&acc)[TM][TN]) {
  constexpr int BM = 16 * TM, BN = 16 * TN;
  using Val = typename SR::Val;
  using T = Tiled<SR>;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t M = int64_t(1) << g.nm, N = int64_t(1) << g.nn, K = int64_t(1) << g.nk;
  const int64_t m0 = tm * BM, n0 = tn_ * BN;
  const int a_k0 = g.nb + g.nm, b_k0 = g.nb, b_n0 = g.nb + g.nk;
  constexpr int lbm = (BM >= 128) ? 7 : (BM >= 64 ? 6 : (BM >= 32 ? 5 : 4));
  constexpr int lbn = (BN >= 128) ? 7 : (BN >= 64 ? 6 : (BN >= 32 ? 5 : 4));
  constexpr int lbk = (BK >= 32) ? 5 : (BK >= 16 ? 4 : 3);
  for (int i = tid; i < BM; i += kBlock) sm.offAm[i] = deposit(i, g.a_pos, g.nb, min(lbm, g.nm));
  for (int i = tid; i < BN; i += kBlock) sm.offBn[i] = deposit(i, g.b_pos, b_n0, min(lbn, g.nn));
  for (int i = tid; i < BK; i += kBlock) {
    sm.offAk[i] = deposit(i, g.a_pos, a_k0, min(lbk, g.nk));
    sm.offBk[i] = deposit(i, g.b_pos, b_k0, min(lbk, g.nk));
  }
  const int64_t baseA = deposit(b, g.a_pos, 0, g.nb) +
                        (g.nm > lbm ? deposit(m0 >> lbm, g.a_pos, g.nb + lbm, g.nm - lbm) : 0);
  const int64_t baseB = deposit(b, g.b_pos, 0, g.nb) +
                        (g.nn > lbn ? deposit(n0 >> lbn, g.b_pos, b_n0 + lbn, g.nn - lbn) : 0);
  __syncthreads();

#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = SR::zero(mp);

  for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
    const int64_t kbaseA = g.nk > lbk ? deposit(k0 >> lbk, g.a_pos, a_k0 + lbk, g.nk - lbk) : 0;
    const int64_t kbaseB = g.nk > lbk ? deposit(k0 >> lbk, g.b_pos, b_k0 + lbk, g.nk - lbk) : 0;
#pragma unroll 4
    for (int e = tid; e < BK * BM; e += kBlock) {
      const int kk = e / BM, mm = e % BM;
      Val v = T::zero_val();
      if (m0 + mm < M && k0 + kk < K) v = SR::template load<CG>(A, baseA + sm.offAm[mm] + kbaseA + sm.offAk[kk], q);
      sm.As[kk * BM + mm] = v;
    }
#pragma unroll 4
    for (int e = tid; e < BK * BN; e += kBlock) {
      const int kk = e / BN, nn = e % BN;
      Val v = T::zero_val();
      if (n0 + nn < N && k0 + kk < K) v = SR::template load<CG>(B, baseB + sm.offBn[nn] + kbaseB + sm.offBk[kk], q);
      sm.Bs[kk * BN + nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      Val a[TM], bv[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = sm.As[kk * BM + ty * TM + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) bv[j] = sm.Bs[kk * BN + tx * TN + j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) T::mac(acc[i][j], a[i], bv[j], mp);
      if ((kk + 1) % FOLD == 0 || kk == BK - 1) {
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) T::fold(acc[i][j], mp);
      }
    }
    __syncthreads();
  }
}

}  // namespace dev
}  // namespace tn
