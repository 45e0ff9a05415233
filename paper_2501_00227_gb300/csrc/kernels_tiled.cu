// kernels_tiled.cu -- register-blocked semiring GEMM for the wide pairwise
// steps of a contraction (Sec. 4.1 of arXiv:2501.00227: a binary step is a
// matricised product; here the product is over a semiring).
//
//   C[b, m, n] = (+)_k A[b, m, k] (x) B[b, k, n]
//
// * Operands are read in place through bit-position maps (no permute pass):
//   the offset of A[b, m, k] is dep_b(b) + dep_m(m) + dep_k(k), each term a
//   scatter of the coordinate's bits to the operand's label positions.  A CTA
//   tile covers the low bits of m, n and k, so the per-tile offsets are small
//   tables in shared memory plus one base per tile.
// * A CTA computes a BM x BN output tile for one batch index; each of its 256
//   threads owns a TM x TN micro-tile held in registers; k advances in chunks
//   of BK staged through shared memory (A as [k][m], B as [k][n]).
// * Split-K: S CTAs of one thread-block cluster share an output tile, each
//   taking 1/S of the k range; the partial tiles are merged through
//   distributed shared memory (DSMEM) with the semiring (+), and each CTA of
//   the cluster writes 1/S of the tile.
#include <cooperative_groups.h>
#include <cstdlib>
#include <cuda_runtime.h>

#include "kernels.h"
#include "semiring.cuh"
#include "tile_device.cuh"

namespace cg = cooperative_groups;

namespace tn {
namespace dev {

struct TiledArgs {
  StepGeom g;
  Operand A, B;
  Output C;
  ModTable mods;
  int32_t split;      // CTAs per output tile (cluster size along x)
  int32_t tiles_m, tiles_n;
};

template <class SR, int TM, int TN, int BK, int FOLD>
__global__ void __launch_bounds__(kBlock) k_step_tiled(const __grid_constant__ TiledArgs args) {
  constexpr int BM = 16 * TM, BN = 16 * TN;
  using Acc = typename SR::Acc;
  extern __shared__ __align__(16) unsigned char smem[];
  auto& sm = *reinterpret_cast<TileSmem<SR, TM, TN, BK>*>(smem);
  const StepGeom& g = args.g;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int split = args.split;
  const int rank = static_cast<int>(blockIdx.x) % split;
  const int tile = static_cast<int>(blockIdx.x) / split;
  const int64_t tm = tile / args.tiles_n, tn_ = tile % args.tiles_n;
  const int64_t b = blockIdx.y;
  const int q = blockIdx.z;
  const ModParams mp = args.mods.q[q];
  const int64_t M = int64_t(1) << g.nm, N = int64_t(1) << g.nn, K = int64_t(1) << g.nk;
  const int64_t kspan = K >= split ? K / split : K;
  const int64_t kbeg = int64_t(rank) * kspan;

  Acc acc[TM][TN];
  tile_mainloop<SR, TM, TN, BK, FOLD, false>(g, args.A, args.B, mp, q, b, tm, tn_, kbeg, kbeg + kspan, sm, acc);

  const int64_t m0 = tm * BM, n0 = tn_ * BN;
  const int64_t cbase = b << (g.nn + g.nm);
  if (split == 1) {
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int64_t m = m0 + ty * TM + i;
      if (m >= M) continue;
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int64_t n = n0 + tx * TN + j;
        if (n < N) SR::store(args.C, cbase + (m << g.nn) + n, q, acc[i][j], mp);
      }
    }
    return;
  }

  // split-K: merge the partial tiles of the cluster through DSMEM
  cg::cluster_group cluster = cg::this_cluster();
  Acc* red = reinterpret_cast<Acc*>(smem);  // [BM][BN], reuses the staging buffers
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) red[(ty * TM + i) * BN + tx * TN + j] = acc[i][j];
  cluster.sync();
  const int per = BM * BN / split;
  for (int e = rank * per + tid; e < (rank + 1) * per; e += kBlock) {
    Acc v = red[e];
    for (int r = 0; r < split; ++r) {
      if (r == rank) continue;
      const Acc* peer = cluster.map_shared_rank(red, r);
      SR::merge(v, peer[e], mp);
    }
    const int64_t m = m0 + e / BN, n = n0 + e % BN;
    if (m < M && n < N) SR::store(args.C, cbase + (m << g.nn) + n, q, v, mp);
  }
  cluster.sync();
}

// --------------------------------------------------------------------------
// host side
// --------------------------------------------------------------------------
template <class SR, int TM, int TN, int BK, int FOLD>
static int launch_tiled_t(const TiledArgs& a, int nprimes, cudaStream_t st) {
  constexpr int BM = 16 * TM, BN = 16 * TN;
  using Acc = typename SR::Acc;
  size_t stage = sizeof(TileSmem<SR, TM, TN, BK>);
  size_t red = a.split > 1 ? sizeof(Acc) * BM * BN : 0;
  size_t smem = stage > red ? stage : red;
  auto kern = k_step_tiled<SR, TM, TN, BK, FOLD>;
  static bool attr_set = false;
  if (!attr_set) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) != cudaSuccess)
      return TN_ECUDA;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
      return TN_ECUDA;
    attr_set = true;
  }
  const int64_t batch = int64_t(1) << a.g.nb;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(a.tiles_m * a.tiles_n * a.split), static_cast<unsigned>(batch),
                     static_cast<unsigned>(nprimes));
  cfg.blockDim = dim3(256, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = static_cast<unsigned>(a.split);
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, kern, a);
  return e == cudaSuccess ? TN_OK : TN_ECUDA;
}

// Tile shapes (TM x TN micro-tiles on a 16 x 16 thread grid).
//   id 0: 128 x 128 (8 x 8), id 1: 64 x 64 (4 x 4)
int tiled_tile_bm(int tile) { return tile == 0 ? 128 : 64; }
int tiled_tile_bn(int tile) { return tile == 0 ? 128 : 64; }
int tiled_tile_bk(int) { return 16; }

int launch_step_tiled(tn_semiring_t s, const StepGeom& g, const Operand& A, const Operand& B,
                      const Output& C, const ModTable& mods, int nprimes, int tile, int split,
                      cudaStream_t st) {
  TiledArgs a;
  a.g = g;
  a.A = A;
  a.B = B;
  a.C = C;
  a.mods = mods;
  a.split = split;
  const int64_t M = int64_t(1) << g.nm, N = int64_t(1) << g.nn;
  const int bm = tiled_tile_bm(tile), bn = tiled_tile_bn(tile);
  a.tiles_m = static_cast<int32_t>((M + bm - 1) / bm);
  a.tiles_n = static_cast<int32_t>((N + bn - 1) / bn);
  switch (s) {
    case TN_TROPICAL_F32:
      return tile == 0 ? launch_tiled_t<SrF32, 8, 8, 16, 1>(a, 1, st)
                       : launch_tiled_t<SrF32, 4, 4, 16, 1>(a, 1, st);
    case TN_TROPICAL_I32:
      return tile == 0 ? launch_tiled_t<SrI32, 8, 8, 16, 1>(a, 1, st)
                       : launch_tiled_t<SrI32, 4, 4, 16, 1>(a, 1, st);
    case TN_COUNTING_TROPICAL:
      return launch_tiled_t<SrCnt, 4, 4, 16, 1>(a, 1, st);
    case TN_COUNT_MODP: {
      bool small_r = true;
      for (int i = 0; i < nprimes; ++i) small_r = small_r && mods.q[i].r32 < (1u << 20);
      return small_r ? launch_tiled_t<SrMod, 4, 4, 16, 3>(a, nprimes, st)
                     : launch_tiled_t<SrMod, 4, 4, 16, 1>(a, nprimes, st);
    }
  }
  return TN_EINVAL;
}

// Heuristic kernel choice (see the step-kernel table in the design notes):
// the tiled GEMM needs some reduction depth (nk >= 2), tiles that are not
// mostly empty (nm, nn >= 3), a batch that fits gridDim.y and enough work to
// beat the general kernel.  Split-K doubles until two waves of CTAs are
// resident or the k range per CTA would drop below one BK chunk.
// TN_KERNEL=naive|tiled in the environment forces one path (tests).
void pick_launch(const StepGeom& g, tn_semiring_t s, int nprimes, int* kernel, int* tile, int* split) {
  const char* force = getenv("TN_KERNEL");
  const bool force_naive = force && force[0] == 'n';
  const bool force_tiled = force && force[0] == 't';
  *kernel = kKernNaive;
  *tile = 1;
  *split = 1;
  if (force_naive || g.nb > 15 || g.rc < 1) return;
  const int ops_bits = g.nb + g.nm + g.nn + g.nk;
  if (!force_tiled && (ops_bits < 15 || g.nk < 2 || g.nm < 3 || g.nn < 3)) return;
  const bool tropical = (s == TN_TROPICAL_F32 || s == TN_TROPICAL_I32);
  *tile = (tropical && g.nm >= 7 && g.nn >= 7) ? 0 : 1;
  const int64_t bm = tiled_tile_bm(*tile), bn = tiled_tile_bn(*tile), bk = tiled_tile_bk(*tile);
  const int64_t tiles = ((int64_t(1) << g.nm) + bm - 1) / bm * (((int64_t(1) << g.nn) + bn - 1) / bn) *
                        (int64_t(1) << g.nb) * (s == TN_COUNT_MODP ? nprimes : 1);
  const int64_t K = int64_t(1) << g.nk;
  int sp = 1;
  while (tiles * sp < 2 * 152 && sp < 8 && K / (2 * sp) >= bk) sp *= 2;
  *split = sp;
  *kernel = kKernTiled;
}

int launch_step(tn_semiring_t s, const StepGeom& g, const Operand& A, const Operand& B,
                const Output& C, const ModTable& mods, int nprimes, cudaStream_t st, int* kernel_used) {
  int kernel, tile, split;
  pick_launch(g, s, nprimes, &kernel, &tile, &split);
  if (kernel_used) *kernel_used = kernel;
  if (kernel == kKernTiled && g.c_identity)
    return launch_step_tiled(s, g, A, B, C, mods, nprimes, tile, split, st);
  if (kernel_used) *kernel_used = kKernNaive;
  return launch_step_naive(s, g, A, B, C, mods, nprimes, st);
}

}  // namespace dev
}  // namespace tn
