// kernels_tiled.cu -- per-step launch of the register-blocked semiring GEMM
// (tile_device.cuh) and the host-side choice of kernel, tile shape and
// split-K for a step.
//
// Split-K in a per-step launch: S CTAs of one thread-block cluster share an
// output tile, each taking 1/S of the k range; the partial tiles are merged
// through distributed shared memory (DSMEM) with the semiring (+), and each
// CTA of the cluster writes 1/S of the tile.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <type_traits>

#include "exec.h"
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
  int32_t split;  // CTAs per output tile (cluster size along x)
  int32_t tiles_m, tiles_n;
};

template <class SR, class Cfg, int FOLD>
__global__ void __launch_bounds__(kBlock, 2) k_step_tiled(const __grid_constant__ TiledArgs args) {
  constexpr int BM = Cfg::BM, BN = Cfg::BN, TM = Cfg::TM, TN = Cfg::TN;
  using Acc = typename SR::Acc;
  extern __shared__ __align__(16) unsigned char smem[];
  auto& sm = *reinterpret_cast<TileSmem<SR, Cfg>*>(smem);
  const StepGeom& g = args.g;
  const int tid = threadIdx.x;
  const int grp = tid / Cfg::GT, gt = tid % Cfg::GT;
  const int tx = gt % Cfg::WN, ty = gt / Cfg::WN;
  const int split = args.split;
  const int rank = static_cast<int>(blockIdx.x) % split;
  const int tile = static_cast<int>(blockIdx.x) / split;
  const int64_t tm = tile / args.tiles_n, tn_ = tile % args.tiles_n;
  const int64_t b = blockIdx.y;
  const int q = blockIdx.z;
  const ModParams mp = args.mods.q[q];
  const int64_t K = int64_t(1) << g.nk;
  // rank r of `split` takes the k chunks [nch r / split, nch (r+1) / split)
  const int64_t nch = K > Cfg::BK ? K / Cfg::BK : 1;
  const int64_t kbeg = nch * rank / split * Cfg::BK;
  const int64_t kend_ = nch * (rank + 1) / split * Cfg::BK;
  const int64_t kstop = kend_ < K ? kend_ : K;
  const Operand A = at_prime(args.A, q, mp), B = at_prime(args.B, q, mp);
  const Output C = at_prime(args.C, q);

  Acc acc[TM][TN];
  if constexpr (std::is_same<SR, SrCnt>::value)
    tile_mainloop_counting<Cfg, false>(g, A, B, mp, b, tm, tn_, kbeg, kstop, smem, acc);
  else
    tile_mainloop<SR, Cfg, FOLD, false>(g, A, B, mp, b, tm, tn_, kbeg, kstop, sm, acc);
  tile_merge_groups<SR, Cfg>(acc, reinterpret_cast<Acc*>(smem), mp);

  const uint32_t M = 1u << g.nm, N = 1u << g.nn;
  const uint32_t m0 = static_cast<uint32_t>(tm) * BM, n0 = static_cast<uint32_t>(tn_) * BN;
  const uint32_t cbase = static_cast<uint32_t>(b) << (g.nn + g.nm);
  if (split == 1) {
    if (grp != 0) return;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const uint32_t m = m0 + ty * TM + i;
      if (m >= M) continue;
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const uint32_t n = n0 + tx * TN + j;
        if (n < N) SR::store(C, cbase + (m << g.nn) + n, acc[i][j], mp);
      }
    }
    return;
  }

  // split-K: merge the partial tiles of the cluster through DSMEM
  cg::cluster_group cluster = cg::this_cluster();
  Acc* red = reinterpret_cast<Acc*>(smem);  // [BM][BN]
  if (grp == 0) {
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) red[(ty * TM + i) * BN + tx * TN + j] = acc[i][j];
  }
  cluster.sync();
  const int per = BM * BN / split;
  for (int e = rank * per + tid; e < (rank + 1) * per; e += kBlock) {
    Acc v = red[e];
    for (int r = 0; r < split; ++r) {
      if (r == rank) continue;
      const Acc* peer = cluster.map_shared_rank(red, r);
      SR::merge(v, peer[e], mp);
    }
    const uint32_t m = m0 + e / BN, n = n0 + e % BN;
    if (m < M && n < N) SR::store(C, cbase + (m << g.nn) + n, v, mp);
  }
  cluster.sync();
}

template <class SR, class Cfg, int FOLD>
static int launch_tiled_t(const TiledArgs& a, int nprimes, cudaStream_t st) {
  using Acc = typename SR::Acc;
  size_t smem = tile_smem_bytes<SR, Cfg>();
  const size_t red = sizeof(Acc) * Cfg::BM * Cfg::BN;
  if (a.split > 1 && red > smem) smem = red;
  auto kern = k_step_tiled<SR, Cfg, FOLD>;
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
  cfg.blockDim = dim3(kBlock, 1, 1);
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

// Tile shapes: see TileC0..TileC5 in tile_device.cuh.
static const int kTileBM[kNumTiles] = {TileC0::BM, TileC1::BM, TileC2::BM, TileC3::BM, TileC4::BM, TileC5::BM};
static const int kTileBN[kNumTiles] = {TileC0::BN, TileC1::BN, TileC2::BN, TileC3::BN, TileC4::BN, TileC5::BN};
static const int kTileBK[kNumTiles] = {TileC0::BK, TileC1::BK, TileC2::BK, TileC3::BK, TileC4::BK, TileC5::BK};
// relative throughput of a fully used tile (register blocking, sliced-K merge)
static const float kTileEff[kNumTiles] = {1.0f, 0.8f, 0.72f, 0.68f, 0.68f, 0.8f};

int tiled_tile_bm(int tile) { return kTileBM[tile]; }
int tiled_tile_bn(int tile) { return kTileBN[tile]; }
int tiled_tile_bk(int tile) { return kTileBK[tile]; }

template <class SR, int FOLD>
static int launch_cfg(const TiledArgs& a, int tile, int nprimes, cudaStream_t st) {
  switch (tile) {
    case 1: return launch_tiled_t<SR, TileC1, FOLD>(a, nprimes, st);
    case 2: return launch_tiled_t<SR, TileC2, FOLD>(a, nprimes, st);
    case 3: return launch_tiled_t<SR, TileC3, FOLD>(a, nprimes, st);
    case 4: return launch_tiled_t<SR, TileC4, FOLD>(a, nprimes, st);
    case 5: return launch_tiled_t<SR, TileC5, FOLD>(a, nprimes, st);
  }
  return TN_EINVAL;
}

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
      return tile == 0 ? launch_tiled_t<SrF32, TileC0, 1>(a, 1, st) : launch_cfg<SrF32, 1>(a, tile, 1, st);
    case TN_TROPICAL_I32:
      return tile == 0 ? launch_tiled_t<SrI32, TileC0, 1>(a, 1, st) : launch_cfg<SrI32, 1>(a, tile, 1, st);
    case TN_COUNTING_TROPICAL:
      return launch_cfg<SrCnt, 1>(a, tile, 1, st);
    case TN_COUNT_MODP: {
      bool fold4 = true;
      for (int i = 0; i < nprimes; ++i) fold4 = fold4 && mod_fold_interval(mods.q[i].p, mods.q[i].r32) == 4;
      return fold4 ? launch_cfg<SrMod, 4>(a, tile, nprimes, st) : launch_cfg<SrMod, 1>(a, tile, nprimes, st);
    }
  }
  return TN_EINVAL;
}

// Heuristic kernel choice.  The tiled GEMM needs some reduction depth
// (K >= 8), an M x N extent that fills at least a 16 x 64 tile, a batch that
// fits gridDim.y and enough work.  Among tile shapes t and split-K factors s
// the choice minimises an estimate of the step's time on 2 CTAs x 152 SMs:
//   waves(tasks) x (kTaskFixed + padded work per task / tile efficiency),
// where waves = ceil(tasks / 304) and kTaskFixed is the fixed cost of one
// task (claim, tables, pipeline fill, epilogue, publication) expressed in
// multiply-adds of the semiring.  Every split keeps at least one k chunk.
// TN_KERNEL=naive|tiled in the environment forces one path (tests).
void pick_launch(const StepGeom& g, tn_semiring_t s, int nprimes, int* kernel, int* tile, int* split,
                 bool batched) {
  const char* force = getenv("TN_KERNEL");
  const bool force_naive = force && force[0] == 'n';
  const bool force_tiled = force && force[0] == 't';
  *kernel = kKernNaive;
  *tile = 1;
  *split = 1;
  if (force_naive || g.nb > 15 || g.rc < 1 || s == TN_SIZE_MAX_K || s == TN_COUNTING_MAX_K) return;
  const int ops_bits = g.nb + g.nm + g.nn + g.nk;
  if (!force_tiled && (ops_bits < 16 || g.nk < 3 || g.nm + g.nn < 10 || g.nm < 2 || g.nn < 2)) return;
  const bool tropical = (s == TN_TROPICAL_F32 || s == TN_TROPICAL_I32);
  const int64_t M = int64_t(1) << g.nm, N = int64_t(1) << g.nn, K = int64_t(1) << g.nk;
  const int64_t batch = (int64_t(1) << g.nb) * (s == TN_COUNT_MODP ? nprimes : 1);
  constexpr double kSlots = 2 * 152;
  // fixed cost of a task in multiply-adds: ~5 us at the per-CTA rate of each
  // semiring's tile (tropical ~20, mod p ~10, counting ~5 Gop/s per CTA)
  const double kTaskFixed = tropical ? 100e3 : (s == TN_COUNT_MODP ? 50e3 : 25e3);
  const double acc_bytes = tropical ? 4.0 : (s == TN_COUNT_MODP ? 8.0 : 16.0);
  const double out_bytes = double(M) * double(N) * double(batch) * acc_bytes;
  double best = -1.0;
  int best_tile = 1, best_split = 1;
  for (int t = 0; t < kNumTiles; ++t) {
    if (t == 0 && !tropical) continue;
    const int64_t bm = kTileBM[t], bn = kTileBN[t], bk = kTileBK[t];
    const int64_t tiles = ((M + bm - 1) / bm) * ((N + bn - 1) / bn) * batch;
    const int64_t nch = K > bk ? K / bk : 1;  // k chunks
    for (int sp = 1; sp <= (batched ? 1 : 16) && sp <= nch; ++sp) {
      // split-K scratch (one partial tile per task; reused by later steps)
      // at most max(2 x the step's output, 4 MiB)
      const double scratch = sp > 1 ? double(tiles) * sp * bm * bn * acc_bytes : 0.0;
      if (scratch > std::max(2.0 * out_bytes, double(4 << 20))) break;
      const double tasks = double(tiles) * sp;
      // batched: the other networks' tasks fill the waves, so the cost is the
      // total over tasks
      const double waves = batched ? tasks / kSlots
                                   : static_cast<double>(static_cast<int64_t>((tasks + kSlots - 1) / kSlots));
      const double work = double(bm) * double(bn) * double(K) / sp / kTileEff[t];
      const double est = waves * (kTaskFixed + work);
      if (best < 0 || est < best) {
        best = est;
        best_tile = t;
        best_split = sp;
      }
    }
  }
  *tile = best_tile;
  *split = best_split;
  *kernel = kKernTiled;
  // a measured shape installed by tn_tune_set replaces the estimate
  int tt, ts;
  if (tune_lookup(s, g, &tt, &ts)) {
    if (tt < 0) {
      *kernel = kKernNaive;
      *tile = 1;
      *split = 1;
      return;
    }
    if (tt < kNumTiles && (tropical || tt != 0)) {
      const int64_t nch = K > kTileBK[tt] ? K / kTileBK[tt] : 1;
      *tile = tt;
      *split = batched ? 1 : static_cast<int>(ts < nch ? ts : nch);
    }
  }
  // TN_TILE / TN_SPLIT in the environment force the tile shape / split-K of
  // every tiled step (measurement and tests)
  static const int force_tile = getenv("TN_TILE") ? atoi(getenv("TN_TILE")) : -1;
  static const int force_split = getenv("TN_SPLIT") ? atoi(getenv("TN_SPLIT")) : -1;
  if (force_tile >= 0 && force_tile < kNumTiles && (tropical || force_tile != 0)) *tile = force_tile;
  if (force_split >= 1) {
    const int64_t nch = K > kTileBK[*tile] ? K / kTileBK[*tile] : 1;
    *split = static_cast<int>(force_split < nch ? force_split : nch);
  }
}

int launch_step(tn_semiring_t s, const StepGeom& g, const Operand& A, const Operand& B,
                const Output& C, const ModTable& mods, int nprimes, cudaStream_t st, int* kernel_used) {
  int kernel, tile, split;
  pick_launch(g, s, nprimes, &kernel, &tile, &split);
  // per-step launch: a power-of-two cluster of at most 8 CTAs (portable size)
  int sp2 = 1;
  while (sp2 * 2 <= split && sp2 < 8) sp2 *= 2;
  split = sp2;
  if (kernel_used) *kernel_used = kernel;
  if (kernel == kKernTiled && g.c_identity)
    return launch_step_tiled(s, g, A, B, C, mods, nprimes, tile, split, st);
  if (kernel_used) *kernel_used = kKernNaive;
  return launch_step_naive(s, g, A, B, C, mods, nprimes, st);
}

}  // namespace dev
}  // namespace tn
