// ablation_limb.cu -- tn_modp_gemm_limb: the batched mod-p GEMM of one
// pairwise step on the integer tensor cores, as an ablation of the CUDA-core
// path (the contraction itself never calls it).
//
//   C[q][b][m][n] = sum_k A[q][b][m][k] * B[q][b][n][k]  mod p_q
//
// Every residue (< 2^31) is cut into four 8-bit limbs, a = sum_i a_i 2^(8i),
// so C = sum_{i,j} 2^(8(i+j)) S_ij with S_ij = sum_k a_i b_j, an exact
// unsigned 8-bit GEMM.  The 16 limb products run as warp-level integer MMAs
// (mma.sync m16n8k32, u8 x u8 -> s32; tcgen05.mma kind::i8 is not available
// for sm_103a), summed per diagonal d = i + j in 32-bit registers (exact for
// k blocks of at most 8192: 4 x 8192 x 255^2 < 2^31), and every k block's
// diagonals are folded into the residue: acc += sum_d (S_d mod p)(2^(8d) mod
// p), with Barrett reductions (Barrett 1986) after each product.
//
// Tiles: a CTA owns a 64 x 32 block of C for one (prime, batch); 8 warps in a
// 4 x 2 grid own 16 x 16 each (two m16n8 fragments).  k advances in chunks of
// 32: the chunk's A (64 x 32) and B (32 x 32) residues are read from global
// memory, split into limb planes in shared memory, and consumed by 32 MMAs
// per warp.
#include <cuda_runtime.h>

#include <cstdint>

#include "semiring.cuh"
#include "tn_internal.h"

namespace tn {
namespace dev {
namespace {

constexpr int kLBM = 64, kLBN = 32, kLBK = 32;  // CTA tile of C, k chunk
constexpr int kLKBlock = 8192;                   // k terms per exact diagonal block

struct LimbArgs {
  const uint32_t* A;
  const uint32_t* B;
  uint32_t* C;
  ModTable mods;
  int32_t batch, m, n, k;
};

__device__ __forceinline__ void mma_u8(int (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k32.row.col.s32.u8.u8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t mulmod(uint32_t a, uint32_t b, const ModParams& mp) {
  return barrett64(static_cast<uint64_t>(a) * b, mp);
}

__global__ void __launch_bounds__(256) k_modp_gemm_limb(const __grid_constant__ LimbArgs args) {
  __shared__ __align__(16) uint8_t As[4][kLBM][kLBK];  // limb planes of the A chunk, [m][k]
  __shared__ __align__(16) uint8_t Bs[4][kLBN][kLBK];  // limb planes of the B chunk, [n][k]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = lane >> 2, t = lane & 3;  // mma fragment coordinates
  const int wm = warp >> 1, wn = warp & 1;
  const int tiles_n = args.n / kLBN;
  const int m0 = (blockIdx.x / tiles_n) * kLBM, n0 = (blockIdx.x % tiles_n) * kLBN;
  const int b = blockIdx.y, q = blockIdx.z;
  const ModParams mp = args.mods.q[q];
  const int64_t mk = int64_t(args.m) * args.k, nk = int64_t(args.n) * args.k;
  const uint32_t* A = args.A + (int64_t(q) * args.batch + b) * mk;
  const uint32_t* B = args.B + (int64_t(q) * args.batch + b) * nk;

  // 2^(8d) mod p for the diagonals d = 0..6
  uint32_t w[7];
  w[0] = 1u % mp.p;
#pragma unroll
  for (int d = 1; d < 7; ++d) w[d] = mulmod(w[d - 1], 256u % mp.p, mp);

  uint32_t res[2][4];  // residues of this warp's two m16n8 fragments
#pragma unroll
  for (int f = 0; f < 2; ++f)
#pragma unroll
    for (int r = 0; r < 4; ++r) res[f][r] = 0u;

  for (int kb = 0; kb < args.k; kb += kLKBlock) {
    const int kb_end = kb + kLKBlock < args.k ? kb + kLKBlock : args.k;
    int s[7][2][4];  // diagonal sums of this k block
#pragma unroll
    for (int d = 0; d < 7; ++d)
#pragma unroll
      for (int f = 0; f < 2; ++f)
#pragma unroll
        for (int r = 0; r < 4; ++r) s[d][f][r] = 0;
    for (int k0 = kb; k0 < kb_end; k0 += kLBK) {
      __syncthreads();
      // stage: A chunk 64 x 32 (8 residues per thread), B chunk 32 x 32 (4)
#pragma unroll
      for (int e = tid; e < kLBM * kLBK; e += 256) {
        const int row = e / kLBK, kk = e % kLBK;
        const uint32_t v = A[int64_t(m0 + row) * args.k + k0 + kk];
#pragma unroll
        for (int i = 0; i < 4; ++i) As[i][row][kk] = static_cast<uint8_t>(v >> (8 * i));
      }
#pragma unroll
      for (int e = tid; e < kLBN * kLBK; e += 256) {
        const int col = e / kLBK, kk = e % kLBK;
        const uint32_t v = B[int64_t(n0 + col) * args.k + k0 + kk];
#pragma unroll
        for (int j = 0; j < 4; ++j) Bs[j][col][kk] = static_cast<uint8_t>(v >> (8 * j));
      }
      __syncthreads();
      const int ra = wm * 16;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        uint32_t a[4];
        a[0] = *reinterpret_cast<const uint32_t*>(&As[i][ra + g][4 * t]);
        a[1] = *reinterpret_cast<const uint32_t*>(&As[i][ra + g + 8][4 * t]);
        a[2] = *reinterpret_cast<const uint32_t*>(&As[i][ra + g][16 + 4 * t]);
        a[3] = *reinterpret_cast<const uint32_t*>(&As[i][ra + g + 8][16 + 4 * t]);
#pragma unroll
        for (int f = 0; f < 2; ++f) {
          const int cb = wn * 16 + f * 8;
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            uint32_t bb[2];
            bb[0] = *reinterpret_cast<const uint32_t*>(&Bs[j][cb + g][4 * t]);
            bb[1] = *reinterpret_cast<const uint32_t*>(&Bs[j][cb + g][16 + 4 * t]);
            mma_u8(s[i + j][f], a, bb);
          }
        }
      }
    }
    // fold the block's diagonals into the residues
#pragma unroll
    for (int f = 0; f < 2; ++f)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        uint32_t acc = res[f][r];
#pragma unroll
        for (int d = 0; d < 7; ++d) {
          const uint32_t sd = barrett64(static_cast<uint32_t>(s[d][f][r]), mp);
          acc = barrett64(static_cast<uint64_t>(acc) + static_cast<uint64_t>(sd) * w[d], mp);
        }
        res[f][r] = acc;
      }
  }
  uint32_t* C = args.C + (int64_t(q) * args.batch + b) * int64_t(args.m) * args.n;
#pragma unroll
  for (int f = 0; f < 2; ++f) {
    const int row = m0 + wm * 16 + g, col = n0 + wn * 16 + f * 8 + 2 * t;
    C[int64_t(row) * args.n + col] = res[f][0];
    C[int64_t(row) * args.n + col + 1] = res[f][1];
    C[int64_t(row + 8) * args.n + col] = res[f][2];
    C[int64_t(row + 8) * args.n + col + 1] = res[f][3];
  }
}

}  // namespace
}  // namespace dev

int make_mod_table_checked(tn_semiring_t s, const uint32_t* primes, int32_t nprimes, void* mods);

}  // namespace tn

extern "C" int tn_modp_gemm_limb(const uint32_t* primes, int32_t nprimes, const void* d_a, const void* d_b,
                                 void* d_c, int32_t batch, int32_t m, int32_t n, int32_t k, void* cuda_stream) {
  using namespace tn;
  if (!d_a || !d_b || !d_c || batch < 1 || batch > 65535 || m < dev::kLBM || n < dev::kLBN || k < dev::kLBK ||
      m % dev::kLBM || n % dev::kLBN || k % dev::kLBK || int64_t(m / dev::kLBM) * (n / dev::kLBN) > (1ll << 30))
    return TN_EINVAL;
  dev::LimbArgs a;
  const int rc = make_mod_table_checked(TN_COUNT_MODP, primes, nprimes, &a.mods);
  if (rc) return rc;
  a.A = static_cast<const uint32_t*>(d_a);
  a.B = static_cast<const uint32_t*>(d_b);
  a.C = static_cast<uint32_t*>(d_c);
  a.batch = batch;
  a.m = m;
  a.n = n;
  a.k = k;
  const dim3 grid(static_cast<unsigned>((m / dev::kLBM) * (n / dev::kLBN)), static_cast<unsigned>(batch),
                  static_cast<unsigned>(nprimes));
  dev::k_modp_gemm_limb<<<grid, 256, 0, static_cast<cudaStream_t>(cuda_stream)>>>(a);
  return cudaGetLastError() == cudaSuccess ? TN_OK : TN_ECUDA;
}
