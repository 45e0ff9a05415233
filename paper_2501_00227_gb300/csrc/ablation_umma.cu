// ablation_umma.cu -- tn_modp_gemm_umma: the batched mod-p GEMM of one
// pairwise step on the 5th-generation tensor cores (tcgen05.mma, operands in
// shared memory, accumulators in tensor memory), as an ablation of the
// CUDA-core path (the contraction itself never calls it).
//
//   C[q][b][m][n] = sum_k A[q][b][m][k] * B[q][b][n][k]  mod p_q
//
// Residues (< 2^31) are cut into four 8-bit limbs.  A limb is an integer
// 0..255, exact in bf16; a limb product is at most 255^2 and a sum of them
// stays exact in fp32 while it is below 2^24.  For every chunk of 64 k the
// 16 limb products (i, j) are accumulated by kind::f16 MMAs (M = 128,
// N = 32, K = 16, bf16 x bf16 -> fp32) into seven tensor-memory
// accumulators, one per diagonal d = i + j (at most 4 x 64 x 255^2 < 2^24,
// so every accumulator is an exact integer).  After each chunk the
// accumulators are read back (tcgen05.ld), converted to integers and folded
// into the residues: res = (res + sum_d S_d (2^(8d) mod p)) mod p, one
// Barrett reduction (Barrett 1986) per entry and chunk.
//
// One CTA of 256 threads owns a 128 x 32 block of C for one (prime, batch);
// warps w and w + 4 read lanes 32 (w % 4) .. + 31 (rows of C), each half of
// the columns.  Shared memory and tensor
// memory are double-buffered: chunk c + 1 is staged (16-byte loads, limbs
// split in registers) while the tensor cores work on chunk c, and chunk c
// is drained while they work on chunk c + 1.  Every wait on an MMA
// completion barrier is bounded (2 s); on a timeout the CTA records it in
// the status word, releases its tensor memory and returns.
#include <cuda_runtime.h>

#include <cstdint>

#include "semiring.cuh"
#include "tn_internal.h"

namespace tn {
namespace dev {
namespace {

constexpr int kUM = 128, kUN = 32, kUK = 64;  // C tile rows, columns; k chunk
constexpr int kUDiag = 7;                     // limb diagonals 0..6
constexpr int kUCols = 512;                   // tensor-memory columns allocated: 2 buffers x 7 x 32 used
// one stage of shared memory: 4 A limb tiles (128 x 64 bf16), 4 B limb tiles (32 x 64)
constexpr int kUATile = kUM * kUK * 2, kUBTile = kUN * kUK * 2;
constexpr int kUStage = 4 * kUATile + 4 * kUBTile;       // 81920
constexpr int kUSmem = 2 * kUStage + 1024;               // two stages + barriers / slot: 1 CTA / SM
constexpr int kUThreads = 256;                           // 8 warps; warps w and w + 4 share lane quadrant w % 4

__device__ uint32_t g_umma_status;

struct UmmaArgs {
  const uint32_t* A;
  const uint32_t* B;
  uint32_t* C;
  ModTable mods;
  int32_t batch, m, n, k;
};

// Byte offset of element (row, kk) of a K-major tile with 8 x (16-byte)
// core matrices: core matrices adjacent in k are 128 bytes apart (leading
// byte offset), row groups of 8 are 1024 bytes apart (stride byte offset).
__device__ __forceinline__ uint32_t umma_off(int row, int kk) {
  return static_cast<uint32_t>((row >> 3) * 1024 + (kk >> 3) * 128 + (row & 7) * 16 + (kk & 7) * 2);
}

// Shared-memory matrix descriptor (no swizzle, K-major): start address,
// leading byte offset 128, stride byte offset 1024, descriptor version 1.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr >> 4) & 0x3FFF);
  d |= static_cast<uint64_t>(128 >> 4) << 16;
  d |= static_cast<uint64_t>(1024 >> 4) << 32;
  d |= static_cast<uint64_t>(1) << 46;
  return d;
}

// Instruction descriptor of kind::f16: fp32 accumulator, bf16 A and B, both
// K-major, N = 32, M = 128.
constexpr uint32_t kUIdesc = (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(kUN >> 3) << 17) |
                             (static_cast<uint32_t>(kUM >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Waits until the barrier's phase `parity` has completed; false after 2 s.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const unsigned long long t0 = now_ns();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (now_ns() - t0 > 2000000000ull) return false;
  }
}

// Element e of a staged chunk (16-byte group k4 of row `row`): the 16 threads
// of a half-warp cover 8 rows x 2 adjacent groups, i.e. 128 distinct bytes
// of one core-matrix column, so their shared-memory stores are free of bank
// conflicts, and a warp reads 64 contiguous bytes of 8 rows from global
// memory.
__device__ __forceinline__ int umma_k4(int e) { return (((e >> 4) & 7) << 1) | (e & 1); }
__device__ __forceinline__ int umma_row(int e) { return ((e >> 1) & 7) | ((e >> 7) << 3); }

// Stages the k chunk starting at k0 into stage buffer `buf` (bf16 limb planes
// in the K-major core-matrix layout).  Every thread issues all its 16-byte
// loads before splitting them.
__device__ __forceinline__ void umma_stage(const uint32_t* A, const uint32_t* B, int lda, int m0, int n0, int k0,
                                           unsigned char* buf) {
  constexpr int kA = kUM * kUK / 4 / kUThreads, kB = kUN * kUK / 4 / kUThreads;  // uint4 per thread: 8, 2
  uint4 va[kA], vb[kB];
#pragma unroll
  for (int u = 0; u < kA; ++u) {
    const int e = threadIdx.x + kUThreads * u, row = umma_row(e), k4 = umma_k4(e);
    va[u] = __ldg(reinterpret_cast<const uint4*>(A + int64_t(m0 + row) * lda + k0) + k4);
  }
#pragma unroll
  for (int u = 0; u < kB; ++u) {
    const int e = threadIdx.x + kUThreads * u, row = umma_row(e), k4 = umma_k4(e);
    vb[u] = __ldg(reinterpret_cast<const uint4*>(B + int64_t(n0 + row) * lda + k0) + k4);
  }
#pragma unroll
  for (int u = 0; u < kA; ++u) {
    const int e = threadIdx.x + kUThreads * u, row = umma_row(e), k4 = umma_k4(e);
    const uint32_t off = umma_off(row, 4 * k4);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const uint32_t b0 = __float_as_uint(static_cast<float>((va[u].x >> (8 * i)) & 0xFFu)) >> 16;
      const uint32_t b1 = __float_as_uint(static_cast<float>((va[u].y >> (8 * i)) & 0xFFu)) >> 16;
      const uint32_t b2 = __float_as_uint(static_cast<float>((va[u].z >> (8 * i)) & 0xFFu)) >> 16;
      const uint32_t b3 = __float_as_uint(static_cast<float>((va[u].w >> (8 * i)) & 0xFFu)) >> 16;
      *reinterpret_cast<uint2*>(buf + i * kUATile + off) = make_uint2(b0 | (b1 << 16), b2 | (b3 << 16));
    }
  }
#pragma unroll
  for (int u = 0; u < kB; ++u) {
    const int e = threadIdx.x + kUThreads * u, row = umma_row(e), k4 = umma_k4(e);
    const uint32_t off = umma_off(row, 4 * k4);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint32_t b0 = __float_as_uint(static_cast<float>((vb[u].x >> (8 * j)) & 0xFFu)) >> 16;
      const uint32_t b1 = __float_as_uint(static_cast<float>((vb[u].y >> (8 * j)) & 0xFFu)) >> 16;
      const uint32_t b2 = __float_as_uint(static_cast<float>((vb[u].z >> (8 * j)) & 0xFFu)) >> 16;
      const uint32_t b3 = __float_as_uint(static_cast<float>((vb[u].w >> (8 * j)) & 0xFFu)) >> 16;
      *reinterpret_cast<uint2*>(buf + 4 * kUATile + j * kUBTile + off) = make_uint2(b0 | (b1 << 16), b2 | (b3 << 16));
    }
  }
}

// Issues the 16 x 4 MMAs of one staged chunk into accumulator buffer `half`
// (columns half * 224 + d * 32) and commits them to barrier `bar` (one thread).
__device__ __forceinline__ void umma_issue(uint32_t tmem, int half, const unsigned char* buf, uint32_t bar) {
  bool first[kUDiag];
#pragma unroll
  for (int d = 0; d < kUDiag; ++d) first[d] = true;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int kk = 0; kk < kUK; kk += 16) {
        const int d = i + j;
        const uint64_t ad = umma_desc(smem_u32(buf + i * kUATile + (kk >> 3) * 128));
        const uint64_t bd = umma_desc(smem_u32(buf + 4 * kUATile + j * kUBTile + (kk >> 3) * 128));
        const uint32_t acc = first[d] ? 0u : 1u;
        first[d] = false;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(
                tmem + static_cast<uint32_t>(half * kUDiag * kUN + d * kUN)),
            "l"(ad), "l"(bd), "r"(kUIdesc), "r"(acc)
            : "memory");
      }
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__global__ void __launch_bounds__(kUThreads, 1) k_modp_gemm_umma(const __grid_constant__ UmmaArgs args) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* stage0 = smem;
  unsigned char* stage1 = smem + kUStage;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + 2 * kUStage);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + 2 * kUStage + 64);
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int tiles_n = args.n / kUN;
  const int m0 = (blockIdx.x / tiles_n) * kUM, n0 = (blockIdx.x % tiles_n) * kUN;
  const int b = blockIdx.y, q = blockIdx.z;
  const ModParams mp = args.mods.q[q];
  const uint32_t* A = args.A + (int64_t(q) * args.batch + b) * int64_t(args.m) * args.k;
  const uint32_t* B = args.B + (int64_t(q) * args.batch + b) * int64_t(args.n) * args.k;
  const uint32_t bar0 = smem_u32(bars), bar1 = smem_u32(bars + 1);

  if (tid == 0) {
    s_fail = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(kUCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;

  // 2^(8d) mod p
  uint32_t w[kUDiag];
  w[0] = 1u % mp.p;
#pragma unroll
  for (int d = 1; d < kUDiag; ++d) w[d] = barrett64(static_cast<uint64_t>(w[d - 1]) * (256u % mp.p), mp);
  constexpr int kUH = kUN / 2;  // columns drained per thread
  uint32_t res[kUH];
#pragma unroll
  for (int c = 0; c < kUH; ++c) res[c] = 0u;
  const int col0 = (warp >> 2) * kUH, row = (warp & 3) * 32 + (tid & 31);

  const int nch = args.k / kUK;
  umma_stage(A, B, args.k, m0, n0, 0, stage0);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (tid == 0) umma_issue(tmem, 0, stage0, bar0);
  const uint32_t lane_addr = tmem + (static_cast<uint32_t>((warp & 3) * 32) << 16);
  for (int c = 0; c < nch; ++c) {
    const int half = c & 1;
    // stage the next chunk while the tensor cores work on this one (its
    // buffer's previous MMAs completed one iteration ago)
    if (c + 1 < nch) umma_stage(A, B, args.k, m0, n0, (c + 1) * kUK, half ? stage0 : stage1);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (!mbar_wait(half ? bar1 : bar0, static_cast<uint32_t>((c >> 1) & 1))) s_fail = 1;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (s_fail) break;
    if (c + 1 < nch && tid == 0) umma_issue(tmem, half ^ 1, half ? stage0 : stage1, half ? bar0 : bar1);
    // drain this chunk's accumulators while the next chunk runs: thread t
    // reads lane 32 (w % 4) + t % 32, columns 16 (w / 4) .. + 15 of each diagonal
    uint64_t t[kUH];
#pragma unroll
    for (int col = 0; col < kUH; ++col) t[col] = res[col];
#pragma unroll 1
    for (int d = 0; d < kUDiag; ++d) {
      uint32_t r[kUH];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(lane_addr + static_cast<uint32_t>(half * kUDiag * kUN + d * kUN + col0))
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int col = 0; col < kUH; ++col)  // exact integers < 2^24; the sum stays below 2^59
        t[col] += static_cast<uint64_t>(static_cast<uint32_t>(__uint_as_float(r[col]))) * w[d];
    }
#pragma unroll
    for (int col = 0; col < kUH; ++col) res[col] = barrett64(t[col], mp);
    // the drained buffer is overwritten by the MMAs issued next iteration
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  if (s_fail) {
    if (tid == 0) atomicOr(&g_umma_status, 1u);
  } else {
    uint32_t* C = args.C + (int64_t(q) * args.batch + b) * int64_t(args.m) * args.n + int64_t(m0 + row) * args.n +
                  n0 + col0;
#pragma unroll
    for (int c = 0; c < kUH; c += 4) *reinterpret_cast<uint4*>(C + c) = make_uint4(res[c], res[c + 1], res[c + 2], res[c + 3]);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kUCols) : "memory");
}

}  // namespace
}  // namespace dev

int make_mod_table_checked(tn_semiring_t s, const uint32_t* primes, int32_t nprimes, void* mods);

}  // namespace tn

extern "C" int tn_modp_gemm_umma(const uint32_t* primes, int32_t nprimes, const void* d_a, const void* d_b,
                                 void* d_c, int32_t batch, int32_t m, int32_t n, int32_t k, void* cuda_stream) {
  using namespace tn;
  if (!d_a || !d_b || !d_c || batch < 1 || batch > 65535 || m < dev::kUM || n < dev::kUN || k < dev::kUK ||
      m % dev::kUM || n % dev::kUN || k % dev::kUK || int64_t(m / dev::kUM) * (n / dev::kUN) > (1ll << 30) ||
      ((reinterpret_cast<uintptr_t>(d_a) | reinterpret_cast<uintptr_t>(d_b) | reinterpret_cast<uintptr_t>(d_c)) & 15))
    return TN_EINVAL;
  dev::UmmaArgs a;
  int rc = make_mod_table_checked(TN_COUNT_MODP, primes, nprimes, &a.mods);
  if (rc) return rc;
  a.A = static_cast<const uint32_t*>(d_a);
  a.B = static_cast<const uint32_t*>(d_b);
  a.C = static_cast<uint32_t*>(d_c);
  a.batch = batch;
  a.m = m;
  a.n = n;
  a.k = k;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(dev::k_modp_gemm_umma, cudaFuncAttributeMaxDynamicSharedMemorySize, dev::kUSmem) !=
        cudaSuccess)
      return TN_ECUDA;
    attr = true;
  }
  const uint32_t zero = 0;
  if (cudaMemcpyToSymbolAsync(dev::g_umma_status, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice, st) !=
      cudaSuccess)
    return TN_ECUDA;
  const dim3 grid(static_cast<unsigned>((m / dev::kUM) * (n / dev::kUN)), static_cast<unsigned>(batch),
                  static_cast<unsigned>(nprimes));
  dev::k_modp_gemm_umma<<<grid, dev::kUThreads, dev::kUSmem, st>>>(a);
  if (cudaGetLastError() != cudaSuccess) return TN_ECUDA;
  uint32_t status = 0;
  if (cudaMemcpyFromSymbolAsync(&status, dev::g_umma_status, sizeof(status), 0, cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return TN_ECUDA;
  return status ? TN_ETIMEOUT : TN_OK;
}
