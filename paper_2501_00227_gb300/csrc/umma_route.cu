// umma_route.cu -- the tensor-core ablation inside a whole contraction.
//
// In the one-launch-per-step mode (TN_EXEC=0) with TN_UMMA=1, every mod-p
// step whose GEMM shape fits the tcgen05 limb kernel (tn_modp_gemm_umma:
// M a multiple of 128, N of 64, K of 64) runs as
//   1. a gather of A into [prime][batch][m][k] and of B into
//      [prime][batch][n][k] (the kernel's row-major layouts),
//   2. tn_modp_gemm_umma (bf16 limbs on the 5th-generation tensor cores),
//   3. a scatter of C from [prime][batch][m][n] into the step's stored
//      layout;
// every other step runs the CUDA-core kernels as usual.  The point is to
// measure the tensor-core product end to end against the CUDA-core path on
// the same plan, with identical residues (Sec. 5.1, the count modulo p).
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdlib>
#include <mutex>

#include "kernels.h"
#include "semiring.cuh"
#include "tn_internal.h"

extern "C" int tn_modp_gemm_umma(const uint32_t* primes, int32_t nprimes, const void* d_a, const void* d_b,
                                 void* d_c, int32_t batch, int32_t m, int32_t n, int32_t k, void* cuda_stream);

namespace tn {
namespace dev {
namespace {

// Bit positions of a permutation between a row-major index (bit t) and the
// stored tensor (bit pos[t]); rank <= 31.
struct BitMap {
  int8_t pos[32];
  int32_t rank;
};

__device__ __forceinline__ uint32_t map_bits(const BitMap& bm, uint32_t idx) {
  uint32_t off = 0;
  for (int t = 0; t < bm.rank; ++t) off |= ((idx >> t) & 1u) << bm.pos[t];
  return off;
}

// dst[q][idx] = src[q][map(idx)] for every prime block q (gather = true), or
// dst[q][map(idx)] = src[q][idx] (gather = false); 2^rank entries per block.
__global__ void k_permute(const uint32_t* __restrict__ src, int64_t src_stride, uint32_t* __restrict__ dst,
                          int64_t dst_stride, int32_t nprimes, const __grid_constant__ BitMap bm, bool gather) {
  const int64_t per = int64_t(1) << bm.rank;
  const int64_t total = per * nprimes;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t q = i / per;
    const uint32_t idx = static_cast<uint32_t>(i - q * per);
    const uint32_t off = map_bits(bm, idx);
    if (gather) dst[q * dst_stride + idx] = src[q * src_stride + off];
    else dst[q * dst_stride + off] = src[q * src_stride + idx];
  }
}

int permute(const uint32_t* src, int64_t src_stride, uint32_t* dst, int64_t dst_stride, int32_t np, const BitMap& bm,
            bool gather, cudaStream_t st) {
  const int64_t total = (int64_t(1) << bm.rank) * np;
  const int64_t blocks = (total + 255) / 256;
  k_permute<<<static_cast<unsigned>(blocks < 152 * 16 ? blocks : 152 * 16), 256, 0, st>>>(
      src, src_stride, dst, dst_stride, np, bm, gather);
  return cudaGetLastError() == cudaSuccess ? TN_OK : TN_ECUDA;
}

// Library-owned scratch for the three row-major tensors (grows, never shrinks).
std::mutex g_mu;
void* g_scratch = nullptr;
size_t g_scratch_bytes = 0;

}  // namespace

bool umma_route_enabled() {
  const char* e = getenv("TN_UMMA");
  return e && e[0] == '1';
}

bool umma_step_fits(const StepGeom& g, const Operand& A, const Operand& B) {
  return A.kind == kOpArena && B.kind == kOpArena && g.nm >= 7 && g.nn >= 6 && g.nk >= 6 && g.nb <= 15 &&
         g.nb + g.nm + g.nk <= 31 && g.nb + g.nk + g.nn <= 31 && g.rc <= 31;
}

int umma_step(const StepGeom& g, const Operand& A, const Operand& B, const Output& C, const ModTable& mods,
              int32_t np, cudaStream_t st) {
  const int64_t ea = int64_t(1) << (g.nb + g.nm + g.nk), eb = int64_t(1) << (g.nb + g.nk + g.nn);
  const int64_t ec = int64_t(1) << g.rc;
  const size_t need = static_cast<size_t>(ea + eb + ec) * np * sizeof(uint32_t) + 64;
  std::lock_guard<std::mutex> lk(g_mu);
  if (need > g_scratch_bytes) {
    if (g_scratch && cudaFree(g_scratch) != cudaSuccess) return TN_ECUDA;
    g_scratch = nullptr;
    g_scratch_bytes = 0;
    if (cudaMalloc(&g_scratch, need) != cudaSuccess) return TN_ENOMEM;
    g_scratch_bytes = need;
  }
  uint32_t* ac = static_cast<uint32_t*>(g_scratch);
  uint32_t* bc = ac + ea * np;
  uint32_t* cc = bc + eb * np;
  // A row-major [b][m][k]: k bits lowest, then m, then batch
  BitMap ma;
  ma.rank = g.nb + g.nm + g.nk;
  for (int t = 0; t < ma.rank; ++t)
    ma.pos[t] = t < g.nk ? g.a_pos[g.nb + g.nm + t] : t < g.nk + g.nm ? g.a_pos[g.nb + t - g.nk] : g.a_pos[t - g.nk - g.nm];
  // B row-major [b][n][k]
  BitMap mb;
  mb.rank = g.nb + g.nk + g.nn;
  for (int t = 0; t < mb.rank; ++t)
    mb.pos[t] = t < g.nk ? g.b_pos[g.nb + t] : t < g.nk + g.nn ? g.b_pos[g.nb + t] : g.b_pos[t - g.nk - g.nn];
  // C row-major [b][m][n] is the output index c; stored at c or through c_pos
  BitMap mc;
  mc.rank = g.rc;
  for (int t = 0; t < mc.rank; ++t) mc.pos[t] = g.c_identity ? static_cast<int8_t>(t) : g.c_pos[t];
  int rc = permute(static_cast<const uint32_t*>(A.p0), A.prime_stride, ac, ea, np, ma, true, st);
  if (!rc) rc = permute(static_cast<const uint32_t*>(B.p0), B.prime_stride, bc, eb, np, mb, true, st);
  if (rc) return rc;
  uint32_t primes[TN_MAX_PRIMES];
  for (int q = 0; q < np; ++q) primes[q] = mods.q[q].p;
  rc = tn_modp_gemm_umma(primes, np, ac, bc, cc, 1 << g.nb, 1 << g.nm, 1 << g.nn, 1 << g.nk, st);
  if (rc) return rc;
  return permute(cc, ec, static_cast<uint32_t*>(C.p0), C.prime_stride, np, mc, false, st);
}

}  // namespace dev
}  // namespace tn
