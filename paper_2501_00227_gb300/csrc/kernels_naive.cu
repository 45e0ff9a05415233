// kernels_naive.cu -- the general pairwise-step kernel of libtn: one thread
// per output entry, operands read through bit-position maps.  It handles any
// step (any label classes, leaves generated on the fly, broadcast labels)
// and is the path for the many small steps of a contraction; wide steps go
// to the tiled kernels in kernels_tiled.cu.
//
// A step (Sec. 4.1 of arXiv:2501.00227) computes
//   C[b, m, n] = (+)_k A[b, m, k] (x) B[b, k, n]
// with C stored contiguously as c = n | m << nn | b << (nn + nm).
#include <cuda_runtime.h>

#include "kernels.h"
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

constexpr int kNaiveKLoBits = 9;

template <class SR>
__global__ void __launch_bounds__(256) k_step_naive(const __grid_constant__ StepGeom g, Operand A,
                                                    Operand B, Output C,
                                                    ModTable mods) {
  __shared__ int64_t s_ka[1 << kNaiveKLoBits];
  __shared__ int64_t s_kb[1 << kNaiveKLoBits];
  const int kl = g.nk < kNaiveKLoBits ? g.nk : kNaiveKLoBits;
  const int64_t nklo = int64_t(1) << kl;
  const int64_t nkhi = int64_t(1) << (g.nk - kl);
  const int a_k0 = g.nb + g.nm;  // first k bit in a_pos
  const int b_k0 = g.nb;         // first k bit in b_pos
  for (int64_t i = threadIdx.x; i < nklo; i += blockDim.x) {
    s_ka[i] = deposit(i, g.a_pos, a_k0, kl);
    s_kb[i] = deposit(i, g.b_pos, b_k0, kl);
  }
  __syncthreads();
  const int q = blockIdx.y;
  const ModParams mp = mods.q[q];
  const int64_t nc = int64_t(1) << g.rc;
  const int64_t mask_n = (int64_t(1) << g.nn) - 1, mask_m = (int64_t(1) << g.nm) - 1;
  for (int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; c < nc;
       c += int64_t(gridDim.x) * blockDim.x) {
    const int64_t n = c & mask_n, m = (c >> g.nn) & mask_m, b = c >> (g.nn + g.nm);
    const int64_t base_a = deposit(b, g.a_pos, 0, g.nb) | deposit(m, g.a_pos, g.nb, g.nm);
    const int64_t base_b = deposit(b, g.b_pos, 0, g.nb) | deposit(n, g.b_pos, g.nb + g.nk, g.nn);
    typename SR::Acc acc = SR::zero(mp);
    for (int64_t kh = 0; kh < nkhi; ++kh) {
      const int64_t oa = base_a | deposit(kh, g.a_pos, a_k0 + kl, g.nk - kl);
      const int64_t ob = base_b | deposit(kh, g.b_pos, b_k0 + kl, g.nk - kl);
      for (int64_t k = 0; k < nklo; ++k)
        SR::mac(acc, SR::load(A, oa | s_ka[k], q), SR::load(B, ob | s_kb[k], q), mp);
    }
    SR::store(C, g.c_identity ? c : deposit(c, g.c_pos, 0, g.rc), q, acc, mp);
  }
}

template <class SR>
static int launch_naive_t(const StepGeom& g, const Operand& A, const Operand& B, const Output& C,
                          const ModTable& mods, int nprimes, cudaStream_t st) {
  const int64_t nc = int64_t(1) << g.rc;
  int64_t blocks = (nc + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  dim3 grid(static_cast<unsigned>(blocks), static_cast<unsigned>(nprimes));
  k_step_naive<SR><<<grid, 256, 0, st>>>(g, A, B, C, mods);
  return cudaGetLastError() == cudaSuccess ? TN_OK : TN_ECUDA;
}

int launch_step_naive(tn_semiring_t s, const StepGeom& g, const Operand& A, const Operand& B,
                      const Output& C, const ModTable& mods, int nprimes, cudaStream_t st) {
  switch (s) {
    case TN_TROPICAL_F32: return launch_naive_t<SrF32>(g, A, B, C, mods, 1, st);
    case TN_TROPICAL_I32: return launch_naive_t<SrI32>(g, A, B, C, mods, 1, st);
    case TN_COUNTING_TROPICAL: return launch_naive_t<SrCnt>(g, A, B, C, mods, 1, st);
    case TN_COUNT_MODP: return launch_naive_t<SrMod>(g, A, B, C, mods, nprimes, st);
  }
  return TN_EINVAL;
}

// Copies the scalar result (entry 0 of the root tensor) and the status word
// into the raw result block:
//   [0..4)   int32 / float value        (tropical, counting max)
//   [8..16)  uint64 count               (counting)
//   [16..80) uint32 residues[16]        (mod p)
//   [96..100) uint32 device status flags
__global__ void k_finalize(tn_semiring_t s, Operand root, int nprimes, const uint32_t* status,
                           unsigned char* raw) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (s == TN_TROPICAL_F32 || s == TN_TROPICAL_I32) {
    *reinterpret_cast<int32_t*>(raw) = static_cast<const int32_t*>(root.p0)[0];
  } else if (s == TN_COUNTING_TROPICAL) {
    *reinterpret_cast<int32_t*>(raw) = static_cast<const int32_t*>(root.p0)[0];
    *reinterpret_cast<uint64_t*>(raw + 8) = static_cast<const uint64_t*>(root.p1)[0];
  } else {
    for (int q = 0; q < nprimes; ++q)
      reinterpret_cast<uint32_t*>(raw + 16)[q] =
          static_cast<const uint32_t*>(root.p0)[q * root.prime_stride];
  }
  *reinterpret_cast<uint32_t*>(raw + 96) = status ? *status : 0u;
}

int launch_finalize(tn_semiring_t s, const Operand& root, int nprimes, const uint32_t* d_status,
                    void* d_raw, cudaStream_t st) {
  k_finalize<<<1, 32, 0, st>>>(s, root, nprimes, d_status, static_cast<unsigned char*>(d_raw));
  return cudaGetLastError() == cudaSuccess ? TN_OK : TN_ECUDA;
}

}  // namespace dev
}  // namespace tn
