// kernels_naive.cu -- the general pairwise-step kernel of libtn: R threads
// per output entry (K-parallel, merged with the semiring (+)), operands read
// through bit-position maps.  It handles any step (any label classes, leaves
// generated on the fly, broadcast labels) and is the path for the many small
// steps of a contraction and for reductions with few outputs; wide steps go
// to the tiled kernels in kernels_tiled.cu.
//
// A step (Sec. 4.1 of arXiv:2501.00227) computes
//   C[b, m, n] = (+)_k A[b, m, k] (x) B[b, k, n]
// with C stored contiguously as c = n | m << nn | b << (nn + nm).
#include <cuda_runtime.h>

#include "kernels.h"
#include "semiring.cuh"
#include "step_device.cuh"

namespace tn {
namespace dev {

template <class SR>
__global__ void __launch_bounds__(kBlock) k_step_naive(const __grid_constant__ StepGeom g, Operand A,
                                                       Operand B, Output C, ModTable mods, int R,
                                                       int64_t chunk) {
  __shared__ NaiveSmem<SR> sm;
  const int kl = g.nk < kNaiveKLoBits ? g.nk : kNaiveKLoBits;
  const int32_t nkhi = 1 << (g.nk - kl);
  naive_tables<SR>(g, sm, 0, nkhi);
  const int q = blockIdx.y;
  const ModParams mp = mods.q[q];
  const Operand Aq = at_prime(A, q, mp), Bq = at_prime(B, q, mp);
  const Output Cq = at_prime(C, q);
  const int32_t E = 1 << g.rc;
  const int32_t c0 = static_cast<int32_t>(blockIdx.x) * static_cast<int32_t>(chunk);
  const int32_t c1 = c0 + chunk < E ? c0 + static_cast<int32_t>(chunk) : E;
  auto la = [&](uint32_t e) { return SR::load(Aq, e); };
  auto lb = [&](uint32_t e) { return SR::load(Bq, e); };
  auto sink = [&](uint32_t c, const typename SR::Acc& acc) {
    SR::store(Cq, g.c_identity ? c : deposit(c, g.c_pos, 0, g.rc), acc, mp);
  };
  naive_chunk<SR>(g, la, lb, sink, mp, c0, c1, 0, nkhi, R, sm);
}

template <class SR>
static int launch_naive_t(const StepGeom& g, const Operand& A, const Operand& B, const Output& C,
                          const ModTable& mods, int nprimes, cudaStream_t st) {
  const NaiveShape sh = naive_shape(g.rc, g.nk, false);
  dim3 grid(static_cast<unsigned>(sh.ntasks), static_cast<unsigned>(nprimes));
  k_step_naive<SR><<<grid, kBlock, 0, st>>>(g, A, B, C, mods, sh.R, sh.chunk);
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
