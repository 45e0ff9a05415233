// peaks.cu -- register-only throughput of the inner arithmetic of the
// contraction kernels, the denominators of their ALU rooflines.
//
//   kind 0  (max,+) multiply-add on int32: acc = max(acc, a + b), one
//           __viaddmax_s32 per term (the tropical tile's inner step)
//   kind 1  mod-p multiply-add: acc += a * b on a 64-bit accumulator, its
//           high word folded back (acc = hi * (2^32 mod p) + lo) every fourth
//           term (the mod-p tile's inner step)
//   kind 2  (max,+) multiply-add on two int16 lanes: acc = max(acc, a + b)
//           per 16-bit half, one __viaddmax_s16x2 per two terms (the packed
//           tropical tile's inner step)
//
// Every thread runs 16 independent chains for `iters` terms each, so the
// pipes, not the latencies, bound the loop; a term is one semiring
// multiply-add.  The results are stored so that the loop is kept.
#include <cuda_runtime.h>

#include <cstdint>

#include "tn_internal.h"

namespace {

constexpr int kChains = 16;

__global__ void __launch_bounds__(256) k_peak_maxplus(int iters, int32_t seed, int32_t* out) {
  int32_t acc[kChains], b[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) {
    acc[j] = seed + j + static_cast<int32_t>(threadIdx.x);
    b[j] = seed * (j + 1);
  }
  const int32_t a = seed ^ static_cast<int32_t>(blockIdx.x);
  for (int i = 0; i < iters; ++i) {
    const int32_t ai = a ^ static_cast<int32_t>(static_cast<uint32_t>(i) * 2654435761u);  // shared by 16 terms
#pragma unroll
    for (int j = 0; j < kChains; ++j) acc[j] = __viaddmax_s32(ai, b[j], acc[j]);
  }
  int32_t r = 0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) r ^= acc[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

__global__ void __launch_bounds__(256) k_peak_maxplus2(int iters, int32_t seed, uint32_t* out) {
  uint32_t acc[kChains], b[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) {
    acc[j] = static_cast<uint32_t>(seed + j) + threadIdx.x;
    b[j] = static_cast<uint32_t>(seed) * (j + 1);
  }
  const uint32_t a = static_cast<uint32_t>(seed) ^ blockIdx.x;
  for (int i = 0; i < iters; ++i) {
    const uint32_t ai = a ^ (static_cast<uint32_t>(i) * 2654435761u);  // shared by 16 instructions
#pragma unroll
    for (int j = 0; j < kChains; ++j) acc[j] = __viaddmax_s16x2(ai, b[j], acc[j]);
  }
  uint32_t r = 0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) r ^= acc[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

__global__ void __launch_bounds__(256) k_peak_modp(int iters, uint32_t seed, uint32_t r32, uint64_t* out) {
  uint64_t acc[kChains];
  uint32_t b[4][kChains];  // a different factor per term of a fold group: no product can be merged
#pragma unroll
  for (int j = 0; j < kChains; ++j) {
    acc[j] = seed + j;
#pragma unroll
    for (int t = 0; t < 4; ++t) b[t][j] = ((seed * 2654435761u) ^ ((j + 16 * t) * 40503u) ^ threadIdx.x) & 0x7fffffffu;
  }
  const uint32_t a = seed ^ blockIdx.x;
  for (int i = 0; i < iters; i += 4) {
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const uint32_t at = (a + static_cast<uint32_t>(i + t)) & 0x7fffffffu;  // shared by 16 terms
#pragma unroll
      for (int j = 0; j < kChains; ++j) acc[j] += static_cast<uint64_t>(at) * b[t][j];
    }
#pragma unroll
    for (int j = 0; j < kChains; ++j)
      acc[j] = static_cast<uint64_t>(static_cast<uint32_t>(acc[j] >> 32)) * r32 + static_cast<uint32_t>(acc[j]);
  }
  uint64_t r = 0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) r ^= acc[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

}  // namespace

extern "C" int tn_alu_peak(int32_t kind, int32_t iters, void* cuda_stream, double* tops_out) {
  if (!tops_out || kind < 0 || kind > 2 || iters < 4 || iters > (1 << 24)) return TN_EINVAL;
  iters -= iters % 4;
  int dev, sms;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return TN_ECUDA;
  const int blocks = sms * 8, threads = 256;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  void* out = nullptr;
  if (cudaMalloc(&out, size_t(blocks) * threads * 8) != cudaSuccess) return TN_ENOMEM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = TN_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = TN_ECUDA;
  float ms = 0.f;
  for (int rep = 0; rep < 2 && rc == TN_OK; ++rep) {  // the first run warms up
    cudaEventRecord(e0, st);
    if (kind == 0)
      k_peak_maxplus<<<blocks, threads, 0, st>>>(iters, 12345 + rep, static_cast<int32_t*>(out));
    else if (kind == 1)
      k_peak_modp<<<blocks, threads, 0, st>>>(iters, 54321u + rep, 20u, static_cast<uint64_t*>(out));
    else
      k_peak_maxplus2<<<blocks, threads, 0, st>>>(iters, 777 + rep, static_cast<uint32_t*>(out));
    cudaEventRecord(e1, st);
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
      rc = TN_ECUDA;
  }
  if (rc == TN_OK)
    *tops_out = double(blocks) * threads * kChains * double(iters) * (kind == 2 ? 2 : 1) / (double(ms) * 1e-3) / 1e12;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  return rc;
}
