// kernels.h -- host-side launchers of the libtn device kernels.
#pragma once

#include <cuda_runtime.h>

#include "semiring.cuh"
#include "tn_internal.h"

namespace tn {
namespace dev {

// General step kernel (any geometry): kernels_naive.cu
int launch_step_naive(tn_semiring_t s, const StepGeom& g, const Operand& A, const Operand& B,
                      const Output& C, const ModTable& mods, int nprimes, cudaStream_t st);

// Register-blocked semiring GEMM (kernels_tiled.cu).  tile: 0 = 128 x 128
// output tile (tropical only), 1 = 64 x 64; split: CTAs of a cluster that
// share one output tile (split-K, power of two <= 8).
int launch_step_tiled(tn_semiring_t s, const StepGeom& g, const Operand& A, const Operand& B,
                      const Output& C, const ModTable& mods, int nprimes, int tile, int split,
                      cudaStream_t st);
int tiled_tile_bm(int tile);
int tiled_tile_bn(int tile);
int tiled_tile_bk(int tile);

// Kernel choice for one step: fills kernel (kKernNaive / kKernTiled), tile
// and split from the step geometry, the semiring and the number of primes.
// batched: the step runs beside the same step of many other networks (a
// batch or a served group), so there is parallelism to spare and k is not
// split.
void pick_launch(const StepGeom& g, tn_semiring_t s, int nprimes, int* kernel, int* tile, int* split,
                 bool batched = false);
int launch_step(tn_semiring_t s, const StepGeom& g, const Operand& A, const Operand& B,
                const Output& C, const ModTable& mods, int nprimes, cudaStream_t st, int* kernel_used);

// Tensor-core ablation inside the one-launch-per-step mode (umma_route.cu):
// TN_UMMA=1 in the environment routes every mod-p step that fits the
// tcgen05 limb GEMM (M % 128, N % 64, K % 64 == 0, stored operands) through
// a gather, tn_modp_gemm_umma and a scatter into the step's stored layout.
bool umma_route_enabled();
bool umma_step_fits(const StepGeom& g, const Operand& A, const Operand& B);
int umma_step(const StepGeom& g, const Operand& A, const Operand& B, const Output& C, const ModTable& mods,
              int32_t nprimes, cudaStream_t st);

// Copies the root scalar and the status word into a TN_RAW_BYTES block.
int launch_finalize(tn_semiring_t s, const Operand& root, int nprimes, const uint32_t* d_status,
                    void* d_raw, cudaStream_t st);

}  // namespace dev
}  // namespace tn
