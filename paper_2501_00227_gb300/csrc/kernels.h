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

// Copies the root scalar and the status word into a TN_RAW_BYTES block.
int launch_finalize(tn_semiring_t s, const Operand& root, int nprimes, const uint32_t* d_status,
                    void* d_raw, cudaStream_t st);

}  // namespace dev
}  // namespace tn
