// Tensor-core (tcgen05) residual of the batched form.
#pragma once

#include "ffs_kernels.cuh"

namespace fermi {

// P[b, y] = |sum_c H[b, c] Ue[j, c]|^2 on tcgen05 tensor cores (operand encoding op).
cudaError_t launch_residual_tc(ffs_ctx* c, const StepArgs& a, int op, cudaStream_t s);
cudaError_t configure_residual_tc();

}  // namespace fermi
