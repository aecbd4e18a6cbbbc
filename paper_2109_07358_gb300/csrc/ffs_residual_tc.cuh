// Tensor-core (tcgen05) residual of the batched form.
#pragma once

#include "ffs_kernels.cuh"

namespace fermi {

// Per-instance parameters of the residual epilogue.
struct TcArgs {
  int64_t bw, L, ldP, ldMask;
  int nK;
  int cplx;
  float* P;
  const uint32_t* mask;
  int* status;
};

// P[b, y] = |sum_c H[b, c] Ue[j, c]|^2 on tcgen05 tensor cores (operand encoding op).
cudaError_t launch_residual_tc(ffs_ctx* c, const StepArgs& a, int op, cudaStream_t s);
cudaError_t configure_residual_tc();
// Encode the tensor maps of c for operand mode op (no-op when already current).
cudaError_t prepare_residual_tc(ffs_ctx* c, int op);
int residual_tile_cols();        // embedding columns per CTA tile
int residual_k_block(int op);    // K elements per 128-byte TMA row

}  // namespace fermi
