// Tensor-core (tcgen05) residual of the batched form.
#pragma once

#include "ffs_kernels.cuh"

namespace fermi {

// Per-instance parameters of the residual epilogue.
struct TcArgs {
  int64_t bw, L, ldP, ldMask;
  int nK;
  int cplx;
  int grp_rows;  // grouped form: rows of one group's copy of Ue (row offset of sample tile t: t x grp_rows)
  float* P;
  float* G = nullptr;  // or the sums of the weights per 32 accumulator columns (32 real, 16 complex sites)
  int64_t ldG = 0;
  const uint32_t* mask;
  int* status;
  uint32_t spin = 1u << 18;  // polls before a wait gives up (FFS_E_TIMEOUT); each may suspend 100 us
  int fault = 0;             // failure-path test: the first CTA's producer skips stage 0
};

// P[b, y] = |sum_c H[b, c] Ue[j, c]|^2 on tcgen05 tensor cores (operand encoding op).
cudaError_t launch_residual_tc(ffs_ctx* c, const StepArgs& a, int op, cudaStream_t s);
cudaError_t configure_residual_tc();
// Encode the tensor maps of c for operand mode op and column tile bn (no-op when current).
cudaError_t prepare_residual_tc(ffs_ctx* c, int op);  // keeps the tile chosen before (256 if none)
cudaError_t prepare_residual_tc_bn(ffs_ctx* c, int op, int bn);
// Column tile (128 or 256) for this size class: autotuned on first use, then cached.
int residual_tile_for(ffs_ctx* c, const StepArgs& a, int op, cudaStream_t s);
int residual_k_block(int op);    // K elements per 128-byte TMA row
// Tensor map of a row-major rows x inner matrix (BF16, or FP32 when f32), boxes of 128
// bytes x box_rows with the 128-byte swizzle.
cudaError_t encode_2d(CUtensorMap* map, const void* base, bool f32, uint64_t inner, uint64_t rows, uint32_t box_rows);

}  // namespace fermi
