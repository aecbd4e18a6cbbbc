// Launchers of the libffs kernels (host side).  All launches are asynchronous on the
// given stream; they check their own launch errors and return cudaError_t.
#pragma once

#include "ffs_internal.cuh"

namespace fermi {

// Operand encodings of the batched residual (what the per-sample state writes for h).
enum OpMode : int {
  kOpNone = 0,    // plain form: no shared operand, the residual reads h from the state
  kOpF32 = 1,     // FP32, for the CUDA-core residual
  kOpBF16x3 = 2,  // BF16 hi and lo planes (hi*hi + hi*lo + lo*hi)
  kOpBF16 = 3,    // BF16 hi plane only
  kOpTF32 = 4     // FP32 container, rounded to TF32
};

struct StepArgs {
  int64_t L, N, Lr, Kr, Kp, ldP, ldMask;
  int64_t bw;              // samples in this wave
  int64_t n_steps;
  uint64_t seed, first;    // Philox key; global index of the wave's first sample
  bool cplx;
  const void* U64;         // L x N (double / cd)
  const void* Ust;         // L x N in the blocked state's type (the FP64 copy for FP64 states)
  const int32_t* m;        // bw x N
  uint32_t* mask;          // bw x ldMask
  void* H;                 // bw x Kp operand planes
  int64_t hplane;          // elements per operand plane (capacity x Kp)
  float* P;                // bw x ldP
  // bw x ldG sums of the weights per group of kGroupSites(cplx) sites, written by the
  // tensor-core residual next to P (null when the residual form does not write them);
  // the draw then reads the sums instead of all L weights
  float* G = nullptr;
  int64_t ldG = 0;
  void* W;                 // bw x N x N state
  double* logp;            // bw
  int32_t* x;              // bw x ldx
  const int32_t* force_x;  // bw x ldx or null
  float* probs;            // bw x ldx x L or null
  int* status;
  int64_t ldx;             // row stride of x / force_x / probs in steps: n_steps, or N when
                           // samples have their own chain lengths
  const double* sel_p;     // L-ensemble: N keep probabilities of the columns, or null
  const int32_t* nlen;     // bw per-sample chain lengths (<= n_steps), or null: all n_steps
  int grouped;             // groups of 128 samples share m; h is stored in the group's order
  int64_t kcols;           // residual K columns in use (grouped form), 0 = all
};

// Sites per weight-group sum: the 32 accumulator columns of one residual epilogue load,
// 32 real sites or 16 complex ones (a site's real and imaginary parts are adjacent columns).
__host__ __device__ __forceinline__ int kGroupSites(bool cplx) { return cplx ? 16 : 32; }

// Operand column of entry j of h: the original column m_j, or position j when the group's
// copy of the embedding is already in its column order.
__device__ __forceinline__ int operand_col(const StepArgs& a, const int32_t* mrow, int64_t j) {
  return a.grouped ? (int)j : mrow[j];
}

// Layout of a sample's blocked elimination state.  The columns are stored in slabs of 32;
// slab s (columns [32 s, 32 s + 32)) holds only the rows it can ever hold, 0 .. 32 s + 31
// (column c is live while at most c fermions are placed, so its rows stay below
// 32 (c / 32 + 1)), contiguously with 32 entries per row: element (j, c) sits at
// slab_offset(c / 32) + 32 j + c % 32, and a sample holds slab_offset(ceil(Nc / 32))
// entries, about half of Nc^2.  The columns of one slab over a range of rows, which the
// per-step and per-panel kernels stream, are one run of memory.
__host__ __device__ __forceinline__ int64_t slab_offset(int64_t s) { return 512 * s * (s + 1); }
__host__ __device__ __forceinline__ int64_t state_stride(int64_t Nc) { return slab_offset((Nc + 31) / 32); }
__host__ __device__ __forceinline__ int64_t sidx(int64_t j, int64_t c) { return slab_offset(c >> 5) + j * 32 + (c & 31); }

// Precision of the per-sample elimination state.
enum StateKind : int { kStateFP64 = 0, kStateFP32 = 1, kStateDF64 = 2 };

// Buffers of the blocked state (per sample: W Nc rows x round_up(Nc, 32) columns in
// 32-column slabs, W0P Nc x 32 panel-start copy of the
// old rows' panel columns, Sinv 32 x 32 inverse of the panel Schur complement).
struct BlockedArgs {
  int64_t Nc;  // state columns kept (= steps taken)
  void* W;
  void* W0P;
  void* Sinv;
  int tc_top;  // the old rows' trailing update (Top) and the next operand are done elsewhere
};

cudaError_t launch_blocked_step(const StepArgs& a, const BlockedArgs& t, int64_t k, int state, int op,
                                cudaStream_t s);
cudaError_t launch_blocked_panel(const StepArgs& a, const BlockedArgs& t, int64_t k0, int64_t k1, int state,
                                 int op, cudaStream_t s);
// The two halves of launch_blocked_panel (timed separately by the profiler): the panel
// Schur complement and its inverse, then the trailing-column update.
cudaError_t launch_blocked_panel_s(const StepArgs& a, const BlockedArgs& t, int64_t k0, int64_t k1, int state,
                                   cudaStream_t s);
cudaError_t launch_blocked_panel_update(const StepArgs& a, const BlockedArgs& t, int64_t k0, int64_t k1, int state,
                                        int op, cudaStream_t s);
// Operand of step k1 from column k1 of the state (after every row of it is updated).
cudaError_t launch_column_operand(const StepArgs& a, const BlockedArgs& t, int64_t k1, int state, int op,
                                  cudaStream_t s);
// Tensor-core Top update (ffs_ozaki.cu): slices of W0_P and Bot, the product, the operand.
cudaError_t launch_oz_top(ffs_ctx* c, const StepArgs& a, const BlockedArgs& t, int64_t k0, int64_t k1, int op,
                          cudaStream_t s);
cudaError_t oz_prepare(ffs_ctx* c, int64_t Bw, int64_t Nc);
size_t oz_bytes_per_sample(int64_t Nc);
cudaError_t configure_oz();
// Tensor-core new rows (ffs_ozaki_y.cu, double-float state): C's slices, then
// Y = U - C W0_T and Bot = S^-1 Y written as the panel's rows of the trailing columns.
cudaError_t launch_oz_y(ffs_ctx* c, const StepArgs& a, const BlockedArgs& t, int64_t k0, int64_t k1, cudaStream_t s);
cudaError_t ozy_prepare(ffs_ctx* c, int64_t Bw, int64_t Nc);
size_t ozy_bytes_per_sample(int64_t Nc, bool cplx);
cudaError_t configure_oz_y();

// Large-L draw of Section S-7: a Metropolis chain of m_cond updates per step, then the
// same per-step state update (no residual); the panel ends are launch_blocked_panel's.
cudaError_t launch_mcmc_step(const StepArgs& a, const BlockedArgs& t, int64_t k, int64_t m_cond, int state,
                             cudaStream_t s);
size_t mcmc_step_smem(int64_t N, bool cplx, int state);
size_t blocked_elem_bytes(bool cplx, int state);
size_t blocked_step_smem(int64_t Nc, bool cplx, int state);
int blocked_panel_width();
int blocked_step_samples_per_cta();
cudaError_t configure_blocked();

cudaError_t launch_perm_init(const StepArgs& a, int op_mode, cudaStream_t s);
// Grouped form: copies of the residual operand planes, one per group of 128 samples, with
// the K columns in the group's order (group g's order is row 128 g of a.m).
cudaError_t launch_group_embed(const void* src0, const void* src1, void* dst, int64_t Lrp, int64_t Kp, int64_t Kr,
                               bool cplx, bool f32, int planes, const int32_t* m, int64_t N, int64_t groups,
                               int64_t plane_groups, cudaStream_t s);  // planes are plane_groups copies apart
// L-ensemble set-up: keep probabilities from the eigenvalues, then the per-sample chain
// lengths of samples first .. first + B - 1 (a.seed, a.first, a.N, a.sel_p) and their max.
cudaError_t launch_keep_prob(const double* lambda, int64_t N, double* p, int* status, cudaStream_t s);
cudaError_t launch_lens_count(const StepArgs& a, int64_t B, int32_t* nlen, int* max_len, cudaStream_t s);
cudaError_t launch_ortho_check(const void* U64, bool cplx, int64_t L, int64_t N, double* maxdev,
                               cudaStream_t s);
cudaError_t launch_derive_operands(ffs_ctx* c, cudaStream_t s);
// Copy of U in the blocked state's arithmetic type (double-float or FP32); FP64 states use U64.
cudaError_t launch_derive_state_copy(const void* U64, bool cplx, int state, int64_t count, void* out, cudaStream_t s);
cudaError_t launch_residual_fp32(const StepArgs& a, const float* Ue32, cudaStream_t s);
cudaError_t launch_residual_plain(const StepArgs& a, const void* UT32, int64_t k, cudaStream_t s);
// state_fp64: FP64 (double / cd) state, else FP32 (float / cf).
cudaError_t launch_tail(const StepArgs& a, int64_t k, bool state_fp64, int op_mode, cudaStream_t s);
size_t tail_smem_bytes(int64_t N, bool cplx, bool state_fp64);
cudaError_t configure_kernels(int64_t N, bool cplx);

}  // namespace fermi
