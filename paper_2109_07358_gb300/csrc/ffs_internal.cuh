// Internal declarations of libffs: the handle, device scalar helpers, Philox.
//
// Fast fermion sampling (arXiv 2109.07358).  Notation follows the paper: U is L x N,
// a sample is x = (x_1..x_N), m is the sample's column order, step k places x_k
// using the normal vector h of Eq. 3.  Internally everything is 0-based.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/ffs.h"

namespace fermi {

// ------------------------------------------------------------------ scalars
struct cd {  // complex double, interleaved like complex128
  double re, im;
};
struct cf {  // complex float, interleaved like complex64
  float re, im;
};

template <typename T> struct real_of { using type = T; };
template <> struct real_of<cd> { using type = double; };
template <> struct real_of<cf> { using type = float; };

__host__ __device__ __forceinline__ double abs2(double a) { return a * a; }
__host__ __device__ __forceinline__ float abs2(float a) { return a * a; }
__host__ __device__ __forceinline__ double abs2(cd a) { return a.re * a.re + a.im * a.im; }
__host__ __device__ __forceinline__ float abs2(cf a) { return a.re * a.re + a.im * a.im; }

__host__ __device__ __forceinline__ cd operator*(cd a, cd b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
__host__ __device__ __forceinline__ cf operator*(cf a, cf b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
__host__ __device__ __forceinline__ cd operator-(cd a, cd b) { return {a.re - b.re, a.im - b.im}; }
__host__ __device__ __forceinline__ cf operator-(cf a, cf b) { return {a.re - b.re, a.im - b.im}; }
__host__ __device__ __forceinline__ cd operator-(cd a) { return {-a.re, -a.im}; }
__host__ __device__ __forceinline__ cf operator-(cf a) { return {-a.re, -a.im}; }
__host__ __device__ __forceinline__ cd operator/(cd a, cd b) {
  double d = b.re * b.re + b.im * b.im;
  return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}
__host__ __device__ __forceinline__ cf operator/(cf a, cf b) {
  float d = b.re * b.re + b.im * b.im;
  return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}

template <typename T> __host__ __device__ __forceinline__ T s_one();
template <> __host__ __device__ __forceinline__ double s_one<double>() { return 1.0; }
template <> __host__ __device__ __forceinline__ float s_one<float>() { return 1.0f; }
template <> __host__ __device__ __forceinline__ cd s_one<cd>() { return {1.0, 0.0}; }
template <> __host__ __device__ __forceinline__ cf s_one<cf>() { return {1.0f, 0.0f}; }

template <typename T> __host__ __device__ __forceinline__ T s_zero();
template <> __host__ __device__ __forceinline__ double s_zero<double>() { return 0.0; }
template <> __host__ __device__ __forceinline__ float s_zero<float>() { return 0.0f; }
template <> __host__ __device__ __forceinline__ cd s_zero<cd>() { return {0.0, 0.0}; }
template <> __host__ __device__ __forceinline__ cf s_zero<cf>() { return {0.0f, 0.0f}; }

// a - b * c  (fused where the hardware has it)
__device__ __forceinline__ double fms(double a, double b, double c) { return fma(-b, c, a); }
__device__ __forceinline__ float fms(float a, float b, float c) { return fmaf(-b, c, a); }
__device__ __forceinline__ cd fms(cd a, cd b, cd c) {
  return {fma(b.im, c.im, fma(-b.re, c.re, a.re)), fma(-b.im, c.re, fma(-b.re, c.im, a.im))};
}
__device__ __forceinline__ cf fms(cf a, cf b, cf c) {
  return {fmaf(b.im, c.im, fmaf(-b.re, c.re, a.re)), fmaf(-b.im, c.re, fmaf(-b.re, c.im, a.im))};
}

template <typename D, typename S> __host__ __device__ __forceinline__ D s_cast(S v);
template <> __host__ __device__ __forceinline__ double s_cast<double, double>(double v) { return v; }
template <> __host__ __device__ __forceinline__ float s_cast<float, double>(double v) { return (float)v; }
template <> __host__ __device__ __forceinline__ float s_cast<float, float>(float v) { return v; }
template <> __host__ __device__ __forceinline__ double s_cast<double, float>(float v) { return v; }
template <> __host__ __device__ __forceinline__ cd s_cast<cd, cd>(cd v) { return v; }
template <> __host__ __device__ __forceinline__ cf s_cast<cf, cd>(cd v) { return {(float)v.re, (float)v.im}; }
template <> __host__ __device__ __forceinline__ cf s_cast<cf, cf>(cf v) { return v; }
template <> __host__ __device__ __forceinline__ cd s_cast<cd, cf>(cf v) { return {v.re, v.im}; }

__device__ __forceinline__ bool s_finite(double a) { return isfinite(a); }
__device__ __forceinline__ bool s_finite(float a) { return isfinite(a); }
__device__ __forceinline__ bool s_finite(cd a) { return isfinite(a.re) && isfinite(a.im); }
__device__ __forceinline__ bool s_finite(cf a) { return isfinite(a.re) && isfinite(a.im); }

// ------------------------------------------------------------------ Philox4x32-10
// Written from the published definition (Salmon, Moraes, Dror, Shaw, SC'11): ten
// rounds of two 32x32->64 multiplies with the Weyl-incremented key.
__host__ __device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
#ifdef __CUDA_ARCH__
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
#else
    const uint64_t p0 = (uint64_t)0xD2511F53u * c.x, p1 = (uint64_t)0xCD9E8D57u * c.z;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
#endif
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

enum { kStreamPerm = 0, kStreamSite = 1, kStreamSelect = 2, kStreamMcmc = 3 };

__host__ __device__ __forceinline__ uint4 philox_block(uint64_t seed, uint32_t block, uint32_t stream,
                                                       uint64_t sample) {
  return philox4x32_10(make_uint4(block, stream, (uint32_t)sample, (uint32_t)(sample >> 32)),
                       make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}

// 53-bit uniform in [0, 1) of step k.
__host__ __device__ __forceinline__ double site_uniform(uint64_t seed, uint64_t sample, int k) {
  const uint4 w = philox_block(seed, (uint32_t)k, kStreamSite, sample);
  const uint64_t bits = ((uint64_t)(w.x >> 5) << 26) | (uint64_t)(w.y >> 6);
  return (double)bits * 0x1p-53;
}

// Uniform in [0, 1) that decides whether eigenvector j of an L-ensemble is kept
// (stream 2, block j; built like the site uniforms).
__host__ __device__ __forceinline__ double select_uniform(uint64_t seed, uint64_t sample, int64_t j) {
  const uint4 w = philox_block(seed, (uint32_t)j, kStreamSelect, sample);
  const uint64_t bits = ((uint64_t)(w.x >> 5) << 26) | (uint64_t)(w.y >> 6);
  return (double)bits * 0x1p-53;
}

// Slice buffers of the tensor-core trailing update: A [b][slice][KP][64] and B
// [b][slice][re/im][TP][64] BF16, row scales As [b][KP] and column scales Bs [b][TP].
struct OzArgs {
  __nv_bfloat16* A;
  __nv_bfloat16* B;
  float* As;
  float* Bs;
  int64_t KP, TP;
};

// C's slices for the tensor-core new-row update: [b][chunk][slice][32][64] BF16 and the
// row scales [b][chunk][32]; n_chunks = chunks of 64 K elements per sample (64 old rows
// of a real state, 32 of a complex one as interleaved real and imaginary parts).
struct OzYArgs {
  __nv_bfloat16* C;
  float* Cs;
  int64_t n_chunks;
};

// ------------------------------------------------------------------ status word
__device__ __forceinline__ void set_status(int* status, int code) { atomicCAS(status, 0, code); }

}  // namespace fermi

// ------------------------------------------------------------------ the handle
struct ffs_ctx {
  int64_t L = 0, N = 0;
  int dtype = 0;
  bool cplx = false;
  unsigned flags = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
  int num_sms = 0;
  std::string last_error;

  // U on the device.
  void* U64 = nullptr;      // L x N double / cd: rows gathered by the per-sample state update
  float* Ue32 = nullptr;    // FP32 residual operand, real embedding Lr x Kr (batched form)
  __nv_bfloat16* Ue_hi = nullptr;  // BF16 hi / lo planes of the real embedding (tensor-core forms)
  __nv_bfloat16* Ue_lo = nullptr;
  float* Ue_tf32 = nullptr;        // TF32-rounded FP32 plane (TF32 form)
  void* UT32 = nullptr;     // N x L float / cf: columns of U, contiguous in y (plain form)
  void* Ust = nullptr;      // L x N in the blocked state's type when it is not FP64 (owned)
  int64_t Lr = 0, Kr = 0;   // real-embedding sizes: (L, N) real, (2L, 2N) complex
  int64_t Kp = 0;           // Kr padded to the tensor-core K tile
  int64_t Lrp = 0;          // Lr padded to the tensor-core site tile

  // Workspace for one wave of samples (grown on demand).
  int64_t ws_B = 0;
  size_t W_bytes = 0, W0P_bytes = 0;  // capacities of the state buffers
  int64_t ws_steps = 0;
  int32_t* m = nullptr;          // Bw x N column orders
  uint32_t* mask = nullptr;      // Bw x ceil(L/32) chosen-site bits
  void* H = nullptr;             // Bw x Kp residual operand (per-mode element type / planes)
  float* P = nullptr;            // Bw x ldP masked weights |u_y^T h|^2 of the current step
  float* G = nullptr;            // Bw x ldG their sums per group of 32 (real) or 16 (complex) sites
  void* W = nullptr;             // elimination state (state precision): Bw x N x N unblocked,
                                 // Bw x Nc x round_up(Nc, 32) in 32-column slabs when blocked
  void* W0P = nullptr;           // Bw x N x 32 old rows' panel columns at the panel start
  void* Sinv = nullptr;          // Bw x 32 x 32 inverse of the panel Schur complement
  double* logp = nullptr;        // Bw
  int32_t* xbuf = nullptr;       // Bw x n_steps when the caller's buffer is on the host
  int32_t* fbuf = nullptr;       // Bw x n_steps teacher-forcing copy
  int32_t* permbuf = nullptr;    // Bw x N
  double* logpbuf = nullptr;     // Bw
  float* probsbuf = nullptr;     // Bw x n_steps x L (only when asked)
  int64_t probs_cap = 0;
  int64_t ldP = 0;
  int64_t ldG = 0;
  int64_t ldMask = 0;

  // TMA descriptors of the tensor-core residual: the two planes of Ue and of H.
  CUtensorMap tmU[2];
  CUtensorMap tmH[2];
  int tm_U_ready = -1;   // operand mode * 1000 + column tile that tmU was encoded for
  int res_bn = 0;        // residual column tile in use (0: not chosen yet)
  int64_t tm_H_B = -1;   // workspace capacity tmH was encoded for
  double* sel_p = nullptr;       // N keep probabilities lambda / (lambda + 1) (L-ensemble calls)
  // Tensor-core trailing update (FFS_TRAILING_TC): BF16 slices of W0_P and Bot, their
  // power-of-two scales, and the tensor maps of the slice planes.
  void* oz_buf = nullptr;
  size_t oz_bytes = 0;
  fermi::OzArgs oz{};
  CUtensorMap ozA, ozB;
  CUtensorMap ozA2, ozB2;  // real states: the packed pair layouts of the same buffers
  int64_t oz_key_B = -1, oz_key_Nc = -1;
  // Tensor-core new-row update (FFS_TRAILING_TC, real U): C's slices and their tensor map.
  void* ozy_buf = nullptr;
  size_t ozy_bytes = 0;
  fermi::OzYArgs ozy{};
  CUtensorMap ozyC;
  int64_t ozy_key_B = -1, ozy_key_Nc = -1;
  // Grouped form: per group of 128 samples a copy of the residual operand planes with the
  // K columns in the group's order ([planes][groups][Lrp][Kp]) and its tensor maps.
  void* Ug = nullptr;
  size_t Ug_bytes = 0;
  int64_t Ug_groups = 0;
  CUtensorMap tmUg[2];
  int tmUg_key = -1;
  int64_t tmUg_groups = 0;
  int* status = nullptr;         // device status word
  int* status_host = nullptr;    // pinned mirror
  int debug_fault = 0;           // FFS_FAULT_*: armed by ffs_debug_inject for the next launch

  // Optional per-phase timing with CUDA events on the launching stream.
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<int> prof_phase;   // phase of event pair i (events 2i, 2i+1)
  double prof_ms[8] = {0};
  int64_t prof_launches[8] = {0};
};

namespace fermi {
// Handle internals shared by the C-ABI file and the multi-instance engine.
int ctx_op_mode(const ffs_ctx* c);
int ctx_state_kind(const ffs_ctx* c);
bool ctx_blocked(const ffs_ctx* c);
int ctx_ensure_workspace(ffs_ctx* c, int64_t B);
size_t ctx_per_sample_bytes(const ffs_ctx* c);
size_t ctx_op_elem_bytes(int op);
int ctx_fail(ffs_ctx* c, int code, const std::string& msg);
bool ptr_is_device(const void* p);
void set_null_handle_error(const std::string& msg);
}  // namespace fermi
