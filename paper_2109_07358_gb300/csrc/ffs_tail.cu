// Blocked per-sample elimination state of the batched form.
//
// The state of a sample after k steps is the Gauss-Jordan form
//   W = A^-1 U[x_<k, m_>=k],  A = U[x_<k, m_<k]
// (Section S-1 carries the elimination of every new base row in the full N-dim space;
// here the base rows are also reduced against each other, so that the next normal
// vector is simply h_{k+1} = (-W[:, k+1] ; 1) in the sample's column order).
//
// Updating all N-k future columns at every step costs a pass over the whole state per
// step.  Instead the columns are processed in panels of NB = 32:
//   per step (tail_step_kernel): draw x_k; reduce the new row u = U[x_k, m] against the
//     state only on the remaining panel columns [k, k1); pivot s_k = the reduced value at
//     column k (the Schur residual of x_k); rank-1 update of the panel columns; save w_k
//     (the old column k, i.e. the current normal vector) and the couplings
//     beta[k][k'] = u_k' - u_<k' . w_k' for the earlier panel steps k'.
//   per panel (tail_panel_kernel), for the trailing columns T = [k1, Nc):
//     Y   = U[x_new, m_T] - U[x_new, m_<k0] W0_T            (GEMM, nb x k0 x |T|)
//     n_i = (Y_i - sum_{i'<i} beta[i][i'] n_i') / s_i       (forward substitution)
//     W[old rows, T] = W0_T - Wsave_old n                    (GEMM, k0 x nb x |T|)
//     W[new row j, T] = n_j - sum_{i>j} w_{k0+i}[k0+j] n_i
//   which is exactly the sequence of per-step updates the unblocked form would apply
//   to T, regrouped.  The state therefore stays identical in exact arithmetic.
// Only the first Nc = n_steps columns are kept (marginal sampling needs no more).
#include <type_traits>

#include "ffs_arith.cuh"
#include "ffs_draw.cuh"
#include "ffs_group.cuh"
#include "ffs_kernels.cuh"

namespace fermi {

constexpr int NB = 32;  // panel width (== warp size: one lane per panel column)

__device__ __forceinline__ void put_out(const StepArgs& a, int op, int64_t b, int col, double v) {
  const size_t idx = (size_t)b * a.Kp + col;
  switch (op) {
    case kOpF32: ((float*)a.H)[idx] = (float)v; break;
    case kOpTF32: {
      uint32_t r;
      asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"((float)v));
      ((float*)a.H)[idx] = __uint_as_float(r);
      break;
    }
    case kOpBF16x3: {
      const __nv_bfloat16 hi = __double2bfloat16(v);
      ((__nv_bfloat16*)a.H)[idx] = hi;
      ((__nv_bfloat16*)a.H)[a.hplane + idx] = __double2bfloat16(v - (double)__bfloat162float(hi));
      break;
    }
    case kOpBF16: ((__nv_bfloat16*)a.H)[idx] = __double2bfloat16(v); break;
    default: break;
  }
}
__device__ __forceinline__ void put_h(const StepArgs& a, int op, int64_t b, int col, double v) {
  put_out(a, op, b, col, v);
}
__device__ __forceinline__ void put_h(const StepArgs& a, int op, int64_t b, int col, cd v) {
  put_out(a, op, b, 2 * col, v.re);
  put_out(a, op, b, 2 * col + 1, v.im);
}

// Step k of sample b of one instance, executed by one 256-thread CTA.
template <typename A>
__device__ __forceinline__ void step_body(const StepArgs& a, const BlockedArgs& t, int64_t b, int64_t k,
                                          int op_mode, unsigned char* smem_raw, DrawShared& dsh) {
  using T = Ar<A>;
  using U = typename T::U;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t N = a.N, Nc = t.Nc;
  const float* __restrict__ prow = a.P + b * a.ldP;

  double Z = 0.0;
  const int x = block_draw(prow, a.L, a.seed, a.first + (uint64_t)b, k, forced_site(a, b, k), a.status, dsh, Z);
  draw_outputs(a, b, k, x, Z, prow);
  if (k + 1 >= a.n_steps) return;

  const int64_t k0 = (k / NB) * NB, i = k - k0, k1 = min(k0 + NB, Nc);
  A* W = (A*)t.W + (size_t)b * N * N;
  A* WsT = (A*)t.WsT + (size_t)b * N * NB;
  A* beta = (A*)t.beta + (size_t)b * NB * NB;
  A* piv = (A*)t.piv + (size_t)b * NB;
  A* r = (A*)smem_raw;
  A* wk = r + Nc;
  A* red = wk + Nc;  // 8 x 32 partial sums
  A* nv = red + 8 * 32;
  int* ms = (int*)(nv + 32);
  const int32_t* mrow = a.m + b * N;
  const U* urow = (const U*)a.U64 + (int64_t)x * N;
  for (int64_t c = tid; c < Nc; c += blockDim.x) {
    const int mc = mrow[c];
    ms[c] = mc;
    r[c] = T::from(urow[mc]);
  }
  for (int64_t j = tid; j < k; j += blockDim.x) {
    const A w = W[j * N + k];
    wk[j] = w;
    WsT[j * NB + i] = w;
  }
  __syncthreads();

  // couplings with the earlier steps of this panel: beta[i][i'] = u_k' - u_<k' . w_k'
  for (int64_t ip = warp; ip < i; ip += 8) {
    const int64_t kp = k0 + ip;
    A acc = T::zero();
    for (int64_t j = lane; j < kp; j += 32) acc = T::fms(acc, r[j], WsT[j * NB + ip]);
    for (int o = 16; o; o >>= 1) acc = T::add(acc, shfl_xor_any(acc, o));
    if (lane == 0) beta[i * NB + ip] = T::add(r[kp], acc);
  }

  // reduce the new row on the panel columns [k, k1): lane = column, warp = row group
  const int64_t c = k + lane;
  const bool cval = c < k1;
  A part = T::zero();
  if (cval)
    for (int64_t j = warp; j < k; j += 8) part = T::fms(part, r[j], W[j * N + c]);
  red[warp * 32 + lane] = part;
  __syncthreads();
  if (warp == 0 && cval) {
    A s = r[c];
    for (int w = 0; w < 8; ++w) s = T::add(s, red[w * 32 + lane]);
    nv[lane] = s;
  }
  __syncthreads();
  const A s = nv[0];  // pivot: the Schur residual of x_k
  if (tid == 0) {
    piv[i] = s;
    const double s2 = T::abs2(s);
    if (!(s2 > 1e-300) || !isfinite(s2)) set_status(a.status, FFS_E_NUMERIC);
  }
  __syncthreads();
  if (warp == 0 && cval && lane > 0) nv[lane] = T::div(nv[lane], s);
  __syncthreads();
  if (cval && lane > 0) {
    const A ncv = nv[lane];
    for (int64_t j = warp; j < k; j += 8) W[j * N + c] = T::fms(W[j * N + c], wk[j], ncv);
    if (warp == 0) W[k * N + c] = ncv;
  }
  __syncthreads();

  // operand of step k+1 while column k+1 is still inside this panel
  if (op_mode != kOpNone && k + 1 < k1) {
    for (int64_t j = tid; j <= k + 1; j += blockDim.x) {
      const A v = (j <= k) ? T::neg(W[j * N + k + 1]) : T::one();
      put_h(a, op_mode, b, ms[j], T::out(v));
    }
  }
}

template <typename A>
__global__ void __launch_bounds__(256) tail_step_kernel(StepArgs a, BlockedArgs t, int64_t k, int op_mode) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ DrawShared dsh;
  step_body<A>(a, t, blockIdx.x, k, op_mode, smem_raw, dsh);
}

// Trailing update of sample b on the 32 columns cb of T = [k1, Nc), one 256-thread CTA.
template <typename A>
__device__ __forceinline__ void panel_body(const StepArgs& a, const BlockedArgs& t, int64_t b, int64_t cb,
                                           int64_t k0, int64_t k1, int op_mode, unsigned char* smem_raw) {
  using T = Ar<A>;
  using U = typename T::U;
  A* Ys = (A*)smem_raw;         // NB x 32: Y, then n
  A* Cs = Ys + NB * 32;         // NB x 32: U[x_new, m_j] chunk
  A* Ws = Cs + NB * 32;         // 32 x 32: W chunk
  A* bs = Ws + 32 * 32;         // NB x NB couplings
  A* ps = bs + NB * NB;         // NB pivots
  int* xs = (int*)(ps + NB);    // NB new sites
  int* mj = xs + NB;            // 32: m of the current K chunk
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t N = a.N, Nc = t.Nc;
  const int nbr = (int)(k1 - k0);
  const int64_t c0 = k1 + cb * 32;
  const int64_t c = c0 + lane;
  const bool cval = c < Nc;
  A* W = (A*)t.W + (size_t)b * N * N;
  const A* WsT = (const A*)t.WsT + (size_t)b * N * NB;
  const int32_t* mrow = a.m + b * N;
  const U* U64 = (const U*)a.U64;

  for (int e = tid; e < NB * NB; e += blockDim.x) bs[e] = ((const A*)t.beta)[(size_t)b * NB * NB + e];
  if (tid < NB) {
    ps[tid] = ((const A*)t.piv)[(size_t)b * NB + tid];
    xs[tid] = tid < nbr ? a.x[b * a.n_steps + k0 + tid] : 0;
  }
  __syncthreads();

  // Y = U[x_new, m_T] - U[x_new, m_<k0] W0_T; thread owns rows warp + 8q, column lane
  const int mc = cval ? mrow[c] : 0;
  A acc[NB / 8];
#pragma unroll
  for (int q = 0; q < NB / 8; ++q) {
    const int ii = warp + 8 * q;
    acc[q] = (ii < nbr && cval) ? T::from(U64[(int64_t)xs[ii] * N + mc]) : T::zero();
  }
  for (int64_t j0 = 0; j0 < k0; j0 += 32) {
    if (tid < 32) mj[tid] = (j0 + tid < k0) ? mrow[j0 + tid] : 0;
    __syncthreads();
    for (int e = tid; e < NB * 32; e += blockDim.x) {
      const int ii = e >> 5, jj = e & 31;
      Cs[e] = (ii < nbr && j0 + jj < k0) ? T::from(U64[(int64_t)xs[ii] * N + mj[jj]]) : T::zero();
    }
    for (int e = tid; e < 32 * 32; e += blockDim.x) {
      const int jj = e >> 5, cc = e & 31;
      Ws[e] = (j0 + jj < k0 && c0 + cc < Nc) ? W[(j0 + jj) * N + c0 + cc] : T::zero();
    }
    __syncthreads();
#pragma unroll 4
    for (int jj = 0; jj < 32; ++jj) {
      const A w = Ws[jj * 32 + lane];
#pragma unroll
      for (int q = 0; q < NB / 8; ++q) acc[q] = T::fms(acc[q], Cs[(warp + 8 * q) * 32 + jj], w);
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < NB / 8; ++q) Ys[(warp + 8 * q) * 32 + lane] = acc[q];
  __syncthreads();

  // n_i = (Y_i - sum_{i'<i} beta[i][i'] n_i') / s_i
  if (warp == 0 && cval) {
    for (int ii = 0; ii < nbr; ++ii) {
      A y = Ys[ii * 32 + lane];
      for (int ip = 0; ip < ii; ++ip) y = T::fms(y, bs[ii * NB + ip], Ys[ip * 32 + lane]);
      Ys[ii * 32 + lane] = T::div(y, ps[ii]);
    }
  }
  __syncthreads();

  if (cval) {
    // old rows: W0_T - Wsave n
    for (int64_t j = warp; j < k0; j += 8) {
      A v = W[j * N + c];
      const A* ws = WsT + j * NB;
      for (int ii = 0; ii < nbr; ++ii) v = T::fms(v, ws[ii], Ys[ii * 32 + lane]);
      W[j * N + c] = v;
    }
    // new rows: n_j - sum_{i>j} w_{k0+i}[k0+j] n_i
    for (int jn = warp; jn < nbr; jn += 8) {
      A v = Ys[jn * 32 + lane];
      const A* ws = WsT + (k0 + jn) * NB;
      for (int ii = jn + 1; ii < nbr; ++ii) v = T::fms(v, ws[ii], Ys[ii * 32 + lane]);
      W[(k0 + jn) * N + c] = v;
    }
  }
  __syncthreads();

  // operand of step k1 (its column is the first of T)
  if (op_mode != kOpNone && cb == 0 && k1 < a.n_steps) {
    for (int64_t j = tid; j <= k1; j += blockDim.x) {
      const A v = (j < k1) ? T::neg(W[j * N + k1]) : T::one();
      put_h(a, op_mode, b, mrow[j], T::out(v));
    }
  }
}

template <typename A>
__global__ void __launch_bounds__(256) tail_panel_kernel(StepArgs a, BlockedArgs t, int64_t k0, int64_t k1,
                                                         int op_mode) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  panel_body<A>(a, t, blockIdx.y, blockIdx.x, k0, k1, op_mode, smem_raw);
}

static size_t step_smem(int64_t Nc, size_t es) { return (size_t)Nc * (2 * es + 4) + (8 * 32 + 32) * es; }
static size_t panel_smem(size_t es) { return (size_t)(NB * 32 * 2 + 32 * 32 + NB * NB + NB) * es + (NB + 32) * 4; }

// Grouped forms: CTA blockIdx.x -> (instance, sample[, column block]) through the entry list.
template <typename A>
__global__ void __launch_bounds__(256)
    step_group_kernel(const GroupInst* __restrict__ inst, const GroupEntry* __restrict__ ent, int n, int op_mode) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ DrawShared dsh;
  const int64_t item = blockIdx.x;
  const int e = group_find(ent, n, item);
  const GroupInst* gi = inst + ent[e].inst;
  const StepArgs a = gi->a;
  const BlockedArgs t = gi->t;
  step_body<A>(a, t, item - ent[e].start, ent[e].k, op_mode, smem_raw, dsh);
}

template <typename A>
__global__ void __launch_bounds__(256)
    panel_group_kernel(const GroupInst* __restrict__ inst, const GroupEntry* __restrict__ ent, int n, int op_mode) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int64_t item = blockIdx.x;
  const int e = group_find(ent, n, item);
  const GroupInst* gi = inst + ent[e].inst;
  const StepArgs a = gi->a;
  const BlockedArgs t = gi->t;
  const int64_t k = ent[e].k;
  const int64_t k0 = (k / NB) * NB, k1 = min(k0 + NB, t.Nc);
  const int64_t ncb = (t.Nc - k1 + 31) / 32;
  const int64_t local = item - ent[e].start;
  panel_body<A>(a, t, local / ncb, local % ncb, k0, k1, op_mode, smem_raw);
}

template <typename A>
static cudaError_t group_step_t(const GroupInst* inst, const GroupEntry* e, int n, int64_t total, int op,
                                int64_t maxNc, cudaStream_t s) {
  step_group_kernel<A><<<(unsigned)total, 256, step_smem(maxNc, sizeof(A)), s>>>(inst, e, n, op);
  return cudaGetLastError();
}
template <typename A>
static cudaError_t group_panel_t(const GroupInst* inst, const GroupEntry* e, int n, int64_t total, int op,
                                 cudaStream_t s) {
  panel_group_kernel<A><<<(unsigned)total, 256, panel_smem(sizeof(A)), s>>>(inst, e, n, op);
  return cudaGetLastError();
}

cudaError_t launch_group_step(const GroupInst* inst, const GroupEntry* e, int n, int64_t total, bool cplx,
                              int state, int op, int64_t maxNc, cudaStream_t s) {
  if (total <= 0) return cudaSuccess;
  if (cplx) {
    if (state == kStateFP64) return group_step_t<cd>(inst, e, n, total, op, maxNc, s);
    if (state == kStateFP32) return group_step_t<cf>(inst, e, n, total, op, maxNc, s);
    return group_step_t<cdf>(inst, e, n, total, op, maxNc, s);
  }
  if (state == kStateFP64) return group_step_t<double>(inst, e, n, total, op, maxNc, s);
  if (state == kStateFP32) return group_step_t<float>(inst, e, n, total, op, maxNc, s);
  return group_step_t<df>(inst, e, n, total, op, maxNc, s);
}

cudaError_t launch_group_panel(const GroupInst* inst, const GroupEntry* e, int n, int64_t total, bool cplx,
                               int state, int op, cudaStream_t s) {
  if (total <= 0) return cudaSuccess;
  if (cplx) {
    if (state == kStateFP64) return group_panel_t<cd>(inst, e, n, total, op, s);
    if (state == kStateFP32) return group_panel_t<cf>(inst, e, n, total, op, s);
    return group_panel_t<cdf>(inst, e, n, total, op, s);
  }
  if (state == kStateFP64) return group_panel_t<double>(inst, e, n, total, op, s);
  if (state == kStateFP32) return group_panel_t<float>(inst, e, n, total, op, s);
  return group_panel_t<df>(inst, e, n, total, op, s);
}

size_t blocked_elem_bytes(bool cplx, int state) {
  const size_t base = (state == kStateFP32) ? 4 : 8;  // FP64 and double-float are both 8 bytes
  return cplx ? 2 * base : base;
}


template <typename A>
static cudaError_t launch_step_t(const StepArgs& a, const BlockedArgs& t, int64_t k, int op, cudaStream_t s) {
  tail_step_kernel<A><<<(unsigned)a.bw, 256, step_smem(t.Nc, sizeof(A)), s>>>(a, t, k, op);
  return cudaGetLastError();
}
template <typename A>
static cudaError_t launch_panel_t(const StepArgs& a, const BlockedArgs& t, int64_t k0, int64_t k1, int op,
                                  cudaStream_t s) {
  dim3 grid((unsigned)((t.Nc - k1 + 31) / 32), (unsigned)a.bw);
  tail_panel_kernel<A><<<grid, 256, panel_smem(sizeof(A)), s>>>(a, t, k0, k1, op);
  return cudaGetLastError();
}

cudaError_t launch_blocked_step(const StepArgs& a, const BlockedArgs& t, int64_t k, int state, int op,
                                cudaStream_t s) {
  if (a.cplx) {
    if (state == kStateFP64) return launch_step_t<cd>(a, t, k, op, s);
    if (state == kStateFP32) return launch_step_t<cf>(a, t, k, op, s);
    return launch_step_t<cdf>(a, t, k, op, s);
  }
  if (state == kStateFP64) return launch_step_t<double>(a, t, k, op, s);
  if (state == kStateFP32) return launch_step_t<float>(a, t, k, op, s);
  return launch_step_t<df>(a, t, k, op, s);
}

cudaError_t launch_blocked_panel(const StepArgs& a, const BlockedArgs& t, int64_t k0, int64_t k1, int state,
                                 int op, cudaStream_t s) {
  if (k1 >= t.Nc) return cudaSuccess;
  if (a.cplx) {
    if (state == kStateFP64) return launch_panel_t<cd>(a, t, k0, k1, op, s);
    if (state == kStateFP32) return launch_panel_t<cf>(a, t, k0, k1, op, s);
    return launch_panel_t<cdf>(a, t, k0, k1, op, s);
  }
  if (state == kStateFP64) return launch_panel_t<double>(a, t, k0, k1, op, s);
  if (state == kStateFP32) return launch_panel_t<float>(a, t, k0, k1, op, s);
  return launch_panel_t<df>(a, t, k0, k1, op, s);
}

int blocked_panel_width() { return NB; }

size_t blocked_step_smem(int64_t Nc, bool cplx, int state) { return step_smem(Nc, blocked_elem_bytes(cplx, state)); }

template <typename K> static cudaError_t allow_smem(K kernel, int optin) {
  cudaFuncAttributes at;
  cudaError_t e = cudaFuncGetAttributes(&at, kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)at.sharedSizeBytes);
}

cudaError_t configure_blocked() {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess) e = allow_smem(tail_step_kernel<double>, optin);
  if (e == cudaSuccess) e = allow_smem(tail_step_kernel<float>, optin);
  if (e == cudaSuccess) e = allow_smem(tail_step_kernel<df>, optin);
  if (e == cudaSuccess) e = allow_smem(tail_step_kernel<cd>, optin);
  if (e == cudaSuccess) e = allow_smem(tail_step_kernel<cf>, optin);
  if (e == cudaSuccess) e = allow_smem(tail_step_kernel<cdf>, optin);
  if (e == cudaSuccess) e = allow_smem(tail_panel_kernel<double>, optin);
  if (e == cudaSuccess) e = allow_smem(tail_panel_kernel<float>, optin);
  if (e == cudaSuccess) e = allow_smem(tail_panel_kernel<df>, optin);
  if (e == cudaSuccess) e = allow_smem(tail_panel_kernel<cd>, optin);
  if (e == cudaSuccess) e = allow_smem(tail_panel_kernel<cf>, optin);
  if (e == cudaSuccess) e = allow_smem(tail_panel_kernel<cdf>, optin);
  if (e == cudaSuccess) e = allow_smem(step_group_kernel<double>, optin);
  if (e == cudaSuccess) e = allow_smem(step_group_kernel<float>, optin);
  if (e == cudaSuccess) e = allow_smem(step_group_kernel<df>, optin);
  if (e == cudaSuccess) e = allow_smem(step_group_kernel<cd>, optin);
  if (e == cudaSuccess) e = allow_smem(step_group_kernel<cf>, optin);
  if (e == cudaSuccess) e = allow_smem(step_group_kernel<cdf>, optin);
  if (e == cudaSuccess) e = allow_smem(panel_group_kernel<double>, optin);
  if (e == cudaSuccess) e = allow_smem(panel_group_kernel<float>, optin);
  if (e == cudaSuccess) e = allow_smem(panel_group_kernel<df>, optin);
  if (e == cudaSuccess) e = allow_smem(panel_group_kernel<cd>, optin);
  if (e == cudaSuccess) e = allow_smem(panel_group_kernel<cf>, optin);
  if (e == cudaSuccess) e = allow_smem(panel_group_kernel<cdf>, optin);
  return e;
}

}  // namespace fermi
