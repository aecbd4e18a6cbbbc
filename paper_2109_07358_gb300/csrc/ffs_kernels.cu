// libffs kernels: permutations, operand derivation, the CUDA-core residuals (plain
// per-sample form and the FP32 batched form), and the per-sample draw + elimination
// state update.  The tensor-core residual lives in ffs_residual_tc.cu.
//
// Fast fermion sampling, arXiv 2109.07358.  Step k (0-based) of sample b:
//   h      = (-w ; 1) in the sample's column order m, w = A^-1 b with A = U[x_<k, m_<k],
//            b = U[x_<k, m_k]                                   (Eq. 3 normal vector)
//   v_y    = u_y^T h = U[y, m_k] - U[y, m_<k] w   for all sites y  (Section S-1 products)
//   p_y    = |v_y|^2, 0 on sites already drawn
//   x_k    = first y with p_y > 0 and C_y > u Z, C the running sum, Z its total
//   state  the Gauss-Jordan form W = A^-1 U[x_<k, m_>=k] (Section S-1: elimination
//          carried in the full N-dim space), updated by the new row x_k.
#include <climits>
#include <cstdio>
#include <type_traits>

#include "ffs_draw.cuh"
#include "ffs_group.cuh"
#include "ffs_kernels.cuh"

namespace fermi {

constexpr unsigned kFull = 0xffffffffu;

template <typename S> struct is_cplx : std::false_type {};
template <> struct is_cplx<cd> : std::true_type {};
template <> struct is_cplx<cf> : std::true_type {};

__device__ __forceinline__ float to_tf32(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return __uint_as_float(r);
}

// Write one real entry e of operand row b (mode-specific encoding).
__device__ __forceinline__ void put_operand_entry(const StepArgs& a, int op, int64_t b, int64_t e,
                                                  double v) {
  const size_t idx = (size_t)b * a.Kp + e;
  switch (op) {
    case kOpF32:
      ((float*)a.H)[idx] = (float)v;
      break;
    case kOpTF32:
      ((float*)a.H)[idx] = to_tf32((float)v);
      break;
    case kOpBF16x3: {
      const __nv_bfloat16 hi = __double2bfloat16(v);
      const __nv_bfloat16 lo = __double2bfloat16(v - (double)__bfloat162float(hi));
      ((__nv_bfloat16*)a.H)[idx] = hi;
      ((__nv_bfloat16*)a.H)[a.hplane + idx] = lo;
      break;
    }
    case kOpBF16:
      ((__nv_bfloat16*)a.H)[idx] = __double2bfloat16(v);
      break;
    default:
      break;
  }
}

__device__ __forceinline__ void put_operand(const StepArgs& a, int op, int64_t b, int col, double v) {
  put_operand_entry(a, op, b, col, v);
}
__device__ __forceinline__ void put_operand(const StepArgs& a, int op, int64_t b, int col, float v) {
  put_operand_entry(a, op, b, col, (double)v);
}
__device__ __forceinline__ void put_operand(const StepArgs& a, int op, int64_t b, int col, cd v) {
  put_operand_entry(a, op, b, 2 * (int64_t)col, v.re);
  put_operand_entry(a, op, b, 2 * (int64_t)col + 1, v.im);
}
__device__ __forceinline__ void put_operand(const StepArgs& a, int op, int64_t b, int col, cf v) {
  put_operand_entry(a, op, b, 2 * (int64_t)col, (double)v.re);
  put_operand_entry(a, op, b, 2 * (int64_t)col + 1, (double)v.im);
}

// ------------------------------------------------------------------------ a1 permutation
// One thread per sample: Fisher-Yates over (0..N-1) driven by Philox stream 0 (block j
// serves shuffle steps N-1-2j and N-2-2j, 64 bits each, index = mulhi(r, i+1)).  Also
// writes the step-0 operand h = e_{m_0} (the operand buffer is zeroed beforehand).
// L-ensemble (sel_p set): column j is kept when its stream-2 uniform is below sel_p[j];
// the kept columns, ascending, are shuffled the same way over their count n, and the
// others follow in ascending order (the chain never reaches them).
__device__ __forceinline__ bool kept_column(const StepArgs& a, uint64_t sample, int64_t j) {
  return select_uniform(a.seed, sample, j) < a.sel_p[j];
}

__device__ __forceinline__ void perm_one(const StepArgs& a, int op_mode, int64_t b) {
  // grouped form: every sample of a group draws the order of the group's first index
  const uint64_t sample = a.grouped ? (a.first + (uint64_t)b) / FFS_GROUP_SIZE * FFS_GROUP_SIZE
                                    : a.first + (uint64_t)b;
  int32_t* m = const_cast<int32_t*>(a.m) + b * a.N;
  int64_t n = a.N;
  if (a.sel_p) {
    n = 0;
    for (int64_t j = 0; j < a.N; ++j)
      if (kept_column(a, sample, j)) m[n++] = (int32_t)j;
    int64_t r = n;
    for (int64_t j = 0; j < a.N; ++j)
      if (!kept_column(a, sample, j)) m[r++] = (int32_t)j;
    if (n == 0) return;
  } else {
    for (int64_t i = 0; i < a.N; ++i) m[i] = (int32_t)i;
  }
  int64_t i = n - 1;
  uint32_t block = 0;
  while (i >= 1) {
    const uint4 w = philox_block(a.seed, block, kStreamPerm, sample);
    {
      const uint64_t r = ((uint64_t)w.x << 32) | w.y;
      const int64_t j = (int64_t)__umul64hi(r, (uint64_t)(i + 1));
      const int32_t t = m[i];
      m[i] = m[j];
      m[j] = t;
      --i;
    }
    if (i >= 1) {
      const uint64_t r = ((uint64_t)w.z << 32) | w.w;
      const int64_t j = (int64_t)__umul64hi(r, (uint64_t)(i + 1));
      const int32_t t = m[i];
      m[i] = m[j];
      m[j] = t;
      --i;
    }
    ++block;
  }
  if (op_mode != kOpNone) {
    const int col = a.grouped ? 0 : m[0];
    if (a.cplx)
      put_operand(a, op_mode, b, col, cd{1.0, 0.0});
    else
      put_operand(a, op_mode, b, col, 1.0);
  }
}

// Grouped form: dst[g] = the operand planes with their K columns in group g's order:
// column pair (2q, 2q + 1) of a complex embedding (column q of a real one) takes the
// source column of U column m_g[q]; the padding columns past Kr are copied as they are.
__global__ void group_embed_kernel(const void* src0, const void* src1, void* dst, int64_t Lrp, int64_t Kp,
                                   int64_t Kr, bool cplx, bool f32, int planes, const int32_t* m, int64_t N,
                                   int64_t plane_groups) {
  const int64_t g = blockIdx.y, y = blockIdx.x;
  const int32_t* mg = m + g * FFS_GROUP_SIZE * N;
  for (int pl = 0; pl < planes; ++pl) {
    const void* src = pl == 0 ? src0 : src1;
    for (int64_t c = threadIdx.x; c < Kp; c += blockDim.x) {
      int64_t sc = c;
      if (c < Kr) sc = cplx ? 2 * (int64_t)mg[c >> 1] + (c & 1) : (int64_t)mg[c];
      const size_t di = (((size_t)pl * plane_groups + g) * Lrp + y) * Kp + c;
      if (f32)
        ((float*)dst)[di] = ((const float*)src)[y * Kp + sc];
      else
        ((__nv_bfloat16*)dst)[di] = ((const __nv_bfloat16*)src)[y * Kp + sc];
    }
  }
}

cudaError_t launch_group_embed(const void* src0, const void* src1, void* dst, int64_t Lrp, int64_t Kp, int64_t Kr,
                               bool cplx, bool f32, int planes, const int32_t* m, int64_t N, int64_t groups,
                               int64_t plane_groups, cudaStream_t s) {
  if (groups <= 0) return cudaSuccess;
  group_embed_kernel<<<dim3((unsigned)Lrp, (unsigned)groups), 256, 0, s>>>(src0, src1, dst, Lrp, Kp, Kr, cplx, f32,
                                                                           planes, m, N, plane_groups);
  return cudaGetLastError();
}

// L-ensemble: the chain length of every sample (the number of kept columns) and its
// maximum over the call.
__global__ void lens_count_kernel(StepArgs a, int64_t B, int32_t* nlen, int* max_len) {
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b >= B) return;
  int n = 0;
  for (int64_t j = 0; j < a.N; ++j) n += kept_column(a, a.first + (uint64_t)b, j) ? 1 : 0;
  nlen[b] = n;
  atomicMax(max_len, n);
}

// Keep probabilities lambda / (lambda + 1) (lambda <= 0: never kept); a non-finite
// lambda is an argument error.
__global__ void keep_prob_kernel(const double* lambda, int64_t N, double* p, int* status) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= N) return;
  const double l = lambda[j];
  if (!isfinite(l)) set_status(status, FFS_E_ARG);
  p[j] = (l > 0.0 && isfinite(l)) ? l / (l + 1.0) : 0.0;
}

cudaError_t launch_lens_count(const StepArgs& a, int64_t B, int32_t* nlen, int* max_len, cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  lens_count_kernel<<<(unsigned)((B + 127) / 128), 128, 0, s>>>(a, B, nlen, max_len);
  return cudaGetLastError();
}

cudaError_t launch_keep_prob(const double* lambda, int64_t N, double* p, int* status, cudaStream_t s) {
  keep_prob_kernel<<<(unsigned)((N + 127) / 128), 128, 0, s>>>(lambda, N, p, status);
  return cudaGetLastError();
}

__global__ void perm_init_kernel(StepArgs a, int op_mode) {
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b >= a.bw) return;
  perm_one(a, op_mode, b);
}

// Grouped start of a wave: per sample, clear its operand row, drawn-site bits and
// log-probability, then draw its column order (128 samples per CTA).
__global__ void group_init_kernel(const GroupInst* __restrict__ inst, const GroupEntry* __restrict__ ent, int n,
                                  int op_mode) {
  const int64_t item = blockIdx.x;
  const int e = group_find(ent, n, item);
  const StepArgs a = inst[ent[e].inst].a;
  const int64_t b = (item - ent[e].start) * 128 + threadIdx.x;
  if (b >= a.bw) return;
  if (op_mode == kOpF32 || op_mode == kOpTF32) {
    float* h = (float*)a.H + b * a.Kp;
    for (int64_t i = 0; i < a.Kp; ++i) h[i] = 0.f;
  } else if (op_mode == kOpBF16x3 || op_mode == kOpBF16) {
    __nv_bfloat16* h = (__nv_bfloat16*)a.H + b * a.Kp;
    for (int64_t i = 0; i < a.Kp; ++i) h[i] = __float2bfloat16(0.f);
    if (op_mode == kOpBF16x3)
      for (int64_t i = 0; i < a.Kp; ++i) h[a.hplane + i] = __float2bfloat16(0.f);
  }
  for (int64_t i = 0; i < a.ldMask; ++i) a.mask[b * a.ldMask + i] = 0u;
  a.logp[b] = 0.0;
  perm_one(a, op_mode, b);
}

cudaError_t launch_group_init(const GroupInst* inst, const GroupEntry* e, int n, int64_t total, int op,
                              cudaStream_t s) {
  if (total <= 0) return cudaSuccess;
  group_init_kernel<<<(unsigned)total, 128, 0, s>>>(inst, e, n, op);
  return cudaGetLastError();
}

cudaError_t launch_perm_init(const StepArgs& a, int op_mode, cudaStream_t s) {
  if (a.bw <= 0) return cudaSuccess;
  const int threads = 128;
  perm_init_kernel<<<(unsigned)((a.bw + threads - 1) / threads), threads, 0, s>>>(a, op_mode);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------ U^dagger U check
// max_ij |(U^dagger U)_ij - delta_ij| in FP64, 32 x 32 tiles of the Gram matrix.
template <bool CPLX>
__global__ void __launch_bounds__(256) ortho_kernel(const void* U64, int64_t L, int64_t N,
                                                    unsigned long long* maxbits) {
  using T = typename std::conditional<CPLX, cd, double>::type;
  const T* U = (const T*)U64;
  __shared__ T Ai[32][33];
  __shared__ T Aj[32][33];
  const int tid = threadIdx.x;
  const int64_t i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  const int ti = tid / 32, tj = tid % 32;  // thread owns rows ti, ti+8, ti+16, ti+24 of the tile
  T acc[4];
  for (int q = 0; q < 4; ++q) acc[q] = s_zero<T>();
  for (int64_t y0 = 0; y0 < L; y0 += 32) {
    for (int e = tid; e < 1024; e += 256) {
      const int yy = e / 32, cc = e % 32;
      const int64_t y = y0 + yy;
      Ai[yy][cc] = (y < L && i0 + cc < N) ? U[y * N + i0 + cc] : s_zero<T>();
      Aj[yy][cc] = (y < L && j0 + cc < N) ? U[y * N + j0 + cc] : s_zero<T>();
    }
    __syncthreads();
    for (int yy = 0; yy < 32; ++yy) {
      const T bj = Aj[yy][tj];
      for (int q = 0; q < 4; ++q) {
        T ai = Ai[yy][ti + 8 * q];
        if constexpr (CPLX) {
          ai.im = -ai.im;  // conj
          acc[q] = fms(acc[q], -ai, bj);
        } else {
          acc[q] = fma(ai, bj, acc[q]);
        }
      }
    }
    __syncthreads();
  }
  double dev = 0.0;
  for (int q = 0; q < 4; ++q) {
    const int64_t i = i0 + ti + 8 * q, j = j0 + tj;
    if (i < N && j < N) {
      T g = acc[q];
      double d;
      if constexpr (CPLX)
        d = sqrt(((i == j) ? (g.re - 1.0) * (g.re - 1.0) : g.re * g.re) + g.im * g.im);
      else
        d = fabs(g - (i == j ? 1.0 : 0.0));
      if (!(d == d)) d = 1e300;  // NaN counts as failure
      dev = fmax(dev, d);
    }
  }
  for (int o = 16; o; o >>= 1) dev = fmax(dev, __shfl_xor_sync(kFull, dev, o));
  if ((tid & 31) == 0) atomicMax(maxbits, (unsigned long long)__double_as_longlong(dev));
}

cudaError_t launch_ortho_check(const void* U64, bool cplx, int64_t L, int64_t N, double* maxdev,
                               cudaStream_t s) {
  unsigned long long* d = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&d, sizeof(*d), s);
  if (e != cudaSuccess) return e;
  cudaMemsetAsync(d, 0, sizeof(*d), s);
  dim3 grid((unsigned)((N + 31) / 32), (unsigned)((N + 31) / 32));
  if (cplx)
    ortho_kernel<true><<<grid, 256, 0, s>>>(U64, L, N, d);
  else
    ortho_kernel<false><<<grid, 256, 0, s>>>(U64, L, N, d);
  e = cudaGetLastError();
  unsigned long long h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFreeAsync(d, s);
  double v;
  memcpy(&v, &h, sizeof(v));
  *maxdev = v;
  return e;
}

// ------------------------------------------------------------------------ operand derivation
// Real embedding of U used by the batched residual: Lr x Kr with (Lr, Kr) = (L, N) for
// real U and (2L, 2N) for complex U, where row 2y = [Re U_yc, -Im U_yc]_c and row
// 2y+1 = [Im U_yc, Re U_yc]_c (column pairs (2c, 2c+1)), so that with the operand row
// [Re h_c, Im h_c]_c the products give (Re v_y, Im v_y) in adjacent columns.  Rows and
// columns beyond (Lr, Kr) up to (Lrp, Kp) are zero.
__global__ void derive_embed_kernel(const void* U64, bool cplx, int64_t L, int64_t N, int64_t Lrp,
                                    int64_t Kp, float* f32, __nv_bfloat16* hi, __nv_bfloat16* lo,
                                    float* tf) {
  const int64_t total = Lrp * Kp;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / Kp, c = e % Kp;
    double v = 0.0;
    if (!cplx) {
      if (r < L && c < N) v = ((const double*)U64)[r * N + c];
    } else {
      const int64_t y = r >> 1, col = c >> 1;
      if (y < L && col < N) {
        const cd u = ((const cd*)U64)[y * N + col];
        const bool rim = r & 1, cim = c & 1;
        v = (!rim) ? (cim ? -u.im : u.re) : (cim ? u.re : u.im);
      }
    }
    if (f32) f32[e] = (float)v;
    if (hi) {
      const __nv_bfloat16 h = __double2bfloat16(v);
      hi[e] = h;
      if (lo) lo[e] = __double2bfloat16(v - (double)__bfloat162float(h));
    }
    if (tf) tf[e] = to_tf32((float)v);
  }
}

// Columns of U contiguous in y (N x L), FP32, for the plain per-sample form.
__global__ void derive_transpose_kernel(const void* U64, bool cplx, int64_t L, int64_t N, void* UT) {
  const int64_t total = L * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / L, y = e % L;
    if (cplx) {
      const cd u = ((const cd*)U64)[y * N + c];
      ((cf*)UT)[e] = cf{(float)u.re, (float)u.im};
    } else {
      ((float*)UT)[e] = (float)((const double*)U64)[y * N + c];
    }
  }
}

cudaError_t launch_derive_operands(ffs_ctx* c, cudaStream_t s) {
  if (c->Ue32 || c->Ue_hi || c->Ue_tf32) {
    derive_embed_kernel<<<4 * c->num_sms, 256, 0, s>>>(c->U64, c->cplx, c->L, c->N, c->Lrp, c->Kp, c->Ue32,
                                                       c->Ue_hi, c->Ue_lo, c->Ue_tf32);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (c->UT32) {
    derive_transpose_kernel<<<4 * c->num_sms, 256, 0, s>>>(c->U64, c->cplx, c->L, c->N, c->UT32);
    return cudaGetLastError();
  }
  return cudaSuccess;
}

// ------------------------------------------------------------------------ residual, FP32 batched
// P[b, y] = |sum_c H[b, c] Ue[j, c]|^2 over the real embedding (one column, or a column
// pair for complex U), 0 on sites already drawn.  64 samples x 64 embedding columns
// per CTA, 4 x 4 per thread, K chunks of 16 through shared memory.
template <bool CPLX>
__global__ void __launch_bounds__(256) residual_fp32_kernel(StepArgs a, const float* __restrict__ Ue) {
  __shared__ float As[16][68];
  __shared__ float Bs[16][68];
  const float* __restrict__ H = (const float*)a.H;
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
  const int64_t b0 = (int64_t)blockIdx.y * 64, j0 = (int64_t)blockIdx.x * 64;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int64_t kc = 0; kc < a.Kr; kc += 16) {
    for (int e = tid; e < 1024; e += 256) {
      const int r = e >> 4, c = e & 15;
      const int64_t bb = b0 + r, jj = j0 + r, kk = kc + c;
      As[c][r] = (bb < a.bw && kk < a.Kr) ? H[bb * a.Kp + kk] : 0.f;
      Bs[c][r] = (jj < a.Lr && kk < a.Kr) ? Ue[jj * a.Kp + kk] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      float av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        av[i] = As[c][ty * 4 + i];
        bv[i] = Bs[c][tx * 4 + i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t bb = b0 + ty * 4 + i;
    if (bb >= a.bw) continue;
    const uint32_t* mk = a.mask + bb * a.ldMask;
#pragma unroll
    for (int j = 0; j < 4; j += (CPLX ? 2 : 1)) {
      const int64_t col = j0 + tx * 4 + j;
      const int64_t y = CPLX ? (col >> 1) : col;
      if (y >= a.L) continue;
      float p = CPLX ? acc[i][j] * acc[i][j] + acc[i][j + 1] * acc[i][j + 1] : acc[i][j] * acc[i][j];
      if ((mk[y >> 5] >> (y & 31)) & 1u) p = 0.f;
      a.P[bb * a.ldP + y] = p;
    }
  }
}

cudaError_t launch_residual_fp32(const StepArgs& a, const float* Ue32, cudaStream_t s) {
  dim3 grid((unsigned)((a.Lr + 63) / 64), (unsigned)((a.bw + 63) / 64));
  if (a.cplx)
    residual_fp32_kernel<true><<<grid, 256, 0, s>>>(a, Ue32);
  else
    residual_fp32_kernel<false><<<grid, 256, 0, s>>>(a, Ue32);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------ residual, plain form
// One CTA per sample: v_y = sum_{j<=k} U[y, m_j] h_j over the sample's own columns, FP32,
// with h = (-W[:, k] ; 1) read from the FP32 state.
template <typename S>
__global__ void __launch_bounds__(256) residual_plain_kernel(StepArgs a, const S* __restrict__ UT, int64_t k) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  S* h = (S*)smem_raw;
  int* mc = (int*)(h + a.N);
  const int64_t b = blockIdx.x;
  const S* W = (const S*)a.W + (size_t)b * a.N * a.N;
  for (int64_t j = threadIdx.x; j <= k; j += blockDim.x) {
    h[j] = (j < k) ? -W[j * a.N + k] : s_one<S>();
    mc[j] = a.m[b * a.N + j];
  }
  __syncthreads();
  const uint32_t* mk = a.mask + b * a.ldMask;
  for (int64_t y = threadIdx.x; y < a.L; y += blockDim.x) {
    S acc = s_zero<S>();
    for (int64_t j = 0; j <= k; ++j) acc = fms(acc, -UT[(int64_t)mc[j] * a.L + y], h[j]);
    float p = (float)abs2(acc);
    if ((mk[y >> 5] >> (y & 31)) & 1u) p = 0.f;
    a.P[b * a.ldP + y] = p;
  }
}

cudaError_t launch_residual_plain(const StepArgs& a, const void* UT32, int64_t k, cudaStream_t s) {
  if (a.cplx) {
    const size_t sm = a.N * (sizeof(cf) + sizeof(int));
    residual_plain_kernel<cf><<<(unsigned)a.bw, 256, sm, s>>>(a, (const cf*)UT32, k);
  } else {
    const size_t sm = a.N * (sizeof(float) + sizeof(int));
    residual_plain_kernel<float><<<(unsigned)a.bw, 256, sm, s>>>(a, (const float*)UT32, k);
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------------ draw + state update
// One CTA (256 threads, 8 warps) per sample.
//  (1) Z and the inverse CDF with a warp-shuffle block scan: warp w owns a contiguous
//      segment of sites; segment totals give each warp its base; each warp then walks
//      its segment 32 sites at a time with an inclusive shuffle scan until the running
//      sum passes t = u Z.  The order of every sum is fixed, so a sample's draw never
//      depends on the batch it runs in.
//  (2) outputs: x_k, the chosen-site mask, log-probability, optional conditional.
//  (3) Gauss-Jordan update of the state with the row U[x_k, m]: r' = r - r_<k W,
//      pivot s = r'_k, n = r'_>k / s, W_<k,>k -= W_<k,k n, new row n.
//  (4) the operand of step k+1: h = (-W[:, k+1] ; 1) scattered to columns m_0..m_{k+1}.
template <typename S>
__global__ void __launch_bounds__(256) tail_kernel(StepArgs a, int64_t k, int op_mode) {
  using Ud = typename std::conditional<is_cplx<S>::value, cd, double>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x;
  const int64_t b = blockIdx.x;
  const uint64_t sample = a.first + (uint64_t)b;
  const int64_t L = a.L, N = a.N;
  const float* __restrict__ prow = a.P + b * a.ldP;

  // (1) normaliser and inverse CDF, (2) outputs
  __shared__ DrawShared dsh;
  double Z = 0.0;
  const int x = block_draw(prow, L, a.seed, sample, k, forced_site(a, b, k), a.status, dsh, Z);
  draw_outputs(a, b, k, x, Z, prow);
  if (k + 1 >= a.n_steps) return;

  // (3) state update
  S* W = (S*)a.W + (size_t)b * N * N;
  S* r = (S*)smem_raw;
  S* nv = r + N;
  S* wc = nv + N;
  int* ms = (int*)(wc + N);
  const int32_t* mrow = a.m + b * N;
  const Ud* urow = (const Ud*)a.U64 + (int64_t)x * N;
  for (int64_t c = tid; c < N; c += blockDim.x) {
    const int mcol = mrow[c];
    ms[c] = mcol;
    r[c] = s_cast<S>(urow[mcol]);
  }
  __syncthreads();
  for (int64_t c = k + tid; c < N; c += blockDim.x) {
    S acc = r[c];
    for (int64_t j = 0; j < k; ++j) acc = fms(acc, r[j], W[j * N + c]);
    nv[c] = acc;
  }
  for (int64_t j = tid; j < k; j += blockDim.x) wc[j] = W[j * N + k];
  __syncthreads();
  const S s = nv[k];
  if (tid == 0 && (!(abs2(s) > 1e-300) || !s_finite(s))) set_status(a.status, FFS_E_NUMERIC);
  for (int64_t c = k + 1 + tid; c < N; c += blockDim.x) {
    const S nc = nv[c] / s;
    for (int64_t j = 0; j < k; ++j) W[j * N + c] = fms(W[j * N + c], wc[j], nc);
    W[k * N + c] = nc;
  }
  __syncthreads();

  // (4) operand of step k+1
  if (op_mode != kOpNone) {
    for (int64_t j = tid; j <= k + 1; j += blockDim.x) {
      const S v = (j <= k) ? -W[j * N + k + 1] : s_one<S>();
      put_operand(a, op_mode, b, ms[j], v);
    }
  }
}

size_t tail_smem_bytes(int64_t N, bool cplx, bool state_fp64) {
  const size_t es = cplx ? (state_fp64 ? sizeof(cd) : sizeof(cf)) : (state_fp64 ? sizeof(double) : sizeof(float));
  return (size_t)N * (3 * es + sizeof(int));
}

cudaError_t launch_tail(const StepArgs& a, int64_t k, bool state_fp64, int op_mode, cudaStream_t s) {
  const size_t sm = tail_smem_bytes(a.N, a.cplx, state_fp64);
  const unsigned grid = (unsigned)a.bw;
  if (a.cplx) {
    if (state_fp64)
      tail_kernel<cd><<<grid, 256, sm, s>>>(a, k, op_mode);
    else
      tail_kernel<cf><<<grid, 256, sm, s>>>(a, k, op_mode);
  } else {
    if (state_fp64)
      tail_kernel<double><<<grid, 256, sm, s>>>(a, k, op_mode);
    else
      tail_kernel<float><<<grid, 256, sm, s>>>(a, k, op_mode);
  }
  return cudaGetLastError();
}

// Allow each kernel the device's opt-in shared memory minus its own static shared memory.
template <typename K> static cudaError_t allow_max_smem(K kernel, int optin) {
  cudaFuncAttributes at;
  cudaError_t e = cudaFuncGetAttributes(&at, kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              optin - (int)at.sharedSizeBytes);
}

cudaError_t configure_kernels(int64_t N, bool cplx) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess) e = allow_max_smem(tail_kernel<cd>, optin);
  if (e == cudaSuccess) e = allow_max_smem(tail_kernel<cf>, optin);
  if (e == cudaSuccess) e = allow_max_smem(tail_kernel<double>, optin);
  if (e == cudaSuccess) e = allow_max_smem(tail_kernel<float>, optin);
  if (e == cudaSuccess) e = allow_max_smem(residual_plain_kernel<cf>, optin);
  if (e == cudaSuccess) e = allow_max_smem(residual_plain_kernel<float>, optin);
  (void)N;
  (void)cplx;
  return e;
}

}  // namespace fermi
