// Slater-Jastrow reweighting (Supplementary Section S-5).
//
// The correlated state is |psi_J> = J |phi_0> with the diagonal Jastrow factor
// J(x) = exp(-1/2 sum_ij v_ij n_i n_j) (Eq. 4 of the main text is the Gutzwiller case
// v_{i up, i down} = v_{i down, i up} = V/2).  For an observable that is diagonal in
// the configuration basis, its local value o_L(x) is the observable itself, here
//   o_L(x) = sum_i o_i n_i + sum_ij q_ij n_i n_j,
// and free-fermion samples x_b of |phi_0> give
//   <O>_J = <J^2 o_L>_0 / <J^2>_0 = sum_b J^2(x_b) o_L(x_b) / sum_b J^2(x_b).
//
// Kernel 1, one warp per sample: the sample's occupation bitmap goes to shared memory,
// then each lane takes occupied orbitals i and adds the stored entries v_ij (and q_ij)
// of row i whose column j is occupied, so the work is sum over occupied i of the row
// lengths (one entry per row for the Gutzwiller factor).  log J^2 = -n^T v n.
// Kernel 2, one CTA: weights w_b = exp(log J^2_b - max_b log J^2_b), then the weighted
// mean, log <J^2>_0, the effective sample size (sum w)^2 / sum w^2 and the first-order
// (delta-method) standard error of the ratio, each summed in a fixed order.
#include <cfloat>
#include <cmath>

#include <math_constants.h>

#include "ffs_internal.cuh"

namespace fermi {

namespace {

constexpr int kTermsWarps = 8;       // samples per CTA (shared bitmap permitting)
constexpr int kReduceThreads = 1024;
constexpr size_t kMaxBitmapBytes = 200u << 10;  // one warp's bitmap must fit in shared memory

struct JastrowArgs {
  const int32_t* x;
  int64_t B, n_occ, n_orb;
  ffs_csr v, q;  // val == nullptr: absent
  const double* o;
  double* logw;
  double* obs;
  int* status;
  int words;  // 32-bit words of one occupation bitmap
};

// Sum of the stored entries of CSR row i whose column is occupied.
// Row pointers outside [0, nnz] or decreasing, and columns outside [0, n_orb), are flagged.
__device__ __forceinline__ double occupied_row_sum(const ffs_csr& m, int32_t i, const uint32_t* occ, int64_t n_orb,
                                                   bool& bad) {
  double s = 0.0;
  const int64_t e0 = m.rowptr[i], e1 = m.rowptr[i + 1];
  if (e0 < 0 || e1 < e0 || e1 > m.nnz) {
    bad = true;
    return 0.0;
  }
  for (int64_t e = e0; e < e1; ++e) {
    const int32_t j = m.col[e];
    if (j < 0 || j >= n_orb) {
      bad = true;
      continue;
    }
    if ((occ[j >> 5] >> (j & 31)) & 1u) s += m.val[e];
  }
  return s;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void jastrow_terms_kernel(JastrowArgs a) {
  extern __shared__ uint32_t occ_all[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  if (b >= a.B) return;  // warp-uniform: no block-wide barrier follows
  uint32_t* occ = occ_all + (size_t)warp * a.words;
  for (int w = lane; w < a.words; w += 32) occ[w] = 0u;
  __syncwarp();
  const int32_t* xb = a.x + b * a.n_occ;
  bool bad = false;
  for (int64_t c = lane; c < a.n_occ; c += 32) {
    const int32_t i = xb[c];
    if (i < 0 || i >= a.n_orb)
      bad = true;
    else
      atomicOr(&occ[i >> 5], 1u << (i & 31));
  }
  __syncwarp();
  // n_i is 0 or 1: a configuration that names an orbital twice is not a fermion state.
  int set = 0;
  for (int w = lane; w < a.words; w += 32) set += __popc(occ[w]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) set += __shfl_xor_sync(0xffffffffu, set, o);
  if (set != a.n_occ) bad = true;
  double lw = 0.0, ob = 0.0;
  if (!__any_sync(0xffffffffu, bad)) {
    for (int64_t c = lane; c < a.n_occ; c += 32) {
      const int32_t i = xb[c];
      if (a.v.val) lw -= occupied_row_sum(a.v, i, occ, a.n_orb, bad);
      if (a.o) ob += a.o[i];
      if (a.q.val) ob += occupied_row_sum(a.q, i, occ, a.n_orb, bad);
    }
    lw = warp_sum(lw);
    ob = warp_sum(ob);
  }
  if (__any_sync(0xffffffffu, bad)) {
    if (lane == 0) set_status(a.status, FFS_E_ARG);
    lw = ob = CUDART_NAN;
  }
  if (lane == 0) {
    a.logw[b] = lw;
    a.obs[b] = ob;
  }
}

// Fixed-order tree over one CTA (the same result on every run).
__device__ double block_combine(double v, double* sh, bool take_max) {
  const int tid = threadIdx.x;
  sh[tid] = v;
  __syncthreads();
  for (int s = kReduceThreads / 2; s > 0; s >>= 1) {
    if (tid < s) sh[tid] = take_max ? fmax(sh[tid], sh[tid + s]) : sh[tid] + sh[tid + s];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kReduceThreads) jastrow_reduce_kernel(const double* logw, const double* obs,
                                                                        int64_t B, double* out) {
  __shared__ double sh[kReduceThreads];
  const int tid = threadIdx.x;
  double mx = -DBL_MAX;
  for (int64_t b = tid; b < B; b += kReduceThreads) mx = fmax(mx, logw[b]);
  mx = block_combine(mx, sh, true);
  double sw = 0.0, swo = 0.0, sw2 = 0.0;
  for (int64_t b = tid; b < B; b += kReduceThreads) {
    const double w = exp(logw[b] - mx);
    sw += w;
    swo += w * obs[b];
    sw2 += w * w;
  }
  sw = block_combine(sw, sh, false);
  swo = block_combine(swo, sh, false);
  sw2 = block_combine(sw2, sh, false);
  const double R = swo / sw;
  double sv = 0.0;
  for (int64_t b = tid; b < B; b += kReduceThreads) {
    const double w = exp(logw[b] - mx), d = obs[b] - R;
    sv += w * w * d * d;
  }
  sv = block_combine(sv, sh, false);
  if (tid == 0) {
    out[0] = R;                        // <O>_J
    out[1] = mx + log(sw / (double)B);  // log <J^2>_0
    out[2] = sw * sw / sw2;            // effective sample size
    out[3] = sqrt(sv) / sw;            // standard error of <O>_J (first order)
  }
}

}  // namespace
}  // namespace fermi

using namespace fermi;

extern "C" int ffs_jastrow_estimate(const int32_t* x, int64_t B, int64_t n_occ, int64_t n_orb, const ffs_csr* v,
                                    const double* o, const ffs_csr* q, double* out_logj2, double* out_obs,
                                    double* result, void* cuda_stream) {
  auto reject = [](const char* msg) {
    set_null_handle_error(std::string("ffs_jastrow_estimate: ") + msg);
    return (int)FFS_E_ARG;
  };
  if (!x || !result) return reject("x and result are required");
  if (B < 1 || n_occ < 1 || n_orb < 1 || n_occ > n_orb || n_orb > INT32_MAX) return reject("bad sizes");
  const ffs_csr none{nullptr, nullptr, nullptr, 0};
  const ffs_csr vv = v ? *v : none, qq = q ? *q : none;
  for (const ffs_csr* m : {&vv, &qq})
    if (m->val || m->col || m->rowptr)
      if (!(m->rowptr && m->col && m->val) || m->nnz < 0) return reject("a CSR matrix needs rowptr, col, val, nnz");
  const void* dev[] = {x, vv.rowptr, vv.col, vv.val, o, qq.rowptr, qq.col, qq.val, out_logj2, out_obs};
  for (const void* p : dev)
    if (p && !ptr_is_device(p)) return reject("x, v, o, q and the per-sample outputs must be device memory");
  const size_t words = (size_t)((n_orb + 31) / 32);
  if (words * 4 > kMaxBitmapBytes) return reject("n_orb above the shared-memory bitmap limit (1638400)");

  cudaStream_t st = (cudaStream_t)cuda_stream;
  double* scratch = nullptr;
  int* status = nullptr;
  const size_t n_scratch = (out_logj2 ? 0 : B) + (out_obs ? 0 : B) + 4;
  cudaError_t e = cudaMallocAsync((void**)&scratch, sizeof(double) * n_scratch, st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&status, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int), st);
  int h_status = 0;
  if (e == cudaSuccess) {
    double* s = scratch;
    JastrowArgs a{};
    a.x = x;
    a.B = B;
    a.n_occ = n_occ;
    a.n_orb = n_orb;
    a.v = vv;
    a.q = qq;
    a.o = o;
    a.logw = out_logj2 ? out_logj2 : s;
    if (!out_logj2) s += B;
    a.obs = out_obs ? out_obs : s;
    if (!out_obs) s += B;
    a.status = status;
    a.words = (int)words;
    int warps = (int)std::min<size_t>(kTermsWarps, kMaxBitmapBytes / (words * 4));
    warps = std::max(warps, 1);
    const size_t smem = (size_t)warps * words * 4;
    if (smem > 48u << 10)
      e = cudaFuncSetAttribute(jastrow_terms_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
      jastrow_terms_kernel<<<(unsigned)((B + warps - 1) / warps), warps * 32, smem, st>>>(a);
      jastrow_reduce_kernel<<<1, kReduceThreads, 0, st>>>(a.logw, a.obs, B, s);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(result, s, 4 * sizeof(double), cudaMemcpyDefault, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  if (scratch) cudaFreeAsync(scratch, st);
  if (status) cudaFreeAsync(status, st);
  if (e != cudaSuccess) {
    set_null_handle_error(std::string("ffs_jastrow_estimate: ") + cudaGetErrorString(e));
    return FFS_E_CUDA;
  }
  if (h_status) {
    set_null_handle_error(
        "ffs_jastrow_estimate: a configuration names an orbital outside [0, n_orb) or twice, or a column "
        "index of v or q is outside [0, n_orb)");
    return h_status;
  }
  return FFS_OK;
}
