// ffs_sample_noalloc: sampling without any device allocation.
//
// Some callers cannot allocate device memory at the point where they want samples:
// code running under an allocator that forbids new cudaMalloc calls (a memory pool
// that has been sized and frozen, or a framework whose caching allocator must not be
// bypassed), plugins that may only use memory handed to them, and paths that must
// not risk an allocation failure mid-run.  For them this entry point draws samples
// with every piece of working memory taken from one fixed array in device global
// memory, declared below.  The caller passes U and the output buffer; nothing else is
// allocated, by this library or by any library it calls.
//
// The arithmetic is the same as ffs_sample_ex with FFS_RES_FP32 | FFS_STATE_FP64 |
// FFS_TAIL_UNBLOCKED (FP32 all-site weights over the real embedding of U, summed in the same order; FP64
// Gauss-Jordan elimination state; the same draw), fused into one kernel in which one
// CTA runs the whole chain of one sample.  It is meant for small problems: the
// per-sample working set must fit in the fixed array.
#include <climits>
#include <mutex>
#include <type_traits>

#include "ffs_draw.cuh"
#include "ffs_internal.cuh"

namespace fermi {

void set_null_handle_error(const std::string& msg);  // defined in ffs_api.cu

// Working memory of ffs_sample_noalloc: FFS_NOALLOC_SCRATCH_BYTES of device global
// memory, reserved on every GPU that loads this library for as long as it stays loaded.
// Host code must not use the symbol as an address (on the host it is only a stand-in);
// it obtains the device address with cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[FFS_NOALLOC_SCRATCH_BYTES];

namespace {

struct NoAllocLayout {
  int64_t L, N, Kr, Kp, ldP, ldMask, B;
  int32_t* m;
  uint32_t* mask;
  float* P;
  float* H;
  void* W;
};

int64_t align256(int64_t v) { return (v + 255) / 256 * 256; }

// Carve the fixed array; returns the bytes needed (the pointers are set when base != 0).
int64_t carve(NoAllocLayout& lay, unsigned char* base, int64_t L, int64_t N, int64_t B, bool cplx) {
  lay.L = L;
  lay.N = N;
  lay.B = B;
  lay.Kr = cplx ? 2 * N : N;
  lay.Kp = (lay.Kr + 63) / 64 * 64;
  lay.ldP = (L + 3) / 4 * 4;
  lay.ldMask = (L + 31) / 32;
  const int64_t es = cplx ? (int64_t)sizeof(cd) : (int64_t)sizeof(double);
  int64_t off = 0;
  const int64_t o_m = off;
  off = align256(off + B * N * 4);
  const int64_t o_mask = off;
  off = align256(off + B * lay.ldMask * 4);
  const int64_t o_P = off;
  off = align256(off + B * lay.ldP * 4);
  const int64_t o_H = off;
  off = align256(off + B * lay.Kp * 4);
  const int64_t o_W = off;
  off = align256(off + B * N * N * es);
  if (base) {
    lay.m = (int32_t*)(base + o_m);
    lay.mask = (uint32_t*)(base + o_mask);
    lay.P = (float*)(base + o_P);
    lay.H = (float*)(base + o_H);
    lay.W = (void*)(base + o_W);
  }
  return off;
}

__device__ __forceinline__ void na_put(float* H, int col, double v) { H[col] = (float)v; }
__device__ __forceinline__ void na_put(float* H, int col, cd v) {
  H[2 * col] = (float)v.re;
  H[2 * col + 1] = (float)v.im;
}

// One CTA (256 threads) runs the whole chain of sample blockIdx.x.  A degenerate step
// (no site with a positive finite weight, a non-finite or non-positive normaliser, or a
// vanishing pivot) ends the sample's chain: that entry and the rest of its row are -1.
template <typename S>
__global__ void __launch_bounds__(256)
    noalloc_kernel(const void* __restrict__ U64, NoAllocLayout lay, uint64_t seed, int32_t* __restrict__ out_x) {
  constexpr bool CPLX = std::is_same<S, cd>::value;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ DrawShared dsh;
  __shared__ int s_status;
  const int tid = threadIdx.x;
  const int64_t b = blockIdx.x;
  const int64_t L = lay.L, N = lay.N, Kr = lay.Kr;
  int32_t* m = lay.m + b * N;
  uint32_t* mask = lay.mask + b * lay.ldMask;
  float* prow = lay.P + b * lay.ldP;
  float* H = lay.H + b * lay.Kp;
  S* W = (S*)lay.W + (size_t)b * N * N;
  S* r = (S*)smem_raw;
  S* nv = r + N;
  S* wc = nv + N;
  int* ms = (int*)(wc + N);

  // The array keeps the previous call's contents: clear what must start at zero.
  for (int64_t i = tid; i < lay.ldMask; i += blockDim.x) mask[i] = 0u;
  for (int64_t i = tid; i < lay.Kp; i += blockDim.x) H[i] = 0.f;
  if (tid == 0) s_status = 0;
  __syncthreads();
  if (tid == 0) {  // column order: Fisher-Yates from Philox stream 0
    for (int64_t i = 0; i < N; ++i) m[i] = (int32_t)i;
    int64_t i = N - 1;
    uint32_t block = 0;
    while (i >= 1) {
      const uint4 w = philox_block(seed, block, kStreamPerm, (uint64_t)b);
      for (int half = 0; half < 2 && i >= 1; ++half) {
        const uint64_t rr = half ? (((uint64_t)w.z << 32) | w.w) : (((uint64_t)w.x << 32) | w.y);
        const int64_t j = (int64_t)__umul64hi(rr, (uint64_t)(i + 1));
        const int32_t t = m[i];
        m[i] = m[j];
        m[j] = t;
        --i;
      }
      ++block;
    }
    if (CPLX)
      na_put(H, m[0], cd{1.0, 0.0});
    else
      na_put(H, m[0], 1.0);
  }
  __syncthreads();
  for (int64_t c = tid; c < N; c += blockDim.x) ms[c] = m[c];
  __syncthreads();

  for (int64_t k = 0; k < N; ++k) {
    // all-site weights, FP32, embedding columns summed in ascending order
    for (int64_t y = tid; y < L; y += blockDim.x) {
      float p;
      if constexpr (CPLX) {
        const cd* U = (const cd*)U64 + y * N;
        float re = 0.f, im = 0.f;
        for (int64_t c = 0; c < N; ++c) {
          const cd u = U[c];
          re = fmaf(H[2 * c], (float)u.re, re);
          im = fmaf(H[2 * c], (float)u.im, im);
          re = fmaf(H[2 * c + 1], (float)(-u.im), re);
          im = fmaf(H[2 * c + 1], (float)u.re, im);
        }
        p = re * re + im * im;
      } else {
        const double* U = (const double*)U64 + y * N;
        float v = 0.f;
        for (int64_t c = 0; c < Kr; ++c) v = fmaf(H[c], (float)U[c], v);
        p = v * v;
      }
      if ((mask[y >> 5] >> (y & 31)) & 1u) p = 0.f;
      prow[y] = p;
    }
    __syncthreads();

    // normaliser and inverse CDF: the draw of the batched forms (ffs_draw.cuh)
    double Z = 0.0;
    const int x = block_draw(prow, L, seed, (uint64_t)b, k, -1, &s_status, dsh, Z);
    __syncthreads();  // s_status is final
    if (s_status != 0 || !(Z > 0.0) || !isfinite(Z)) {
      for (int64_t j = k + tid; j < N; j += blockDim.x) out_x[b * N + j] = -1;
      return;  // uniform over the CTA
    }
    if (tid == 0) {
      out_x[b * N + k] = x;
      mask[x >> 5] |= 1u << (x & 31);
    }
    if (k + 1 >= N) break;

    // Gauss-Jordan update of the FP64 state with the row U[x, m]
    using Ud = typename std::conditional<CPLX, cd, double>::type;
    const Ud* urow = (const Ud*)U64 + (int64_t)x * N;
    for (int64_t c = tid; c < N; c += blockDim.x) r[c] = urow[ms[c]];
    __syncthreads();
    for (int64_t c = k + tid; c < N; c += blockDim.x) {
      S acc = r[c];
      for (int64_t j = 0; j < k; ++j) acc = fms(acc, r[j], W[j * N + c]);
      nv[c] = acc;
    }
    for (int64_t j = tid; j < k; j += blockDim.x) wc[j] = W[j * N + k];
    __syncthreads();
    const S s = nv[k];
    const double s2 = abs2(s);
    if (!(s2 > 1e-300) || !isfinite(s2)) {  // the pivot vanished: x_{k+1} has no weight left
      for (int64_t j = k + 1 + tid; j < N; j += blockDim.x) out_x[b * N + j] = -1;
      return;  // uniform over the CTA
    }
    for (int64_t c = k + 1 + tid; c < N; c += blockDim.x) {
      const S nc = nv[c] / s;
      for (int64_t j = 0; j < k; ++j) W[j * N + c] = fms(W[j * N + c], wc[j], nc);
      W[k * N + c] = nc;
    }
    __syncthreads();
    for (int64_t j = tid; j <= k + 1; j += blockDim.x) {
      const S v = (j <= k) ? -W[j * N + k + 1] : s_one<S>();
      na_put(H, ms[j], v);
    }
    __syncthreads();
  }
}

// Device or managed memory (what the kernel may dereference); pageable or pinned host
// memory is refused.  cudaPointerGetAttributes allocates nothing.
bool na_is_device(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

std::mutex g_setup_mutex;
void* g_scratch_ptr[64] = {nullptr};   // device address of the array, per device
bool g_configured[64] = {false};

}  // namespace
}  // namespace fermi

using namespace fermi;

extern "C" int ffs_sample_noalloc(const void* U, int dtype, int64_t L, int64_t N, int64_t B, uint64_t seed,
                                  int32_t* out_x, void* cuda_stream) {
  if (B == 0) return FFS_OK;
  if (!U || !out_x || B < 0 || N < 1 || L < N || (dtype != FFS_F64 && dtype != FFS_C128)) {
    set_null_handle_error("ffs_sample_noalloc: need device U (FFS_F64 or FFS_C128), 1 <= N <= L, B >= 0, out_x");
    return FFS_E_ARG;
  }
  // The smallest working set is 288 bytes per sample (L = N = 1); a larger B cannot fit,
  // and refusing it here keeps the size arithmetic below from overflowing.
  if (B > (int64_t)(FFS_NOALLOC_SCRATCH_BYTES / 288) || N > 4096 || L > ((int64_t)1 << 24)) {
    set_null_handle_error("ffs_sample_noalloc: B = " + std::to_string((long long)B) + ", L = " +
                          std::to_string((long long)L) + ", N = " + std::to_string((long long)N) +
                          " cannot fit the fixed " + std::to_string((long long)FFS_NOALLOC_SCRATCH_BYTES) +
                          "-byte array");
    return FFS_E_NOMEM;
  }
  const bool cplx = dtype == FFS_C128;
  NoAllocLayout lay;
  const int64_t need = carve(lay, nullptr, L, N, B, cplx);
  if (need > (int64_t)FFS_NOALLOC_SCRATCH_BYTES) {
    set_null_handle_error("ffs_sample_noalloc: B, L, N need " + std::to_string(need) +
                          " bytes of working memory, more than the fixed " +
                          std::to_string((long long)FFS_NOALLOC_SCRATCH_BYTES) + "-byte array");
    return FFS_E_NOMEM;
  }
  const size_t smem = (size_t)N * (3 * (cplx ? sizeof(cd) : sizeof(double)) + sizeof(int));
  if (smem > 200 * 1024) {
    set_null_handle_error("ffs_sample_noalloc: N too large");
    return FFS_E_ARG;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64) {
    set_null_handle_error("ffs_sample_noalloc: no usable current device");
    return FFS_E_CUDA;
  }
  if (!na_is_device(U) || !na_is_device(out_x)) {
    set_null_handle_error("ffs_sample_noalloc: U and out_x must be device (or managed) memory");
    return FFS_E_ARG;
  }
  {
    // First call on a device: look up the array's device address (and allow the
    // kernel its shared memory).  This set-up should happen before any stream capture.
    std::lock_guard<std::mutex> lk(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess || !ptr) {
        set_null_handle_error(std::string("ffs_sample_noalloc: cudaGetSymbolAddress failed: ") +
                              cudaGetErrorString(e));
        return FFS_E_CUDA;
      }
      g_scratch_ptr[dev] = ptr;
    }
    if (!g_configured[dev]) {
      e = cudaFuncSetAttribute(noalloc_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(noalloc_kernel<cd>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      if (e != cudaSuccess) {
        set_null_handle_error(std::string("ffs_sample_noalloc: ") + cudaGetErrorString(e));
        return FFS_E_CUDA;
      }
      g_configured[dev] = true;
    }
  }
  carve(lay, (unsigned char*)g_scratch_ptr[dev], L, N, B, cplx);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (cplx)
    noalloc_kernel<cd><<<(unsigned)B, 256, smem, st>>>(U, lay, seed, out_x);
  else
    noalloc_kernel<double><<<(unsigned)B, 256, smem, st>>>(U, lay, seed, out_x);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_null_handle_error(std::string("ffs_sample_noalloc: launch failed: ") + cudaGetErrorString(e));
    return FFS_E_CUDA;
  }
  return FFS_OK;
}
