// libffs C ABI: handle lifecycle, memory, and the per-step launch sequence.
// The declarations and the contract of every entry point are in include/ffs.h.
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "ffs_kernels.cuh"
#include "ffs_residual_tc.cuh"

using namespace fermi;

static thread_local std::string g_null_handle_error;

namespace fermi {
// Error message of a call that has no handle (read back by ffs_last_error(NULL)).
void set_null_handle_error(const std::string& msg) { g_null_handle_error = msg; }
}  // namespace fermi

static int fail(ffs_ctx* c, int code, const std::string& msg) {
  if (c)
    c->last_error = msg;
  else
    g_null_handle_error = msg;
  return code;
}

#define FFS_CUDA_TRY(ctx, expr)                                                                 \
  do {                                                                                          \
    cudaError_t _e = (expr);                                                                    \
    if (_e != cudaSuccess)                                                                      \
      return fail((ctx), _e == cudaErrorMemoryAllocation ? FFS_E_NOMEM : FFS_E_CUDA,            \
                  std::string(#expr) + ": " + cudaGetErrorString(_e));                          \
  } while (0)

static bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

static int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

static int op_mode_of(unsigned flags) {
  if ((flags & FFS_FORM_MASK) == FFS_FORM_PLAIN) return kOpNone;
  switch (flags & FFS_RES_MASK) {
    case FFS_RES_FP32: return kOpF32;
    case FFS_RES_BF16X3: return kOpBF16x3;
    case FFS_RES_BF16: return kOpBF16;
    case FFS_RES_TF32: return kOpTF32;
  }
  return -1;
}

static size_t op_elem_bytes(int op) {
  switch (op) {
    case kOpF32:
    case kOpTF32: return 4;
    case kOpBF16x3: return 4;  // two BF16 planes
    case kOpBF16: return 2;
    default: return 0;
  }
}

static bool state_fp64(const ffs_ctx* c) { return (c->flags & FFS_STATE_MASK) == FFS_STATE_FP64; }

static int state_kind(const ffs_ctx* c) {
  switch (c->flags & FFS_STATE_MASK) {
    case FFS_STATE_FP32: return kStateFP32;
    case FFS_STATE_DF64: return kStateDF64;
    default: return kStateFP64;
  }
}

static bool blocked(const ffs_ctx* c) {
  return op_mode_of(c->flags) != kOpNone && !(c->flags & FFS_TAIL_UNBLOCKED);
}

static size_t state_elem_bytes(const ffs_ctx* c) { return blocked_elem_bytes(c->cplx, state_kind(c)); }

// Device bytes per sample of a wave (not counting optional outputs) for a chain of Nc
// steps: the blocked state keeps Nc rows of round_up(Nc, 32) columns (32-column slabs),
// the unblocked one N x N.
static size_t state_cols(const ffs_ctx* c, int64_t Nc) { return blocked(c) ? (size_t)Nc : (size_t)c->N; }
static size_t state_entries(const ffs_ctx* c, int64_t Nc) {
  const size_t sc = state_cols(c, Nc);
  return blocked(c) ? (size_t)state_stride((int64_t)sc) : sc * sc;
}
static size_t per_sample_bytes_nc(const ffs_ctx* c, int64_t Nc) {
  const int op = op_mode_of(c->flags);
  const size_t sc = state_cols(c, Nc);
  size_t b = 0;
  b += (size_t)c->N * 4;                           // m
  b += (size_t)c->ldMask * 4;                      // mask
  b += (size_t)c->Kp * op_elem_bytes(op);          // operand planes
  b += (size_t)c->ldP * 4;                         // weights
  b += (size_t)c->ldG * 4;                         // their group sums
  b += state_entries(c, Nc) * state_elem_bytes(c);  // elimination state
  b += 8;                                          // logp
  if (blocked(c)) {                                // panel-start columns, panel inverse
    const size_t nb = blocked_panel_width();
    b += (sc * nb + nb * nb) * state_elem_bytes(c);
  }
  return b;
}
static size_t per_sample_bytes(const ffs_ctx* c) { return per_sample_bytes_nc(c, c->N); }

static void free_workspace(ffs_ctx* c) {
  cudaFree(c->m);
  cudaFree(c->mask);
  cudaFree(c->H);
  cudaFree(c->P);
  cudaFree(c->G);
  cudaFree(c->W);
  cudaFree(c->W0P);
  cudaFree(c->Sinv);
  cudaFree(c->logp);
  c->W0P = nullptr;
  c->Sinv = nullptr;
  c->m = nullptr;
  c->mask = nullptr;
  c->H = nullptr;
  c->P = nullptr;
  c->G = nullptr;
  c->W = nullptr;
  c->logp = nullptr;
  c->ws_B = 0;
  c->W_bytes = 0;
  c->W0P_bytes = 0;
}

// Buffers for Bw samples of a chain of Nc steps; the state buffers are sized in bytes so
// that short (marginal) chains fit more samples.
static int ensure_workspace_nc(ffs_ctx* c, int64_t Bw, int64_t Nc) {
  const size_t sc = state_cols(c, Nc), es = state_elem_bytes(c), nb = blocked_panel_width();
  const size_t w_need = (size_t)Bw * state_entries(c, Nc) * es;
  const size_t w0_need = blocked(c) ? (size_t)Bw * sc * nb * es : 0;
  if (Bw <= c->ws_B && w_need <= c->W_bytes && w0_need <= c->W0P_bytes) return FFS_OK;
  cudaStreamSynchronize(c->stream);
  const int64_t B = Bw > c->ws_B ? Bw : c->ws_B;
  const size_t wb = w_need > c->W_bytes ? w_need : c->W_bytes;
  const size_t w0b = w0_need > c->W0P_bytes ? w0_need : c->W0P_bytes;
  free_workspace(c);
  const int op = op_mode_of(c->flags);
  FFS_CUDA_TRY(c, cudaMalloc((void**)&c->m, (size_t)B * c->N * 4));
  FFS_CUDA_TRY(c, cudaMalloc((void**)&c->mask, (size_t)B * c->ldMask * 4));
  if (op != kOpNone) FFS_CUDA_TRY(c, cudaMalloc(&c->H, (size_t)B * c->Kp * op_elem_bytes(op)));
  FFS_CUDA_TRY(c, cudaMalloc((void**)&c->P, (size_t)B * c->ldP * 4));
  FFS_CUDA_TRY(c, cudaMalloc((void**)&c->G, (size_t)B * c->ldG * 4));
  FFS_CUDA_TRY(c, cudaMalloc(&c->W, wb));
  FFS_CUDA_TRY(c, cudaMalloc((void**)&c->logp, (size_t)B * 8));
  if (blocked(c)) {
    FFS_CUDA_TRY(c, cudaMalloc(&c->W0P, w0b));
    FFS_CUDA_TRY(c, cudaMalloc(&c->Sinv, (size_t)B * nb * nb * es));
  }
  c->ws_B = B;
  c->W_bytes = wb;
  c->W0P_bytes = w0b;
  return FFS_OK;
}
static int ensure_workspace(ffs_ctx* c, int64_t Bw) { return ensure_workspace_nc(c, Bw, c->N); }

static void release(ffs_ctx* c) {
  if (!c) return;
  if (c->stream || true) cudaStreamSynchronize(c->stream);
  free_workspace(c);
  cudaFree(c->U64);
  cudaFree(c->Ue32);
  cudaFree(c->Ue_hi);
  cudaFree(c->Ue_lo);
  cudaFree(c->Ue_tf32);
  cudaFree(c->UT32);
  cudaFree(c->Ust);
  cudaFree(c->sel_p);
  cudaFree(c->Ug);
  cudaFree(c->oz_buf);
  cudaFree(c->ozy_buf);
  cudaFree(c->status);
  if (c->status_host) cudaFreeHost(c->status_host);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  delete c;
}

// Widen a (possibly strided, host or device) U of any supported dtype into the
// contiguous FP64 copy.
__global__ void widen_kernel(const void* src, int dtype, int64_t L, int64_t N, int64_t ld, void* dst) {
  const int64_t total = L * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t y = e / N, c = e % N;
    switch (dtype) {
      case FFS_F64: ((double*)dst)[e] = ((const double*)src)[y * ld + c]; break;
      case FFS_F32: ((double*)dst)[e] = ((const float*)src)[y * ld + c]; break;
      case FFS_C128: ((cd*)dst)[e] = ((const cd*)src)[y * ld + c]; break;
      case FFS_C64: {
        const cf v = ((const cf*)src)[y * ld + c];
        ((cd*)dst)[e] = cd{v.re, v.im};
        break;
      }
    }
  }
}

// Per-phase CUDA-event timing (enabled by ffs_profile).
static void prof_begin(ffs_ctx* c, int phase, cudaStream_t st) {
  if (!c->prof) return;
  while (c->ev_pool.size() < c->ev_used + 2) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    c->ev_pool.push_back(e);
  }
  cudaEventRecord(c->ev_pool[c->ev_used], st);
  c->prof_phase.push_back(phase);
}
static void prof_end(ffs_ctx* c, cudaStream_t st) {
  if (!c->prof) return;
  cudaEventRecord(c->ev_pool[c->ev_used + 1], st);
  c->ev_used += 2;
}
static void prof_fold(ffs_ctx* c) {
  for (size_t i = 0; i < c->prof_phase.size(); ++i) {
    float ms = 0.f;
    cudaEventSynchronize(c->ev_pool[2 * i + 1]);
    cudaEventElapsedTime(&ms, c->ev_pool[2 * i], c->ev_pool[2 * i + 1]);
    c->prof_ms[c->prof_phase[i]] += ms;
    c->prof_launches[c->prof_phase[i]] += 1;
  }
  c->prof_phase.clear();
  c->ev_used = 0;
}

#define TIMED(ctx, phase, st, expr)                                                             \
  do {                                                                                          \
    prof_begin((ctx), (phase), (st));                                                           \
    cudaError_t _e2 = (expr);                                                                   \
    prof_end((ctx), (st));                                                                      \
    if (_e2 != cudaSuccess)                                                                     \
      return fail((ctx), FFS_E_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e2));     \
  } while (0)

extern "C" {

const char* ffs_last_error(ffs_handle h) {
  return h ? h->last_error.c_str() : g_null_handle_error.c_str();
}

int ffs_create_ex(const void* U, int dtype, int64_t L, int64_t N, int64_t ldU, unsigned flags,
                  void* cuda_stream, ffs_handle* out) {
  if (!out) return fail(nullptr, FFS_E_ARG, "ffs_create_ex: out is NULL");
  *out = nullptr;
  if (!U) return fail(nullptr, FFS_E_ARG, "ffs_create_ex: U is NULL");
  if (dtype < FFS_F64 || dtype > FFS_C64) return fail(nullptr, FFS_E_ARG, "ffs_create_ex: bad dtype");
  if (N < 1 || L < N) return fail(nullptr, FFS_E_ARG, "ffs_create_ex: need 1 <= N <= L");
  if (ldU < N) return fail(nullptr, FFS_E_ARG, "ffs_create_ex: need ldU >= N");
  if (L > (int64_t)1 << 30) return fail(nullptr, FFS_E_ARG, "ffs_create_ex: L too large");
  const bool cplx = (dtype == FFS_C128 || dtype == FFS_C64);
  if ((flags & FFS_TRAILING_TC) &&
      ((flags & FFS_STATE_MASK) != FFS_STATE_DF64 || (flags & FFS_TAIL_UNBLOCKED) ||
       (flags & FFS_FORM_MASK) == FFS_FORM_PLAIN || (flags & FFS_RES_MASK) == FFS_RES_FP32))
    return fail(nullptr, FFS_E_UNSUPPORTED,
                "ffs_create_ex: the tensor-core trailing update needs the double-float state, the blocked "
                "state and a tensor-core residual");
  if ((flags & FFS_FORM_MASK) == FFS_FORM_PLAIN)
    flags = (flags & ~(FFS_RES_MASK | FFS_STATE_MASK)) | FFS_RES_FP32 | FFS_STATE_FP32 | FFS_TAIL_UNBLOCKED;
  if ((flags & FFS_FORM_MASK) > FFS_FORM_GROUPED || (flags & FFS_STATE_MASK) > FFS_STATE_DF64 ||
      (flags & ~(FFS_RES_MASK | FFS_STATE_MASK | FFS_FORM_MASK | FFS_NO_ORTHO_CHECK | FFS_TAIL_UNBLOCKED |
                 FFS_TRAILING_TC)) ||
      op_mode_of(flags) < 0)
    return fail(nullptr, FFS_E_ARG, "ffs_create_ex: bad flags");
  if ((flags & FFS_FORM_MASK) == FFS_FORM_GROUPED &&
      ((flags & FFS_TAIL_UNBLOCKED) || (flags & FFS_RES_MASK) == FFS_RES_FP32))
    return fail(nullptr, FFS_E_ARG,
                "ffs_create_ex: the grouped form needs a tensor-core residual and the blocked state");
  if ((flags & FFS_TAIL_UNBLOCKED) && (flags & FFS_STATE_MASK) == FFS_STATE_DF64)
    return fail(nullptr, FFS_E_ARG, "ffs_create_ex: the unblocked state update has no double-float form");

  ffs_ctx* c = new ffs_ctx();
  c->L = L;
  c->N = N;
  c->dtype = dtype;
  c->cplx = cplx;
  c->flags = flags;
  c->stream = (cudaStream_t)cuda_stream;
  const size_t smem_need = blocked(c) ? blocked_step_smem(N, cplx, state_kind(c))
                                     : tail_smem_bytes(N, cplx, state_fp64(c));
  if (smem_need > 224 * 1024) {
    int r = fail(nullptr, FFS_E_UNSUPPORTED, "ffs_create_ex: N too large for the per-sample state kernel");
    release(c);
    return r;
  }
#define CREATE_TRY(expr)                                                                            \
  do {                                                                                              \
    cudaError_t _e = (expr);                                                                        \
    if (_e != cudaSuccess) {                                                                        \
      int r = fail(nullptr, _e == cudaErrorMemoryAllocation ? FFS_E_NOMEM : FFS_E_CUDA,             \
                   std::string(#expr) + ": " + cudaGetErrorString(_e));                             \
      release(c);                                                                                   \
      return r;                                                                                     \
    }                                                                                               \
  } while (0)
  CREATE_TRY(cudaGetDevice(&c->device));
  CREATE_TRY(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
  {
    // Kernel attributes are set once per device (callers may create handles from several threads).
    static std::mutex mu;
    static bool configured[64] = {false};
    std::lock_guard<std::mutex> lk(mu);
    if (c->device >= 0 && c->device < 64 && !configured[c->device]) {
      CREATE_TRY(configure_kernels(N, cplx));
      CREATE_TRY(configure_residual_tc());
      CREATE_TRY(configure_blocked());
      CREATE_TRY(configure_oz());
      CREATE_TRY(configure_oz_y());
      configured[c->device] = true;
    }
  }
  c->Lr = cplx ? 2 * L : L;
  c->Kr = cplx ? 2 * N : N;
  c->Kp = round_up(c->Kr, 64);
  c->Lrp = round_up(c->Lr, 256);
  c->ldP = round_up(L, 4);
  c->ldG = round_up((L + 15) / 16, 4);  // group sums of at most 16 sites each
  c->ldMask = (L + 31) / 32;

  // FP64 copy of U
  const size_t es64 = cplx ? sizeof(cd) : sizeof(double);
  const size_t es_in = (dtype == FFS_F64) ? 8 : (dtype == FFS_C128) ? 16 : (dtype == FFS_F32) ? 4 : 8;
  CREATE_TRY(cudaMalloc(&c->U64, (size_t)L * N * es64));
  if ((dtype == FFS_F64 || dtype == FFS_C128) && ldU == N) {
    CREATE_TRY(cudaMemcpyAsync(c->U64, U, (size_t)L * N * es64, cudaMemcpyDefault, c->stream));
  } else {
    void* stage = nullptr;
    CREATE_TRY(cudaMalloc(&stage, (size_t)L * N * es_in));
    cudaError_t e = cudaMemcpy2DAsync(stage, N * es_in, U, ldU * es_in, N * es_in, L, cudaMemcpyDefault,
                                      c->stream);
    if (e == cudaSuccess) {
      widen_kernel<<<4 * c->num_sms, 256, 0, c->stream>>>(stage, dtype, L, N, N, c->U64);
      e = cudaGetLastError();
    }
    cudaStreamSynchronize(c->stream);
    cudaFree(stage);
    CREATE_TRY(e);
  }
  if (!(flags & FFS_NO_ORTHO_CHECK)) {
    double dev = 0.0;
    CREATE_TRY(launch_ortho_check(c->U64, cplx, L, N, &dev, c->stream));
    if (!(dev <= FFS_ORTHO_TOL)) {
      char msg[160];
      snprintf(msg, sizeof msg, "ffs_create_ex: U^dagger U deviates from 1 by %.3e (tolerance %.1e)", dev,
               FFS_ORTHO_TOL);
      int r = fail(nullptr, FFS_E_NOT_ORTHONORMAL, msg);
      release(c);
      return r;
    }
  }
  const int op = op_mode_of(flags);
  const size_t emb = (size_t)c->Lrp * c->Kp;
  if (op == kOpF32) CREATE_TRY(cudaMalloc((void**)&c->Ue32, emb * 4));
  if (op == kOpBF16x3 || op == kOpBF16) CREATE_TRY(cudaMalloc((void**)&c->Ue_hi, emb * 2));
  if (op == kOpBF16x3) CREATE_TRY(cudaMalloc((void**)&c->Ue_lo, emb * 2));
  if (op == kOpTF32) CREATE_TRY(cudaMalloc((void**)&c->Ue_tf32, emb * 4));
  if (op == kOpNone) CREATE_TRY(cudaMalloc(&c->UT32, (size_t)L * N * (cplx ? 8 : 4)));
  CREATE_TRY(launch_derive_operands(c, c->stream));
  if (blocked(c) && state_kind(c) != kStateFP64) {
    const size_t es = blocked_elem_bytes(cplx, state_kind(c));
    CREATE_TRY(cudaMalloc(&c->Ust, (size_t)L * N * es));
    CREATE_TRY(launch_derive_state_copy(c->U64, cplx, state_kind(c), L * N, c->Ust, c->stream));
  }
  CREATE_TRY(cudaMalloc((void**)&c->status, sizeof(int)));
  CREATE_TRY(cudaMemsetAsync(c->status, 0, sizeof(int), c->stream));
  CREATE_TRY(cudaMallocHost((void**)&c->status_host, sizeof(int)));
  CREATE_TRY(cudaStreamSynchronize(c->stream));
#undef CREATE_TRY
  *out = c;
  return FFS_OK;
}

int ffs_create(const double* U, int64_t L, int64_t N, ffs_handle* out) {
  return ffs_create_ex(U, FFS_F64, L, N, N, 0u, nullptr, out);
}

int ffs_query(ffs_handle h, int64_t* L, int64_t* N, int* dtype, unsigned* flags, int64_t B,
              int64_t* bytes_for_B) {
  if (!h) return fail(nullptr, FFS_E_ARG, "ffs_query: NULL handle");
  if (L) *L = h->L;
  if (N) *N = h->N;
  if (dtype) *dtype = h->dtype;
  if (flags) *flags = h->flags;
  if (bytes_for_B) *bytes_for_B = (int64_t)(B * per_sample_bytes(h));
  return FFS_OK;
}

}  // extern "C"

// The sampling loop shared by ffs_sample_ex and ffs_sample_lensemble: waves of samples,
// each a permutation launch and then n_steps residual + state launches.  Rows of out_x,
// force_x and out_probs are ldx steps apart.  sel_p / nlen: L-ensemble keep probabilities
// and per-sample chain lengths (device; null for ordinary calls).
static bool grouped_form(const ffs_ctx* c) { return (c->flags & FFS_FORM_MASK) == FFS_FORM_GROUPED; }

// Bytes of one group's copy of the residual operand planes (grouped form).
static size_t group_copy_bytes(const ffs_ctx* c) {
  const int op = op_mode_of(c->flags);
  const size_t planes = op == kOpBF16x3 ? 2 : 1;
  return planes * (size_t)c->Lrp * c->Kp * (op == kOpTF32 ? 4 : 2);
}

static int sample_core(ffs_ctx* h, int64_t B, uint64_t seed, uint64_t first_sample_index, int64_t n_steps,
                       int64_t ldx, int32_t* out_x, int32_t* out_perm, double* out_logp, const int32_t* force_x,
                       float* out_probs, cudaStream_t st, const double* sel_p, const int32_t* nlen) {
  const int op = op_mode_of(h->flags);
  const bool plain = op == kOpNone;
  const bool grouped = grouped_form(h);
  const bool tc_top = (h->flags & FFS_TRAILING_TC) && blocked(h);
  const bool tc_new = tc_top;  // the new rows (Y, Bot) on the tensor cores too
  const int64_t G = FFS_GROUP_SIZE;
  if (grouped && (first_sample_index % G) != 0)
    return fail(h, FFS_E_ARG, "grouped form: first_sample_index must be a multiple of 128");

  const bool x_dev = is_device_ptr(out_x);
  const bool perm_dev = is_device_ptr(out_perm);
  const bool logp_dev = is_device_ptr(out_logp);
  const bool force_dev = is_device_ptr(force_x);
  const bool probs_dev = is_device_ptr(out_probs);
  const bool any_host = !x_dev || (out_perm && !perm_dev) || (out_logp && !logp_dev) ||
                        (out_probs && !probs_dev);

  // Wave size from free device memory.
  size_t per = per_sample_bytes_nc(h, n_steps);
  if (!x_dev) per += ldx * 4;
  if (force_x && !force_dev) per += ldx * 4;
  if (out_probs && !probs_dev) per += (size_t)ldx * h->L * 4;
  if (grouped) per += group_copy_bytes(h) / G + 1;  // a group's operand copy, shared by its 128 samples
  if (tc_top) per += oz_bytes_per_sample(n_steps);   // slices of the tensor-core trailing update
  if (tc_new) per += ozy_bytes_per_sample(n_steps, h->cplx);  // C's slices of the tensor-core new rows
  size_t free_b = 0, total_b = 0;
  FFS_CUDA_TRY(h, cudaMemGetInfo(&free_b, &total_b));
  const size_t reserve = (size_t)512 << 20;
  size_t have = free_b > reserve ? free_b - reserve : 0;
  have += (size_t)h->ws_B * per_sample_bytes_nc(h, n_steps);  // the workspace we already hold is reusable
  int64_t Bw = (int64_t)(have / per);
  if (grouped && Bw < B) Bw = Bw / G * G;  // waves hold whole groups
  if (Bw < 1) return fail(h, FFS_E_NOMEM, "ffs_sample_ex: not enough device memory for one sample");
  if (Bw > B) Bw = B;
  if (grouped) {
    const int64_t groups = (Bw + G - 1) / G;
    const size_t need = (size_t)groups * group_copy_bytes(h);
    if (need > h->Ug_bytes) {
      cudaStreamSynchronize(h->stream);
      cudaStreamSynchronize(st);
      cudaFree(h->Ug);
      h->Ug = nullptr;
      h->Ug_bytes = 0;
      FFS_CUDA_TRY(h, cudaMalloc(&h->Ug, need));
      h->Ug_bytes = need;
      h->tmUg_key = -1;
    }
    h->Ug_groups = groups;
  }
  {
    int r = ensure_workspace_nc(h, Bw, n_steps);
    if (r != FFS_OK) return r;
  }
  if (tc_top) FFS_CUDA_TRY(h, oz_prepare(h, Bw, n_steps));
  if (tc_new) FFS_CUDA_TRY(h, ozy_prepare(h, Bw, n_steps));
  int32_t* xbuf = nullptr;
  int32_t* fbuf = nullptr;
  float* pbuf = nullptr;
  if (!x_dev) FFS_CUDA_TRY(h, cudaMallocAsync((void**)&xbuf, (size_t)Bw * ldx * 4, st));
  if (force_x && !force_dev) FFS_CUDA_TRY(h, cudaMallocAsync((void**)&fbuf, (size_t)Bw * ldx * 4, st));
  if (out_probs && !probs_dev)
    FFS_CUDA_TRY(h, cudaMallocAsync((void**)&pbuf, (size_t)Bw * ldx * h->L * 4, st));

  int rc = FFS_OK;
  for (int64_t b0 = 0; b0 < B && rc == FFS_OK; b0 += Bw) {
    const int64_t bw = (B - b0 < Bw) ? B - b0 : Bw;
    StepArgs a{};
    a.L = h->L;
    a.N = h->N;
    a.Lr = h->Lr;
    a.Kr = h->Kr;
    a.Kp = h->Kp;
    a.ldP = h->ldP;
    a.ldMask = h->ldMask;
    a.bw = bw;
    a.n_steps = n_steps;
    a.seed = seed;
    a.first = first_sample_index + (uint64_t)b0;
    a.cplx = h->cplx;
    a.U64 = h->U64;
    a.Ust = h->Ust ? h->Ust : h->U64;
    a.m = h->m;
    a.mask = h->mask;
    a.H = h->H;
    a.hplane = h->ws_B * h->Kp;
    a.P = h->P;
    if (!plain && op != kOpF32) {  // the tensor-core residual writes the weights' group sums
      a.G = h->G;
      a.ldG = h->ldG;
    }
    a.W = h->W;
    a.logp = h->logp;
    a.x = x_dev ? out_x + b0 * ldx : xbuf;
    a.probs = out_probs ? (probs_dev ? out_probs + (size_t)b0 * ldx * h->L : pbuf) : nullptr;
    a.status = h->status;
    a.ldx = ldx;
    a.sel_p = sel_p;
    a.nlen = nlen ? nlen + b0 : nullptr;
    a.grouped = grouped ? 1 : 0;
    if (force_x) {
      if (force_dev) {
        a.force_x = force_x + b0 * ldx;
      } else {
        FFS_CUDA_TRY(h, cudaMemcpyAsync(fbuf, force_x + b0 * ldx, (size_t)bw * ldx * 4,
                                        cudaMemcpyHostToDevice, st));
        a.force_x = fbuf;
      }
    }
    BlockedArgs bt{};
    bt.Nc = n_steps;
    bt.W = h->W;
    bt.W0P = h->W0P;
    bt.Sinv = h->Sinv;
    if (!plain) FFS_CUDA_TRY(h, cudaMemsetAsync(h->H, 0, (size_t)h->ws_B * h->Kp * op_elem_bytes(op), st));
    FFS_CUDA_TRY(h, cudaMemsetAsync(h->mask, 0, (size_t)bw * h->ldMask * 4, st));
    FFS_CUDA_TRY(h, cudaMemsetAsync(h->logp, 0, (size_t)bw * 8, st));
    TIMED(h, FFS_PHASE_PERM, st, launch_perm_init(a, op, st));
    if (grouped) {  // each group's copy of the operand planes, in the group's column order
      const bool f32 = op == kOpTF32;
      const void* s0 = f32 ? (const void*)h->Ue_tf32 : (const void*)h->Ue_hi;
      const void* s1 = op == kOpBF16x3 ? (const void*)h->Ue_lo : s0;
      TIMED(h, FFS_PHASE_PERM, st,
            launch_group_embed(s0, s1, h->Ug, h->Lrp, h->Kp, h->Kr, h->cplx, f32, op == kOpBF16x3 ? 2 : 1, h->m, h->N,
                               (bw + G - 1) / G, h->Ug_groups, st));
    }
    if (!plain && op != kOpF32 && b0 == 0) {
      // column tile of the tensor-core residual: autotuned once per size class
      const int bn = residual_tile_for(h, a, op, st);
      FFS_CUDA_TRY(h, prepare_residual_tc_bn(h, op, bn));
    }
    for (int64_t k = 0; k < n_steps; ++k) {
      if (plain)
        TIMED(h, FFS_PHASE_RESIDUAL, st, launch_residual_plain(a, h->UT32, k, st));
      else if (op == kOpF32)
        TIMED(h, FFS_PHASE_RESIDUAL, st, launch_residual_fp32(a, h->Ue32, st));
      else {
        a.kcols = grouped ? (k + 1) * (h->cplx ? 2 : 1) : 0;  // grouped: only the leading columns
        TIMED(h, FFS_PHASE_RESIDUAL, st, launch_residual_tc(h, a, op, st));
      }
      if (blocked(h)) {
        TIMED(h, FFS_PHASE_TAIL, st, launch_blocked_step(a, bt, k, state_kind(h), op, st));
        const int64_t nb = blocked_panel_width();
        const int64_t k0 = (k / nb) * nb, k1 = (k0 + nb < n_steps) ? k0 + nb : n_steps;
        if (k + 1 == k1 && k1 < n_steps) {
          TIMED(h, FFS_PHASE_PANEL_S, st, launch_blocked_panel_s(a, bt, k0, k1, state_kind(h), st));
          bt.tc_top = tc_top ? 1 : 0;  // then the old rows and the next operand are the tensor-core pass's
          if (tc_new)
            TIMED(h, FFS_PHASE_PANEL, st, launch_oz_y(h, a, bt, k0, k1, st));
          else
            TIMED(h, FFS_PHASE_PANEL, st, launch_blocked_panel_update(a, bt, k0, k1, state_kind(h), op, st));
          if (tc_top) TIMED(h, FFS_PHASE_PANEL_TC, st, launch_oz_top(h, a, bt, k0, k1, op, st));
          bt.tc_top = 0;
        }
      } else {
        TIMED(h, FFS_PHASE_TAIL, st, launch_tail(a, k, state_fp64(h), op, st));
      }
    }
    if (!x_dev)
      FFS_CUDA_TRY(h, cudaMemcpyAsync(out_x + b0 * ldx, xbuf, (size_t)bw * ldx * 4,
                                      cudaMemcpyDeviceToHost, st));
    if (out_perm)
      FFS_CUDA_TRY(h, cudaMemcpyAsync(out_perm + b0 * h->N, h->m, (size_t)bw * h->N * 4, cudaMemcpyDefault, st));
    if (out_logp)
      FFS_CUDA_TRY(h, cudaMemcpyAsync(out_logp + b0, h->logp, (size_t)bw * 8, cudaMemcpyDefault, st));
    if (out_probs && !probs_dev)
      FFS_CUDA_TRY(h, cudaMemcpyAsync(out_probs + (size_t)b0 * ldx * h->L, pbuf,
                                      (size_t)bw * ldx * h->L * 4, cudaMemcpyDeviceToHost, st));
    if (any_host) FFS_CUDA_TRY(h, cudaStreamSynchronize(st));
  }
  if (xbuf) cudaFreeAsync(xbuf, st);
  if (fbuf) cudaFreeAsync(fbuf, st);
  if (pbuf) cudaFreeAsync(pbuf, st);
  if (any_host) {
    FFS_CUDA_TRY(h, cudaStreamSynchronize(st));
    FFS_CUDA_TRY(h, cudaMemcpy(h->status_host, h->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (*h->status_host != 0) {
      const int code = *h->status_host;
      cudaMemset(h->status, 0, sizeof(int));
      return fail(h, code, "device reported an error (see ffs.h status codes)");
    }
  }
  return rc;
}

extern "C" {

int ffs_sample_ex(ffs_handle h, int64_t B, uint64_t seed, uint64_t first_sample_index, int64_t n_steps,
                  int32_t* out_x, int32_t* out_perm, double* out_logp, const int32_t* force_x,
                  float* out_probs, void* cuda_stream) {
  if (!h) return fail(nullptr, FFS_E_ARG, "ffs_sample_ex: NULL handle");
  if (B < 0) return fail(h, FFS_E_ARG, "ffs_sample_ex: B < 0");
  if (n_steps == 0) n_steps = h->N;
  if (n_steps < 1 || n_steps > h->N) return fail(h, FFS_E_ARG, "ffs_sample_ex: need 0 <= n_steps <= N");
  if (B == 0) return FFS_OK;
  if (!out_x) return fail(h, FFS_E_ARG, "ffs_sample_ex: out_x is NULL");
  cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : h->stream;
  return sample_core(h, B, seed, first_sample_index, n_steps, n_steps, out_x, out_perm, out_logp, force_x,
                     out_probs, st, nullptr, nullptr);
}

int ffs_sample_lensemble(ffs_handle h, const double* lambda, int64_t B, uint64_t seed,
                         uint64_t first_sample_index, int32_t* out_x, int32_t* out_n, int32_t* out_perm,
                         double* out_logp, const int32_t* force_x, float* out_probs, void* cuda_stream) {
  if (!h) return fail(nullptr, FFS_E_ARG, "ffs_sample_lensemble: NULL handle");
  if (B < 0) return fail(h, FFS_E_ARG, "ffs_sample_lensemble: B < 0");
  if (B == 0) return FFS_OK;
  if (!lambda || !out_x) return fail(h, FFS_E_ARG, "ffs_sample_lensemble: lambda and out_x are required");
  if (!blocked(h) || op_mode_of(h->flags) == kOpNone || grouped_form(h))
    return fail(h, FFS_E_UNSUPPORTED, "ffs_sample_lensemble: needs the batched form with the blocked state");
  for (const void* p : {(const void*)out_x, (const void*)out_n, (const void*)out_perm, (const void*)out_logp,
                        (const void*)force_x, (const void*)out_probs})
    if (p && !is_device_ptr(p))
      return fail(h, FFS_E_ARG, "ffs_sample_lensemble: out_x, out_n, out_perm, out_logp, force_x and "
                                "out_probs must be device memory");
  cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : h->stream;
  const int64_t N = h->N;
  if (!h->sel_p) FFS_CUDA_TRY(h, cudaMalloc((void**)&h->sel_p, (size_t)N * sizeof(double)));
  if (is_device_ptr(lambda)) {
    FFS_CUDA_TRY(h, launch_keep_prob(lambda, N, h->sel_p, h->status, st));
  } else {
    FFS_CUDA_TRY(h, cudaMemcpyAsync(h->sel_p, lambda, (size_t)N * sizeof(double), cudaMemcpyHostToDevice, st));
    FFS_CUDA_TRY(h, launch_keep_prob(h->sel_p, N, h->sel_p, h->status, st));  // in place, per entry
  }
  // chain lengths of all samples, and the longest (the number of steps the call runs)
  int32_t* nlen = out_n;
  int* dmax = nullptr;
  if (!nlen) FFS_CUDA_TRY(h, cudaMallocAsync((void**)&nlen, (size_t)B * 4, st));
  FFS_CUDA_TRY(h, cudaMallocAsync((void**)&dmax, sizeof(int), st));
  FFS_CUDA_TRY(h, cudaMemsetAsync(dmax, 0, sizeof(int), st));
  StepArgs a{};
  a.N = N;
  a.seed = seed;
  a.first = first_sample_index;
  a.sel_p = h->sel_p;
  FFS_CUDA_TRY(h, launch_lens_count(a, B, nlen, dmax, st));
  FFS_CUDA_TRY(h, cudaMemcpyAsync(h->status_host, dmax, sizeof(int), cudaMemcpyDeviceToHost, st));
  FFS_CUDA_TRY(h, cudaStreamSynchronize(st));
  const int64_t longest = *h->status_host;
  FFS_CUDA_TRY(h, cudaMemcpy(h->status_host, h->status, sizeof(int), cudaMemcpyDeviceToHost));
  if (*h->status_host != 0) {
    cudaMemset(h->status, 0, sizeof(int));
    if (!out_n) cudaFreeAsync(nlen, st);
    cudaFreeAsync(dmax, st);
    return fail(h, FFS_E_ARG, "ffs_sample_lensemble: an eigenvalue is not finite");
  }
  // positions past a sample's chain: site -1, conditional 0
  FFS_CUDA_TRY(h, cudaMemsetAsync(out_x, 0xff, (size_t)B * N * 4, st));
  if (out_probs) FFS_CUDA_TRY(h, cudaMemsetAsync(out_probs, 0, (size_t)B * N * h->L * 4, st));
  if (out_logp) FFS_CUDA_TRY(h, cudaMemsetAsync(out_logp, 0, (size_t)B * 8, st));
  int rc = FFS_OK;
  if (longest > 0) {
    rc = sample_core(h, B, seed, first_sample_index, longest, N, out_x, out_perm, out_logp, force_x, out_probs,
                     st, h->sel_p, nlen);
  } else if (out_perm) {  // nothing kept anywhere: the column orders are the columns in order
    a.bw = B;
    a.m = out_perm;
    FFS_CUDA_TRY(h, launch_perm_init(a, kOpNone, st));
  }
  if (!out_n) cudaFreeAsync(nlen, st);
  cudaFreeAsync(dmax, st);
  return rc;
}

int ffs_sample_metropolis(ffs_handle h, int64_t B, uint64_t seed, uint64_t first_sample_index, int64_t n_steps,
                          int64_t m_cond, int32_t* out_x, int32_t* out_perm, void* cuda_stream) {
  if (!h) return fail(nullptr, FFS_E_ARG, "ffs_sample_metropolis: NULL handle");
  if (B < 0 || m_cond < 0) return fail(h, FFS_E_ARG, "ffs_sample_metropolis: B < 0 or m_cond < 0");
  if (n_steps == 0) n_steps = h->N;
  if (n_steps < 1 || n_steps > h->N) return fail(h, FFS_E_ARG, "ffs_sample_metropolis: need 0 <= n_steps <= N");
  if ((double)n_steps * (double)(m_cond + 1) > 4294967295.0)
    return fail(h, FFS_E_ARG, "ffs_sample_metropolis: n_steps x (m_cond + 1) must stay below 2^32");
  if (B == 0) return FFS_OK;
  if (!out_x || !is_device_ptr(out_x) || (out_perm && !is_device_ptr(out_perm)))
    return fail(h, FFS_E_ARG, "ffs_sample_metropolis: out_x (and out_perm) must be device memory");
  if (!blocked(h) || grouped_form(h))
    return fail(h, FFS_E_UNSUPPORTED, "ffs_sample_metropolis: needs the blocked state and no grouped form");
  int optin = 0;
  FFS_CUDA_TRY(h, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
  if (mcmc_step_smem(h->N, h->cplx, state_kind(h)) > (size_t)optin - 1024)
    return fail(h, FFS_E_UNSUPPORTED, "ffs_sample_metropolis: N too large for the shared-memory normal vectors");
  cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : h->stream;
  const int state = state_kind(h);
  const size_t es = state_elem_bytes(h), nb = blocked_panel_width(), Nc = (size_t)n_steps;
  // per sample: m, drawn-site bits, the blocked state (no residual operand, no weights)
  const size_t st_entries = (size_t)state_stride((int64_t)Nc);  // the blocked state's slabs
  const size_t per = (size_t)h->N * 4 + (size_t)h->ldMask * 4 + (st_entries + Nc * nb + nb * nb) * es;
  size_t free_b = 0, total_b = 0;
  FFS_CUDA_TRY(h, cudaMemGetInfo(&free_b, &total_b));
  const size_t reserve = (size_t)512 << 20;
  int64_t Bw = (int64_t)((free_b > reserve ? free_b - reserve : 0) / per);
  if (Bw < 1) return fail(h, FFS_E_NOMEM, "ffs_sample_metropolis: not enough device memory for one sample");
  if (Bw > B) Bw = B;
  int32_t* m = nullptr;
  uint32_t* mask = nullptr;
  void *W = nullptr, *W0P = nullptr, *Sinv = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&m, (size_t)Bw * h->N * 4, st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&mask, (size_t)Bw * h->ldMask * 4, st);
  if (e == cudaSuccess) e = cudaMallocAsync(&W, (size_t)Bw * st_entries * es, st);
  if (e == cudaSuccess) e = cudaMallocAsync(&W0P, (size_t)Bw * Nc * nb * es, st);
  if (e == cudaSuccess) e = cudaMallocAsync(&Sinv, (size_t)Bw * nb * nb * es, st);
  for (int64_t b0 = 0; b0 < B && e == cudaSuccess; b0 += Bw) {
    const int64_t bw = (B - b0 < Bw) ? B - b0 : Bw;
    StepArgs a{};
    a.L = h->L;
    a.N = h->N;
    a.ldMask = h->ldMask;
    a.bw = bw;
    a.n_steps = n_steps;
    a.seed = seed;
    a.first = first_sample_index + (uint64_t)b0;
    a.cplx = h->cplx;
    a.U64 = h->U64;
    a.Ust = h->Ust ? h->Ust : h->U64;
    a.m = m;
    a.mask = mask;
    a.x = out_x + b0 * n_steps;
    a.ldx = n_steps;
    a.status = h->status;
    BlockedArgs bt{};
    bt.Nc = n_steps;
    bt.W = W;
    bt.W0P = W0P;
    bt.Sinv = Sinv;
    e = cudaMemsetAsync(mask, 0, (size_t)bw * h->ldMask * 4, st);
    if (e == cudaSuccess) e = launch_perm_init(a, kOpNone, st);
    for (int64_t k = 0; k < n_steps && e == cudaSuccess; ++k) {
      prof_begin(h, FFS_PHASE_TAIL, st);
      e = launch_mcmc_step(a, bt, k, m_cond, state, st);
      prof_end(h, st);
      const int64_t k0 = (k / (int64_t)nb) * (int64_t)nb;
      const int64_t k1 = (k0 + (int64_t)nb < n_steps) ? k0 + (int64_t)nb : n_steps;
      if (e == cudaSuccess && k + 1 == k1 && k1 < n_steps) {
        prof_begin(h, FFS_PHASE_PANEL_S, st);
        e = launch_blocked_panel_s(a, bt, k0, k1, state, st);
        prof_end(h, st);
        if (e == cudaSuccess) {
          prof_begin(h, FFS_PHASE_PANEL, st);
          e = launch_blocked_panel_update(a, bt, k0, k1, state, kOpNone, st);
          prof_end(h, st);
        }
      }
    }
    if (e == cudaSuccess && out_perm)
      e = cudaMemcpyAsync(out_perm + b0 * h->N, m, (size_t)bw * h->N * 4, cudaMemcpyDeviceToDevice, st);
  }
  if (m) cudaFreeAsync(m, st);
  if (mask) cudaFreeAsync(mask, st);
  if (W) cudaFreeAsync(W, st);
  if (W0P) cudaFreeAsync(W0P, st);
  if (Sinv) cudaFreeAsync(Sinv, st);
  if (e != cudaSuccess) return fail(h, FFS_E_CUDA, std::string("ffs_sample_metropolis: ") + cudaGetErrorString(e));
  return FFS_OK;
}

int ffs_sample(ffs_handle h, int64_t B, uint64_t seed, int32_t* out_x) {
  return ffs_sample_ex(h, B, seed, 0, 0, out_x, nullptr, nullptr, nullptr, nullptr, nullptr);
}

int ffs_sync(ffs_handle h) {
  if (!h) return fail(nullptr, FFS_E_ARG, "ffs_sync: NULL handle");
  FFS_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  FFS_CUDA_TRY(h, cudaMemcpy(h->status_host, h->status, sizeof(int), cudaMemcpyDeviceToHost));
  const int code = *h->status_host;
  if (code != 0) {
    cudaMemset(h->status, 0, sizeof(int));
    return fail(h, code, "device reported an error (see ffs.h status codes)");
  }
  return FFS_OK;
}

void ffs_destroy(ffs_handle h) { release(h); }

}  // extern "C"

namespace fermi {
int ctx_op_mode(const ffs_ctx* c) { return op_mode_of(c->flags); }
int ctx_state_kind(const ffs_ctx* c) { return state_kind(c); }
bool ctx_blocked(const ffs_ctx* c) { return blocked(c); }
int ctx_ensure_workspace(ffs_ctx* c, int64_t B) { return ensure_workspace(c, B); }
size_t ctx_per_sample_bytes(const ffs_ctx* c) { return per_sample_bytes(c); }
size_t ctx_op_elem_bytes(int op) { return op_elem_bytes(op); }
int ctx_fail(ffs_ctx* c, int code, const std::string& msg) { return fail(c, code, msg); }
bool ptr_is_device(const void* p) { return is_device_ptr(p); }
}  // namespace fermi

extern "C" {

int ffs_profile(ffs_handle h, int enable) {
  if (!h) return fail(nullptr, FFS_E_ARG, "ffs_profile: NULL handle");
  if (h->prof) prof_fold(h);
  h->prof = enable != 0;
  for (int p = 0; p < 8; ++p) {
    h->prof_ms[p] = 0.0;
    h->prof_launches[p] = 0;
  }
  return FFS_OK;
}

int ffs_debug_inject(ffs_handle h, int fault) {
  if (!h) return fail(nullptr, FFS_E_ARG, "ffs_debug_inject: NULL handle");
  if (fault != FFS_FAULT_NONE && fault != FFS_FAULT_SKIP_ARRIVAL)
    return fail(h, FFS_E_ARG, "ffs_debug_inject: unknown fault");
  const int op = op_mode_of(h->flags);
  if (fault != FFS_FAULT_NONE && (op == kOpNone || op == kOpF32))
    return fail(h, FFS_E_UNSUPPORTED, "ffs_debug_inject: the handle has no tensor-core residual");
  h->debug_fault = fault;
  return FFS_OK;
}

int ffs_profile_read(ffs_handle h, double* ms, int64_t* launches, int n) {
  if (!h) return fail(nullptr, FFS_E_ARG, "ffs_profile_read: NULL handle");
  if (n < 0 || n > FFS_NUM_PHASES) return fail(h, FFS_E_ARG, "ffs_profile_read: bad n");
  prof_fold(h);
  for (int p = 0; p < n; ++p) {
    if (ms) ms[p] = h->prof_ms[p];
    if (launches) launches[p] = h->prof_launches[p];
  }
  return FFS_OK;
}

}  // extern "C"
