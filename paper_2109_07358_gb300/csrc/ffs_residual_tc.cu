// Tensor-core (tcgen05) residual of the batched form.
//
// Step k of every sample in a wave needs the weights of all L sites (Section S-1:
// the inner products u_y^T h), p[b, y] = |v_y|^2 with v = U h_b.  Across the wave this
// is one contraction D = H Ue^T: H (wave x Kp) holds each sample's h scattered into its
// column order m (real embedding for complex U), Ue (Lrp x Kp) is the real embedding
// of U.  Both operands are K-major in global memory, loaded by TMA with the 128-byte
// swizzle, multiplied by tcgen05.mma into an FP32 accumulator in tensor memory, and
// the epilogue squares, pairs (complex), masks the sites already drawn and writes the
// weights.  V itself is never stored.
//
// Precision modes:
//   BF16x3: H = Hh + Hl, Ue = Uh + Ul (BF16 hi/lo split); D = Hh Uh + Hh Ul + Hl Uh
//   BF16:   D = Hh Uh
//   TF32:   D = H Ue with TF32-rounded operands
//
// CTA: 128 samples x BN embedding columns; 6 warps: warp 0 issues TMA loads into a
// ring of STAGES shared-memory stages, warp 1 allocates tensor memory and issues the
// MMAs (one thread), warps 2-5 drain the accumulator (each warp owns the 32 TMEM
// lanes of its rank mod 4).
#include <cudaTypedefs.h>

#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>

#include "ffs_group.cuh"
#include "ffs_residual_tc.cuh"
#include "ffs_sm100.cuh"

namespace fermi {

using namespace sm100;

enum { kKindBF16x3 = 0, kKindBF16 = 1, kKindTF32 = 2 };

template <int BN, int STAGES, int KIND>
struct TcCfg {
  static constexpr int BM = 128;
  static constexpr int NA = (KIND == kKindBF16x3) ? 2 : 1;
  static constexpr int NB = NA;
  static constexpr uint32_t A_BYTES = BM * 128;  // one plane: 128 rows x 128 bytes
  static constexpr uint32_t B_BYTES = BN * 128;
  static constexpr uint32_t STAGE_BYTES = NA * A_BYTES + NB * B_BYTES;
  static constexpr int BK = (KIND == kKindTF32) ? 32 : 64;  // elements per 128-byte row
  static constexpr uint32_t SMEM = STAGES * STAGE_BYTES + 1024 + 256;
  static constexpr uint32_t IDESC = (KIND == kKindTF32) ? idesc_tf32(BM, BN) : idesc_bf16(BM, BN);
};

// Sum of the n weights of one site group by a balanced tree (the draw adds these group
// sums in site order for the normaliser and the search).
template <int n>
__device__ __forceinline__ float group_sum_w(const float (&w)[n]) {
  float t[n / 2];
#pragma unroll
  for (int i = 0; i < n / 2; ++i) t[i] = w[2 * i] + w[2 * i + 1];
#pragma unroll
  for (int m = n / 4; m >= 1; m /= 2) {
#pragma unroll
    for (int i = 0; i < m; ++i) t[i] = t[2 * i] + t[2 * i + 1];
  }
  return t[0];
}

// One output tile (samples [b0, b0+128) x embedding columns [j0, j0+BN)) of one
// instance; the tensor maps may live in kernel parameters or in global memory.
template <int BN, int STAGES, int KIND>
__device__ __forceinline__ void residual_body(const CUtensorMap* tmA0p, const CUtensorMap* tmA1p,
                                              const CUtensorMap* tmB0p, const CUtensorMap* tmB1p, const TcArgs& p,
                                              int32_t b0, int32_t j0, uint8_t* smem_raw, bool global_maps) {
  using C = TcCfg<BN, STAGES, KIND>;
  const CUtensorMap& tmA0 = *tmA0p;
  const CUtensorMap& tmA1 = *tmA1p;
  const CUtensorMap& tmB0 = *tmB0p;
  const CUtensorMap& tmB1 = *tmB1p;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t sbase = (raw + 1023u) & ~1023u;
  uint8_t* gbase = smem_raw + (sbase - raw);
  uint64_t* bars = (uint64_t*)(gbase + STAGES * C::STAGE_BYTES);
  const uint32_t bar0 = smem_u32(bars);
  auto full = [&](int s) { return bar0 + 8u * s; };
  auto empty = [&](int s) { return bar0 + 8u * (STAGES + s); };
  const uint32_t accum = bar0 + 8u * (2 * STAGES);
  uint32_t* tmem_slot = (uint32_t*)(bars + 2 * STAGES + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    mbar_init(accum, 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 1) {
    tmem_alloc(smem_u32(tmem_slot), BN);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int nK = p.nK;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer
    if (global_maps) {
      acquire_tmap(&tmA0);
      acquire_tmap(&tmA1);
      acquire_tmap(&tmB0);
      acquire_tmap(&tmB1);
    }
    prefetch_tmap(&tmA0);
    prefetch_tmap(&tmB0);
    if (C::NA == 2) {
      prefetch_tmap(&tmA1);
      prefetch_tmap(&tmB1);
    }
    int issued = 0;
    // failure-path test: the first CTA skips stage 0 (no arrival, no copy), so the MMA
    // warp's wait for it runs out
    const bool skip0 = p.fault && b0 == 0 && j0 == 0;
    const int32_t jg = j0 + (b0 / 128) * p.grp_rows;  // row of Ue (or of the sample group's copy)
    for (int kb = 0; kb < nK; ++kb) {
      const int s = kb % STAGES;
      const uint32_t round = kb / STAGES;
      if (kb >= STAGES && !mbar_wait_lim(empty(s), (round - 1) & 1, abort_flag, p.spin)) {
        *abort_flag = 1;
        set_status(p.status, FFS_E_TIMEOUT);
        break;
      }
      if (skip0 && kb == 0) {
        ++issued;
        continue;
      }
      const uint32_t st = sbase + s * C::STAGE_BYTES;
      mbar_arrive_expect_tx(full(s), C::STAGE_BYTES);
      const int32_t x = kb * C::BK;
      tma_load_2d(st, &tmA0, full(s), x, b0);
      if (C::NA == 2) tma_load_2d(st + C::A_BYTES, &tmA1, full(s), x, b0);
      tma_load_2d(st + C::NA * C::A_BYTES, &tmB0, full(s), x, jg);
      if (C::NB == 2) tma_load_2d(st + C::NA * C::A_BYTES + C::B_BYTES, &tmB1, full(s), x, jg);
      ++issued;
    }
    // Never leave with copies in flight: wait (bounded, even after an abort) for the last
    // loads to land.
    for (int kb = (issued > STAGES ? issued - STAGES : 0); kb < issued; ++kb)
      if (!(skip0 && kb == 0)) mbar_drain(full(kb % STAGES), (kb / STAGES) & 1, p.spin);
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    for (int kb = 0; kb < nK; ++kb) {
      const int s = kb % STAGES;
      const uint32_t round = kb / STAGES;
      if (!mbar_wait_lim(full(s), round & 1, abort_flag, p.spin)) {
        *abort_flag = 1;
        set_status(p.status, FFS_E_TIMEOUT);
        break;
      }
      tc_fence_after();
      const uint32_t st = sbase + s * C::STAGE_BYTES;
      const uint32_t sa0 = st, sa1 = st + C::A_BYTES;
      const uint32_t sb0 = st + C::NA * C::A_BYTES, sb1 = sb0 + C::B_BYTES;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint32_t koff = kk * 32;  // 32 bytes = one MMA's K (16 BF16 or 8 TF32)
        const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
        const uint64_t da0 = smem_desc_sw128(sa0 + koff), db0 = smem_desc_sw128(sb0 + koff);
        if (KIND == kKindTF32) {
          mma_tf32(tmem, da0, db0, C::IDESC, acc);
        } else if (KIND == kKindBF16) {
          mma_bf16(tmem, da0, db0, C::IDESC, acc);
        } else {
          const uint64_t da1 = smem_desc_sw128(sa1 + koff), db1 = smem_desc_sw128(sb1 + koff);
          mma_bf16(tmem, da0, db0, C::IDESC, acc);
          mma_bf16(tmem, da0, db1, C::IDESC, 1u);
          mma_bf16(tmem, da1, db0, C::IDESC, 1u);
        }
      }
      mma_commit(empty(s));
    }
    mma_commit(accum);
  } else if (warp >= 2) {
    // ---- epilogue: weights of 128 samples x BN embedding columns
    const bool ok = mbar_wait_lim(accum, 0, abort_flag, p.spin);
    tc_fence_after();
    const int q = warp & 3;
    const int row = 32 * q + lane;
    const int64_t b = (int64_t)b0 + row;
    const bool live = ok && b < p.bw;
    float* prow = p.P + b * p.ldP;
    const uint32_t* mrow = p.mask + b * p.ldMask;
#pragma unroll 1
    for (int c = 0; c < BN / 32; ++c) {
      uint32_t r[32];
      tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(c * 32), r);
      tmem_ld_wait();
      if (!live) continue;
      if (p.cplx) {
        const int64_t y0 = ((int64_t)j0 + 32 * c) >> 1;  // 16 sites
        if (y0 >= p.L) continue;
        const uint32_t mbits = mrow[y0 >> 5] >> (y0 & 31);
        float w[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const float re = __uint_as_float(r[2 * i]), im = __uint_as_float(r[2 * i + 1]);
          w[i] = ((mbits >> i) & 1u) ? 0.f : fmaf(re, re, im * im);
        }
        if (y0 + 16 <= p.L) {
#pragma unroll
          for (int i = 0; i < 16; i += 4)
            *(float4*)(prow + y0 + i) = make_float4(w[i], w[i + 1], w[i + 2], w[i + 3]);
        } else {
          for (int i = 0; i < 16; ++i)
            if (y0 + i < p.L) prow[y0 + i] = w[i];
            else w[i] = 0.f;
        }
        if (p.G) p.G[b * p.ldG + (y0 >> 4)] = group_sum_w<16>(w);
      } else {
        const int64_t y0 = (int64_t)j0 + 32 * c;  // 32 sites
        if (y0 >= p.L) continue;
        const uint32_t mbits = mrow[y0 >> 5];
        float w[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const float v = __uint_as_float(r[i]);
          w[i] = ((mbits >> i) & 1u) ? 0.f : v * v;
        }
        if (y0 + 32 <= p.L) {
#pragma unroll
          for (int i = 0; i < 32; i += 4)
            *(float4*)(prow + y0 + i) = make_float4(w[i], w[i + 1], w[i + 2], w[i + 3]);
        } else {
          for (int i = 0; i < 32; ++i)
            if (y0 + i < p.L) prow[y0 + i] = w[i];
            else w[i] = 0.f;
        }
        if (p.G) p.G[b * p.ldG + (y0 >> 5)] = group_sum_w<32>(w);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem, BN);
  }
}

template <int BN, int STAGES, int KIND>
__global__ void __launch_bounds__(192, 1)
    residual_tc_kernel(const __grid_constant__ CUtensorMap tmA0, const __grid_constant__ CUtensorMap tmA1,
                       const __grid_constant__ CUtensorMap tmB0, const __grid_constant__ CUtensorMap tmB1,
                       TcArgs p) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  residual_body<BN, STAGES, KIND>(&tmA0, &tmA1, &tmB0, &tmB1, p, (int32_t)blockIdx.y * 128,
                                  (int32_t)blockIdx.x * BN, smem_raw, false);
}

// Grouped form: CTA blockIdx.x -> (instance, tile) through the entry list.
template <int BN, int STAGES, int KIND>
__global__ void __launch_bounds__(192, 1)
    residual_group_kernel(const GroupInst* __restrict__ inst, const GroupEntry* __restrict__ ent, int n) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  const int64_t item = blockIdx.x;
  const int e = group_find(ent, n, item);
  const GroupInst* gi = inst + ent[e].inst;
  const int64_t local = item - ent[e].start;
  const int64_t bt = local / gi->n_jtiles, jt = local - bt * gi->n_jtiles;
  const TcArgs p = gi->tc;
  residual_body<BN, STAGES, KIND>(&gi->tm[0], &gi->tm[1], &gi->tm[2], &gi->tm[3], p, (int32_t)(bt * 128),
                                  (int32_t)(jt * BN), smem_raw, true);
}

// ------------------------------------------------------------------ host side
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)ptr;
  }
  return fn;
}

// Row-major rows x inner matrix, 128-byte-swizzled boxes of (128 bytes) x box_rows.
cudaError_t encode_2d(CUtensorMap* map, const void* base, bool f32, uint64_t inner, uint64_t rows,
                             uint32_t box_rows) {
  auto fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  const uint32_t es = f32 ? 4 : 2;
  cuuint64_t dims[2] = {inner, rows};
  cuuint64_t strides[1] = {inner * es};
  cuuint32_t box[2] = {128 / es, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                  const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Tile configurations (embedding columns per CTA, pipeline stages) for each precision;
// the autotuner picks the column tile per size class.
template <int KIND, int BN> struct StagesOf;
template <> struct StagesOf<kKindBF16x3, 256> { static constexpr int v = 2; };
template <> struct StagesOf<kKindBF16x3, 128> { static constexpr int v = 3; };
template <> struct StagesOf<kKindBF16, 256> { static constexpr int v = 4; };
template <> struct StagesOf<kKindBF16, 128> { static constexpr int v = 6; };
template <> struct StagesOf<kKindTF32, 256> { static constexpr int v = 4; };
template <> struct StagesOf<kKindTF32, 128> { static constexpr int v = 6; };

static int kind_of(int op) { return op == kOpBF16x3 ? kKindBF16x3 : op == kOpBF16 ? kKindBF16 : kKindTF32; }

cudaError_t prepare_residual_tc_bn(ffs_ctx* c, int op, int bn) {
  const bool f32 = (op == kOpTF32);
  const int key = op * 1000 + bn;
  if (c->tm_U_ready != key) {
    const void* u0 = f32 ? (const void*)c->Ue_tf32 : (const void*)c->Ue_hi;
    cudaError_t e = encode_2d(&c->tmU[0], u0, f32, c->Kp, c->Lrp, bn);
    if (e != cudaSuccess) return e;
    if (op == kOpBF16x3) {
      e = encode_2d(&c->tmU[1], c->Ue_lo, false, c->Kp, c->Lrp, bn);
      if (e != cudaSuccess) return e;
    } else {
      c->tmU[1] = c->tmU[0];
    }
    c->tm_U_ready = key;
  }
  if (c->Ug && (c->tmUg_key != key || c->tmUg_groups != c->Ug_groups)) {
    // grouped form: one map per plane over all groups' copies (groups x Lrp rows)
    const uint64_t rows = (uint64_t)c->Ug_groups * c->Lrp;
    const size_t es = f32 ? 4 : 2;
    cudaError_t e = encode_2d(&c->tmUg[0], c->Ug, f32, c->Kp, rows, bn);
    if (e != cudaSuccess) return e;
    if (op == kOpBF16x3) {
      e = encode_2d(&c->tmUg[1], (const char*)c->Ug + rows * c->Kp * es, false, c->Kp, rows, bn);
      if (e != cudaSuccess) return e;
    } else {
      c->tmUg[1] = c->tmUg[0];
    }
    c->tmUg_key = key;
    c->tmUg_groups = c->Ug_groups;
  }
  if (c->tm_H_B != c->ws_B) {
    const uint64_t plane = (uint64_t)c->ws_B * c->Kp;
    cudaError_t e = encode_2d(&c->tmH[0], c->H, f32, c->Kp, c->ws_B, 128);
    if (e != cudaSuccess) return e;
    if (op == kOpBF16x3) {
      e = encode_2d(&c->tmH[1], (const __nv_bfloat16*)c->H + plane, false, c->Kp, c->ws_B, 128);
      if (e != cudaSuccess) return e;
    } else {
      c->tmH[1] = c->tmH[0];
    }
    c->tm_H_B = c->ws_B;
  }
  c->res_bn = bn;
  return cudaSuccess;
}

cudaError_t prepare_residual_tc(ffs_ctx* c, int op) {
  return prepare_residual_tc_bn(c, op, c->res_bn ? c->res_bn : 256);
}

template <int BN, int KIND>
static cudaError_t launch_cfg(ffs_ctx* c, const StepArgs& a, cudaStream_t s) {
  constexpr int STAGES = StagesOf<KIND, BN>::v;
  using Cf = TcCfg<BN, STAGES, KIND>;
  TcArgs p;
  p.bw = a.bw;
  p.L = a.L;
  p.ldP = a.ldP;
  p.ldMask = a.ldMask;
  p.nK = (int)(a.Kp / Cf::BK);
  if (a.grouped && a.kcols > 0) p.nK = (int)((a.kcols + Cf::BK - 1) / Cf::BK);  // the leading K columns
  p.cplx = a.cplx ? 1 : 0;
  p.grp_rows = a.grouped ? (int)c->Lrp : 0;
  p.P = a.P;
  p.G = a.G;
  p.ldG = a.ldG;
  p.mask = a.mask;
  p.status = a.status;
  if (c->debug_fault == FFS_FAULT_SKIP_ARRIVAL) {  // one-shot, armed by ffs_debug_inject
    p.fault = 1;
    p.spin = 1u << 12;
    c->debug_fault = FFS_FAULT_NONE;
  }
  dim3 grid((unsigned)(c->Lrp / BN), (unsigned)((a.bw + 127) / 128));
  const CUtensorMap* tu = a.grouped ? c->tmUg : c->tmU;
  residual_tc_kernel<BN, STAGES, KIND><<<grid, 192, Cf::SMEM, s>>>(c->tmH[0], c->tmH[1], tu[0], tu[1], p);
  return cudaGetLastError();
}

static cudaError_t launch_bn(ffs_ctx* c, const StepArgs& a, int op, int bn, cudaStream_t s) {
  switch (kind_of(op) * 2 + (bn == 128 ? 1 : 0)) {
    case kKindBF16x3 * 2: return launch_cfg<256, kKindBF16x3>(c, a, s);
    case kKindBF16x3 * 2 + 1: return launch_cfg<128, kKindBF16x3>(c, a, s);
    case kKindBF16 * 2: return launch_cfg<256, kKindBF16>(c, a, s);
    case kKindBF16 * 2 + 1: return launch_cfg<128, kKindBF16>(c, a, s);
    case kKindTF32 * 2: return launch_cfg<256, kKindTF32>(c, a, s);
    default: return launch_cfg<128, kKindTF32>(c, a, s);
  }
}

// ------------------------------------------------------------------ autotuner
// Size class -> column tile, measured once per process (CUDA events on the launching
// stream, two candidates, best of three launches each) and optionally kept in the file
// named by FFS_TUNE_CACHE ("key tile" lines).  FFS_RES_BN=128|256 forces a tile.
static std::mutex g_tune_mu;
static std::map<std::string, int> g_tune;
static bool g_tune_loaded = false;

// Size classes: power-of-two buckets of the embedding rows, K and sample tiles, so that a
// stream of requests of varied sizes reuses a handful of measurements.
static int64_t pow2_ceil(int64_t v) {
  int64_t b = 1;
  while (b < v) b <<= 1;
  return b;
}
static std::string tune_key(int op, int64_t Lrp, int64_t Kp, int64_t bw) {
  return std::to_string(op) + ":" + std::to_string(pow2_ceil(Lrp)) + ":" + std::to_string(pow2_ceil(Kp)) + ":" +
         std::to_string(pow2_ceil((bw + 127) / 128));
}

static void tune_load() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* path = getenv("FFS_TUNE_CACHE");
  if (!path) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  char key[128];
  int bn;
  while (fscanf(f, "%127s %d", key, &bn) == 2)
    if (bn == 128 || bn == 256) g_tune[key] = bn;
  fclose(f);
}

static void tune_store(const std::string& key, int bn) {
  const char* path = getenv("FFS_TUNE_CACHE");
  if (!path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s %d\n", key.c_str(), bn);
  fclose(f);
}

int residual_tile_for(ffs_ctx* c, const StepArgs& a, int op, cudaStream_t s) {
  const char* forced = getenv("FFS_RES_BN");
  if (forced && (atoi(forced) == 128 || atoi(forced) == 256)) return atoi(forced);
  const std::string key = tune_key(op, c->Lrp, c->Kp, a.bw);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_load();
    auto it = g_tune.find(key);
    if (it != g_tune.end()) return it->second;
  }
  int best = 256;
  float best_ms = 1e30f;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return best;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return best;
  }
  for (int bn : {256, 128}) {
    if (prepare_residual_tc_bn(c, op, bn) != cudaSuccess || launch_bn(c, a, op, bn, s) != cudaSuccess) continue;
    float ms_min = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      cudaEventRecord(e0, s);
      launch_bn(c, a, op, bn, s);
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      ms_min = ms < ms_min ? ms : ms_min;
    }
    if (ms_min < best_ms) {
      best_ms = ms_min;
      best = bn;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (!g_tune.count(key)) {
    g_tune[key] = best;
    tune_store(key, best);
  }
  return best;
}

cudaError_t launch_residual_tc(ffs_ctx* c, const StepArgs& a, int op, cudaStream_t s) {
  const int bn = c->res_bn ? c->res_bn : 256;
  cudaError_t e = prepare_residual_tc_bn(c, op, bn);
  if (e != cudaSuccess) return e;
  return launch_bn(c, a, op, bn, s);
}

template <int BN, int KIND>
static void group_launch(const GroupInst* inst, const GroupEntry* e, int n, unsigned grid, cudaStream_t s) {
  constexpr int STAGES = StagesOf<KIND, BN>::v;
  residual_group_kernel<BN, STAGES, KIND><<<grid, 192, TcCfg<BN, STAGES, KIND>::SMEM, s>>>(inst, e, n);
}

cudaError_t launch_group_residual(const GroupInst* inst, const GroupEntry* e, int n, int64_t total, int op, int bn,
                                  cudaStream_t s) {
  if (total <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)total;
  switch (kind_of(op) * 2 + (bn == 128 ? 1 : 0)) {
    case kKindBF16x3 * 2: group_launch<256, kKindBF16x3>(inst, e, n, grid, s); break;
    case kKindBF16x3 * 2 + 1: group_launch<128, kKindBF16x3>(inst, e, n, grid, s); break;
    case kKindBF16 * 2: group_launch<256, kKindBF16>(inst, e, n, grid, s); break;
    case kKindBF16 * 2 + 1: group_launch<128, kKindBF16>(inst, e, n, grid, s); break;
    case kKindTF32 * 2: group_launch<256, kKindTF32>(inst, e, n, grid, s); break;
    default: group_launch<128, kKindTF32>(inst, e, n, grid, s); break;
  }
  return cudaGetLastError();
}

int residual_k_block(int op) { return op == kOpTF32 ? 32 : 64; }

template <int BN, int KIND> static cudaError_t allow_cfg() {
  constexpr int STAGES = StagesOf<KIND, BN>::v;
  constexpr int SM = TcCfg<BN, STAGES, KIND>::SMEM;
  cudaError_t e = cudaFuncSetAttribute(residual_tc_kernel<BN, STAGES, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, SM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(residual_group_kernel<BN, STAGES, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, SM);
  return e;
}

cudaError_t configure_residual_tc() {
  cudaError_t e = allow_cfg<256, kKindBF16x3>();
  if (e == cudaSuccess) e = allow_cfg<128, kKindBF16x3>();
  if (e == cudaSuccess) e = allow_cfg<256, kKindBF16>();
  if (e == cudaSuccess) e = allow_cfg<128, kKindBF16>();
  if (e == cudaSuccess) e = allow_cfg<256, kKindTF32>();
  if (e == cudaSuccess) e = allow_cfg<128, kKindTF32>();
  return e;
}

}  // namespace fermi
