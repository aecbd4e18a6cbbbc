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
    for (int kb = 0; kb < nK; ++kb) {
      const int s = kb % STAGES;
      const uint32_t round = kb / STAGES;
      if (kb >= STAGES && !mbar_wait(empty(s), (round - 1) & 1, abort_flag)) {
        *abort_flag = 1;
        set_status(p.status, FFS_E_TIMEOUT);
        break;
      }
      const uint32_t st = sbase + s * C::STAGE_BYTES;
      mbar_arrive_expect_tx(full(s), C::STAGE_BYTES);
      const int32_t x = kb * C::BK;
      tma_load_2d(st, &tmA0, full(s), x, b0);
      if (C::NA == 2) tma_load_2d(st + C::A_BYTES, &tmA1, full(s), x, b0);
      tma_load_2d(st + C::NA * C::A_BYTES, &tmB0, full(s), x, j0);
      if (C::NB == 2) tma_load_2d(st + C::NA * C::A_BYTES + C::B_BYTES, &tmB1, full(s), x, j0);
      ++issued;
    }
    // Never leave with copies in flight: wait (bounded) for the last loads to land.
    for (int kb = (issued > STAGES ? issued - STAGES : 0); kb < issued; ++kb)
      mbar_wait(full(kb % STAGES), (kb / STAGES) & 1, abort_flag);
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    for (int kb = 0; kb < nK; ++kb) {
      const int s = kb % STAGES;
      const uint32_t round = kb / STAGES;
      if (!mbar_wait(full(s), round & 1, abort_flag)) {
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
    const bool ok = mbar_wait(accum, 0, abort_flag);
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
          for (int i = 0; i < 16 && y0 + i < p.L; ++i) prow[y0 + i] = w[i];
        }
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
          for (int i = 0; i < 32 && y0 + i < p.L; ++i) prow[y0 + i] = w[i];
        }
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
static cudaError_t encode_2d(CUtensorMap* map, const void* base, bool f32, uint64_t inner, uint64_t rows,
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

constexpr int kBN = 256;

cudaError_t prepare_residual_tc(ffs_ctx* c, int op) {
  const bool f32 = (op == kOpTF32);
  if (c->tm_U_ready != op) {
    const void* u0 = f32 ? (const void*)c->Ue_tf32 : (const void*)c->Ue_hi;
    cudaError_t e = encode_2d(&c->tmU[0], u0, f32, c->Kp, c->Lrp, kBN);
    if (e != cudaSuccess) return e;
    if (op == kOpBF16x3) {
      e = encode_2d(&c->tmU[1], c->Ue_lo, false, c->Kp, c->Lrp, kBN);
      if (e != cudaSuccess) return e;
    } else {
      c->tmU[1] = c->tmU[0];
    }
    c->tm_U_ready = op;
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
  return cudaSuccess;
}

template <int BN, int STAGES, int KIND>
static cudaError_t launch_cfg(ffs_ctx* c, const StepArgs& a, cudaStream_t s) {
  using Cf = TcCfg<BN, STAGES, KIND>;
  TcArgs p;
  p.bw = a.bw;
  p.L = a.L;
  p.ldP = a.ldP;
  p.ldMask = a.ldMask;
  p.nK = (int)(a.Kp / Cf::BK);
  p.cplx = a.cplx ? 1 : 0;
  p.P = a.P;
  p.mask = a.mask;
  p.status = a.status;
  dim3 grid((unsigned)(c->Lrp / BN), (unsigned)((a.bw + 127) / 128));
  residual_tc_kernel<BN, STAGES, KIND><<<grid, 192, Cf::SMEM, s>>>(c->tmH[0], c->tmH[1], c->tmU[0], c->tmU[1], p);
  return cudaGetLastError();
}

cudaError_t launch_residual_tc(ffs_ctx* c, const StepArgs& a, int op, cudaStream_t s) {
  cudaError_t e = prepare_residual_tc(c, op);
  if (e != cudaSuccess) return e;
  switch (op) {
    case kOpBF16x3: return launch_cfg<kBN, 2, kKindBF16x3>(c, a, s);
    case kOpBF16: return launch_cfg<kBN, 4, kKindBF16>(c, a, s);
    case kOpTF32: return launch_cfg<kBN, 4, kKindTF32>(c, a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_group_residual(const GroupInst* inst, const GroupEntry* e, int n, int64_t total, int op,
                                  cudaStream_t s) {
  if (total <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)total;
  switch (op) {
    case kOpBF16x3:
      residual_group_kernel<kBN, 2, kKindBF16x3><<<grid, 192, TcCfg<kBN, 2, kKindBF16x3>::SMEM, s>>>(inst, e, n);
      break;
    case kOpBF16:
      residual_group_kernel<kBN, 4, kKindBF16><<<grid, 192, TcCfg<kBN, 4, kKindBF16>::SMEM, s>>>(inst, e, n);
      break;
    case kOpTF32:
      residual_group_kernel<kBN, 4, kKindTF32><<<grid, 192, TcCfg<kBN, 4, kKindTF32>::SMEM, s>>>(inst, e, n);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

int residual_tile_cols() { return kBN; }
int residual_k_block(int op) { return op == kOpTF32 ? 32 : 64; }

cudaError_t configure_residual_tc() {
  {
    cudaError_t e = cudaFuncSetAttribute(residual_group_kernel<kBN, 2, kKindBF16x3>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, TcCfg<kBN, 2, kKindBF16x3>::SMEM);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(residual_group_kernel<kBN, 4, kKindBF16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               TcCfg<kBN, 4, kKindBF16>::SMEM);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(residual_group_kernel<kBN, 4, kKindTF32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               TcCfg<kBN, 4, kKindTF32>::SMEM);
    if (e != cudaSuccess) return e;
  }
  cudaError_t e;
  e = cudaFuncSetAttribute(residual_tc_kernel<kBN, 2, kKindBF16x3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           TcCfg<kBN, 2, kKindBF16x3>::SMEM);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(residual_tc_kernel<kBN, 4, kKindBF16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           TcCfg<kBN, 4, kKindBF16>::SMEM);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(residual_tc_kernel<kBN, 4, kKindTF32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              TcCfg<kBN, 4, kKindTF32>::SMEM);
}

}  // namespace fermi
