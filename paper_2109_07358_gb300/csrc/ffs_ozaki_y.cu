// New rows of the trailing update on tensor cores (FFS_TRAILING_TC, double-float state).
//
// At a panel end (panel rows k0..k1-1, trailing columns T = [k1, Nc)) the new rows of the
// blocked state are (Supplementary Section S-1's elimination, in panels)
//   Y   = U[x_new, m_T] - C W0_T,   C = U[x_new, m_<k0]   (32 x |T|, K = k0)
//   Bot = S^-1 Y                                          (written as state rows k0..k1-1)
// Y holds most of the panel end's multiply-adds (32 k0 |T| per sample).  Here it runs on
// tcgen05 as Y^T = D^T - W0_T^T C^T through a split of both double-float operands into
// BF16 slices (Ozaki, Ogita, Oishi & Rump, Numer. Algorithms 59, 2012):
//   * K (the old rows j < k0) is cut into chunks of 64.  Within a chunk, trailing column c
//     of W0_T is scaled by a power of two sigma_{c,t} >= its largest entry and cut into six
//     8-bit integer slices, W0_T[j, c] / sigma = sum_i a_i 2^(-7 - 8(i-1)) + r, |r| <=
//     2^-47 (three exact digits of the high part, then the low part folded into the
//     remainder by one FMA; |a_i| <= 128 except |a_4| <= 256, all exact in BF16); row i
//     of C likewise with sigma_{i,t}, by error-free steps (|r| <= 2^-48);
//   * the 26 slice products a_i b_j with i + j = d <= 8 accumulate in one FP32 accumulator
//     per d in tensor memory: 64 products of at most 2^15 each, integers of at most 2^23,
//     so the tensor-core accumulation is exact;
//   * per chunk the epilogue adds the seven accumulators (oz_group_sum), scales by
//     sigma_{c,t} sigma_{i,t} 2^-14 and accumulates the chunk into Y;
//   * the accumulators are double-buffered, so one chunk's epilogue overlaps the next
//     chunk's products.
// The remainders (3/4 of 2^-46 sigma sigma per term), the dropped products (i + j > 8,
// below 2^-53 sigma sigma per term) and the FP32 rounding of the three smallest groups
// (2^-47 sigma sigma per chunk) keep each chunk's product within 2^-46 sigma sigma K of
// the exact one, next to the double-float rounding of the direct update.
//
// CTA: one sample, 128 trailing columns.  Warp 0 issues the TMA loads of C's slices (made
// once per sample and panel by ozc_slice_kernel), warp 1 allocates tensor memory and
// issues the MMAs, warps 2-9 load W0_T from the state and write its slices straight into
// the swizzled shared-memory operand tiles (two threads per trailing column, 32 old rows
// each), warps 10-17 drain the accumulators (two per tensor-memory lane quarter, 16 new
// rows each); then warps 2-17 together form Bot = S^-1 Y and write the new rows.
#include <type_traits>

#include "ffs_arith.cuh"
#include "ffs_kernels.cuh"
#include "ffs_residual_tc.cuh"
#include "ffs_sm100.cuh"

namespace fermi {

using namespace sm100;

namespace {

constexpr int kYS = 6;                      // slices per operand (48 bits)
constexpr int kYD = 8;                      // products a_i b_j kept: i + j <= kYD
constexpr int YM = 128;                     // trailing columns per CTA
constexpr int YN = 32;                      // new rows (real)
constexpr int YKC = 64;                     // old rows per K chunk
constexpr uint32_t kYATile = YM * 128;      // one slice of A: 128 rows x 64 BF16 (16 KB)
constexpr uint32_t kYAHalf = 3 * kYATile;   // three slices (48 KB)
constexpr int kYAHalves = 3;                // ring of half-chunk stages
constexpr uint32_t kYBTile = YN * 128;      // one slice of B: 32 rows x 64 BF16 (4 KB)
constexpr uint32_t kYBStage = kYS * kYBTile;  // the six slices of a chunk (24 KB)
constexpr int kYBStages = 2;
constexpr int kYProdWarps = 8, kYEpiWarps = 8;
constexpr int kYThreads = 32 * (2 + kYProdWarps + kYEpiWarps);  // 576
constexpr uint32_t kYAccCols = 256;         // one accumulator set: 7 groups x 32 columns (+ pad)
constexpr uint32_t kYTmemCols = 512;        // two sets
constexpr uint32_t kYSigRing = 4;           // chunks of column scales kept for the epilogue
constexpr uint32_t kYSmem = kYAHalves * kYAHalf + kYBStages * kYBStage + kYSigRing * YM * 4 + 1024 + 256;
static_assert(YN * YM * 8 + YN * YN * 16 <= kYAHalves * kYAHalf, "Y and S^-1 staging fit the operand ring");
constexpr uint32_t kYIdesc = idesc_bf16(YM, YN);

// Power-of-two scale sigma > max (as sigma, 1/sigma); 1 for an all-zero chunk.  A
// subnormal max takes sigma = 2^-125 so that 1/sigma stays finite; a max at or above
// 2^127 takes sigma = 2^127 (then |x| / sigma < 2 and the first slice is at most 256,
// still exact in BF16, and the group sums stay below 2^22).
__device__ __forceinline__ void ypow2(float mx, float& sigma, float& inv) {
  if (!(mx > 0.f)) {
    sigma = inv = 1.f;
    return;
  }
  int e;
  frexpf(mx, &e);  // mx = m 2^e, m in [0.5, 1)
  e = min(max(e, -125), 127);
  sigma = ldexpf(1.f, e);
  inv = ldexpf(1.f, -e);
}

// One slicing step of a scaled value held as an unevaluated pair (th, tl), |tl| <=
// ulp(th) / 2: the next 8-bit digit a = rint(th), and the remainder, scaled by 2^8, again
// as such a pair.  th - a is exact (|th| <= 2^7 + 1/2) and a multiple of ulp(th), so the
// sum with tl is error-free by the fast two-sum (its magnitude condition holds, or
// th - a = 0).
__device__ __forceinline__ float slice_step(float& th, float& tl) {
  const float a = rintf(th);
  const float d = __fsub_rn(th, a);
  const float s = __fadd_rn(d, tl);
  const float e = __fsub_rn(tl, __fsub_rn(s, d));
  th = __fmul_rn(s, 256.f);
  tl = __fmul_rn(e, 256.f);
  return a;
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // exact: integers of magnitude <= 128
  return *reinterpret_cast<const uint32_t*>(&v);
}

// Byte offset of the 16-byte chunk kc (elements 8 kc .. 8 kc + 7) of row r in a K-major tile
// of 128-byte rows stored with the 128-byte swizzle (the layout TMA writes and the MMA
// descriptors of ffs_sm100.cuh describe).
__device__ __forceinline__ uint32_t sw128_chunk(uint32_t r, uint32_t kc) {
  return (r >> 3) * 1024u + (r & 7u) * 128u + ((kc ^ (r & 7u)) << 4);
}

// C's slices for one sample, panel and K chunk: rows i < 32 of C = U[x_new, m_<k0]
// (Ust in double-float), layout [b][chunk][slice][32 rows][64] BF16 with the row scales
// in [b][chunk][32].  One warp per (row, chunk, sample).  Real: a chunk is 64 old rows,
// lane l takes columns 2l, 2l+1.  Complex: a chunk is 32 old rows as 64 interleaved
// K elements (Re C, Im C); lane l takes old row l of the chunk.
template <bool CX>
__global__ void __launch_bounds__(256) ozc_slice_kernel(StepArgs a, BlockedArgs t, OzYArgs z, int64_t k0,
                                                        int64_t k1) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t b = blockIdx.z;
  const int64_t tc = blockIdx.y;                 // chunk
  const int i = blockIdx.x * 8 + warp;           // row of C
  if (i >= YN) return;
  if (a.nlen && a.nlen[b] <= k1) return;
  const int32_t* mrow = a.m + b * a.N;
  const int xi = a.x[b * a.ldx + k0 + i];
  df v[2];
  if constexpr (CX) {
    const int64_t j = tc * (YKC / 2) + lane;
    const cdf u = (j < k0) ? ((const cdf*)a.Ust)[(int64_t)xi * a.N + mrow[j]] : cdf{df{0.f, 0.f}, df{0.f, 0.f}};
    v[0] = u.re;
    v[1] = u.im;
  } else {
    const df* urow = (const df*)a.Ust + (int64_t)xi * a.N;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int64_t j = tc * YKC + 2 * lane + q;
      v[q] = (j < k0) ? urow[mrow[j]] : df{0.f, 0.f};
    }
  }
  float mx = fmaxf(fabsf(v[0].hi), fabsf(v[1].hi));
#pragma unroll
  for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  float sigma, inv;
  ypow2(mx, sigma, inv);
  float th[2], tl[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    th[q] = __fmul_rn(__fmul_rn(v[q].hi, inv), 128.f);
    tl[q] = __fmul_rn(__fmul_rn(v[q].lo, inv), 128.f);
  }
  __nv_bfloat16* base = z.C + ((size_t)(b * z.n_chunks + tc) * kYS) * YN * YKC;
#pragma unroll
  for (int s = 0; s < kYS; ++s) {
    const float a0 = slice_step(th[0], tl[0]), a1 = slice_step(th[1], tl[1]);
    *(uint32_t*)(base + ((size_t)s * YN + i) * YKC + 2 * lane) = pack_bf16x2(a0, a1);
  }
  if (lane == 0) z.Cs[(b * z.n_chunks + tc) * YN + i] = sigma;
}

// Y, Bot and the new rows for one sample: 128 trailing columns of a real double-float
// state, or 64 of a complex one.  A complex column c becomes two real operand rows over
// K elements interleaved per old row j, (Re W, -Im W) and (Im W, Re W), so that against
// the rows (Re C, Im C) of B they give Re and Im of (C W0_T)[i, c]; the MMAs, the tensor
// memory and the pipeline are those of the real kernel.
template <bool CX>
__global__ void __launch_bounds__(kYThreads, 1)
    ozy_kernel(const __grid_constant__ CUtensorMap tmC, StepArgs a, BlockedArgs t, OzYArgs z, int64_t k0, int64_t k1) {
  using E = typename std::conditional<CX, cdf, df>::type;  // the state's element type
  constexpr int YCOL = CX ? YM / 2 : YM;                   // trailing columns per CTA
  constexpr int JC = CX ? YKC / 2 : YKC;                   // old rows per K chunk
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t b = blockIdx.y;
  if (a.nlen && a.nlen[b] <= k1) return;  // uniform over the CTA
  const int64_t Nc = t.Nc;
  const int64_t c0 = k1 + (int64_t)blockIdx.x * YCOL;
  const int nch = (int)((k0 + JC - 1) / JC);
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t sbase = (raw + 1023u) & ~1023u;
  uint8_t* gbase = smem_raw + (sbase - raw);
  const uint32_t sA = sbase, sB = sbase + kYAHalves * kYAHalf;
  float* sSig = (float*)(gbase + kYAHalves * kYAHalf + kYBStages * kYBStage);
  uint64_t* bars = (uint64_t*)(sSig + kYSigRing * YM);
  const uint32_t bar0 = smem_u32(bars);
  auto a_full = [&](int s) { return bar0 + 8u * s; };
  auto a_empty = [&](int s) { return bar0 + 8u * (3 + s); };
  auto b_full = [&](int s) { return bar0 + 8u * (6 + s); };
  auto b_empty = [&](int s) { return bar0 + 8u * (8 + s); };
  auto acc_full = [&](int u) { return bar0 + 8u * (10 + u); };
  auto acc_empty = [&](int u) { return bar0 + 8u * (12 + u); };
  auto sig_full = [&](int r) { return bar0 + 8u * (14 + r); };
  const uint32_t mma_done = bar0 + 8u * 18;
  uint32_t* tmem_slot = (uint32_t*)(bars + 19);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  if (threadIdx.x == 0) {
    for (int s = 0; s < kYAHalves; ++s) {
      mbar_init(a_full(s), kYProdWarps);
      mbar_init(a_empty(s), 1);
    }
    for (int s = 0; s < kYBStages; ++s) {
      mbar_init(b_full(s), 1);
      mbar_init(b_empty(s), 1);
    }
    for (int u = 0; u < 2; ++u) {
      mbar_init(acc_full(u), 1);
      mbar_init(acc_empty(u), kYEpiWarps);
    }
    for (int r = 0; r < (int)kYSigRing; ++r) mbar_init(sig_full(r), kYProdWarps);
    mbar_init(mma_done, 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 1) {
    tmem_alloc(smem_u32(tmem_slot), kYTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  auto fail = [&]() {
    *abort_flag = 1;
    set_status(a.status, FFS_E_TIMEOUT);
  };

  if (warp == 0) {
    // ---- TMA: the six slices of C for every chunk (one box of 6 x 32 rows)
    if (lane == 0 && nch > 0) {
      prefetch_tmap(&tmC);
      int issued = 0;
      for (int tc = 0; tc < nch; ++tc) {
        const int s = tc % kYBStages;
        if (tc >= kYBStages && !mbar_wait(b_empty(s), ((tc / kYBStages) - 1) & 1, abort_flag)) {
          fail();
          break;
        }
        mbar_arrive_expect_tx(b_full(s), kYBStage);
        tma_load_2d(sB + s * kYBStage, &tmC, b_full(s), 0, (int32_t)((b * z.n_chunks + tc) * kYS * YN));
        ++issued;
      }
      for (int tc = (issued > kYBStages ? issued - kYBStages : 0); tc < issued; ++tc)
        mbar_drain(b_full(tc % kYBStages), (tc / kYBStages) & 1, kSpinLimit);
    }
  } else if (warp == 1) {
    // ---- MMA issuer: group d of accumulator set u at columns u * 256 + 32 (d - 2)
    if (lane == 0) {
      bool ok = true;
      for (int tc = 0; tc < nch && ok; ++tc) {
        const int u = tc & 1;
        if ((tc >= 2 && !mbar_wait(acc_empty(u), ((tc >> 1) - 1) & 1, abort_flag)) ||
            !mbar_wait(b_full(tc % kYBStages), (tc / kYBStages) & 1, abort_flag)) {
          fail();
          break;
        }
        const uint32_t accb = tmem + (uint32_t)u * kYAccCols;
        const uint32_t stB = sB + (tc % kYBStages) * kYBStage;
        uint32_t started = 0;
        for (int hf = 0; hf < 2 && ok; ++hf) {
          const int hidx = 2 * tc + hf, slot = hidx % kYAHalves;
          if (!mbar_wait(a_full(slot), (hidx / kYAHalves) & 1, abort_flag)) {
            fail();
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t stA = sA + slot * kYAHalf;
#pragma unroll 1
          for (int i = 3 * hf + 1; i <= 3 * hf + 3; ++i) {
#pragma unroll 1
            for (int j = 1; j <= kYS && i + j <= kYD; ++j) {
              const int d = i + j;
              const uint32_t ta = stA + (i - 1 - 3 * hf) * kYATile, tb = stB + (j - 1) * kYBTile;
#pragma unroll
              for (int kk = 0; kk < 4; ++kk) {
                const uint32_t acc = ((started >> d) & 1u) | (kk > 0 ? 1u : 0u);
                mma_bf16(accb + (uint32_t)(32 * (d - 2)), smem_desc_sw128(ta + kk * 32), smem_desc_sw128(tb + kk * 32),
                         kYIdesc, acc);
              }
              started |= 1u << d;
            }
          }
          mma_commit(a_empty(slot));
        }
        if (!ok) break;
        mma_commit(b_empty(tc % kYBStages));
        mma_commit(acc_full(u));
      }
      // every MMA issued has completed before tensor memory is released (also after an abort)
      mma_commit(mma_done);
      mbar_drain(mma_done, 0, kSpinLimit);
    }
  } else if (warp < 2 + kYProdWarps) {
    // ---- producers: thread pair (2 r, 2 r + 1) owns operand row r (real: trailing column
    // c0 + r; complex: column c0 + r / 2, its (Re, -Im) or (Im, Re) row), K elements
    // [32 q, 32 q + 32) of each chunk (q = the thread's parity)
    const int pid = threadIdx.x - 64;
    const int q = pid & 1, ar = pid >> 1;
    const int cl = CX ? (ar >> 1) : ar;
    const int rpart = CX ? (ar & 1) : 0;
    const int64_t c = c0 + cl;
    const bool cval = c < Nc;
    const E* Wc = (const E*)t.W + (size_t)b * state_stride(Nc) + (size_t)slab_offset(c >> 5) + (c & 31);
    // one thread keeps the next two chunks of the CTA's slabs (JC rows each, contiguous) on
    // their way into L2 while the current chunk is sliced
    const E* Wb = (const E*)t.W + (size_t)b * state_stride(Nc);
    auto prefetch_chunk = [&](int tcp) {
      if (pid != 0 || tcp >= nch) return;
      const int64_t r0 = (int64_t)tcp * JC, rn = min((int64_t)JC, k0 - r0);
      for (int sl = 0; sl < YCOL / 32; ++sl) {
        const int64_t cs = c0 + 32 * sl;
        if (cs < Nc) prefetch_l2_bulk(Wb + slab_offset(cs >> 5) + r0 * 32, (uint32_t)(rn * 32 * sizeof(E)));
      }
    };
    prefetch_chunk(0);
    prefetch_chunk(1);
    for (int tc = 0; tc < nch; ++tc) {
      prefetch_chunk(tc + 2);
      float th[32], tl[32];
      float mx = 0.f;
      if constexpr (CX) {
        const int64_t j0 = (int64_t)tc * JC + 16 * q;
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const cdf v = (cval && j0 + e < k0) ? Wc[(j0 + e) * 32] : cdf{df{0.f, 0.f}, df{0.f, 0.f}};
          const df x0 = rpart ? v.im : v.re, x1 = rpart ? v.re : df_neg(v.im);
          th[2 * e] = x0.hi;
          tl[2 * e] = x0.lo;
          th[2 * e + 1] = x1.hi;
          tl[2 * e + 1] = x1.lo;
          mx = fmaxf(mx, fmaxf(fabsf(v.re.hi), fabsf(v.im.hi)));
        }
      } else {
        const int64_t j0 = (int64_t)tc * JC + 32 * q;
#pragma unroll
        for (int e = 0; e < 32; ++e) {
          const df v = (cval && j0 + e < k0) ? Wc[(j0 + e) * 32] : df{0.f, 0.f};
          th[e] = v.hi;
          tl[e] = v.lo;
          mx = fmaxf(mx, fabsf(v.hi));
        }
      }
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
      if constexpr (CX) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));  // both rows of the column
      float sigma, inv;
      ypow2(mx, sigma, inv);
      // The six slices with three instructions each (against seven for slice_step): the
      // first three digits come from th = hi / sigma 2^7 alone (each remainder th - a is
      // exact and, scaled by 2^8, again at most 2^7); then the low part joins the remainder
      // in one FMA, th + (lo / sigma) 2^31, whose rounding (half an ulp, at most 2^-48 sigma)
      // and the remainder dropped after the sixth digit (at most 2^-48 sigma) are the only
      // errors.  That sum is at most 256, so the fourth digit is too: still exact in BF16.
      // x / sigma first, then 2^7: inv alone can be 2^125, so inv 2^7 would overflow.
#pragma unroll
      for (int e = 0; e < 32; ++e) {
        th[e] = __fmul_rn(__fmul_rn(th[e], inv), 128.f);
        tl[e] = __fmul_rn(tl[e], inv);
      }
      const int rs = tc & (kYSigRing - 1);
      if (q == 0) sSig[rs * YM + ar] = sigma;
      __syncwarp();
      if (lane == 0) mbar_arrive(sig_full(rs));
      bool ok = true;
#pragma unroll 1
      for (int hf = 0; hf < 2; ++hf) {
        const int hidx = 2 * tc + hf, slot = hidx % kYAHalves;
        if (hidx >= kYAHalves && !mbar_wait(a_empty(slot), ((hidx / kYAHalves) - 1) & 1, abort_flag)) {
          ok = false;
          break;
        }
        if (hf == 1) {  // digits 4..6: the remainder of hi with the low part
#pragma unroll
          for (int e = 0; e < 32; ++e) th[e] = __fmaf_rn(tl[e], 0x1p31f, th[e]);
        }
        const uint32_t stA = sA + slot * kYAHalf;
#pragma unroll
        for (int s = 0; s < 3; ++s) {
#pragma unroll
          for (int g = 0; g < 4; ++g) {
            uint32_t w4[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              float x[2];
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                float& v = th[8 * g + 2 * e + h];
                x[h] = rintf(v);
                if (3 * hf + s < kYS - 1) v = __fmul_rn(__fsub_rn(v, x[h]), 256.f);
              }
              w4[e] = pack_bf16x2(x[0], x[1]);
            }
            const uint32_t addr = stA + s * kYATile + sw128_chunk((uint32_t)ar, (uint32_t)(4 * q + g));
            asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(w4[0]), "r"(w4[1]), "r"(w4[2]),
                         "r"(w4[3])
                         : "memory");
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(a_full(slot));
      }
      if (!ok) {
        fail();
        break;
      }
    }
  } else {
    // ---- epilogue: thread = trailing column (its tensor-memory lane), 16 of the 32 new
    // rows; after the chunks, Y, Bot = S^-1 Y and the new rows
    const int ew = warp - (2 + kYProdWarps);
    const int qd = warp & 3;                   // tensor-memory lane quarter of this warp
    const int hh = ew >> 2;                    // new rows [16 hh, 16 hh + 16)
    const int ar = 32 * qd + lane;             // operand row = tensor-memory lane
    const int cl = CX ? (ar >> 1) : ar;        // trailing column within the CTA
    const int rpart = CX ? (ar & 1) : 0;       // complex: 0 = Re, 1 = Im of the product
    const int64_t c = c0 + cl;
    const bool cval = c < Nc;
    lzf yacc[16];
#pragma unroll
    for (int n = 0; n < 16; ++n) yacc[n] = lzf{0.f, 0.f};
    bool dead = false;
    for (int tc = 0; tc < nch; ++tc) {
      const int u = tc & 1;
      const int rs = tc & (kYSigRing - 1);
      const bool ok = !dead && mbar_wait(acc_full(u), (tc >> 1) & 1, abort_flag) &&
                      mbar_wait(sig_full(rs), (tc / kYSigRing) & 1, abort_flag);
      if (!ok) {
        if (!dead) fail();
        dead = true;
        break;
      }
      tc_fence_after();
      lzf S[16];
      oz_group_sum<16>(
          [&](int d, uint32_t(&r)[16]) {
            tmem_ld16(tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)u * kYAccCols + (uint32_t)(32 * (d - 2) + 16 * hh),
                      r);
            tmem_ld_wait();
          },
          S);
      // the chunk's column scale is read before the accumulators are released: a producer
      // can overwrite its ring slot only after that release (four chunks later)
      const float sc = sSig[rs * YM + ar] * 0x1p-14f;
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acc_empty(u));
      const float* cs = z.Cs + (size_t)(b * z.n_chunks + tc) * YN + 16 * hh;
#pragma unroll
      for (int n = 0; n < 16; ++n) {
        const float f = sc * cs[n];  // a power of two
        lz_add(yacc[n], S[n].hi * f);
        yacc[n].lo = __fmaf_rn(S[n].lo, f, yacc[n].lo);
      }
    }
    // Y = U[x_new, m_c] - (C W0_T)[:, c], staged for Bot = S^-1 Y
    const int32_t* mrow = a.m + b * a.N;
    const int mc = cval ? mrow[c] : 0;
    const int et = threadIdx.x - 32 * (2 + kYProdWarps);  // 0 .. 255
    if constexpr (CX) {
      cdf* Ys = (cdf*)gbase;                   // [32 new rows][64 columns]
      cdf* Si = Ys + YN * YCOL;                // [32][32]
#pragma unroll
      for (int n = 0; n < 16; ++n) {
        const int i = 16 * hh + n;
        df y = df{0.f, 0.f};
        if (cval) {
          const int xi = a.x[b * a.ldx + k0 + i];
          const cdf d = ((const cdf*)a.Ust)[(int64_t)xi * a.N + mc];
          y = df_sub(rpart ? d.im : d.re, lz_get(yacc[n]));
        }
        ((df*)&Ys[i * YCOL + cl])[rpart] = y;
      }
      for (int e = et; e < YN * YN; e += 32 * kYEpiWarps) Si[e] = ((const cdf*)t.Sinv)[(size_t)b * YN * YN + e];
    } else {
      df* Ys = (df*)gbase;                     // [32 new rows][128 columns]
      df* Si = Ys + YN * YM;                   // [32][32]
#pragma unroll
      for (int n = 0; n < 16; ++n) {
        const int i = 16 * hh + n;
        df y = df{0.f, 0.f};
        if (cval) {
          const int xi = a.x[b * a.ldx + k0 + i];
          y = df_sub(((const df*)a.Ust)[(int64_t)xi * a.N + mc], lz_get(yacc[n]));
        }
        Ys[i * YM + cl] = y;
      }
      for (int e = et; e < YN * YN; e += 32 * kYEpiWarps) Si[e] = ((const df*)t.Sinv)[(size_t)b * YN * YN + e];
    }
    (void)dead;
  }
  if (warp >= 2) {
    // Bot = S^-1 Y and the new rows, on the producer and epilogue warps together (512
    // threads; the producers are done with their chunks).  Every one of them reaches
    // this barrier exactly once, also after a failed wait.
    named_sync(1, 32 * (kYProdWarps + kYEpiWarps));
    const int u = threadIdx.x - 64;  // 0 .. 511
    if constexpr (CX) {
      const cdf* Ys = (const cdf*)gbase;  // [32 new rows][64 columns]
      const cdf* Si = Ys + YN * YCOL;     // [32][32]
      const int cl = u & (YCOL - 1), rg = u >> 6;  // column, rows 4 rg .. 4 rg + 3
      const int64_t c = c0 + cl;
      if (c < Nc) {
        cdf* Wn = (cdf*)t.W + (size_t)b * state_stride(Nc) + (size_t)slab_offset(c >> 5) + (c & 31);
        // two rows at a time (four independent accumulation chains)
#pragma unroll 1
        for (int n0 = 0; n0 < 4; n0 += 2) {
          const int i0 = 4 * rg + n0;
          lzf re[2], im[2];
#pragma unroll
          for (int r = 0; r < 2; ++r) re[r] = im[r] = lzf{0.f, 0.f};
#pragma unroll 1
          for (int ip = 0; ip < YN; ++ip) {
            const cdf yv = Ys[ip * YCOL + cl];
#pragma unroll
            for (int r = 0; r < 2; ++r) {
              const cdf sv = Si[(i0 + r) * YN + ip];
              lz_mac(re[r], sv.re, yv.re);
              lz_mac(re[r], df_neg(sv.im), yv.im);
              lz_mac(im[r], sv.re, yv.im);
              lz_mac(im[r], sv.im, yv.re);
            }
          }
#pragma unroll
          for (int r = 0; r < 2; ++r) Wn[(k0 + i0 + r) * 32] = cdf{lz_get(re[r]), lz_get(im[r])};
        }
      }
    } else {
      const df* Ys = (const df*)gbase;  // [32 new rows][128 columns]
      const df* Si = Ys + YN * YM;      // [32][32]
      const int cl = u & (YM - 1), rg = u >> 7;  // column, rows 8 rg .. 8 rg + 7
      const int64_t c = c0 + cl;
      if (c < Nc) {
        df* Wn = (df*)t.W + (size_t)b * state_stride(Nc) + (size_t)slab_offset(c >> 5) + (c & 31);
        // four rows at a time: four independent accumulation chains share each Y entry
#pragma unroll 1
        for (int n0 = 0; n0 < 8; n0 += 4) {
          const int i0 = 8 * rg + n0;
          lzf acc[4];
#pragma unroll
          for (int r = 0; r < 4; ++r) acc[r] = lzf{0.f, 0.f};
#pragma unroll 2
          for (int ip = 0; ip < YN; ++ip) {
            const df yv = Ys[ip * YM + cl];
#pragma unroll
            for (int r = 0; r < 4; ++r) lz_mac(acc[r], Si[(i0 + r) * YN + ip], yv);
          }
#pragma unroll
          for (int r = 0; r < 4; ++r) Wn[(k0 + i0 + r) * 32] = lz_get(acc[r]);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem, kYTmemCols);
  }
}

}  // namespace

// Old rows per K chunk: 64 real or 32 complex (64 interleaved K elements).
static int64_t ozy_chunk_rows(bool cplx) { return cplx ? YKC / 2 : YKC; }

size_t ozy_bytes_per_sample(int64_t Nc, bool cplx) {
  const int64_t nch = (Nc + ozy_chunk_rows(cplx) - 1) / ozy_chunk_rows(cplx);
  return (size_t)nch * kYS * YN * YKC * 2 + (size_t)nch * YN * 4;
}

cudaError_t ozy_prepare(ffs_ctx* c, int64_t Bw, int64_t Nc) {
  const int64_t nch = (Nc + ozy_chunk_rows(c->cplx) - 1) / ozy_chunk_rows(c->cplx);
  const size_t need = (size_t)Bw * ozy_bytes_per_sample(Nc, c->cplx);
  if (need > c->ozy_bytes) {
    cudaFree(c->ozy_buf);
    c->ozy_buf = nullptr;
    c->ozy_bytes = 0;
    cudaError_t e = cudaMalloc(&c->ozy_buf, need);
    if (e != cudaSuccess) return e;
    c->ozy_bytes = need;
    c->ozy_key_B = -1;
  }
  if (c->ozy_key_B != Bw || c->ozy_key_Nc != Nc) {
    char* p = (char*)c->ozy_buf;
    c->ozy.C = (__nv_bfloat16*)p;
    c->ozy.Cs = (float*)(p + (size_t)Bw * nch * kYS * YN * YKC * 2);
    c->ozy.n_chunks = nch;
    // one box = the six slices of one chunk (6 x 32 rows of 64 BF16)
    cudaError_t e = encode_2d(&c->ozyC, c->ozy.C, false, YKC, (uint64_t)Bw * nch * kYS * YN, kYS * YN);
    if (e != cudaSuccess) return e;
    c->ozy_key_B = Bw;
    c->ozy_key_Nc = Nc;
  }
  return cudaSuccess;
}

template <bool CX>
static void ozy_launch(ffs_ctx* c, const StepArgs& a, const BlockedArgs& t, int64_t k0, int64_t k1, cudaStream_t s) {
  constexpr int64_t YCOL = CX ? YM / 2 : YM, JC = CX ? YKC / 2 : YKC;
  const OzYArgs z = c->ozy;
  const int64_t nch = (k0 + JC - 1) / JC;
  if (nch > 0) {
    const dim3 gc((unsigned)(YN / 8), (unsigned)nch, (unsigned)a.bw);
    ozc_slice_kernel<CX><<<gc, 256, 0, s>>>(a, t, z, k0, k1);
  }
  const dim3 gy((unsigned)((t.Nc - k1 + YCOL - 1) / YCOL), (unsigned)a.bw);
  ozy_kernel<CX><<<gy, kYThreads, kYSmem, s>>>(c->ozyC, a, t, z, k0, k1);
}

cudaError_t launch_oz_y(ffs_ctx* c, const StepArgs& a, const BlockedArgs& t, int64_t k0, int64_t k1, cudaStream_t s) {
  if (k1 >= t.Nc || a.bw <= 0) return cudaSuccess;
  if (a.cplx)
    ozy_launch<true>(c, a, t, k0, k1, s);
  else
    ozy_launch<false>(c, a, t, k0, k1, s);
  return cudaGetLastError();
}

cudaError_t configure_oz_y() {
  cudaError_t e = cudaFuncSetAttribute(ozy_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kYSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(ozy_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kYSmem);
  return e;
}

}  // namespace fermi
