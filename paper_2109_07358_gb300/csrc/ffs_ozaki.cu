// Trailing update of the old rows on tensor cores (opt-in, double-float state).
//
// At a panel end the old rows' trailing columns take Top = W0_T - W0_P Bot (the
// block-inverse identity of the blocked state, see ffs_tail.cu): per sample a
// (k0 x 32) by (32 x |T|) complex product in double-float precision.  Here the product
// runs on tcgen05 tensor cores through an error-free split of the operands into BF16
// slices (Ozaki, Ogita, Oishi & Rump, "Error-free transformations of matrix
// multiplication by using fast routines of matrix multiplication and its applications",
// Numer. Algorithms 59, 2012):
//   * each row r of A = [Re W0_P | Im W0_P] (64 reals) is scaled by a power of two
//     sigma_r >= its largest entry and cut into six 8-bit integer slices,
//     A_r / sigma_r = sum_i a_i 2^(-7 - 8(i-1)), |a_i| <= 128 (exact in BF16);
//   * each trailing column c of B, [Re Bot ; -Im Bot] for the real part of the product
//     and [Im Bot ; Re Bot] for the imaginary part, likewise with sigma_c;
//   * the slice products a_i b_j with i + j = d <= 8 accumulate in one FP32 tensor-memory
//     accumulator per d: every partial sum is an integer below 2^23, so the tensor-core
//     accumulation is exact;
//   * the epilogue adds the seven accumulators (oz_group_sum: FP32 for the three
//     smallest, lazy error-free sums for the rest), scales by sigma_r sigma_c 2^-14 and
//     subtracts from W0_T.
// A real state uses the same kernels with [values | 0] rows and the real part only.
// The dropped slice products (i + j > 8) and the group sums' rounding stay below 2^-46 of
// sigma_r sigma_c K, the order of the double-float rounding of the direct update.
//
// Kernels per panel end: slices of A (one warp per row), slices of B (one warp per
// column), the product (one CTA per sample and 128 old rows, looping over the trailing
// 32-column slabs; warp 0 issues TMA, warp 1 the MMAs, warps 2-17 the epilogue, four
// per 32-lane quarter of tensor memory, each for 8 of the 32 columns), and the operand of
// the next step from the updated column.
#include <cfloat>
#include <type_traits>

#include "ffs_arith.cuh"
#include "ffs_kernels.cuh"
#include "ffs_residual_tc.cuh"
#include "ffs_sm100.cuh"

namespace fermi {

using namespace sm100;

namespace {

constexpr int kSlices = 6;      // 8-bit slices per operand (48 bits)
constexpr int kDmax = 8;        // slice products a_i b_j kept: i + j <= kDmax
constexpr int kNumD = kDmax - 1;  // accumulator groups d = 2 .. kDmax
constexpr int MT = 128;         // old rows per CTA
constexpr int NT = 32;          // trailing columns per tile (one slab)
constexpr uint32_t kARows = MT, kBRows = NT;
constexpr uint32_t kATile = kARows * 128;     // one slice tile: 128 rows x 64 BF16
constexpr uint32_t kBTile = kBRows * 128;     // one slice tile: 32 rows x 64 BF16
constexpr uint32_t kABytes = kSlices * kATile;                 // 96 KB
constexpr uint32_t kBStage = kSlices * 2 * kBTile;             // 48 KB (six slices, re and im columns)
constexpr int kBStages = 1;
// Epilogue staging of the product, one 32-row block per TMEM lane quarter, rows padded
// by 16 bytes against bank conflicts: the quarter's warps then update its rows of W0_T
// with lanes over columns (coalesced 512-byte rows; measured faster than each thread
// updating its own row directly, which leaves two B stages room in shared memory).
constexpr uint32_t kPRow = NT * 16 + 16;
constexpr int kEpiWarps = 16;
constexpr int kEpiCols = NT / (kEpiWarps / 4);  // columns (and staged rows) per epilogue warp
constexpr int kThreads = 32 * (2 + kEpiWarps);
constexpr uint32_t kPStage = 4 * 32 * kPRow;
constexpr uint32_t kSmem = kABytes + kBStages * kBStage + kPStage + 1024 + 256;
constexpr uint32_t kTmemCols = 512;             // 2 x 7 accumulators of 32 columns = 448
constexpr uint32_t kIdesc = idesc_bf16(MT, NT);

// The six slices of x (|x| < 1): x 2^7 = a_1 + 2^-8 (a_2 + 2^-8 (a_3 + ...)), each a_i an
// integer in [-128, 128].  Every step is exact in double-float arithmetic.
__device__ __forceinline__ void df_slices(df x, float (&s)[kSlices]) {
  float th = x.hi * 128.f, tl = x.lo * 128.f;
#pragma unroll
  for (int i = 0; i < kSlices; ++i) {
    const float a = rintf(th);
    const df r = two_sum(th - a, tl);  // th - a is exact (|th| <= 2^7 + 1)
    s[i] = a;
    th = r.hi * 256.f;
    tl = r.lo * 256.f;
  }
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Power-of-two scale sigma >= max, as (sigma, 1/sigma); 1 for an all-zero vector.  A
// subnormal max (localised orbitals leave rows of order 1e-40) takes sigma = 2^-125, so
// that 1/sigma stays finite; v / sigma >= 2^-24 is then still exact in the 48 slice bits.
__device__ __forceinline__ void pow2_scale(float mx, float& sigma, float& inv) {
  if (!(mx > 0.f)) {
    sigma = inv = 1.f;
    return;
  }
  int e;
  frexpf(mx, &e);  // mx = m 2^e, m in [0.5, 1): mx < 2^e
  e = min(max(e, -125), 127);  // at 2^127: |v| / sigma < 2, first slice <= 256 (exact in BF16)
  sigma = ldexpf(1.f, e);
  inv = ldexpf(1.f, -e);
}

__device__ __forceinline__ df df_scale(df v, float p2) { return {v.hi * p2, v.lo * p2}; }  // exact (power of 2)

// A slices: rows r < k0 of W0_P.  Layout [b][slice][KP][64] BF16, sigma_r in As[b][KP];
// a complex row is [Re | Im], a real one [values | 0].
template <bool CX>
__global__ void __launch_bounds__(256) oz_slice_a_kernel(StepArgs a, BlockedArgs t, OzArgs z, int64_t k0,
                                                          int64_t k1) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t b = blockIdx.y;
  const int64_t r = (int64_t)blockIdx.x * 8 + warp;
  if (r >= k0) return;
  if (a.nlen && a.nlen[b] <= k1) return;
  df wre, wim = df{0.f, 0.f};
  if constexpr (CX) {
    const cdf w = ((const cdf*)t.W0P)[((size_t)b * t.Nc + r) * 32 + lane];
    wre = w.re;
    wim = w.im;
  } else {
    wre = ((const df*)t.W0P)[((size_t)b * t.Nc + r) * 32 + lane];
  }
  float sigma, inv;
  pow2_scale(warp_max(fmaxf(fabsf(wre.hi), fabsf(wim.hi))), sigma, inv);
  float sr[kSlices], si[kSlices];
  df_slices(df_scale(wre, inv), sr);
  df_slices(df_scale(wim, inv), si);
  __nv_bfloat16* A = z.A + (size_t)b * kSlices * z.KP * 64;
#pragma unroll
  for (int i = 0; i < kSlices; ++i) {
    __nv_bfloat16* row = A + ((size_t)i * z.KP + r) * 64;
    row[lane] = __float2bfloat16_rn(sr[i]);
    row[32 + lane] = __float2bfloat16_rn(si[i]);
  }
  if (lane == 0) z.As[(size_t)b * z.KP + r] = sigma;
}

// B slices: trailing columns c of Bot (rows k0 .. k0+31 of the state).  Layout
// [b][slice][re/im][TP][64] BF16 (row c), sigma_c in Bs[b][TP]; a real column is
// [values ; 0] in the first plane only.
template <bool CX>
__global__ void __launch_bounds__(256) oz_slice_b_kernel(StepArgs a, BlockedArgs t, OzArgs z, int64_t k0,
                                                          int64_t k1) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;  // lane = row of the panel
  const int64_t b = blockIdx.y;
  const int64_t c = k1 + (int64_t)blockIdx.x * 8 + warp;
  if (c >= t.Nc) return;
  if (a.nlen && a.nlen[b] <= k1) return;
  const int64_t Nc = t.Nc;
  const size_t idx = (size_t)b * state_stride(Nc) + sidx(k0 + lane, c);
  df vre, vim = df{0.f, 0.f};
  if constexpr (CX) {
    const cdf v = ((const cdf*)t.W)[idx];
    vre = v.re;
    vim = v.im;
  } else {
    vre = ((const df*)t.W)[idx];
  }
  float sigma, inv;
  pow2_scale(warp_max(fmaxf(fabsf(vre.hi), fabsf(vim.hi))), sigma, inv);
  float sr[kSlices], si[kSlices];
  df_slices(df_scale(vre, inv), sr);
  df_slices(df_scale(vim, inv), si);
  __nv_bfloat16* B = z.B + (size_t)b * kSlices * 2 * z.TP * 64;
#pragma unroll
  for (int j = 0; j < kSlices; ++j) {
    __nv_bfloat16* re_row = B + (((size_t)j * 2 + 0) * z.TP + c) * 64;  // [Re ; -Im]
    re_row[lane] = __float2bfloat16_rn(sr[j]);
    re_row[32 + lane] = __float2bfloat16_rn(-si[j]);
    if constexpr (CX) {
      __nv_bfloat16* im_row = B + (((size_t)j * 2 + 1) * z.TP + c) * 64;  // [Im ; Re]
      im_row[lane] = __float2bfloat16_rn(si[j]);
      im_row[32 + lane] = __float2bfloat16_rn(sr[j]);
    }
  }
  if (lane == 0) z.Bs[(size_t)b * z.TP + c] = sigma;
}

// Top = W0_T - W0_P Bot for 128 old rows of one sample, every trailing slab.
template <bool CX>
__global__ void __launch_bounds__(kThreads, 1) oz_top_kernel(const __grid_constant__ CUtensorMap tmA,
                                                        const __grid_constant__ CUtensorMap tmB, StepArgs a,
                                                        BlockedArgs t, OzArgs z, int64_t k0, int64_t k1) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t b = blockIdx.y;
  const int64_t mt = blockIdx.x;
  if (a.nlen && a.nlen[b] <= k1) return;  // uniform over the CTA
  using E = typename std::conditional<CX, cdf, df>::type;  // the state's element type
  const int64_t Nc = t.Nc;
  const int n_tiles = (int)((Nc - k1 + NT - 1) / NT);
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t sbase = (raw + 1023u) & ~1023u;
  uint8_t* gbase = smem_raw + (sbase - raw);
  uint8_t* pstage = gbase + kABytes + kBStages * kBStage;
  uint64_t* bars = (uint64_t*)(pstage + kPStage);
  const uint32_t bar0 = smem_u32(bars);
  const uint32_t a_full = bar0;
  auto b_full = [&](int s) { return bar0 + 8u * (1 + s); };
  auto b_empty = [&](int s) { return bar0 + 8u * (1 + kBStages + s); };
  const uint32_t acc_full = bar0 + 8u * (1 + 2 * kBStages);
  const uint32_t acc_empty = acc_full + 8u;
  uint32_t* tmem_slot = (uint32_t*)(bars + 3 + 2 * kBStages);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  const uint32_t sA = sbase, sB = sbase + kABytes;

  if (threadIdx.x == 0) {
    mbar_init(a_full, 1);
    for (int s = 0; s < kBStages; ++s) {
      mbar_init(b_full(s), 1);
      mbar_init(b_empty(s), 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, kEpiWarps);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 1) {
    tmem_alloc(smem_u32(tmem_slot), kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer: the A slices once, then the B slices of every slab
    prefetch_tmap(&tmA);
    prefetch_tmap(&tmB);
    mbar_arrive_expect_tx(a_full, kABytes);
    for (int i = 0; i < kSlices; ++i)
      tma_load_2d(sA + i * kATile, &tmA, a_full, 0, (int32_t)((b * kSlices + i) * z.KP + mt * MT));
    const E* Wb = (const E*)t.W + (size_t)b * state_stride(Nc);
    const int64_t r_rows = min((int64_t)MT, k0 - mt * MT);
    auto prefetch_slab = [&](int ntp) {  // the epilogue's old rows of slab ntp into L2
      if (ntp < n_tiles && r_rows > 0)
        prefetch_l2_bulk(Wb + slab_offset(((k1 >> 5) + ntp)) + mt * MT * 32, (uint32_t)(r_rows * 32 * sizeof(E)));
    };
    prefetch_slab(0);
    prefetch_slab(1);
    int issued = 0;
    for (int nt = 0; nt < n_tiles; ++nt) {
      prefetch_slab(nt + 2);
      const int s = nt % kBStages;
      if (nt >= kBStages && !mbar_wait(b_empty(s), ((nt / kBStages) - 1) & 1, abort_flag)) {
        *abort_flag = 1;
        set_status(a.status, FFS_E_TIMEOUT);
        break;
      }
      const int32_t c0 = (int32_t)(k1 + (int64_t)nt * NT);
      const uint32_t st = sB + s * kBStage;
      mbar_arrive_expect_tx(b_full(s), CX ? kBStage : kBStage / 2);
      for (int j = 0; j < kSlices; ++j)
        for (int ri = 0; ri < (CX ? 2 : 1); ++ri)
          tma_load_2d(st + (j * 2 + ri) * kBTile, &tmB, b_full(s), 0,
                      (int32_t)(((b * kSlices + j) * 2 + ri) * z.TP + c0));
      ++issued;
    }
    // never leave with copies in flight
    mbar_wait(a_full, 0, abort_flag);
    for (int nt = (issued > kBStages ? issued - kBStages : 0); nt < issued; ++nt)
      mbar_wait(b_full(nt % kBStages), (nt / kBStages) & 1, abort_flag);
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer: accumulator d of the real part at columns 32 (d-2), of the
    // imaginary part at 32 (kNumD + d - 2)
    bool ok = mbar_wait(a_full, 0, abort_flag);
    if (!ok) {
      *abort_flag = 1;
      set_status(a.status, FFS_E_TIMEOUT);
    }
    for (int nt = 0; nt < n_tiles && ok; ++nt) {
      const int s = nt % kBStages;
      if (!mbar_wait(b_full(s), (nt / kBStages) & 1, abort_flag) ||
          (nt >= 1 && !mbar_wait(acc_empty, (nt - 1) & 1, abort_flag))) {
        *abort_flag = 1;
        set_status(a.status, FFS_E_TIMEOUT);
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t st = sB + s * kBStage;
#pragma unroll 1  // unrolled, the 42 slice pairs' descriptors spill in the real kernel
      for (int d = 2; d <= kDmax; ++d) {
        bool first = true;
        for (int i = 1; i <= kSlices; ++i) {
          const int j = d - i;
          if (j < 1 || j > kSlices) continue;
          const uint32_t ta = sA + (i - 1) * kATile;
          const uint32_t tre = st + ((j - 1) * 2 + 0) * kBTile, tim = st + ((j - 1) * 2 + 1) * kBTile;
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint32_t koff = kk * 32;
            const uint32_t acc = (first && kk == 0) ? 0u : 1u;
            const uint64_t da = smem_desc_sw128(ta + koff);
            mma_bf16(tmem + (uint32_t)(32 * (d - 2)), da, smem_desc_sw128(tre + koff), kIdesc, acc);
            if (CX) mma_bf16(tmem + (uint32_t)(32 * (kNumD + d - 2)), da, smem_desc_sw128(tim + koff), kIdesc, acc);
          }
          first = false;
        }
      }
      mma_commit(b_empty(s));
      mma_commit(acc_full);
    }
  } else if (warp >= 2) {
    // ---- epilogue: thread = old row (its TMEM lane) and kEpiCols columns while reading
    // the accumulators; then lanes over columns while updating W0_T, kEpiCols rows per warp
    const int q = warp & 3;             // TMEM lane quarter
    const int h = (warp - 2) >> 2;      // column group of the slab
    const uint32_t quarter_bar = 1 + q; // the warps of a quarter
    const uint32_t quarter_threads = 32 * (kEpiWarps / 4);
    const int64_t j = mt * MT + 32 * q + lane;
    const bool live_row = j < k0;
    const float sr = live_row ? z.As[(size_t)b * z.KP + j] : 1.f;
    uint8_t* Pq = pstage + (size_t)q * 32 * kPRow;  // the quarter's 32 rows
    // All warps of a quarter pass the two quarter barriers of every slab even after a wait
    // has failed (they then skip the work), so that none can be left at a barrier.
    bool dead = false;
    for (int nt = 0; nt < n_tiles; ++nt) {
      const bool ok = !dead && mbar_wait(acc_full, nt & 1, abort_flag);
      if (!ok && !dead) {
        set_status(a.status, FFS_E_TIMEOUT);
        *abort_flag = 1;
        dead = true;
      }
      const int64_t c0 = k1 + (int64_t)nt * NT;
      if (ok) tc_fence_after();
      for (int part = 0; part < (CX ? 2 : 1) && ok; ++part) {  // real, then imaginary part of the product
        lzf S[kEpiCols];
        oz_group_sum<kEpiCols>(
            [&](int d, uint32_t(&r)[kEpiCols]) {
              tmem_ld8(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * (part * kNumD + d - 2) + kEpiCols * h), r);
              tmem_ld_wait();
            },
            S);
#pragma unroll
        for (int n = 0; n < kEpiCols; ++n) {
          const int64_t c = c0 + kEpiCols * h + n;
          const float scale = (c < Nc) ? sr * z.Bs[(size_t)b * z.TP + c] * 0x1p-14f : 0.f;
          *(df*)(Pq + lane * kPRow + (kEpiCols * h + n) * 16 + part * 8) = df_scale(lz_get(S[n]), scale);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0 && ok) mbar_arrive(acc_empty);  // the accumulators may be overwritten now
      named_sync(quarter_bar, quarter_threads);     // all the quarter's columns are staged
      const size_t slab = (size_t)b * state_stride(Nc) + (size_t)slab_offset(c0 >> 5);
      const bool col_ok = ok && c0 + lane < Nc;
      // all the warp's rows are loaded before any is stored, so that their loads overlap
      E wv[kEpiCols];
      E* Wc = (E*)t.W + slab;
#pragma unroll
      for (int n = 0; n < kEpiCols; ++n) {
        const int64_t jr = mt * MT + 32 * q + kEpiCols * h + n;
        if (jr < k0 && col_ok) wv[n] = Wc[jr * 32 + lane];
      }
#pragma unroll
      for (int n = 0; n < kEpiCols; ++n) {
        const int rr = kEpiCols * h + n;
        const int64_t jr = mt * MT + 32 * q + rr;
        if (jr < k0 && col_ok) {
          const cdf p = *(const cdf*)(Pq + rr * kPRow + lane * 16);
          if constexpr (CX) {
            cdf w = wv[n];
            w.re = df_sub(w.re, p.re);
            w.im = df_sub(w.im, p.im);
            Wc[jr * 32 + lane] = w;
          } else {
            Wc[jr * 32 + lane] = df_sub(wv[n], p.re);
          }
        }
      }
      named_sync(quarter_bar, quarter_threads);  // before the next slab overwrites the staging rows
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

// ------------------------------------------------------------------ real states: packed pairs
// For a real state the panel dimension K is 32, half of a 128-byte operand row.  Instead of
// padding each slice row with zeros, two slices share one row: A rows hold the pairs
// [a_p | a_p+1] (p = 1, 3, 5), B rows the shifted pairs [b_q | b_q-1] (q = 1 .. 7, b_0 =
// b_7 = 0), so that one K = 64 product [a_p | a_p+1] . [b_q | b_q-1] = a_p b_q + a_p+1 b_q-1
// adds two slice products of the same weight d = p + q.  The 26 products with d <= 8 take 15
// packed products (60 MMAs per 128 x 32 tile instead of 104); each accumulator still sums 64
// products below 2^14, so it stays exact.  The accumulators are double-buffered (2 x 7
// groups x 32 columns), so a slab's epilogue overlaps the next slab's products.
constexpr int kPairA = 3, kPairB = 7;
constexpr uint32_t kRABytes = kPairA * kATile;       // 48 KB
constexpr uint32_t kRBStage = kPairB * kBTile;       // 28 KB: the seven pair tiles of a slab
constexpr int kRBStages = 3;
constexpr uint32_t kRPRow = NT * 8 + 16;             // staged row: 32 double-floats + pad
constexpr uint32_t kRPStage = 4 * 32 * kRPRow;
constexpr uint32_t kRSmem = kRABytes + kRBStages * kRBStage + kRPStage + 1024 + 256;
constexpr uint32_t kRAccCols = 256;                  // one accumulator set (7 x 32 columns used)

// A pairs: row r < k0 of W0_P; layout [b][pair][KP][64] BF16, sigma_r in As[b][KP].
__global__ void __launch_bounds__(256) oz_pair_a_kernel(StepArgs a, BlockedArgs t, OzArgs z, int64_t k0,
                                                        int64_t k1) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;  // lane = panel column
  const int64_t b = blockIdx.y;
  const int64_t r = (int64_t)blockIdx.x * 8 + warp;
  if (r >= k0) return;
  if (a.nlen && a.nlen[b] <= k1) return;
  const df w = ((const df*)t.W0P)[((size_t)b * t.Nc + r) * 32 + lane];
  float sigma, inv;
  pow2_scale(warp_max(fabsf(w.hi)), sigma, inv);
  float sl[kSlices];
  df_slices(df_scale(w, inv), sl);
  __nv_bfloat16* A = z.A + (size_t)b * kPairA * z.KP * 64;
#pragma unroll
  for (int p = 0; p < kPairA; ++p) {
    __nv_bfloat16* row = A + ((size_t)p * z.KP + r) * 64;
    row[lane] = __float2bfloat16_rn(sl[2 * p]);
    row[32 + lane] = __float2bfloat16_rn(sl[2 * p + 1]);
  }
  if (lane == 0) z.As[(size_t)b * z.KP + r] = sigma;
}

// B shifted pairs: trailing column c of Bot (state rows k0 .. k0+31); layout
// [b][slab][pair][32 columns][64] BF16 (slab = (c - k1) / 32), sigma_c in Bs[b][TP].
__global__ void __launch_bounds__(256) oz_pair_b_kernel(StepArgs a, BlockedArgs t, OzArgs z, int64_t k0,
                                                        int64_t k1) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;  // lane = panel row
  const int64_t b = blockIdx.y;
  const int64_t c = k1 + (int64_t)blockIdx.x * 8 + warp;
  if (c >= t.Nc) return;
  if (a.nlen && a.nlen[b] <= k1) return;
  const df v = ((const df*)t.W)[(size_t)b * state_stride(t.Nc) + sidx(k0 + lane, c)];
  float sigma, inv;
  pow2_scale(warp_max(fabsf(v.hi)), sigma, inv);
  float sl[kSlices];
  df_slices(df_scale(v, inv), sl);
  const int64_t nt = (c - k1) >> 5, rr = (c - k1) & 31;
  __nv_bfloat16* B = z.B + ((size_t)b * (z.TP / NT) + nt) * kPairB * NT * 64;
#pragma unroll
  for (int q = 1; q <= kPairB; ++q) {
    __nv_bfloat16* row = B + ((size_t)(q - 1) * NT + rr) * 64;
    row[lane] = __float2bfloat16_rn(q <= kSlices ? sl[q - 1] : 0.f);
    row[32 + lane] = __float2bfloat16_rn(q >= 2 ? sl[q - 2] : 0.f);
  }
  if (lane == 0) z.Bs[(size_t)b * z.TP + c] = sigma;
}

// Top = W0_T - W0_P Bot for 128 old rows of one sample (real state), every trailing slab.
__global__ void __launch_bounds__(kThreads, 1) oz_top_real_kernel(const __grid_constant__ CUtensorMap tmA,
                                                                  const __grid_constant__ CUtensorMap tmB, StepArgs a,
                                                                  BlockedArgs t, OzArgs z, int64_t k0, int64_t k1) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t b = blockIdx.y;
  const int64_t mt = blockIdx.x;
  if (a.nlen && a.nlen[b] <= k1) return;  // uniform over the CTA
  const int64_t Nc = t.Nc;
  const int n_tiles = (int)((Nc - k1 + NT - 1) / NT);
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t sbase = (raw + 1023u) & ~1023u;
  uint8_t* gbase = smem_raw + (sbase - raw);
  uint8_t* pstage = gbase + kRABytes + kRBStages * kRBStage;
  uint64_t* bars = (uint64_t*)(pstage + kRPStage);
  const uint32_t bar0 = smem_u32(bars);
  const uint32_t a_full = bar0;
  auto b_full = [&](int s) { return bar0 + 8u * (1 + s); };
  auto b_empty = [&](int s) { return bar0 + 8u * (1 + kRBStages + s); };
  auto acc_full = [&](int u) { return bar0 + 8u * (1 + 2 * kRBStages + u); };
  auto acc_empty = [&](int u) { return bar0 + 8u * (3 + 2 * kRBStages + u); };
  const uint32_t mma_done = bar0 + 8u * (5 + 2 * kRBStages);
  uint32_t* tmem_slot = (uint32_t*)(bars + 6 + 2 * kRBStages);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  const uint32_t sA = sbase, sB = sbase + kRABytes;

  if (threadIdx.x == 0) {
    mbar_init(a_full, 1);
    for (int s = 0; s < kRBStages; ++s) {
      mbar_init(b_full(s), 1);
      mbar_init(b_empty(s), 1);
    }
    for (int u = 0; u < 2; ++u) {
      mbar_init(acc_full(u), 1);
      mbar_init(acc_empty(u), kEpiWarps);
    }
    mbar_init(mma_done, 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 1) {
    tmem_alloc(smem_u32(tmem_slot), kTmemCols);
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

  if (warp == 0 && lane == 0) {
    // ---- TMA: the A pairs once, then the seven B pair tiles of every slab (one box)
    prefetch_tmap(&tmA);
    prefetch_tmap(&tmB);
    mbar_arrive_expect_tx(a_full, kRABytes);
    for (int p = 0; p < kPairA; ++p)
      tma_load_2d(sA + p * kATile, &tmA, a_full, 0, (int32_t)((b * kPairA + p) * z.KP + mt * MT));
    const int64_t nslab = z.TP / NT;
    const df* Wb = (const df*)t.W + (size_t)b * state_stride(Nc);
    const int64_t r_rows = min((int64_t)MT, k0 - mt * MT);
    for (int nt = 0; nt < 2 && nt < n_tiles; ++nt)
      prefetch_l2_bulk(Wb + slab_offset(((k1 >> 5) + nt)) + mt * MT * 32, (uint32_t)(r_rows * 32 * sizeof(df)));
    int issued = 0;
    for (int nt = 0; nt < n_tiles; ++nt) {
      const int s = nt % kRBStages;
      if (nt >= kRBStages && !mbar_wait(b_empty(s), ((nt / kRBStages) - 1) & 1, abort_flag)) {
        fail();
        break;
      }
      mbar_arrive_expect_tx(b_full(s), kRBStage);
      tma_load_2d(sB + s * kRBStage, &tmB, b_full(s), 0, (int32_t)((b * nslab + nt) * kPairB * NT));
      ++issued;
      // the epilogue's old rows of slab nt + 2 (128 rows x 256 bytes, contiguous) into L2
      if (nt + 2 < n_tiles && r_rows > 0)
        prefetch_l2_bulk(Wb + slab_offset(((k1 >> 5) + nt + 2)) + mt * MT * 32, (uint32_t)(r_rows * 32 * sizeof(df)));
    }
    mbar_drain(a_full, 0, kSpinLimit);
    for (int nt = (issued > kRBStages ? issued - kRBStages : 0); nt < issued; ++nt)
      mbar_drain(b_full(nt % kRBStages), (nt / kRBStages) & 1, kSpinLimit);
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer: group d of accumulator set u at columns u * 256 + 32 (d - 2)
    bool ok = mbar_wait(a_full, 0, abort_flag);
    if (!ok) fail();
    for (int nt = 0; nt < n_tiles && ok; ++nt) {
      const int s = nt % kRBStages, u = nt & 1;
      if ((nt >= 2 && !mbar_wait(acc_empty(u), ((nt >> 1) - 1) & 1, abort_flag)) ||
          !mbar_wait(b_full(s), (nt / kRBStages) & 1, abort_flag)) {
        fail();
        break;
      }
      tc_fence_after();
      const uint32_t stB = sB + s * kRBStage, accb = tmem + (uint32_t)u * kRAccCols;
#pragma unroll 1
      for (int p = 1; p <= 5; p += 2) {
#pragma unroll 1
        for (int q = 1; q <= kPairB && p + q <= kDmax; ++q) {
          const int d = p + q;
          const uint32_t ta = sA + ((p - 1) / 2) * kATile, tb = stB + (q - 1) * kBTile;
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            mma_bf16(accb + (uint32_t)(32 * (d - 2)), smem_desc_sw128(ta + kk * 32), smem_desc_sw128(tb + kk * 32),
                     kIdesc, (p > 1 || kk > 0) ? 1u : 0u);
        }
      }
      mma_commit(b_empty(s));
      mma_commit(acc_full(u));
    }
    mma_commit(mma_done);
    mbar_drain(mma_done, 0, kSpinLimit);
  } else if (warp >= 2) {
    // ---- epilogue: thread = old row (its TMEM lane) and 8 columns while reading the
    // accumulators, then lanes over columns while updating W0_T (8 rows per warp)
    const int q = warp & 3;
    const int h = (warp - 2) >> 2;
    const uint32_t quarter_bar = 1 + q;
    const uint32_t quarter_threads = 32 * (kEpiWarps / 4);
    const int64_t j = mt * MT + 32 * q + lane;
    const float sr = j < k0 ? z.As[(size_t)b * z.KP + j] : 1.f;
    uint8_t* Pq = pstage + (size_t)q * 32 * kRPRow;
    bool dead = false;
    for (int nt = 0; nt < n_tiles; ++nt) {
      const int u = nt & 1;
      const int64_t c0 = k1 + (int64_t)nt * NT;
      // this warp's rows of the slab (lanes over columns) are loaded before the wait for the
      // accumulators: they do not depend on the products, so their latency overlaps the MMAs
      // and the group sums
      df* Wc = (df*)t.W + (size_t)b * state_stride(Nc) + (size_t)slab_offset(c0 >> 5);
      df wv[kEpiCols];
#pragma unroll
      for (int n = 0; n < kEpiCols; ++n) {
        const int64_t jr = mt * MT + 32 * q + kEpiCols * h + n;
        wv[n] = (jr < k0 && c0 + lane < Nc) ? Wc[jr * 32 + lane] : df{0.f, 0.f};
      }
      const bool ok = !dead && mbar_wait(acc_full(u), (nt >> 1) & 1, abort_flag);
      if (!ok && !dead) {
        fail();
        dead = true;
      }
      if (ok) {
        tc_fence_after();
        lzf S[kEpiCols];
        oz_group_sum<kEpiCols>(
            [&](int d, uint32_t(&r)[kEpiCols]) {
              tmem_ld8(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)u * kRAccCols + (uint32_t)(32 * (d - 2) + kEpiCols * h),
                       r);
              tmem_ld_wait();
            },
            S);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(acc_empty(u));  // the accumulators may be overwritten now
#pragma unroll
        for (int n = 0; n < kEpiCols; ++n) {
          const int64_t c = c0 + kEpiCols * h + n;
          const float scale = (c < Nc) ? sr * z.Bs[(size_t)b * z.TP + c] * 0x1p-14f : 0.f;
          *(df*)(Pq + lane * kRPRow + (kEpiCols * h + n) * 8) = df_scale(lz_get(S[n]), scale);
        }
      }
      named_sync(quarter_bar, quarter_threads);  // all the quarter's columns are staged
      const bool col_ok = ok && c0 + lane < Nc;
#pragma unroll
      for (int n = 0; n < kEpiCols; ++n) {
        const int rr = kEpiCols * h + n;
        const int64_t jr = mt * MT + 32 * q + rr;
        if (jr < k0 && col_ok) Wc[jr * 32 + lane] = df_sub(wv[n], *(const df*)(Pq + rr * kRPRow + lane * 8));
      }
      named_sync(quarter_bar, quarter_threads);  // before the next slab overwrites the staging rows
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

}  // namespace

size_t oz_bytes_per_sample(int64_t Nc) {
  const int64_t KP = (Nc + MT - 1) / MT * MT, TP = (Nc + NT - 1) / NT * NT;
  return (size_t)kSlices * KP * 64 * 2 + (size_t)KP * 4 + (size_t)kSlices * 2 * TP * 64 * 2 + (size_t)TP * 4;
}

cudaError_t oz_prepare(ffs_ctx* c, int64_t Bw, int64_t Nc) {
  const int64_t KP = (Nc + MT - 1) / MT * MT, TP = (Nc + NT - 1) / NT * NT;
  const size_t need = (size_t)Bw * oz_bytes_per_sample(Nc);
  if (need > c->oz_bytes) {
    cudaFree(c->oz_buf);
    c->oz_buf = nullptr;
    c->oz_bytes = 0;
    cudaError_t e = cudaMalloc(&c->oz_buf, need);
    if (e != cudaSuccess) return e;
    c->oz_bytes = need;
    c->oz_key_B = -1;
  }
  if (c->oz_key_B != Bw || c->oz_key_Nc != Nc) {
    char* p = (char*)c->oz_buf;
    c->oz.A = (__nv_bfloat16*)p;
    p += (size_t)Bw * kSlices * KP * 64 * 2;
    c->oz.B = (__nv_bfloat16*)p;
    p += (size_t)Bw * kSlices * 2 * TP * 64 * 2;
    c->oz.As = (float*)p;
    p += (size_t)Bw * KP * 4;
    c->oz.Bs = (float*)p;
    c->oz.KP = KP;
    c->oz.TP = TP;
    cudaError_t e = encode_2d(&c->ozA, c->oz.A, false, 64, (uint64_t)Bw * kSlices * KP, kARows);
    if (e == cudaSuccess) e = encode_2d(&c->ozB, c->oz.B, false, 64, (uint64_t)Bw * kSlices * 2 * TP, kBRows);
    // real states: the packed pair layouts in the same buffers (A pairs [b][3][KP], one
    // box of 128 rows; B shifted pairs [b][slab][7][32], one box = the seven tiles of a slab)
    if (e == cudaSuccess) e = encode_2d(&c->ozA2, c->oz.A, false, 64, (uint64_t)Bw * kPairA * KP, kARows);
    if (e == cudaSuccess) e = encode_2d(&c->ozB2, c->oz.B, false, 64, (uint64_t)Bw * (TP / NT) * kPairB * NT, kPairB * NT);
    if (e != cudaSuccess) return e;
    c->oz_key_B = Bw;
    c->oz_key_Nc = Nc;
  }
  return cudaSuccess;
}

cudaError_t launch_oz_top(ffs_ctx* c, const StepArgs& a, const BlockedArgs& t, int64_t k0, int64_t k1, int op,
                          cudaStream_t s) {
  if (k1 >= t.Nc || a.bw <= 0) return cudaSuccess;
  const OzArgs z = c->oz;
  if (k0 > 0) {
    const dim3 ga((unsigned)((k0 + 7) / 8), (unsigned)a.bw), gb((unsigned)((t.Nc - k1 + 7) / 8), (unsigned)a.bw);
    const dim3 gt((unsigned)((k0 + MT - 1) / MT), (unsigned)a.bw);
    if (a.cplx) {
      oz_slice_a_kernel<true><<<ga, 256, 0, s>>>(a, t, z, k0, k1);
      oz_slice_b_kernel<true><<<gb, 256, 0, s>>>(a, t, z, k0, k1);
      oz_top_kernel<true><<<gt, kThreads, kSmem, s>>>(c->ozA, c->ozB, a, t, z, k0, k1);
    } else {
      oz_pair_a_kernel<<<ga, 256, 0, s>>>(a, t, z, k0, k1);
      oz_pair_b_kernel<<<gb, 256, 0, s>>>(a, t, z, k0, k1);
      oz_top_real_kernel<<<gt, kThreads, kRSmem, s>>>(c->ozA2, c->ozB2, a, t, z, k0, k1);
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && op != kOpNone && k1 < a.n_steps) e = launch_column_operand(a, t, k1, kStateDF64, op, s);
  return e;
}

cudaError_t configure_oz() {
  cudaError_t e = cudaFuncSetAttribute(oz_top_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(oz_top_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(oz_top_real_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRSmem);
  return e;
}

}  // namespace fermi
