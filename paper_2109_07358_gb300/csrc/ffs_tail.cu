// Blocked per-sample elimination state of the batched form.
//
// The state of a sample after k steps is the Gauss-Jordan form
//   W = A^-1 U[x_<k, m_>=k],  A = U[x_<k, m_<k]
// (Section S-1 carries the elimination of every new base row in the full N-dim space;
// here the base rows are also reduced against each other, so that the next normal
// vector is simply h_{k+1} = (-W[:, k+1] ; 1) in the sample's column order).
//
// Updating all remaining columns at every step would stream the whole state once per
// step.  The columns are instead processed in panels P = [k0, k1) of 32:
//   per step (tail_step_kernel, one warp per sample): draw x_k; reduce the new row
//     u = U[x_k, m] against the state on the panel columns [k, k1) only (lane = column);
//     pivot s_k = the reduced value at column k (the Schur residual of x_k); rank-1
//     update of the panel columns; the first step of a panel keeps a copy W0_P of the
//     old rows' panel columns.
//   per panel, for the trailing columns T = [k1, Nc), by the block-inverse identity:
//     S   = U[x_new, m_P] - U[x_new, m_<k0] W0_P            (panel Schur complement)
//     Y   = U[x_new, m_T] - U[x_new, m_<k0] W0_T
//     Bot = S^-1 Y                                          (new rows)
//     Top = W0_T - W0_P Bot                                 (old rows)
//   tail_panel_s_kernel forms S and inverts it (Gauss-Jordan, pivots in draw order, as
//   the per-step updates do); tail_panel_kernel applies the two GEMM-shaped updates.
//   In exact arithmetic this is the same state the per-step updates would produce.
// Only the first Nc = n_steps columns are kept (marginal sampling needs no more).
//
// Layout of a sample's state: slabs of 32 columns, each holding only the rows it can ever
// hold (slab_offset and sidx in ffs_kernels.cuh), about Nc^2 / 2 entries per sample.
#include <type_traits>

#include "ffs_arith.cuh"
#include "ffs_draw.cuh"
#include "ffs_group.cuh"
#include "ffs_kernels.cuh"
#include "ffs_sm100.cuh"

namespace fermi {

constexpr int NB = 32;           // panel width (== warp size: one lane per panel column)

constexpr int kStepWarps = 8;    // samples per CTA of the step kernel
// Rows of the state whose loads a step-kernel warp issues together.  Small groups keep
// the kernel at 64 registers, so that four 256-thread CTAs fit an SM and a 4096-sample
// step runs as one wave (measured on the 64x64 lattice workload: groups of 2 rows at 4
// CTAs/SM 601 ms per step, groups of 8 rows at 2 CTAs/SM 670 ms).
constexpr int kStepRowGroup = 2;

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
// Double-float value straight to the operand encoding, on the FP32 pipes: the BF16 low
// part is the rounded remainder (hi_f - hi_bf16) + lo_f, whose FP32 rounding is far below
// a BF16 ulp of the low part.
__device__ __forceinline__ void put_out_df(const StepArgs& a, int op, int64_t b, int col, df v) {
  const size_t idx = (size_t)b * a.Kp + col;
  switch (op) {
    case kOpF32: ((float*)a.H)[idx] = __fadd_rn(v.hi, v.lo); break;
    case kOpTF32: {
      uint32_t r;
      asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(__fadd_rn(v.hi, v.lo)));
      ((float*)a.H)[idx] = __uint_as_float(r);
      break;
    }
    case kOpBF16x3: {
      const __nv_bfloat16 hi = __float2bfloat16_rn(v.hi);
      ((__nv_bfloat16*)a.H)[idx] = hi;
      ((__nv_bfloat16*)a.H)[a.hplane + idx] =
          __float2bfloat16_rn(__fadd_rn(__fsub_rn(v.hi, __bfloat162float(hi)), v.lo));
      break;
    }
    case kOpBF16: ((__nv_bfloat16*)a.H)[idx] = __float2bfloat16_rn(v.hi); break;
    default: break;
  }
}
template <typename A> __device__ __forceinline__ void put_state(const StepArgs& a, int op, int64_t b, int col, A v) {
  if constexpr (std::is_same<A, df>::value) {
    put_out_df(a, op, b, col, v);
  } else if constexpr (std::is_same<A, cdf>::value) {
    put_out_df(a, op, b, 2 * col, v.re);
    put_out_df(a, op, b, 2 * col + 1, v.im);
  } else {
    put_h(a, op, b, col, Ar<A>::out(v));
  }
}

template <typename A> __device__ __forceinline__ A shfl_idx_any(A v, int src) {
  constexpr int Wd = sizeof(A) / 4;
  uint32_t w[Wd];
  memcpy(w, &v, sizeof(A));
#pragma unroll
  for (int q = 0; q < Wd; ++q) w[q] = __shfl_sync(0xffffffffu, w[q], src);
  memcpy(&v, w, sizeof(A));
  return v;
}

// ------------------------------------------------------------------ warp draw
// Sum of the 128 weights of chunk ch (each lane loads 4), identical in every lane.
__device__ __forceinline__ double chunk_sum(const float* __restrict__ p, int64_t L, int64_t ch, int lane) {
  const int64_t y0 = ch * 128 + 4 * lane;
  float v0 = 0.f, v1 = 0.f, v2 = 0.f, v3 = 0.f;
  if (y0 + 3 < L) {
    const float4 v = *(const float4*)(p + y0);
    v0 = v.x, v1 = v.y, v2 = v.z, v3 = v.w;
  } else {
    if (y0 < L) v0 = p[y0];
    if (y0 + 1 < L) v1 = p[y0 + 1];
    if (y0 + 2 < L) v2 = p[y0 + 2];
  }
  float s = (v0 + v1) + (v2 + v3);
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return (double)s;
}

// First site of chunk ch with a nonzero weight whose running sum, started at base,
// exceeds t; -1 when rounding leaves none in the chunk.
__device__ __forceinline__ int chunk_find(const float* __restrict__ p, int64_t L, int64_t ch, int lane, double base,
                                          double t) {
  const int64_t y0 = ch * 128 + 4 * lane;
  float w[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) w[q] = (y0 + q < L) ? p[y0 + q] : 0.f;
  float run[4];
  float acc = 0.f;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    acc += w[q];
    run[q] = acc;
  }
  float incl = acc;
  for (int o = 1; o < 32; o <<= 1) {
    const float v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  // running sums within the chunk in FP32 (128 terms), the chunk base in FP64
  const float excl = incl - acc;
  const float tl = (float)(t - base);
  int q_hit = -1;
#pragma unroll
  for (int q = 3; q >= 0; --q)
    if (w[q] > 0.f && excl + run[q] > tl) q_hit = q;
  const unsigned hit = __ballot_sync(0xffffffffu, q_hit >= 0);
  if (!hit) return -1;
  const int src = __ffs(hit) - 1;
  const int qs = __shfl_sync(0xffffffffu, q_hit, src);
  return (int)(ch * 128 + 4 * src + qs);
}

// The same chunk sum in two parts, so that the loads of several chunks can be issued
// before any of their warp reductions: lane's four weights, then (v0 + v1) + (v2 + v3)
// reduced over the warp in the order chunk_sum uses.
__device__ __forceinline__ float4 chunk_load(const float* __restrict__ p, int64_t L, int64_t ch, int lane) {
  const int64_t y0 = ch * 128 + 4 * lane;
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  if (y0 + 3 < L) {
    v = *(const float4*)(p + y0);
  } else {
    if (y0 < L) v.x = p[y0];
    if (y0 + 1 < L) v.y = p[y0 + 1];
    if (y0 + 2 < L) v.z = p[y0 + 2];
  }
  return v;
}
__device__ __forceinline__ double chunk_reduce(float4 v) {
  float s = (v.x + v.y) + (v.z + v.w);
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return (double)s;
}
// Normaliser from the residual's group sums g[0 .. ng): lane l adds groups l, l + 32, ...
// in FP64, then a butterfly over the warp (the same value in every lane).
__device__ __forceinline__ double gsum_total(const float* __restrict__ g, int64_t ng, int lane) {
  double z = 0.0;
  int64_t i = lane;
  for (; i + 96 < ng; i += 128) {  // four loads in flight
    const float a0 = g[i], a1 = g[i + 32], a2 = g[i + 64], a3 = g[i + 96];
    z += ((double)a0 + (double)a1) + ((double)a2 + (double)a3);
  }
  for (; i < ng; i += 32) z += (double)g[i];
  for (int o = 16; o; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
  return z;
}

// Inverse-CDF search over the group sums: blocks of 32 groups (a warp scan in FP64), the
// first group with a positive sum whose running sum passes t, then the first site of that
// group (gs sites, one per lane) with a positive weight whose running sum passes t.  When
// rounding leaves no site of the chosen group past t, its last site with a positive
// weight; -1 when no group passes t.
__device__ __forceinline__ int gsum_find(const float* __restrict__ g, const float* __restrict__ p, int64_t L,
                                         int gs, int lane, double t) {
  const int64_t ng = (L + gs - 1) / gs;
  double base = 0.0;
  for (int64_t g0 = 0; g0 < ng; g0 += 32) {
    const int64_t gi = g0 + lane;
    const double v = gi < ng ? (double)g[gi] : 0.0;
    double incl = v;
    for (int o = 1; o < 32; o <<= 1) {
      const double u = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += u;
    }
    const unsigned hit = __ballot_sync(0xffffffffu, v > 0.0 && base + incl > t);
    if (hit) {
      const int src = __ffs(hit) - 1;
      const double gb = base + __shfl_sync(0xffffffffu, incl - v, src);
      const int64_t y = (g0 + src) * gs + lane;
      const double w = (lane < gs && y < L) ? (double)p[y] : 0.0;
      double run = w;
      for (int o = 1; o < 32; o <<= 1) {
        const double u = __shfl_up_sync(0xffffffffu, run, o);
        if (lane >= o) run += u;
      }
      const unsigned in = __ballot_sync(0xffffffffu, w > 0.0 && gb + run > t);
      const unsigned pos = __ballot_sync(0xffffffffu, w > 0.0);
      if (in) return (int)((g0 + src) * gs + __ffs(in) - 1);
      if (pos) return (int)((g0 + src) * gs + 31 - __clz(pos));
    }
    base += __shfl_sync(0xffffffffu, incl, 31);
  }
  return -1;
}

// Chunk sums of the normaliser pass kept in shared memory for the search pass: up to
// kCsMax chunks per warp, i.e. L <= 16384; longer rows take the two-pass form.
constexpr int kCsMax = 128;

__device__ __forceinline__ int last_nonzero(const float* __restrict__ p, int64_t L, int lane) {
  int last = -1;
  for (int64_t y = lane; y < L; y += 32)
    if (p[y] > 0.f) last = (int)y;
  for (int o = 16; o; o >>= 1) last = max(last, __shfl_xor_sync(0xffffffffu, last, o));
  return last;
}

template <typename A>
__device__ __forceinline__ void step_update(const StepArgs& a, const BlockedArgs& t, int64_t b, int64_t k, int x,
                                            int64_t len, int op_mode);

// ------------------------------------------------------------------ per-step body (one warp)
template <typename A>
__device__ __forceinline__ void step_warp(const StepArgs& a, const BlockedArgs& t, int64_t b, int64_t k,
                                          int op_mode, double* csm) {
  using T = Ar<A>;
  const int lane = threadIdx.x & 31;
  const int64_t L = a.L, N = a.N, Nc = t.Nc;
  const float* __restrict__ prow = a.P + b * a.ldP;
  const int64_t len = a.nlen ? (int64_t)a.nlen[b] : a.n_steps;  // this sample's chain length
  if (k >= len) {  // the chain has ended (an L-ensemble sample that kept fewer columns)
    if (lane == 0) a.x[b * a.ldx + k] = -1;
    if (a.probs) {
      float* pr = a.probs + ((size_t)b * a.ldx + k) * L;
      for (int64_t y = lane; y < L; y += 32) pr[y] = 0.f;
    }
    return;
  }

  // draw: Z over 128-site chunks, then the first chunk whose running sum passes t (both
  // sums in chunk order; with the chunk sums cached, the search reads only the chosen chunk).
  // When the residual wrote the weights' group sums, Z and the search read those instead
  // (L / 32 or L / 16 sums) and then the weights of the chosen group alone.
  const int64_t nch = (L + 127) / 128;
  const bool grouped_sums = a.G != nullptr;
  const bool cached = !grouped_sums && nch <= kCsMax;
  double Z = 0.0;
  if (grouped_sums) {
    Z = gsum_total(a.G + b * a.ldG, (L + kGroupSites(a.cplx) - 1) / kGroupSites(a.cplx), lane);
  } else if (cached) {
    for (int64_t ch0 = 0; ch0 < nch; ch0 += 4) {  // four chunks' loads in flight together
      float4 v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        v[q] = (ch0 + q < nch) ? chunk_load(prow, L, ch0 + q, lane) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (ch0 + q < nch) {
          const double sq = chunk_reduce(v[q]);
          Z += sq;
          if (lane == 0) csm[ch0 + q] = sq;
        }
      }
    }
    __syncwarp();
  } else {
    for (int64_t ch = 0; ch < nch; ++ch) Z += chunk_sum(prow, L, ch, lane);
  }
  int x;
  const int f = forced_site(a, b, k);
  if (f != -1) {
    if (f == -2 && lane == 0) set_status(a.status, FFS_E_ARG);
    x = f < 0 ? 0 : f;
  } else {
    const double tt = site_uniform(a.seed, a.first + (uint64_t)b, (int)k) * Z;
    x = -1;
    double base = 0.0;
    if (grouped_sums) {
      x = gsum_find(a.G + b * a.ldG, prow, L, kGroupSites(a.cplx), lane, tt);
    } else if (cached) {
      for (int64_t ch = 0; ch < nch && x < 0; ++ch) {
        const double cs = csm[ch];
        if (base + cs > tt) x = chunk_find(prow, L, ch, lane, base, tt);
        base += cs;
      }
    } else {
      for (int64_t ch = 0; ch < nch && x < 0; ++ch) {
        const double cs = chunk_sum(prow, L, ch, lane);
        if (base + cs > tt) x = chunk_find(prow, L, ch, lane, base, tt);
        base += cs;
      }
    }
    if (x < 0) x = last_nonzero(prow, L, lane);
    if (x < 0) {
      if (lane == 0) set_status(a.status, FFS_E_NUMERIC);
      x = 0;
    }
  }
  if (lane == 0) {
    a.x[b * a.ldx + k] = x;
    a.mask[b * a.ldMask + (x >> 5)] |= 1u << (x & 31);
    const double px = (double)prow[x];
    a.logp[b] += (px > 0.0 && Z > 0.0) ? log(px / Z) : -INFINITY;
    if (!(Z > 0.0) || !isfinite(Z)) set_status(a.status, FFS_E_NUMERIC);
  }
  if (a.probs) {
    float* pr = a.probs + ((size_t)b * a.ldx + k) * L;
    const double iz = Z > 0.0 ? 1.0 / Z : 0.0;
    for (int64_t y = lane; y < L; y += 32) pr[y] = (float)((double)prow[y] * iz);
  }
  step_update<A>(a, t, b, k, x, len, op_mode);
}

// ------------------------------------------------------------------ per-step state update
// After x_k is placed: reduce its row of U against the state on the panel columns, take
// the pivot, and write the operand of step k+1.  The rank-1 update of the panel columns
// that the pivot implies is applied lazily: each step's single pass over the rows first
// applies the previous step's update (W[j][c] -= W[j][k-1] W[k-1][c], row k-1 being that
// step's new row), writes the row back and uses it for the reduction, so every row is
// read and written once per step.  The arithmetic per entry is that of the eager update.
// Lane l owns panel column k0 + l.
template <typename A>
__device__ __forceinline__ void step_update(const StepArgs& a, const BlockedArgs& t, int64_t b, int64_t k, int x,
                                            int64_t len, int op_mode) {
  using T = Ar<A>;
  const int lane = threadIdx.x & 31;
  const int64_t N = a.N, Nc = t.Nc;
  if (k + 1 >= len) return;

  const int64_t k0 = (k / NB) * NB, k1 = min(k0 + NB, Nc);
  const int i = (int)(k - k0);
  // this panel's slab: element (j, k0 + l) at Wp[j * 32 + l]
  A* Wp = (A*)t.W + (size_t)b * state_stride(Nc) + (size_t)slab_offset(k0 >> 5);
  A* W0P = (A*)t.W0P + (size_t)b * Nc * NB;
  const int32_t* mrow = a.m + b * N;
  const A* urow = (const A*)a.Ust + (int64_t)x * N;  // U in the state type
  const bool live = lane < k1 - k0;                  // the column exists
  const bool gem = live && lane >= i;                // columns k .. k1-1 are reduced
  const bool pend = i >= 1;                          // an update of step k-1 is pending
  const bool keep = i == 0 && k0 > 0;                // first step of a panel: save W0_P

  // one pass over the rows: pending update, write-back, reduction
  // r'[c] = u[c] - sum_{j<k} u[j] W[j][c].  Only the columns from k-1 on are read (all of
  // them at a panel's first step), so a warp takes P = 32 / S rows at a time, S the
  // smallest power of two >= the number of those columns: lane = (row slot rr, column
  // cs + cc).  Late in a panel, with few columns left, one instruction then covers
  // several rows.
  const int cs = i >= 1 ? i - 1 : 0;                 // first column read (k-1 when pending)
  const int ncol = (int)(k1 - k0) - cs;              // columns cs .. k1-k0-1
  const int lgS = ncol > 16 ? 5 : ncol > 8 ? 4 : ncol > 4 ? 3 : ncol > 2 ? 2 : ncol > 1 ? 1 : 0;
  const int S = 1 << lgS, P = 32 >> lgS;
  const int rr = lane >> lgS, cc = lane & (S - 1);
  const int lc = cs + cc;                            // this lane's column
  const bool live_c = cc < ncol;
  const bool gem_c = live_c && lc >= i;
  const A nprev = (pend && gem_c) ? Wp[(k - 1) * 32 + lc] : T::zero();  // new row of step k-1
  const int src = rr << lgS;                         // lane of column k-1 in this row slot

  // rows in groups of G passes whose loads are issued together (one group of lookahead for
  // 4- and 8-byte entries: the next group's loads go out before this group's stores, which
  // the compiler cannot do on its own; 16-byte entries take one pass per group, loaded in
  // turn, which keeps them at 64 registers); two accumulation chains
  constexpr bool kAhead = sizeof(A) <= 8;
  constexpr int G = kAhead ? kStepRowGroup : 1;      // 16-byte entries: one pass per group
  const int64_t grp = (int64_t)P * G;                // rows per group
  A acc = T::zero(), acc2 = T::zero();
  // rows stream from DRAM: keep the next 32-row blocks on their way into L2, two blocks
  // ahead of the loads; lane l prefetches row j + l from the first column read (rounded
  // down to 16 bytes) to the end of the row, so late in a panel, when few columns are
  // live, the prefetch does not drag the dead part of each row out of DRAM
  constexpr int kColAlign = sizeof(A) >= 16 ? 1 : (int)(16 / sizeof(A));
  const int cpf = cs & ~(kColAlign - 1);
  const uint32_t pf_bytes = (uint32_t)((32 - cpf) * sizeof(A));
  auto prefetch_rows = [&](int64_t j) {
    if (j + lane < k) sm100::prefetch_l2_bulk(Wp + (j + lane) * 32 + cpf, pf_bytes);
  };
  auto ld_w = [&](int64_t j) { return (j < k && live_c) ? Wp[j * 32 + lc] : T::zero(); };
  auto ld_u = [&](int64_t j) { return j < k ? urow[mrow[j]] : T::zero(); };
  int64_t pf = 0;
  A wv[G];
  if constexpr (kAhead) {
#pragma unroll
    for (int g = 0; g < G; ++g) wv[g] = ld_w((int64_t)g * P + rr);
  }
  for (int64_t jb = 0; jb < k; jb += grp) {
    for (; pf < jb + grp + 64 && pf < k; pf += 32) prefetch_rows(pf);
    A wn[G], uv[G];
    if constexpr (kAhead) {
#pragma unroll
      for (int g = 0; g < G; ++g) wn[g] = ld_w(jb + grp + (int64_t)g * P + rr);
    } else {
#pragma unroll
      for (int g = 0; g < G; ++g) wv[g] = ld_w(jb + (int64_t)g * P + rr);
    }
#pragma unroll
    for (int g = 0; g < G; ++g) uv[g] = ld_u(jb + (int64_t)g * P + rr);  // cached: U's row x
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int64_t j = jb + (int64_t)g * P + rr;
      if (keep && live_c && j < k) W0P[j * NB + lc] = wv[g];
      if (pend) {
        const A wk = shfl_idx_any(wv[g], src);
        if (gem_c && j < k - 1) {
          wv[g] = T::fms(wv[g], wk, nprev);
          Wp[j * 32 + lc] = wv[g];
        }
      }
    }
#pragma unroll
    for (int g = 0; g < G; g += 2) {
      acc = T::fms(acc, uv[g], gem_c ? wv[g] : T::zero());
      if (g + 1 < G) acc2 = T::fms(acc2, uv[g + 1], gem_c ? wv[g + 1] : T::zero());
    }
    if constexpr (kAhead) {
#pragma unroll
      for (int g = 0; g < G; ++g) wv[g] = wn[g];
    }
  }
  acc = T::add(acc, acc2);
  // the row slots' partial sums of each column (the same total in every slot), then
  // column l's total into lane l
  for (int o = S; o < 32; o <<= 1) acc = T::add(acc, shfl_xor_any(acc, o));
  const int from = lane - cs;
  acc = shfl_idx_any(acc, (from >= 0 && from < S) ? from : 0);
  const A rc = gem ? T::add(urow[mrow[k0 + lane]], acc) : T::zero();
  const A s = shfl_idx_any(rc, i);  // pivot: the Schur residual of x_k
  if (lane == 0) {
    const double s2 = T::abs2(s);
    if (!(s2 > 1e-300) || !isfinite(s2)) set_status(a.status, FFS_E_NUMERIC);
  }
  const bool upd = gem && lane > i;
  const A ncv = upd ? T::div(rc, s) : T::zero();
  if (upd) Wp[k * 32 + lane] = ncv;  // the new row; its update of the other rows is pending
  const A nk1 = shfl_idx_any(ncv, min(i + 1, 31));
  __syncwarp();

  // operand of step k+1 while column k+1 is still inside this panel: column k+1 after
  // this step's (pending) update
  if (op_mode != kOpNone && k + 1 < k1) {
    for (int64_t j = lane; j <= k + 1; j += 32) {
      A v;
      if (j < k)
        v = T::neg(T::fms(Wp[j * 32 + i + 1], Wp[j * 32 + i], nk1));
      else if (j == k)
        v = T::neg(nk1);
      else
        v = T::one();
      put_state<A>(a, op_mode, b, operand_col(a, mrow, j), v);
    }
  }
}

template <typename A>
__global__ void __launch_bounds__(256, 4) tail_step_kernel(StepArgs a, BlockedArgs t, int64_t k, int op_mode) {
  __shared__ double csm[kStepWarps][kCsMax];
  const int64_t b = (int64_t)blockIdx.x * kStepWarps + (threadIdx.x >> 5);
  if (b >= a.bw) return;
  step_warp<A>(a, t, b, k, op_mode, csm[threadIdx.x >> 5]);
}

// ------------------------------------------------------------------ large-L draw (Section S-7)
// x_k from a Metropolis chain instead of the all-site weights: the chain starts at a
// uniform site, proposes uniform sites and accepts a move y -> y' when
// u |u_y^T h|^2 < |u_{y'}^T h|^2 (the acceptance ratio of Section S-7; a drawn site has
// weight 0 and is never accepted).  Iteration it of step k takes Philox stream 3, block
// k (m_cond + 1) + it: words 0-1 give the site mulhi(r, L), words 2-3 the 53-bit uniform.
// A site's weight is its whole row of U against h scattered to the original column
// order (-h kept in shared memory), summed by the warp and taken from lane 0, so that
// every lane takes the same decision.
constexpr int kMcmcWarps = 4;

template <typename A>
__device__ __forceinline__ int mcmc_draw(const StepArgs& a, const BlockedArgs& t, int64_t b, int64_t k,
                                         int64_t m_cond, A* hs) {
  using T = Ar<A>;
  const int lane = threadIdx.x & 31;
  const int64_t N = a.N, Nc = t.Nc;
  const A* W = (const A*)t.W + (size_t)b * state_stride(Nc);
  const int32_t* mrow = a.m + b * N;
  for (int64_t c = lane; c < N; c += 32) hs[c] = T::zero();
  __syncwarp();
  // -h: h_j = -W[j][k] (j < k), h_k = 1, with the update of step k-1 (pending in the
  // state, see step_update) applied to column k when k-1 is in the same panel
  const bool pend = (k & 31) != 0;
  const A nk = pend ? W[sidx(k - 1, k)] : T::zero();
  for (int64_t j = lane; j <= k; j += 32) {
    A v = T::neg(T::one());
    if (j < k) {
      v = W[sidx(j, k)];
      if (pend && j < k - 1) v = T::fms(v, W[sidx(j, k - 1)], nk);
    }
    hs[mrow[j]] = v;
  }
  __syncwarp();
  const uint32_t* mk = a.mask + b * a.ldMask;
  const A* Us = (const A*)a.Ust;
  const uint64_t sample = a.first + (uint64_t)b;
  auto weight = [&](int64_t y) -> double {
    if ((mk[y >> 5] >> (y & 31)) & 1u) return 0.0;
    const A* row = Us + y * N;
    A acc = T::zero();
    for (int64_t c = lane; c < N; c += 32) acc = T::fms(acc, row[c], hs[c]);
#pragma unroll
    for (int o = 16; o; o >>= 1) acc = T::add(acc, shfl_xor_any(acc, o));
    return T::abs2(shfl_idx_any(acc, 0));
  };
  const uint32_t base = (uint32_t)(k * (m_cond + 1));
  uint4 w = philox_block(a.seed, base, kStreamMcmc, sample);
  int64_t cur = (int64_t)__umul64hi(((uint64_t)w.x << 32) | w.y, (uint64_t)a.L);
  double pc = weight(cur);
  for (int64_t it = 1; it <= m_cond; ++it) {
    w = philox_block(a.seed, base + (uint32_t)it, kStreamMcmc, sample);
    const int64_t y = (int64_t)__umul64hi(((uint64_t)w.x << 32) | w.y, (uint64_t)a.L);
    const double u = (double)(((uint64_t)(w.z >> 5) << 26) | (uint64_t)(w.w >> 6)) * 0x1p-53;
    const double py = weight(y);
    if (u * pc < py) {
      cur = y;
      pc = py;
    }
  }
  if (!(pc > 0.0) && lane == 0) set_status(a.status, FFS_E_NUMERIC);  // no site with weight reached
  return (int)cur;
}

template <typename A>
__global__ void __launch_bounds__(32 * kMcmcWarps) mcmc_step_kernel(StepArgs a, BlockedArgs t, int64_t k,
                                                                   int64_t m_cond) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t b = (int64_t)blockIdx.x * kMcmcWarps + warp;
  if (b >= a.bw) return;
  A* hs = (A*)smem_raw + (size_t)warp * a.N;
  const int x = mcmc_draw<A>(a, t, b, k, m_cond, hs);
  if (lane == 0) {
    a.x[b * a.ldx + k] = x;
    a.mask[b * a.ldMask + (x >> 5)] |= 1u << (x & 31);
  }
  __syncwarp();
  step_update<A>(a, t, b, k, x, a.n_steps, kOpNone);
}

// ------------------------------------------------------------------ panel end: S^-1
// S = U[x_new, m_P] - U[x_new, m_<k0] W0_P, inverted in shared memory (one CTA per sample).
template <typename A>
__device__ __forceinline__ void panel_s_body(const StepArgs& a, const BlockedArgs& t, int64_t b, int64_t k0,
                                             int64_t k1, unsigned char* smem_raw) {
  using T = Ar<A>;
  // the product phase's chunks and the Gauss-Jordan matrix share one region
  A* Cs = (A*)smem_raw;         // NB x 32 chunk of U[x_new, m_j]
  A* Ws = Cs + NB * 32;         // 32 x NB chunk of W0_P
  df* Csum = (df*)(Ws + 32 * NB);  // double-float: re + im of Cs and Ws (Karatsuba)
  df* Wsum = Csum + NB * 32;
  A* Aug = (A*)smem_raw;        // NB x 2NB: [S | I] -> [I | S^-1], after the products
  unsigned char* end1 = (unsigned char*)(Wsum + 32 * NB);
  unsigned char* end2 = (unsigned char*)(Aug + NB * 2 * NB);
  A* fac = (A*)(end1 > end2 ? end1 : end2);  // NB elimination factors, then the pivot
  int* xs = (int*)(fac + NB + 1);
  int* mj = xs + NB;
  const int tid = threadIdx.x;
  const int64_t N = a.N;
  const int nbr = (int)(k1 - k0);
  if (a.nlen && a.nlen[b] <= k1) return;  // chain ends in this panel (uniform over the CTA)
  const int32_t* mrow = a.m + b * N;
  const A* Us = (const A*)a.Ust;  // U in the state type
  const A* W0P = (const A*)t.W0P + (size_t)b * t.Nc * NB;
  if (tid < NB) xs[tid] = tid < nbr ? a.x[b * a.ldx + k0 + tid] : 0;
  __syncthreads();
  // thread owns entries (ii, cc) = (tid / 32 + 8 q, tid % 32)
  const int cc = tid & 31, r0 = tid >> 5;
  A acc[NB / 8];
#pragma unroll
  for (int q = 0; q < NB / 8; ++q) {
    const int ii = r0 + 8 * q;
    acc[q] = (ii < nbr && cc < nbr) ? Us[(int64_t)xs[ii] * N + mrow[k0 + cc]] : T::zero();
  }
  if constexpr (std::is_same<A, cdf>::value || std::is_same<A, df>::value) {
    // double-float: lazily renormalised accumulators; complex products by Karatsuba, as
    // in the trailing update
    constexpr bool CX = std::is_same<A, cdf>::value;
    lzf S1[NB / 8], S2[NB / 8], S3[NB / 8];
#pragma unroll
    for (int q = 0; q < NB / 8; ++q) S1[q] = S2[q] = S3[q] = lzf{0.f, 0.f};
    for (int64_t j0 = 0; j0 < k0; j0 += 32) {
      if (tid < 32) mj[tid] = (j0 + tid < k0) ? mrow[j0 + tid] : 0;
      __syncthreads();
      for (int e = tid; e < NB * 32; e += blockDim.x) {
        const int ii = e >> 5, jj = e & 31;
        const A cv = (ii < nbr && j0 + jj < k0) ? Us[(int64_t)xs[ii] * N + mj[jj]] : T::zero();
        const A wv = (j0 + ii < k0 && jj < nbr) ? W0P[(j0 + ii) * NB + jj] : T::zero();  // row ii of the chunk
        Cs[e] = cv;
        Ws[e] = wv;
        if constexpr (CX) {
          Csum[e] = df_add(cv.re, cv.im);
          Wsum[e] = df_add(wv.re, wv.im);
        }
      }
      __syncthreads();
#pragma unroll 2
      for (int jj = 0; jj < 32; ++jj) {
        const A w = Ws[jj * NB + cc];
        if constexpr (CX) {
          const df wsum = Wsum[jj * NB + cc];
#pragma unroll
          for (int q = 0; q < NB / 8; ++q) {
            const int ci = (r0 + 8 * q) * 32 + jj;
            const A cv = Cs[ci];
            lz_mac(S1[q], cv.re, w.re);
            lz_mac(S2[q], cv.im, w.im);
            lz_mac(S3[q], Csum[ci], wsum);
          }
        } else {
#pragma unroll
          for (int q = 0; q < NB / 8; ++q) lz_mac(S1[q], Cs[(r0 + 8 * q) * 32 + jj], w);
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < NB / 8; ++q) {
      if constexpr (CX) {
        const df p1 = lz_get(S1[q]), p2 = lz_get(S2[q]), p3 = lz_get(S3[q]);
        const df re = df_sub(p1, p2), im = df_sub(df_sub(p3, p1), p2);
        acc[q] = A{df_sub(acc[q].re, re), df_sub(acc[q].im, im)};
      } else {
        acc[q] = df_sub(acc[q], lz_get(S1[q]));
      }
    }
  } else {
    for (int64_t j0 = 0; j0 < k0; j0 += 32) {
      if (tid < 32) mj[tid] = (j0 + tid < k0) ? mrow[j0 + tid] : 0;
      __syncthreads();
      for (int e = tid; e < NB * 32; e += blockDim.x) {
        const int ii = e >> 5, jj = e & 31;
        Cs[e] = (ii < nbr && j0 + jj < k0) ? Us[(int64_t)xs[ii] * N + mj[jj]] : T::zero();
        Ws[e] = (j0 + ii < k0 && jj < nbr) ? W0P[(j0 + ii) * NB + jj] : T::zero();  // row ii of the chunk
      }
      __syncthreads();
#pragma unroll 4
      for (int jj = 0; jj < 32; ++jj) {
        const A w = Ws[jj * NB + cc];
#pragma unroll
        for (int q = 0; q < NB / 8; ++q) acc[q] = T::fms(acc[q], Cs[(r0 + 8 * q) * 32 + jj], w);
      }
      __syncthreads();
    }
  }
  __syncthreads();  // the product buffers become the Gauss-Jordan matrix
#pragma unroll
  for (int q = 0; q < NB / 8; ++q) {
    const int ii = r0 + 8 * q;
    Aug[ii * 2 * NB + cc] = acc[q];
    Aug[ii * 2 * NB + NB + cc] = (ii == cc) ? T::one() : T::zero();
  }
  __syncthreads();
  // Gauss-Jordan without pivot search: the pivots are taken in draw order
  for (int p = 0; p < nbr; ++p) {
    if (tid == 0) {
      fac[NB] = Aug[p * 2 * NB + p];
      const double p2 = T::abs2(fac[NB]);
      if (!(p2 > 1e-300) || !isfinite(p2)) set_status(a.status, FFS_E_NUMERIC);
    }
    __syncthreads();
    if (tid < 2 * NB) Aug[p * 2 * NB + tid] = T::div(Aug[p * 2 * NB + tid], fac[NB]);
    if (tid < NB) fac[tid] = Aug[tid * 2 * NB + p];
    __syncthreads();
    for (int e = tid; e < NB * 2 * NB; e += blockDim.x) {
      const int rr = e / (2 * NB), col = e % (2 * NB);
      if (rr != p && rr < nbr) Aug[e] = T::fms(Aug[e], fac[rr], Aug[p * 2 * NB + col]);
    }
    __syncthreads();
  }
  A* Sinv = (A*)t.Sinv + (size_t)b * NB * NB;
  for (int e = tid; e < NB * NB; e += blockDim.x) Sinv[e] = Aug[(e / NB) * 2 * NB + NB + (e % NB)];
}

template <typename A>
__global__ void __launch_bounds__(256) tail_panel_s_kernel(StepArgs a, BlockedArgs t, int64_t k0, int64_t k1) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  panel_s_body<A>(a, t, blockIdx.x, k0, k1, smem_raw);
}

// ------------------------------------------------------------------ panel end: trailing columns
// Sample b, columns [k1 + 32 cb, +32) of T: Y, Bot = S^-1 Y, Top = W0_T - W0_P Bot.
template <typename A>
__device__ __forceinline__ void panel_body(const StepArgs& a, const BlockedArgs& t, int64_t b, int64_t cb,
                                           int64_t k0, int64_t k1, int op_mode, unsigned char* smem_raw) {
  using T = Ar<A>;
  // Shared memory is reused between the phases (kept small so that three CTAs fit an SM):
  //   Y phase:        Cs (NB x 32: U[x_new, m_j] chunk), Ws (32 x 32: W0_T chunk), and for
  //                   double-float their re + im sums Csum, Wsum;
  //   Bot/Top phases: Ys (NB x 32: Y), Si (NB x NB: S^-1), Bs (NB x 32: Bot), and for
  //                   complex double-float Bsum and the per-warp W0_P rows Wrow, Wrs.
  A* Cs = (A*)smem_raw;
  A* Ws = Cs + NB * 32;
  df* Csum = (df*)(Ws + 32 * 32);
  df* Wsum = Csum + NB * 32;
  A* Ys = (A*)smem_raw;
  A* Si = Ys + NB * 32;
  A* Bs = Si + NB * NB;
  df* Bsum = (df*)(Bs + NB * 32);
  A* Wrow_all = (A*)(Bsum + NB * 32);
  df* Wrs_all = (df*)(Wrow_all + 8 * 32);
  unsigned char* end1 = (unsigned char*)(Wsum + 32 * 32);
  unsigned char* end2 = (unsigned char*)(Wrs_all + 8 * 32);
  int* xs = (int*)(end1 > end2 ? end1 : end2);
  int* mj = xs + NB;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t N = a.N, Nc = t.Nc;
  const int nbr = (int)(k1 - k0);
  if (a.nlen && a.nlen[b] <= k1) return;  // chain ends in this panel (uniform over the CTA)
  const int64_t c0 = k1 + cb * 32;
  const int64_t c = c0 + lane;
  const bool cval = c < Nc;
  // slab of the columns [c0, c0 + 32) (c0 is a multiple of 32): element (j, c0 + cc) at Wc[j * 32 + cc]
  A* Wc = (A*)t.W + (size_t)b * state_stride(Nc) + (size_t)slab_offset(c0 >> 5);
  const A* W0P = (const A*)t.W0P + (size_t)b * Nc * NB;
  const int32_t* mrow = a.m + b * N;
  const A* Us = (const A*)a.Ust;  // U in the state type

  if (tid < NB) xs[tid] = tid < nbr ? a.x[b * a.ldx + k0 + tid] : 0;
  __syncthreads();

  // Y = U[x_new, m_T] - U[x_new, m_<k0] W0_T; thread owns rows warp + 8q, column lane
  const int mc = cval ? mrow[c] : 0;
  A acc[NB / 8];
#pragma unroll
  for (int q = 0; q < NB / 8; ++q) {
    const int ii = warp + 8 * q;
    acc[q] = (ii < nbr && cval) ? Us[(int64_t)xs[ii] * N + mc] : T::zero();
  }
  if constexpr (std::is_same<A, cdf>::value || std::is_same<A, df>::value) {
    // double-float: lazily renormalised accumulators; complex products by Karatsuba
    // (re = S1 - S2, im = S3 - S1 - S2 with S1 = sum c.re w.re, S2 = sum c.im w.im,
    // S3 = sum (c.re + c.im)(w.re + w.im)): three real products instead of four.
    constexpr bool CX = std::is_same<A, cdf>::value;
    lzf S1[NB / 8], S2[NB / 8], S3[NB / 8];
#pragma unroll
    for (int q = 0; q < NB / 8; ++q) S1[q] = S2[q] = S3[q] = lzf{0.f, 0.f};
    for (int64_t j0 = 0; j0 < k0; j0 += 32) {
      if (tid < 32) mj[tid] = (j0 + tid < k0) ? mrow[j0 + tid] : 0;
      __syncthreads();
      for (int e = tid; e < NB * 32; e += blockDim.x) {
        const int ii = e >> 5, jj = e & 31;
        const A v = (ii < nbr && j0 + jj < k0) ? Us[(int64_t)xs[ii] * N + mj[jj]] : T::zero();
        Cs[e] = v;
        if constexpr (CX) Csum[e] = df_add(v.re, v.im);
      }
      for (int e = tid; e < 32 * 32; e += blockDim.x) {
        const int jj = e >> 5, cc = e & 31;
        const A v = (j0 + jj < k0 && c0 + cc < Nc) ? Wc[(j0 + jj) * 32 + cc] : T::zero();
        Ws[e] = v;
        if constexpr (CX) Wsum[e] = df_add(v.re, v.im);
      }
      __syncthreads();
#pragma unroll 2
      for (int jj = 0; jj < 32; ++jj) {
        const A w = Ws[jj * 32 + lane];
        if constexpr (CX) {
          const df wsum = Wsum[jj * 32 + lane];
#pragma unroll
          for (int q = 0; q < NB / 8; ++q) {
            const int ci = (warp + 8 * q) * 32 + jj;
            const A cv = Cs[ci];
            lz_mac(S1[q], cv.re, w.re);
            lz_mac(S2[q], cv.im, w.im);
            lz_mac(S3[q], Csum[ci], wsum);
          }
        } else {
#pragma unroll
          for (int q = 0; q < NB / 8; ++q) lz_mac(S1[q], Cs[(warp + 8 * q) * 32 + jj], w);
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < NB / 8; ++q) {
      if constexpr (CX) {
        const df p1 = lz_get(S1[q]), p2 = lz_get(S2[q]), p3 = lz_get(S3[q]);
        const df re = df_sub(p1, p2), im = df_sub(df_sub(p3, p1), p2);
        acc[q] = A{df_sub(acc[q].re, re), df_sub(acc[q].im, im)};
      } else {
        acc[q] = df_sub(acc[q], lz_get(S1[q]));
      }
    }
  } else {
    for (int64_t j0 = 0; j0 < k0; j0 += 32) {
      if (tid < 32) mj[tid] = (j0 + tid < k0) ? mrow[j0 + tid] : 0;
      __syncthreads();
      for (int e = tid; e < NB * 32; e += blockDim.x) {
        const int ii = e >> 5, jj = e & 31;
        Cs[e] = (ii < nbr && j0 + jj < k0) ? Us[(int64_t)xs[ii] * N + mj[jj]] : T::zero();
      }
      for (int e = tid; e < 32 * 32; e += blockDim.x) {
        const int jj = e >> 5, cc = e & 31;
        Ws[e] = (j0 + jj < k0 && c0 + cc < Nc) ? Wc[(j0 + jj) * 32 + cc] : T::zero();
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
  }
  __syncthreads();  // the Y-phase buffers are reused from here on
#pragma unroll
  for (int q = 0; q < NB / 8; ++q) Ys[(warp + 8 * q) * 32 + lane] = acc[q];
  for (int e = tid; e < NB * NB; e += blockDim.x) Si[e] = ((const A*)t.Sinv)[(size_t)b * NB * NB + e];
  __syncthreads();

  // Bot = S^-1 Y
#pragma unroll
  for (int q = 0; q < NB / 8; ++q) {
    const int ii = warp + 8 * q;
    A v = T::zero();
    for (int ip = 0; ip < nbr; ++ip) v = T::fms(v, Si[ii * NB + ip], Ys[ip * 32 + lane]);
    Bs[ii * 32 + lane] = T::neg(v);
  }
  __syncthreads();

  if constexpr (std::is_same<A, cdf>::value) {
    // old rows, Karatsuba with lazy accumulators (as for Y): Top = W0_T - W0_P Bot
    A* Wrow = Wrow_all + warp * 32;  // this warp's W0_P row
    df* Wrs = Wrs_all + warp * 32;
    for (int e = tid; e < NB * 32; e += blockDim.x) Bsum[e] = df_add(Bs[e].re, Bs[e].im);
    __syncthreads();
    for (int64_t j = warp; j < (t.tc_top ? 0 : k0); j += 8) {
      if (lane < nbr) {
        const A wv = W0P[j * NB + lane];
        Wrow[lane] = wv;
        Wrs[lane] = df_add(wv.re, wv.im);
      }
      __syncwarp();
      lzf S1{0.f, 0.f}, S2{0.f, 0.f}, S3{0.f, 0.f};
      for (int ii = 0; ii < nbr; ++ii) {
        const A bv = Bs[ii * 32 + lane];
        const A wv = Wrow[ii];
        lz_mac(S1, wv.re, bv.re);
        lz_mac(S2, wv.im, bv.im);
        lz_mac(S3, Wrs[ii], Bsum[ii * 32 + lane]);
      }
      if (cval) {
        const df p1 = lz_get(S1), p2 = lz_get(S2), p3 = lz_get(S3);
        const A v = Wc[j * 32 + lane];
        Wc[j * 32 + lane] = A{df_sub(v.re, df_sub(p1, p2)), df_sub(v.im, df_sub(df_sub(p3, p1), p2))};
      }
      __syncwarp();
    }
    if (cval)
      for (int jn = warp; jn < nbr; jn += 8) Wc[(k0 + jn) * 32 + lane] = Bs[jn * 32 + lane];
  } else if constexpr (std::is_same<A, df>::value) {
    // old rows with a lazy accumulator, the warp's W0_P row staged in shared memory
    A* Wrow = Wrow_all + warp * 32;
    for (int64_t j = warp; j < (t.tc_top ? 0 : k0); j += 8) {
      if (lane < nbr) Wrow[lane] = W0P[j * NB + lane];
      __syncwarp();
      lzf S1{0.f, 0.f};
      for (int ii = 0; ii < nbr; ++ii) lz_mac(S1, Wrow[ii], Bs[ii * 32 + lane]);
      if (cval) Wc[j * 32 + lane] = df_sub(Wc[j * 32 + lane], lz_get(S1));
      __syncwarp();
    }
    if (cval)
      for (int jn = warp; jn < nbr; jn += 8) Wc[(k0 + jn) * 32 + lane] = Bs[jn * 32 + lane];
  } else if (cval) {
    // old rows: Top = W0_T - W0_P Bot
    for (int64_t j = warp; j < (t.tc_top ? 0 : k0); j += 8) {
      A v = Wc[j * 32 + lane];
      const A* wp = W0P + j * NB;
      for (int ii = 0; ii < nbr; ++ii) v = T::fms(v, wp[ii], Bs[ii * 32 + lane]);
      Wc[j * 32 + lane] = v;
    }
    // new rows: Bot
    for (int jn = warp; jn < nbr; jn += 8) Wc[(k0 + jn) * 32 + lane] = Bs[jn * 32 + lane];
  }
  __syncthreads();

  // operand of step k1 (its column is the first of T)
  if (op_mode != kOpNone && cb == 0 && k1 < a.n_steps && !t.tc_top) {
    for (int64_t j = tid; j <= k1; j += blockDim.x) {
      const A v = (j < k1) ? T::neg(Wc[j * 32]) : T::one();  // column k1 = c0 (cb == 0)
      put_state<A>(a, op_mode, b, operand_col(a, mrow, j), v);
    }
  }
}

template <typename A>
__global__ void __launch_bounds__(256, 3) tail_panel_kernel(StepArgs a, BlockedArgs t, int64_t k0, int64_t k1,
                                                         int op_mode) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  panel_body<A>(a, t, blockIdx.y, blockIdx.x, k0, k1, op_mode, smem_raw);
}

static size_t panel_s_smem(size_t es) {
  const size_t products = (size_t)(NB * 32 + 32 * NB) * es + (size_t)(NB * 32 + 32 * NB) * 8;
  const size_t gj = (size_t)NB * 2 * NB * es;
  return (products > gj ? products : gj) + (size_t)(NB + 1) * es + 2 * NB * 4;
}
// Ys, Bs, Cs, Ws, S^-1, the two index arrays, then (double-float) the Karatsuba sums of
// C, W and Bot and the per-warp staged W0_P rows with their sums.
static size_t panel_smem(size_t es) {
  const size_t y_phase = (size_t)(NB * 32 + 32 * 32) * es + (size_t)(NB * 32 + 32 * 32) * 8;
  const size_t bot_phase = (size_t)(NB * 32 + NB * NB + NB * 32) * es + (size_t)NB * 32 * 8 + (size_t)8 * 32 * (es + 8);
  return (y_phase > bot_phase ? y_phase : bot_phase) + (size_t)(NB + 32) * 4;
}

// ------------------------------------------------------------------ grouped forms
template <typename A>
__global__ void __launch_bounds__(256, 4)
    step_group_kernel(const GroupInst* __restrict__ inst, const GroupEntry* __restrict__ ent, int n, int op_mode) {
  __shared__ double csm[kStepWarps][kCsMax];
  const int64_t item = blockIdx.x;
  const int e = group_find(ent, n, item);
  const GroupInst* gi = inst + ent[e].inst;
  const StepArgs a = gi->a;
  const BlockedArgs t = gi->t;
  const int64_t b = (item - ent[e].start) * kStepWarps + (threadIdx.x >> 5);
  if (b >= a.bw) return;
  step_warp<A>(a, t, b, ent[e].k, op_mode, csm[threadIdx.x >> 5]);
}

template <typename A>
__global__ void __launch_bounds__(256)
    panel_s_group_kernel(const GroupInst* __restrict__ inst, const GroupEntry* __restrict__ ent, int n) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int64_t item = blockIdx.x;
  const int e = group_find(ent, n, item);
  const GroupInst* gi = inst + ent[e].inst;
  const StepArgs a = gi->a;
  const BlockedArgs t = gi->t;
  const int64_t k = ent[e].k;
  const int64_t k0 = (k / NB) * NB, k1 = min(k0 + NB, t.Nc);
  panel_s_body<A>(a, t, item - ent[e].start, k0, k1, smem_raw);
}

template <typename A>
__global__ void __launch_bounds__(256, 3)
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

// ------------------------------------------------------------------ launchers
#define FFS_DISPATCH_STATE(cplx, state, F, ...)                       \
  ((cplx) ? ((state) == kStateFP64   ? F<cd>(__VA_ARGS__)            \
             : (state) == kStateFP32 ? F<cf>(__VA_ARGS__)            \
                                     : F<cdf>(__VA_ARGS__))          \
          : ((state) == kStateFP64   ? F<double>(__VA_ARGS__)        \
             : (state) == kStateFP32 ? F<float>(__VA_ARGS__)         \
                                     : F<df>(__VA_ARGS__)))

template <typename A>
static cudaError_t step_t(const StepArgs& a, const BlockedArgs& t, int64_t k, int op, cudaStream_t s) {
  tail_step_kernel<A><<<(unsigned)((a.bw + kStepWarps - 1) / kStepWarps), 32 * kStepWarps, 0, s>>>(a, t, k, op);
  return cudaGetLastError();
}
template <typename A>
static cudaError_t panel_t(const StepArgs& a, const BlockedArgs& t, int64_t k0, int64_t k1, int op, cudaStream_t s) {
  tail_panel_s_kernel<A><<<(unsigned)a.bw, 256, panel_s_smem(sizeof(A)), s>>>(a, t, k0, k1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)((t.Nc - k1 + 31) / 32), (unsigned)a.bw);
  tail_panel_kernel<A><<<grid, 256, panel_smem(sizeof(A)), s>>>(a, t, k0, k1, op);
  return cudaGetLastError();
}
template <typename A>
static cudaError_t group_step_t(const GroupInst* inst, const GroupEntry* e, int n, int64_t total, int op,
                                cudaStream_t s) {
  step_group_kernel<A><<<(unsigned)total, 32 * kStepWarps, 0, s>>>(inst, e, n, op);
  return cudaGetLastError();
}
template <typename A>
static cudaError_t group_panel_s_t(const GroupInst* inst, const GroupEntry* e, int n, int64_t total, cudaStream_t s) {
  panel_s_group_kernel<A><<<(unsigned)total, 256, panel_s_smem(sizeof(A)), s>>>(inst, e, n);
  return cudaGetLastError();
}
template <typename A>
static cudaError_t group_panel_t(const GroupInst* inst, const GroupEntry* e, int n, int64_t total, int op,
                                 cudaStream_t s) {
  panel_group_kernel<A><<<(unsigned)total, 256, panel_smem(sizeof(A)), s>>>(inst, e, n, op);
  return cudaGetLastError();
}

// Operand of step k1 from the state's column k1 (all rows updated): h = (-W[:, k1] ; 1).
template <typename A>
__global__ void column_operand_kernel(StepArgs a, BlockedArgs t, int64_t k1, int op_mode) {
  using T = Ar<A>;
  const int64_t b = blockIdx.x;
  if (b >= a.bw || (a.nlen && a.nlen[b] <= k1)) return;
  const int64_t Nc = t.Nc;
  const A* W = (const A*)t.W + (size_t)b * state_stride(Nc);
  const int32_t* mrow = a.m + b * a.N;
  for (int64_t j = threadIdx.x; j <= k1; j += blockDim.x) {
    const A v = (j < k1) ? T::neg(W[sidx(j, k1)]) : T::one();
    put_state<A>(a, op_mode, b, operand_col(a, mrow, j), v);
  }
}

template <typename A>
static cudaError_t column_operand_t(const StepArgs& a, const BlockedArgs& t, int64_t k1, int op, cudaStream_t s) {
  column_operand_kernel<A><<<(unsigned)a.bw, 128, 0, s>>>(a, t, k1, op);
  return cudaGetLastError();
}

cudaError_t launch_column_operand(const StepArgs& a, const BlockedArgs& t, int64_t k1, int state, int op,
                                  cudaStream_t s) {
  if (a.bw <= 0) return cudaSuccess;
  return FFS_DISPATCH_STATE(a.cplx, state, column_operand_t, a, t, k1, op, s);
}

template <typename A>
static cudaError_t mcmc_t(const StepArgs& a, const BlockedArgs& t, int64_t k, int64_t m_cond, cudaStream_t s) {
  mcmc_step_kernel<A><<<(unsigned)((a.bw + kMcmcWarps - 1) / kMcmcWarps), 32 * kMcmcWarps,
                        (size_t)kMcmcWarps * a.N * sizeof(A), s>>>(a, t, k, m_cond);
  return cudaGetLastError();
}

cudaError_t launch_mcmc_step(const StepArgs& a, const BlockedArgs& t, int64_t k, int64_t m_cond, int state,
                             cudaStream_t s) {
  return FFS_DISPATCH_STATE(a.cplx, state, mcmc_t, a, t, k, m_cond, s);
}

size_t mcmc_step_smem(int64_t N, bool cplx, int state) {
  return (size_t)kMcmcWarps * N * blocked_elem_bytes(cplx, state);
}

cudaError_t launch_blocked_step(const StepArgs& a, const BlockedArgs& t, int64_t k, int state, int op,
                                cudaStream_t s) {
  return FFS_DISPATCH_STATE(a.cplx, state, step_t, a, t, k, op, s);
}

cudaError_t launch_blocked_panel(const StepArgs& a, const BlockedArgs& t, int64_t k0, int64_t k1, int state,
                                 int op, cudaStream_t s) {
  if (k1 >= t.Nc) return cudaSuccess;
  return FFS_DISPATCH_STATE(a.cplx, state, panel_t, a, t, k0, k1, op, s);
}

template <typename A>
static cudaError_t panel_s_only_t(const StepArgs& a, const BlockedArgs& t, int64_t k0, int64_t k1, cudaStream_t s) {
  tail_panel_s_kernel<A><<<(unsigned)a.bw, 256, panel_s_smem(sizeof(A)), s>>>(a, t, k0, k1);
  return cudaGetLastError();
}
template <typename A>
static cudaError_t panel_update_only_t(const StepArgs& a, const BlockedArgs& t, int64_t k0, int64_t k1, int op,
                                       cudaStream_t s) {
  dim3 grid((unsigned)((t.Nc - k1 + 31) / 32), (unsigned)a.bw);
  tail_panel_kernel<A><<<grid, 256, panel_smem(sizeof(A)), s>>>(a, t, k0, k1, op);
  return cudaGetLastError();
}

cudaError_t launch_blocked_panel_s(const StepArgs& a, const BlockedArgs& t, int64_t k0, int64_t k1, int state,
                                   cudaStream_t s) {
  if (k1 >= t.Nc) return cudaSuccess;
  return FFS_DISPATCH_STATE(a.cplx, state, panel_s_only_t, a, t, k0, k1, s);
}

cudaError_t launch_blocked_panel_update(const StepArgs& a, const BlockedArgs& t, int64_t k0, int64_t k1, int state,
                                        int op, cudaStream_t s) {
  if (k1 >= t.Nc) return cudaSuccess;
  return FFS_DISPATCH_STATE(a.cplx, state, panel_update_only_t, a, t, k0, k1, op, s);
}

cudaError_t launch_group_step(const GroupInst* inst, const GroupEntry* e, int n, int64_t total, bool cplx,
                              int state, int op, int64_t maxNc, cudaStream_t s) {
  (void)maxNc;
  if (total <= 0) return cudaSuccess;
  return FFS_DISPATCH_STATE(cplx, state, group_step_t, inst, e, n, total, op, s);
}

cudaError_t launch_group_panel_s(const GroupInst* inst, const GroupEntry* e, int n, int64_t total, bool cplx,
                                 int state, cudaStream_t s) {
  if (total <= 0) return cudaSuccess;
  return FFS_DISPATCH_STATE(cplx, state, group_panel_s_t, inst, e, n, total, s);
}

cudaError_t launch_group_panel(const GroupInst* inst, const GroupEntry* e, int n, int64_t total, bool cplx,
                               int state, int op, cudaStream_t s) {
  if (total <= 0) return cudaSuccess;
  return FFS_DISPATCH_STATE(cplx, state, group_panel_t, inst, e, n, total, op, s);
}

__global__ void state_copy_kernel(const void* U64, bool cplx, int state, int64_t count, void* out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    if (cplx) {
      const cd u = ((const cd*)U64)[e];
      if (state == kStateDF64)
        ((cdf*)out)[e] = cdf{df_from(u.re), df_from(u.im)};
      else
        ((cf*)out)[e] = cf{(float)u.re, (float)u.im};
    } else {
      const double u = ((const double*)U64)[e];
      if (state == kStateDF64)
        ((df*)out)[e] = df_from(u);
      else
        ((float*)out)[e] = (float)u;
    }
  }
}

cudaError_t launch_derive_state_copy(const void* U64, bool cplx, int state, int64_t count, void* out, cudaStream_t s) {
  state_copy_kernel<<<1024, 256, 0, s>>>(U64, cplx, state, count, out);
  return cudaGetLastError();
}

size_t blocked_elem_bytes(bool cplx, int state) {
  const size_t base = (state == kStateFP32) ? 4 : 8;  // FP64 and double-float are both 8 bytes
  return cplx ? 2 * base : base;
}

int blocked_panel_width() { return NB; }
int blocked_step_samples_per_cta() { return kStepWarps; }

size_t blocked_step_smem(int64_t Nc, bool cplx, int state) {
  (void)Nc;
  return panel_smem(blocked_elem_bytes(cplx, state));
}

template <typename K> static cudaError_t allow_smem(K kernel, int optin) {
  cudaFuncAttributes at;
  cudaError_t e = cudaFuncGetAttributes(&at, kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)at.sharedSizeBytes);
}

template <typename A> static cudaError_t allow_all(int optin) {
  cudaError_t e = allow_smem(tail_panel_s_kernel<A>, optin);
  if (e == cudaSuccess) e = allow_smem(tail_panel_kernel<A>, optin);
  if (e == cudaSuccess) e = allow_smem(panel_s_group_kernel<A>, optin);
  if (e == cudaSuccess) e = allow_smem(panel_group_kernel<A>, optin);
  if (e == cudaSuccess) e = allow_smem(mcmc_step_kernel<A>, optin);
  return e;
}

cudaError_t configure_blocked() {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess) e = allow_all<double>(optin);
  if (e == cudaSuccess) e = allow_all<float>(optin);
  if (e == cudaSuccess) e = allow_all<df>(optin);
  if (e == cudaSuccess) e = allow_all<cd>(optin);
  if (e == cudaSuccess) e = allow_all<cf>(optin);
  if (e == cudaSuccess) e = allow_all<cdf>(optin);
  return e;
}

}  // namespace fermi
