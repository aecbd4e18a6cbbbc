// The draw of step k for one sample, executed by one 256-thread CTA, and its outputs.
//
// Normaliser Z and inverse CDF with a warp-shuffle block scan: warp w owns a contiguous
// segment of sites; segment totals give each warp its base; each warp then walks its
// segment 32 sites at a time with an inclusive shuffle scan until the running sum
// passes t = u Z.  x_k is the first site with a nonzero weight whose running sum
// exceeds t; if rounding leaves none, the last site with a nonzero weight.  The order
// of every sum is fixed, so a sample's draw never depends on the batch it runs in.
#pragma once

#include <climits>

#include "ffs_kernels.cuh"

namespace fermi {

struct DrawShared {
  double wsum[8], wbase[8];
  int cand[8];
  int x;
  double Z;
};

__device__ __forceinline__ double draw_warp_sum(double v) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double draw_warp_scan(double v, int lane) {
  for (int o = 1; o < 32; o <<= 1) {
    const double t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Returns x_k (the same value in every thread).  force >= 0 places that site instead
// (teacher forcing); force == -2 marks an invalid forced site (recorded as FFS_E_ARG).
__device__ __forceinline__ int block_draw(const float* __restrict__ prow, int64_t L, uint64_t seed,
                                          uint64_t sample, int64_t k, int force, int* status, DrawShared& sh,
                                          double& Z_out) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t seg = ((L + 255) / 256) * 32;
  const int64_t w0 = min(L, (int64_t)warp * seg), w1 = min(L, w0 + seg);
  double ws = 0.0;
  for (int64_t i = w0 + lane; i < w1; i += 32) ws += (double)prow[i];
  ws = draw_warp_sum(ws);
  if (lane == 0) sh.wsum[warp] = ws;
  __syncthreads();
  if (tid == 0) {
    double acc = 0.0;
    for (int w = 0; w < 8; ++w) {
      sh.wbase[w] = acc;
      acc += sh.wsum[w];
    }
    sh.Z = acc;
  }
  __syncthreads();
  const double Z = sh.Z;
  Z_out = Z;
  if (force != -1) {
    if (force < 0 || force >= L) {
      if (tid == 0) set_status(status, FFS_E_ARG);
      return 0;
    }
    return force;
  }
  const double t = site_uniform(seed, sample, (int)k) * Z;
  int cand = INT_MAX;
  double carry = sh.wbase[warp];
  for (int64_t i0 = w0; i0 < w1; i0 += 32) {
    const int64_t i = i0 + lane;
    const double v = (i < w1) ? (double)prow[i] : 0.0;
    const double inc = draw_warp_scan(v, lane);
    const unsigned hit = __ballot_sync(0xffffffffu, (i < w1) && v > 0.0 && (carry + inc > t));
    if (hit) {
      cand = (int)(i0 + __ffs(hit) - 1);
      break;
    }
    carry += __shfl_sync(0xffffffffu, inc, 31);
  }
  if (lane == 0) sh.cand[warp] = cand;
  __syncthreads();
  if (tid == 0) {
    int xs = INT_MAX;
    for (int w = 0; w < 8; ++w) xs = min(xs, sh.cand[w]);
    sh.x = xs;
  }
  __syncthreads();
  int x = sh.x;
  if (x == INT_MAX) {  // rounding left no site above t: the last site with weight
    int last = -1;
    for (int64_t i = tid; i < L; i += blockDim.x)
      if (prow[i] > 0.f) last = (int)i;
    for (int o = 16; o; o >>= 1) last = max(last, __shfl_xor_sync(0xffffffffu, last, o));
    if (lane == 0) sh.cand[warp] = last;
    __syncthreads();
    if (tid == 0) {
      int l = -1;
      for (int w = 0; w < 8; ++w) l = max(l, sh.cand[w]);
      sh.x = l;
    }
    __syncthreads();
    x = sh.x;
    if (x < 0) {
      if (tid == 0) set_status(status, FFS_E_NUMERIC);
      x = 0;
    }
  }
  return x;
}

// x_k, the chosen-site mask, log-probability and (optionally) the conditional.
__device__ __forceinline__ void draw_outputs(const StepArgs& a, int64_t b, int64_t k, int x, double Z,
                                             const float* __restrict__ prow) {
  const int tid = threadIdx.x;
  if (tid == 0) {
    a.x[b * a.ldx + k] = x;
    a.mask[b * a.ldMask + (x >> 5)] |= 1u << (x & 31);
    const double px = (double)prow[x];
    a.logp[b] += (px > 0.0 && Z > 0.0) ? log(px / Z) : -INFINITY;
    if (!(Z > 0.0) || !isfinite(Z)) set_status(a.status, FFS_E_NUMERIC);
  }
  if (a.probs) {
    float* pr = a.probs + ((size_t)b * a.ldx + k) * a.L;
    const double iz = Z > 0.0 ? 1.0 / Z : 0.0;
    for (int64_t i = tid; i < a.L; i += blockDim.x) pr[i] = (float)((double)prow[i] * iz);
  }
}

__device__ __forceinline__ int forced_site(const StepArgs& a, int64_t b, int64_t k) {
  if (!a.force_x) return -1;
  const int f = a.force_x[b * a.ldx + k];
  return (f < 0 || f >= a.L) ? -2 : f;
}

}  // namespace fermi
