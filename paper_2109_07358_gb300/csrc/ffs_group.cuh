// Grouped launches: one kernel launch serves many independent sampling instances
// (different U, L, N, sample counts, each at its own step).  Work items of a launch
// are numbered 0..total-1; a sorted entry list maps item ranges to (instance, step),
// and each CTA finds its entry by binary search.
#pragma once

#include "ffs_kernels.cuh"
#include "ffs_residual_tc.cuh"

namespace fermi {

struct GroupEntry {
  int64_t start;  // first work item of this entry
  int32_t inst;   // index into the instance table
  int32_t k;      // step of that instance this launch serves
};

// Everything a CTA needs about one instance.  64-byte aligned: the tensor maps are
// read by TMA straight from global memory.
struct alignas(64) GroupInst {
  CUtensorMap tm[4];   // H hi, H lo, Ue hi, Ue lo
  StepArgs a;
  BlockedArgs t;
  TcArgs tc;
  int64_t n_jtiles;    // residual tiles along the embedding columns
  int64_t n_btiles;    // residual tiles along the samples
  int64_t bn;          // residual column tile of this instance (128 or 256)
};

__device__ __forceinline__ int group_find(const GroupEntry* __restrict__ e, int n, int64_t item) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (e[mid].start <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Items per instance: init ceil(bw/128) CTAs; residual n_btiles*n_jtiles; step
// ceil(bw/8) (a warp per sample); panel S bw; panel bw * ceil((Nc - k1)/32).
cudaError_t launch_group_init(const GroupInst* inst, const GroupEntry* e, int n, int64_t total, int op,
                              cudaStream_t s);
cudaError_t launch_group_residual(const GroupInst* inst, const GroupEntry* e, int n, int64_t total, int op, int bn,
                                  cudaStream_t s);
cudaError_t launch_group_step(const GroupInst* inst, const GroupEntry* e, int n, int64_t total, bool cplx,
                              int state, int op, int64_t maxNc, cudaStream_t s);
cudaError_t launch_group_panel_s(const GroupInst* inst, const GroupEntry* e, int n, int64_t total, bool cplx,
                                 int state, cudaStream_t s);
cudaError_t launch_group_panel(const GroupInst* inst, const GroupEntry* e, int n, int64_t total, bool cplx,
                               int state, int op, cudaStream_t s);
cudaError_t configure_group();

}  // namespace fermi
