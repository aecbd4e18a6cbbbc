/*
 * ffs.h - C ABI of the GB300 fast-fermion-sampling library (libffs.so).
 *
 * Fast fermion sampling (FFS), Sun, Zou & Li, arXiv 2109.07358.  Given an L x N
 * matrix U with orthonormal columns (U^dagger U = 1), draw ordered configurations
 * x = (x_1..x_N), x_j in {0..L-1}, from P(x) = |det U_{x,n}|^2 / N!   (Eq. 1).
 * Each sample draws its own uniformly random column order m and then places one
 * fermion per step k by the chain rule (Eq. 2); the conditional weight of site y at
 * step k is |u_y^T h|^2 with h the normal vector of Eq. 3, evaluated for all L sites
 * at once (Supplementary Section S-1).
 *
 * Conventions shared by every entry point
 *   - Every call returns an ffs_status; FFS_OK is 0.  The message of the last error
 *     of a handle is ffs_last_error(handle).
 *   - Sites and columns are 0-based (the paper is 1-based).  Matrices are row-major.
 *   - Pointers may be host or device memory unless stated; the library tells them
 *     apart with cudaPointerGetAttributes.  Host output buffers are written before
 *     the call returns; device output buffers are written in stream order.
 *   - Sample b of a call is fully determined by (U, seed, first_sample_index + b,
 *     the precision flags): it does not depend on B, on how a batch is split into
 *     waves, or on other work sharing the GPU.
 *   - Random numbers: Philox4x32-10 (Salmon et al., SC'11) with key (seed lo32,
 *     seed hi32) and counter (block, stream, sample lo32, sample hi32).  Stream 0
 *     drives a Fisher-Yates shuffle that gives m; stream 1, block k gives the
 *     53-bit uniform of step k.
 *   - Device-detected numeric failures (a non-finite or non-positive normaliser, a
 *     vanishing pivot) are recorded in a status word that ffs_sync returns.
 *   - Nothing here traps or hangs the GPU: every device-side wait is bounded and
 *     reports FFS_E_TIMEOUT instead.
 */
#ifndef FFS_H
#define FFS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ffs_ctx* ffs_handle;

typedef enum {
  FFS_OK = 0,
  FFS_E_ARG = 1,              /* invalid argument (sizes, null pointers, flags)        */
  FFS_E_NOT_ORTHONORMAL = 2,  /* max |U^dagger U - 1| above the tolerance (Eq. 1 text)  */
  FFS_E_NOMEM = 3,            /* device allocation failed or budget exceeded            */
  FFS_E_CUDA = 4,             /* a CUDA runtime call failed (message in ffs_last_error) */
  FFS_E_NUMERIC = 5,          /* normaliser <= 0 or non-finite, or |pivot|^2 < 1e-300   */
  FFS_E_TIMEOUT = 6,          /* a bounded wait ran out                                 */
  FFS_E_BUSY = 7,             /* the engine cannot take the request now                 */
  FFS_E_UNSUPPORTED = 8       /* option not available in this build / on this device    */
} ffs_status;

/* Element type of U as passed to ffs_create_ex. */
typedef enum {
  FFS_F64 = 0,   /* double, L x N                        */
  FFS_C128 = 1,  /* interleaved (re, im) double pairs    */
  FFS_F32 = 2,   /* float                                */
  FFS_C64 = 3    /* interleaved (re, im) float pairs     */
} ffs_dtype;

/* Flags of ffs_create_ex (bitwise OR of one value from each group).
 *
 * Residual arithmetic (the all-site inner products u_y^T h of step k):
 *   FFS_RES_FP32    FP32 CUDA-core arithmetic                 (the "FP32 path")
 *   FFS_RES_BF16X3  tensor cores, operands split into BF16 hi+lo, three products
 *                   hi*hi + hi*lo + lo*hi, FP32 accumulation   (default)
 *   FFS_RES_BF16    tensor cores, one BF16 product, FP32 accumulation
 *   FFS_RES_TF32    tensor cores, one TF32 product, FP32 accumulation
 * Per-sample elimination state (the normal vector h, the pivots):
 *   FFS_STATE_FP64  IEEE double                                 (default)
 *   FFS_STATE_DF64  double-float: pairs of FP32 numbers, about 48 significant bits,
 *                   computed on the FP32 pipes (FP64-class precision)
 *   FFS_STATE_FP32  IEEE float (used by the plain form)
 * State update schedule:
 *   (default)           blocked: per step the new row is reduced on a 32-column panel,
 *                       the remaining columns are updated once per panel
 *   FFS_TAIL_UNBLOCKED  every step updates all remaining columns (FP64 or FP32 state)
 * Form:
 *   FFS_FORM_BATCHED  all samples of a wave share one contraction per step (default)
 *   FFS_FORM_PLAIN    the plain per-sample form: per sample, an FP32 CUDA-core
 *                     product with the columns U[:, m_1..m_k] and an FP32 state
 *   FFS_FORM_GROUPED  opt-in: the 128 samples of each group share one column order m, so
 *                     that step k contracts only the k+1 leading columns of the group's
 *                     order (K = k+1: the paper's 2Lk count instead of 2LN).  A group is
 *                     the 128 consecutive sample indices starting at a multiple of 128;
 *                     its m is the one the group's first index would draw alone.  Each
 *                     sample still follows P(x) exactly, but samples of a group are
 *                     dependent through their shared m.  Needs a tensor-core residual
 *                     (BF16x3, BF16 or TF32) and the blocked state; first_sample_index must
 *                     be a multiple of 128; not available to ffs_sample_batched, the serving
 *                     engine, ffs_sample_lensemble or ffs_sample_metropolis.
 * Trailing update:
 *   FFS_TRAILING_TC  opt-in: the once-per-panel trailing update (the new rows
 *                    Y = U[x_new, m_T] - C W0_T with Bot = S^-1 Y, and the old rows
 *                    Top = W0_T - W0_P Bot) runs on the tensor cores through a split of the
 *                    double-float operands into six BF16 slices each (slice products exact
 *                    in FP32 accumulation, each block's product within 2^-46 of its scales
 *                    times K).  FFS_STATE_DF64, the blocked state and a tensor-core
 *                    residual only (else FFS_E_UNSUPPORTED at creation).  Real and complex
 *                    U; the benchmark's chosen form.
 * Checks:
 *   FFS_NO_ORTHO_CHECK  skip the U^dagger U = 1 check in ffs_create_ex
 */
#define FFS_RES_BF16X3 0x0u
#define FFS_RES_FP32 0x1u
#define FFS_RES_BF16 0x2u
#define FFS_RES_TF32 0x3u
#define FFS_RES_MASK 0xFu
#define FFS_STATE_FP64 0x00u
#define FFS_STATE_FP32 0x10u
#define FFS_STATE_DF64 0x20u
#define FFS_STATE_MASK 0xF0u
#define FFS_FORM_BATCHED 0x000u
#define FFS_FORM_PLAIN 0x100u
#define FFS_FORM_GROUPED 0x200u
#define FFS_GROUP_SIZE 128
#define FFS_FORM_MASK 0xF00u
#define FFS_NO_ORTHO_CHECK 0x1000u
#define FFS_TAIL_UNBLOCKED 0x2000u
#define FFS_TRAILING_TC 0x4000u

/* Tolerance of the orthonormality check: max_ij |(U^dagger U)_ij - delta_ij|. */
#define FFS_ORTHO_TOL 1e-6

/*
 * ffs_create - set up a sampler for one U (Eq. 1: L x N, U^dagger U = 1).
 *   U     real FP64, row-major L x N (leading dimension N), host or device memory.
 *         The library copies it; the caller keeps ownership and may free it on return.
 *   L, N  1 <= N <= L.
 *   out   receives the handle (owning all device memory it allocates).
 * Equivalent to ffs_create_ex(U, FFS_F64, L, N, N, 0, NULL, out).  Synchronous.
 * Errors: FFS_E_ARG, FFS_E_NOT_ORTHONORMAL, FFS_E_NOMEM, FFS_E_CUDA.
 */
int ffs_create(const double* U, int64_t L, int64_t N, ffs_handle* out);

/*
 * ffs_create_ex - as ffs_create with an element type, a leading dimension ldU >= N
 * (in elements), flags (above) and a CUDA stream (cudaStream_t, NULL = legacy default
 * stream) on which every later call of this handle is ordered.  A device U is read on
 * that stream: work that produces it on another stream must be complete or ordered
 * before it (e.g. with an event).
 */
int ffs_create_ex(const void* U, int dtype, int64_t L, int64_t N, int64_t ldU, unsigned flags,
                  void* cuda_stream, ffs_handle* out);

/*
 * ffs_sample - draw B configurations (Eq. 1 via the chain of Eq. 2-3).
 *   B      number of samples, B >= 0 (B = 0 is a no-op).
 *   seed   Philox key; sample b uses sample index b.
 *   out_x  B x N int32, row-major, sites in draw order (x_1..x_N); host or device.
 * Asynchronous on the handle's stream when out_x is device memory; device-detected
 * errors surface at ffs_sync or at the next call.
 */
int ffs_sample(ffs_handle h, int64_t B, uint64_t seed, int32_t* out_x);

/*
 * ffs_sample_ex - ffs_sample with options.
 *   first_sample_index  sample b uses index first_sample_index + b (disjoint index
 *                       ranges give independent samples; this is how a job is sharded).
 *   n_steps             fermions to place, 1..N (N = the full configuration; fewer
 *                       gives the marginal of the first n_steps positions, the
 *                       paper's marginal-sampling case).  0 means N.
 *   out_x               B x n_steps int32 (host or device).
 *   out_perm            nullable; B x N int32 column orders m.
 *   out_logp            nullable; B doubles, log of the chain's probability of x
 *                       given m (sum over steps of log(|s_k|^2 / Z_k)).
 *   force_x             nullable; B x n_steps int32 teacher-forcing sites: step k
 *                       places force_x[b][k] instead of drawing (weights are still
 *                       evaluated).  Used to compare conditionals step by step.
 *   out_probs           nullable; B x n_steps x L float32, the normalised conditional
 *                       of every step (debug/parity output; large).
 *   cuda_stream         NULL = the handle's stream.
 */
int ffs_sample_ex(ffs_handle h, int64_t B, uint64_t seed, uint64_t first_sample_index,
                  int64_t n_steps, int32_t* out_x, int32_t* out_perm, double* out_logp,
                  const int32_t* force_x, float* out_probs, void* cuda_stream);

/* ffs_sync - wait for the handle's stream; return and clear the device status word. */
int ffs_sync(ffs_handle h);

/* ffs_last_error - message of the last failed call on h (never NULL; h may be NULL). */
const char* ffs_last_error(ffs_handle h);

/* ffs_destroy - release everything the handle owns.  NULL-safe. */
void ffs_destroy(ffs_handle h);

/* ffs_query - sizes and settings of a handle: L, N, dtype, flags, and the device bytes
 * a batch of B samples needs (the per-sample state, the operands, the buffers). */
int ffs_query(ffs_handle h, int64_t* L, int64_t* N, int* dtype, unsigned* flags,
              int64_t B, int64_t* bytes_for_B);

/*
 * ffs_sample_noalloc - draw B configurations without allocating any device memory.
 * The paper has no counterpart: this entry point is for callers that cannot allocate
 * device memory at the moment they sample, such as code running inside a memory pool
 * that has been sized and frozen, a framework whose caching allocator must not be
 * bypassed, or a plugin that may only touch the memory it is handed.  ffs_create
 * allocates (copies of U, per-wave working memory), so such callers use this call
 * instead.  All working memory comes from one fixed array of FFS_NOALLOC_SCRATCH_BYTES
 * in device global memory that the library declares statically: every GPU that loads
 * the library holds that memory until the process exits.
 *   U          device (or managed) pointer, row-major L x N, dtype FFS_F64 or FFS_C128
 *              (U^dagger U = 1 is assumed, not checked).  Host memory is FFS_E_ARG.
 *   L, N, B    1 <= N <= L, B >= 0 samples; sample b uses Philox sample index b.
 *   seed       Philox key, as in ffs_sample.
 *   out_x      device (or managed) pointer, B x N int32, sites in draw order.  A sample
 *              whose chain reaches a degenerate step (no site with a positive finite
 *              weight, a non-finite or zero normaliser, or a vanishing pivot) has -1 from
 *              that step to the end of its row: there is no status word, so -1 is how a
 *              caller detects it.
 *   cuda_stream  cudaStream_t or NULL.
 * The samples equal those of ffs_sample_ex with FFS_RES_FP32 | FFS_STATE_FP64 |
 * FFS_TAIL_UNBLOCKED (the same arithmetic in the same order, fused into one kernel;
 * meant for small problems).
 * A size whose working set (about B (8 N^2 + 4 L + 8 N) bytes, twice the N^2 term for
 * complex U; at least 288 bytes per sample) does not fit the array is rejected with
 * FFS_E_NOMEM and a message naming the limit.  The first call on a device looks up the array's device address; make that
 * first call before any stream capture.  Every call works in the same array, which
 * keeps the previous call's contents (the kernel clears what must start at zero), so
 * calls that overlap on the GPU, from different streams or threads, race.  Asynchronous;
 * returns argument and launch errors only (there is no device status word).
 */
#define FFS_NOALLOC_SCRATCH_BYTES (16u << 20)
int ffs_sample_noalloc(const void* U, int dtype, int64_t L, int64_t N, int64_t B, uint64_t seed,
                       int32_t* out_x, void* cuda_stream);

/*
 * ffs_sample_lensemble - draw B samples of the L-ensemble DPP whose correlation matrix is
 * C = sum_j lambda_j u_j u_j^dagger (main text, text-summarisation example): each
 * eigenvector u_j (column j of the handle's U, so U holds the eigenvectors of C with
 * nonzero eigenvalue, orthonormal) is kept with probability lambda_j / (lambda_j + 1),
 * and the kept columns form the U of Eq. 1, sampled by the chain rule with N = the
 * number kept.  Sample b is keyed like ffs_sample_ex; its keep decision for column j
 * uses Philox stream 2, block j (a 53-bit uniform built like the site uniforms; kept
 * when it is below lambda_j / (lambda_j + 1), never when lambda_j <= 0).  The kept
 * columns in ascending order are then shuffled by the stream-0 Fisher-Yates shuffle
 * over their count.  All samples advance together for as many steps as the longest
 * chain; shorter chains stop early.
 *   lambda     host or device, N eigenvalues (a non-finite value is FFS_E_ARG).
 *   out_x      device, B x N int32: the n_b sites of sample b in draw order, then -1.
 *   out_n      device, B int32, or NULL: n_b, the number of kept eigenvectors.
 *   out_perm   device, B x N int32, or NULL: the kept columns in the order the chain
 *              used them, then the other columns ascending.
 *   out_logp   device, B doubles, or NULL: log of the chain's probability of x given
 *              the kept columns and their order (0 for an empty sample).
 *   force_x    device, B x N int32, or NULL: teacher forcing of the first n_b entries.
 *   out_probs  device, B x N x L float, or NULL: the normalised conditionals (zero rows
 *              past n_b).
 * Needs a handle in the batched form with the blocked state (the default flags), else
 * FFS_E_UNSUPPORTED.  The call reads the longest chain length back to the host
 * (it synchronises cuda_stream once, before the sampling launches).
 */
int ffs_sample_lensemble(ffs_handle h, const double* lambda, int64_t B, uint64_t seed,
                         uint64_t first_sample_index, int32_t* out_x, int32_t* out_n, int32_t* out_perm,
                         double* out_logp, const int32_t* force_x, float* out_probs, void* cuda_stream);

/*
 * ffs_sample_metropolis - the large-L (and continuous-model) variant of Supplementary
 * Section S-7: the column order m is drawn as usual, but x_k is drawn by a Metropolis
 * chain of m_cond updates over sites instead of from all L conditional weights, so a
 * step costs O(m_cond N + N k) and the sample O(m_cond N^2 + N^3), independent of L.
 * The chain of step k starts at a uniform site and proposes uniform sites y'; a move
 * y -> y' is accepted when u |u_y^T h|^2 < |u_{y'}^T h|^2 (the ratio of S-7; drawn sites
 * have weight 0, so a chain that starts on one leaves it at the first proposal with
 * weight).  Random numbers: Philox stream 3, block k (m_cond + 1) + t for iteration t
 * (t = 0: the starting site): words 0-1 give the site floor(r L / 2^64) of their 64-bit
 * concatenation r, words 2-3 a 53-bit uniform built like the site uniforms.  The result
 * is exact only as m_cond grows (the chain must equilibrate; the paper leaves m_cond to
 * the user).  A chain that ends on a site of weight 0 sets FFS_E_NUMERIC.
 *   n_steps   fermions to place (0 = N), as ffs_sample_ex.
 *   m_cond    Metropolis updates per step, >= 0; n_steps x (m_cond + 1) < 2^32.
 *   out_x     device, B x n_steps int32, sites in draw order.
 *   out_perm  device, B x N int32, or NULL: column orders m.
 * Needs a handle with the blocked state (default flags; the residual flags are unused).
 * Asynchronous on cuda_stream; device errors surface at ffs_sync.
 */
int ffs_sample_metropolis(ffs_handle h, int64_t B, uint64_t seed, uint64_t first_sample_index, int64_t n_steps,
                          int64_t m_cond, int32_t* out_x, int32_t* out_perm, void* cuda_stream);

/*
 * ffs_sample_batched - sample many independent instances together (the batching
 * pattern: many U of uneven L and N).  Instance i draws Bs[i] samples of handle hs[i]
 * with seed seeds[i] (sample indices 0..Bs[i]-1) into the device buffer outs[i]
 * (Bs[i] x N_i int32).  All instances advance step by step through grouped launches
 * (one kernel launch serves every instance still running), and the whole schedule is
 * captured once into a CUDA graph and launched as one graph on cuda_stream.  The
 * samples are identical to separate ffs_sample calls.  All handles must use the batched
 * tensor-core form with the blocked state, the same flags and the same real/complex
 * type; a handle may appear once; every instance's wave must fit in memory at once.
 * Asynchronous; errors of the set-up are returned, device errors surface at ffs_sync
 * of the handles.
 */
int ffs_sample_batched(ffs_handle* hs, const int64_t* Bs, const uint64_t* seeds, int32_t** outs, int n,
                       void* cuda_stream);

/*
 * Serving engine (continuous batching).  Requests with their own U, L, N, sample count
 * and seed arrive at any time (ffs_submit copies U, so the caller may free it on
 * return).  A host thread admits queued requests in arrival order while their device
 * footprint (copies of U, operand, per-sample state and buffers) fits the HBM budget
 * and an active slot is free; every engine iteration advances each active request by
 * one step with grouped launches, so requests at different steps share the GPU and a
 * new request starts while older ones are mid-chain.  A request's samples are the same
 * as a standalone ffs_sample of its U and seed.  ffs_wait blocks until the request is
 * done (timeout_ms < 0: no limit; FFS_E_TIMEOUT when it runs out) and reports the
 * latency from submission to completion.
 *   hbm_budget   bytes the engine may hold for requests; 0 = 80% of free memory.
 *   flags        as ffs_create_ex; the tensor-core residual and the blocked state.
 *   max_active   requests in flight at once (<= 0: no limit besides memory).
 *   out_x        host or device, n_samples x N int32, written before ffs_wait returns.
 */
typedef struct ffs_server ffs_server;
int ffs_server_create(size_t hbm_budget, unsigned flags, int max_active, void* cuda_stream, ffs_server** out);
int ffs_submit(ffs_server* s, const void* U, int dtype, int64_t L, int64_t N, int64_t n_samples, uint64_t seed,
               int32_t* out_x, uint64_t* req_id);
int ffs_wait(ffs_server* s, uint64_t req_id, int timeout_ms, double* latency_ms);
/* ffs_server_stats - queued and active requests, engine iterations so far, device bytes
 * held for requests, and peak_active: the most requests one engine iteration advanced
 * (requests advanced together share every launch of that iteration).  Any pointer may be
 * NULL. */
int ffs_server_stats(ffs_server* s, int64_t* pending, int64_t* active, int64_t* iterations, size_t* bytes_in_use,
                     int64_t* peak_active);
void ffs_server_destroy(ffs_server* s);

/*
 * Slater-Jastrow reweighting (Supplementary Section S-5; Eq. 4 of the main text).
 *
 * A Jastrow state |psi_J> = J |phi_0>, J(x) = exp(-1/2 sum_ij v_ij n_i n_j), is not a
 * determinant, but J is diagonal in the configuration basis, so expectations in it follow
 * from samples x_b of the free-fermion state |phi_0> (drawn by ffs_sample) by reweighting:
 *   <O>_J = <J^2 o_L>_0 / <J^2>_0,   J^2(x) = exp(-n^T v n).
 * Observables are those diagonal in the configuration basis, whose local value is
 *   o_L(x) = sum_i o_i n_i + sum_ij q_ij n_i n_j
 * (densities, double occupancy, density-density correlations).
 *
 * Orbitals are the rows of U: for spinful fermions, sample each spin species with its
 * own handle and offset the down-spin indices by the number of sites, so that the
 * Gutzwiller factor of Eq. 4 is v_{i, L+i} = v_{L+i, i} = V/2.
 *
 *   x          device, B x n_occ int32, each row n_occ distinct orbitals in [0, n_orb)
 *              in any order (an ffs_sample output, or several side by side).
 *   v, q       sparse n_orb x n_orb matrices (struct below, all arrays device memory) or
 *              NULL; the cost per sample is the summed row lengths of its orbitals, so
 *              the Gutzwiller factor costs one entry per orbital and a dense matrix n_orb.
 *   o          device, n_orb doubles, or NULL.
 *   out_logj2  device, B doubles, or NULL: log J^2(x_b) per sample.
 *   out_obs    device, B doubles, or NULL: o_L(x_b) per sample.
 *   result     host or device, 4 doubles: <O>_J; log <J^2>_0; the effective sample size
 *              (sum w)^2 / sum w^2 of the weights w_b = J^2(x_b); and the first-order
 *              standard error sqrt(sum_b w_b^2 (o_L(x_b) - <O>_J)^2) / sum_b w_b.
 * Reductions run in a fixed order, so equal inputs give equal results.  The call
 * allocates stream-ordered scratch (2B + 4 doubles), runs on cuda_stream and
 * synchronises it before returning.  FFS_E_ARG if a row of x names an orbital twice or
 * outside [0, n_orb), or a CSR row pointer or column is out of range (the message is in
 * ffs_last_error(NULL)); n_orb is limited to 1638400 (one bitmap per sample in shared
 * memory).
 */
typedef struct {
  const int64_t* rowptr; /* n_orb + 1 entries, non-decreasing, rowptr[n_orb] <= nnz */
  const int32_t* col;    /* nnz column indices in [0, n_orb)                       */
  const double* val;     /* nnz values                                             */
  int64_t nnz;
} ffs_csr;
int ffs_jastrow_estimate(const int32_t* x, int64_t B, int64_t n_occ, int64_t n_orb, const ffs_csr* v,
                         const double* o, const ffs_csr* q, double* out_logj2, double* out_obs, double* result,
                         void* cuda_stream);

/*
 * ffs_debug_inject - failure-path testing.  Arms a one-shot fault for the next
 * tensor-core residual launch of h (the paper has no counterpart: this exercises the
 * library's bounded waits).  FFS_FAULT_SKIP_ARRIVAL: the TMA producer of that launch's
 * first CTA skips its first pipeline stage (no arrival, no copy) and every wait of the
 * launch gives up after 4096 polls instead of 262144 (a poll suspends the waiting thread
 * for at most 100 microseconds), so the MMA issuer's wait
 * runs out, the launch records FFS_E_TIMEOUT in the status word (ffs_sync returns it)
 * and every role of the CTA leaves without a copy in flight and with its tensor memory
 * freed.  The samples of that call are invalid; the handle stays usable and its next
 * call samples normally.  Nothing faults, traps or hangs the GPU.  FFS_FAULT_NONE
 * disarms.  FFS_E_UNSUPPORTED for a handle without a tensor-core residual.
 */
#define FFS_FAULT_NONE 0
#define FFS_FAULT_SKIP_ARRIVAL 1
int ffs_debug_inject(ffs_handle h, int fault);

/* Phases reported by ffs_profile_read. */
#define FFS_PHASE_PERM 0      /* column orders m and the step-0 operand              */
#define FFS_PHASE_RESIDUAL 1  /* all-site weights |u_y^T h|^2 (Section S-1 products) */
#define FFS_PHASE_TAIL 2      /* draw, pivot and per-step elimination-state update   */
#define FFS_PHASE_PANEL 3     /* once-per-panel update of the remaining state columns */
#define FFS_PHASE_PANEL_S 4   /* once-per-panel Schur complement and its inverse      */
#define FFS_PHASE_PANEL_TC 5  /* FFS_TRAILING_TC: slices and tensor-core old-row update */
#define FFS_NUM_PHASES 6

/*
 * ffs_profile - enable (1) or disable (0) per-phase timing of h: every kernel launch
 * of h is bracketed by two CUDA events on its stream.  Enabling clears the totals.
 * ffs_profile_read - synchronise, fold the recorded events into per-phase totals and
 * return them: ms[p] total device milliseconds and launches[p] kernel launches of phase
 * p since profiling was enabled (arrays of n entries, n <= FFS_NUM_PHASES).
 */
int ffs_profile(ffs_handle h, int enable);
int ffs_profile_read(ffs_handle h, double* ms, int64_t* launches, int n);

#ifdef __cplusplus
}
#endif

#endif /* FFS_H */
