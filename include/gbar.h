/*
 * gbar.h -- C ABI of the GB300 (sm_103a) library for parallel
 * acceptance-rejection (AR) selection of the next reaction to occur in the
 * Stochastic Simulation Algorithm (Neri & Mestivier, 2014).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Pointers named d_* are caller-owned DEVICE memory; h_* are host memory.
 *   The library never allocates in these calls and keeps no pointer after
 *   the call returns (the network handle of the SSA calls is the exception:
 *   it owns device copies of the network until ssa_net_destroy).
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  Every call is asynchronous with respect to the host: it
 *   validates its arguments, enqueues kernels and returns.
 * - Return value: AR_OK (0) or a negative AR_ERR_* code for an error found
 *   on the host before anything was enqueued (AR_ERR_CUDA: a launch failed;
 *   cudaGetLastError() has been consumed and its code is returned by
 *   ar_last_cuda_error()).
 * - Conditions found on the device are OR-ed into the caller's uint32_t
 *   status word(s) as AR_STATUS_* bits; the caller zeroes them beforehand
 *   and reads them back when it wants them.
 * - Indices are 0-based.  The rejection sentinel is M (the paper's M+1,
 *   Section "Implementation", made 0-based).
 * - dtype: AR_F32 or AR_F64 propensities.  cmp: AR_CMP_F32 (comparison in
 *   FP32, bulk fast path) or AR_CMP_F64 (the exact FP64 test below; the
 *   kernels decide it in FP32 wherever proven error margins make that the
 *   FP64 decision and run the FP64 product for the rest, about one trial in
 *   10^5, so its results are those of the FP64 test exactly).
 *
 * The random stream (bit-exact contract, Philox4x32-10, Salmon et al. SC'11)
 * -----------------------------------------------------------------------
 * key = (seed mod 2^32, seed / 2^32).  Trial t (t = 0, 1, ...) of selection s
 * of realization b reads the Philox block of counter (t/2, s, b, 0) and, in
 * it, words 2(t mod 2) (candidate) and 2(t mod 2)+1 (uniform):
 *     j = floor(w_a * M / 2^32)
 *     FP64 comparison: accept iff fl64((w_b * 2^-32) * T) < alpha_j
 *     FP32 comparison: accept iff fl32((floor(w_b/2^8) * 2^-24) * fl32(T))
 *                                  < fl32(alpha_j)
 * A selection returns the candidate of its first accepted trial, or M (and
 * AR_STATUS_TRIAL_CAP) when trials 0 .. trial_cap-1 all reject.  This is the
 * sequential AR method of Section "A GPU acceptance-rejection algorithm"
 * (choose j at random and u in [0,T) until u < alpha_j) with T = max_j
 * alpha_j (Section "Election step"; experiments' T_w = w max alpha, w = 1).
 * Conditioned on acceptance the law is alpha_j / sum(alpha) up to the
 * 2^-32 candidate lattice and the 2^-24 / 2^-32 uniform lattice.
 *
 * Runs (the batched entry points ar_select_batched and
 * ar_select_batched_bounded): selection ids are grouped in runs of 64,
 * run g = floor(s / 64) holding selections 64 g .. 64 g + 63, and each run
 * is one sequence of trials n = 0, 1, 2, ...: with G = floor(n / 64),
 * h = floor(n / 32) mod 2, i = n mod 32, trial n reads words 2h and 2h+1 of
 * the Philox block q = 32 G + i of counter
 * (q mod 2^32, g, b, 256 floor(q / 2^32)), with j and the test as above.
 * Selection 64 g + r is the first accepted trial after the one that decided
 * selection 64 g + r - 1 (the classical AR loop run over consecutive
 * selections), or M (AR_STATUS_TRIAL_CAP) after trial_cap consecutive
 * rejected trials; the next selection then starts at the following trial.
 * A selection's trials are those from the trial after the previous
 * decision to its own.  Results do not depend on how the selections of a
 * run are split over calls (sel_offset).
 */
#ifndef GBAR_H
#define GBAR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---------------------------------------------------- */
#define AR_OK 0
#define AR_ERR_ARG (-1)       /* bad size, null pointer or enum value     */
#define AR_ERR_ALIGN (-2)     /* a pointer lacks its required alignment   */
#define AR_ERR_CUDA (-3)      /* a CUDA call failed (see ar_last_cuda_error) */
#define AR_ERR_WORKSPACE (-4) /* workspace too small                       */
#define AR_ERR_UNSUPPORTED (-5) /* size beyond what this build supports   */

/* ---- device status bits ---------------------------------------------- */
#define AR_STATUS_BAD_ALPHA 1u  /* a propensity is NaN, +-inf or < 0       */
#define AR_STATUS_ALL_ZERO 2u   /* every propensity is 0 (paper's rejection) */
#define AR_STATUS_TRIAL_CAP 4u  /* a selection hit trial_cap; sentinel M   */
#define AR_STATUS_BAD_BOUND 8u  /* bound NaN, inf, < 0 (or inf in FP32)    */
#define AR_STATUS_ABSORBED 16u  /* SSA realization reached a0 = 0          */
#define AR_STATUS_WAIT_LIMIT 32u  /* ar_select_batched, one-launch form: a bounded wait
                                     for a realization's reduction gave up (not expected);
                                     its selections are the sentinel M_b              */
#define AR_STATUS_UNSUPPORTED 64u /* a batched realization with M_b >= 2^31 */
#define AR_STATUS_T_END 128u      /* SSA realization reached its time limit    */

typedef enum { AR_F32 = 0, AR_F64 = 1 } ar_dtype;
typedef enum { AR_CMP_F32 = 0, AR_CMP_F64 = 1 } ar_cmp;

/* Selection bookkeeping (Section "Assessing the qualities": rejection rate).
 * trials = sum over selections of trials consumed (t_accept + 1, or
 * trial_cap when capped); accepted / capped = counts.  Added atomically. */
typedef struct {
    uint64_t trials;
    uint64_t accepted;
    uint64_t capped;
} ar_stats;

/* Library version (major*10000 + minor*100 + patch). */
int ar_version(void);
/* Last CUDA error code seen by a call that returned AR_ERR_CUDA. */
int ar_last_cuda_error(void);

/* ---------------------------------------------------------------------
 * ar_bound -- threshold and total propensity of one vector.
 * Paper: T = max_j alpha_j (Section "Election step"; experiments T_w with
 * w = 1, Section "Quality of the selection"); alpha_0 = sum_j alpha_j
 * (Section "The Stochastic Simulation Algorithm").
 *   d_alpha      [M] FP32 or FP64 (dtype), 4- or 8-byte aligned.
 *   d_bound_sum  [2] double out: {max (exact), sum (FP64-grade: within
 *                (M + 8) * 2^-53 * sum of the exact sum)}.
 *   d_status     OR-ed with BAD_ALPHA (any NaN/inf/negative; -0 is 0) or
 *                ALL_ZERO (max = 0, including M = 0).  Outputs are
 *                unspecified when BAD_ALPHA is set.
 *   d_work       scratch of ar_bound_workspace_size(M, dtype) bytes (may be
 *                NULL when that size is 0), 16-byte aligned.  It must be
 *                zero-filled before its first use; every call leaves it
 *                zero-filled again, so one call is exactly one kernel
 *                launch.  Calls sharing a workspace must not overlap.
 * Errors: AR_ERR_ARG (M < 0, null pointers, bad dtype), AR_ERR_ALIGN,
 * AR_ERR_WORKSPACE.
 * ------------------------------------------------------------------- */
size_t ar_bound_workspace_size(int64_t M, int dtype);
int ar_bound(const void *d_alpha, int dtype, int64_t M, double *d_bound_sum,
             uint32_t *d_status, void *d_work, size_t work_bytes, void *stream);

/* ---------------------------------------------------------------------
 * ar_bound_noalloc -- ar_bound for callers that cannot allocate device
 * memory.  The paper has no counterpart: this is an interface convenience.
 * Some callers can neither call cudaMalloc nor hand over a workspace: a
 * plug-in that a host simulator gives only its input and output buffers, a
 * component whose host application owns every device allocation through
 * its own pool, or a stepping loop that must not meet the implicit device
 * synchronisation of cudaMalloc/cudaFree.  This entry point computes exactly
 * what ar_bound computes, with its scratch in a file-scope device array of
 * 16 + 16 * 4096 bytes that every GPU loading the library keeps until the
 * process exits; it calls no allocating routine.
 *   Arguments as in ar_bound, without the workspace.
 *   M is limited to AR_BOUND_NOALLOC_MAX_M_F32 (FP32) or
 *   AR_BOUND_NOALLOC_MAX_M_F64 (FP64) elements; larger M returns
 *   AR_ERR_UNSUPPORTED before anything is enqueued.
 *   Every call looks up the array's device address (cudaGetSymbolAddress,
 *   which allocates nothing) with the caller's device current, so a device
 *   reset or another context never leaves a stale address behind.  The
 *   first call on a device may load the library's device code: make it
 *   before any stream capture.
 *   All argument checks (ARG, UNSUPPORTED, ALIGN) come before anything is
 *   enqueued.
 *   All calls share the one array (each clears the part that must start at
 *   zero): calls that overlap on the GPU -- on different streams, or from
 *   different host threads -- race on it and must be serialised.
 * ------------------------------------------------------------------- */
#define AR_BOUND_NOALLOC_MAX_M_F32 33554432LL /* 4096 CTAs x 8192 elements */
#define AR_BOUND_NOALLOC_MAX_M_F64 16777216LL /* 4096 CTAs x 4096 elements */
int ar_bound_noalloc(const void *d_alpha, int dtype, int64_t M, double *d_bound_sum,
                     uint32_t *d_status, void *stream);

/* ---------------------------------------------------------------------
 * ar_select_k -- K independent selections from one propensity vector
 * (Section "A GPU acceptance-rejection algorithm": select the K next
 * reactions; the paper's K parallel realizations sharing one D in its
 * quality experiment, Section "Test and validation").
 *   d_alpha      [M] FP32/FP64.  1 <= M < 2^31 (M = 0: every index is 0).
 *   d_bound      NULL: the kernel uses T = max_j alpha_j, computed in each
 *                CTA from its shared-memory copy (requires M *
 *                element size <= ar_select_k_smem_limit()); else a device
 *                double T >= max alpha (T = w max, w >= 1 keeps the law).
 *   K            number of selections, 0 <= K, sel_offset + K <= 2^32.
 *   seed, sel_offset, realization  the random stream (see top).  Output i
 *                is selection s = sel_offset + i.
 *   cmp          AR_CMP_F32 or AR_CMP_F64.
 *   trial_cap    1 <= trial_cap <= 2^32 trials per selection.
 *   d_idx        [K] int32 out, selected indices (M = sentinel).
 *   d_stats      nullable ar_stats accumulator.
 *   d_status     OR-ed with ALL_ZERO, TRIAL_CAP, BAD_BOUND.
 * ------------------------------------------------------------------- */
size_t ar_select_k_smem_limit(void);
int ar_select_k(const void *d_alpha, int dtype, int64_t M, const double *d_bound,
                int64_t K, uint64_t seed, uint64_t sel_offset, uint32_t realization,
                int cmp, uint64_t trial_cap, int32_t *d_idx, ar_stats *d_stats,
                uint32_t *d_status, void *stream);

/* ---------------------------------------------------------------------
 * ar_select_batched -- many realizations with uneven M_b and K_b:
 * ar_bound_batched followed by ar_select_batched_bounded with each
 * realization's own maximum as its bound (Section "A GPU acceptance-rejection
 * algorithm": K realizations as K blocks; the text's extension to M beyond
 * one block).  With a plan whose realizations all sit in CTA home lists
 * (global share 0, the plan's default; at most 4096 per CTA) and 16-byte
 * aligned FP32 data, one kernel is enqueued: each persistent CTA reduces the chunks of its own
 * realizations, then selects them (a bounded wait covers a realization
 * still being reduced; past it AR_STATUS_WAIT_LIMIT is raised and that
 * realization's indices are the sentinel -- not expected).  Otherwise two
 * kernels: the reduction, then the selections, which combine each
 * realization's chunk results themselves.  The results are the same.
 * Realization b owns alpha_cat[offsets[b] .. offsets[b+1]) and writes
 * K_b = out_offsets[b+1] - out_offsets[b] indices at d_idx[out_offsets[b]].
 * Its bound is its own maximum, computed in the kernel; its Philox
 * realization id is realization_base + b; its selection ids are
 * sel_offset + 0 .. K_b-1, drawn from runs of 64 (the random stream, top).
 *   d_alpha_cat      FP32 or FP64 (dtype).
 *   d_offsets        [B+1] int64, non-decreasing, offsets[0] = 0.
 *   d_out_offsets    [B+1] int64, non-decreasing, out_offsets[0] = 0.
 *   d_bound_sum      [B][2] double out: {max, sum} per realization.  FP32
 *                    data: sum is the exact total rounded once to FP64 (each
 *                    chunk drops terms below 2^-73 of its maximum); FP64
 *                    data: FP64 additions.  NaN for invalid realizations.
 *   plan             nullable handle from ar_plan_create for these offsets on
 *                    this device (NULL: one work item per realization, claimed
 *                    from a global queue in the workspace; realizations
 *                    longer than 1024 elements are then reduced by a single
 *                    warp).  Either way the results are the same.
 *   Realizations with M_b >= 2^31 (or decreasing offsets) are not
 *   processed: AR_STATUS_UNSUPPORTED is raised.
 *   d_work           (plan == NULL only; ignored with a plan) scratch of
 *                    ar_select_batched_workspace_size(B) = 16 + 32 B bytes,
 *                    16-byte aligned.  Its first 16 bytes must be zero before
 *                    the first use and every call leaves them zero again (the
 *                    claim counter, reset by the launch itself); the rest is
 *                    rewritten by every call.  Calls sharing a workspace must
 *                    not overlap.
 *   d_idx, d_stats, d_status   as in ar_select_k (status also collects
 *                    BAD_ALPHA and ALL_ZERO of any realization).  An
 *                    invalid realization (BAD_ALPHA) gets no selections:
 *                    its indices are the sentinel M_b.
 * ------------------------------------------------------------------- */
typedef struct ar_plan ar_plan;
size_t ar_select_batched_workspace_size(int64_t B);

/* ---------------------------------------------------------------------
 * ar_bound_batched -- the reduction step alone (Section "A GPU
 * acceptance-rejection algorithm": T = max_j alpha_j per realization; the
 * total alpha_0 = sum_j alpha_j of Section "The Stochastic Simulation
 * Algorithm").  Arguments as in ar_select_batched; d_bound_sum [B][2]
 * receives {max, sum} (NaN, NaN for an invalid realization).  d_status
 * collects BAD_ALPHA, UNSUPPORTED and ALL_ZERO (a valid realization whose
 * propensities are all zero, including M_b = 0).  Two kernels.
 * ------------------------------------------------------------------- */
int ar_bound_batched(const void *d_alpha_cat, int dtype, const int64_t *d_offsets, int64_t B,
                     const struct ar_plan *plan, double *d_bound_sum, uint32_t *d_status,
                     void *d_work, size_t work_bytes, void *stream);

/* ---------------------------------------------------------------------
 * ar_select_batched_bounded -- the selection step with the caller's bounds:
 * realization b uses T_b = d_bound[b * bound_stride] (bound_stride = 2
 * reads the maxima of a bound_sum array).  The paper's threshold
 * experiment T_w = w * max_j alpha_j (Section "Test and validation"):
 * any T_b >= max_j alpha_j keeps the law exact and lowers the acceptance
 * rate by the factor max / T_b; a T_b below the maximum biases the law
 * (not checked).  Per realization, as ar_select_k with d_bound: T_b NaN,
 * negative or infinite (or infinite in FP32 with AR_CMP_F32) raises
 * BAD_BOUND and gives the sentinel M_b; T_b = 0 or M_b = 0 raises ALL_ZERO
 * (when K_b > 0) and gives M_b.  Other arguments as in ar_select_batched.
 * One kernel.
 * ------------------------------------------------------------------- */
int ar_select_batched_bounded(const void *d_alpha_cat, int dtype, const int64_t *d_offsets,
                              const int64_t *d_out_offsets, int64_t B, const double *d_bound,
                              int64_t bound_stride, uint64_t seed, uint64_t sel_offset,
                              uint32_t realization_base, int cmp, uint64_t trial_cap,
                              const struct ar_plan *plan, int32_t *d_idx, ar_stats *d_stats,
                              uint32_t *d_status, void *d_work, size_t work_bytes,
                              void *stream);

/* ---------------------------------------------------------------------
 * ar_plan_create -- tuning handle for repeated ar_select_batched calls on
 * one batch shape (the paper's K realizations of fixed sizes, iterated
 * over SSA steps).  Built on the host from the shape alone (no
 * propensities):
 *   - the reduction chunks: each realization cut into ceil(M_b / 1024)
 *     chunks of equal length (16 bytes each);
 *   - the selection work: ranges of 64 selections.  The costliest
 *     realizations (estimated cost K_b (0.6 + ln M_b) + 0.05 M_b) are
 *     assigned to the persistent CTAs of the selection kernel by
 *     longest-processing-time-first list scheduling (each CTA's home list);
 *     the cheapest ones, a chosen share of the estimated cost, may form a
 *     global queue that balances the CTAs' finishing times (48 bytes per
 *     range; each CTA's list of chunks to reduce comes with the one-launch
 *     form).  Default tile: 32 warps per CTA (one CTA per SM) with no
 *     global queue, which makes ar_select_batched one launch for FP32 data;
 *     ar_plan_autotune picks tile and share on the caller's data;
 *   - device scratch for the chunk partials (32 bytes per chunk).
 * Results are identical with or without a plan.  Calls sharing a plan must
 * not overlap on the GPU (they share its scratch).
 *   h_offsets, h_out_offsets  [B+1] int64 HOST arrays, as passed (on the
 *                device) to ar_select_batched.  A plan is valid only for
 *                calls whose offsets have exactly these values, on the device
 *                current when it was built.
 *   *out         receives the handle; it owns device memory until
 *                ar_plan_destroy.
 * Errors: AR_ERR_ARG (B <= 0, decreasing offsets, null pointers),
 * AR_ERR_CUDA (allocation or copy failed).
 * ------------------------------------------------------------------- */
int ar_plan_create(const int64_t *h_offsets, const int64_t *h_out_offsets, int64_t B,
                   ar_plan **out);
void ar_plan_destroy(ar_plan *plan);

/* ---------------------------------------------------------------------
 * ar_plan_autotune -- picks the selection kernel's tile shape for a plan
 * by timing it on the caller's data (the batched workload's block/warp
 * tiles): warps per CTA in {16, 32, 8} (1024 threads per SM) times the
 * share of the estimated cost left to the global queue in {0, 0.3, 0.6}.
 * Each candidate rebuilds the plan's selection schedule (host), runs two
 * warm-up calls and `reps` timed calls of ar_select_batched (seed,
 * sel_offset 0, realization_base 0, trial_cap 2^20, the given cmp) on
 * `stream`, timed with CUDA events; the fastest is kept.  Results of
 * ar_select_batched do not depend on the choice.  Synchronous (blocks the
 * host; not capturable).  d_bound_sum, d_idx, d_stats, d_status receive the
 * tuning calls' outputs (stats and status accumulate).
 *   h_choice   nullable host int32[3]: warps per CTA, global share per
 *              mille, mean nanoseconds per call of the choice.
 * Errors: as ar_select_batched; AR_ERR_ARG for reps outside 1..10000.
 * ------------------------------------------------------------------- */
int ar_plan_autotune(ar_plan *plan, const void *d_alpha_cat, int dtype,
                     const int64_t *d_offsets, const int64_t *d_out_offsets, uint64_t seed,
                     int cmp, double *d_bound_sum, int32_t *d_idx, ar_stats *d_stats,
                     uint32_t *d_status, int reps, int32_t *h_choice, void *stream);

/* ---------------------------------------------------------------------
 * ar_plan_set_tile -- sets the plan's selection tile directly (a choice
 * ar_plan_autotune made earlier, or one known to suit the caller's launch
 * pattern): warps_per_cta in {8, 16, 32}, global_share_pm in 0..1000 (the
 * estimated cost per mille left to the global queue).  Rebuilds the
 * selection schedule on the host and uploads it (synchronous; not
 * capturable; no call with this plan may be running).  Results of
 * ar_select_batched do not depend on the tile.  CUDA graphs captured with
 * this plan before the change launch the old tile: recapture them (the
 * same holds after ar_plan_autotune).
 * Errors: AR_ERR_ARG for a NULL plan or values outside those sets;
 * AR_ERR_CUDA when the upload fails.
 * ------------------------------------------------------------------- */
int ar_plan_set_tile(ar_plan *plan, int warps_per_cta, int global_share_pm);

/* ---------------------------------------------------------------------
 * ar_plan_set_grid -- the persistent grid of the plan's selection
 * schedule, for callers that keep several independent calls in flight on
 * other streams (each with a plan of its own).
 *   ctas_per_sm    0 (the default) = as many CTAs per SM as the tile's
 *                  register budget allows (1, 2 or 4 for tiles of 32, 16 or
 *                  8 warps); 1..4 = at most that many, so that a call's CTAs
 *                  occupy only part of each SM and the calls in flight share
 *                  the SMs -- one call's reduction then overlaps another's
 *                  selections.  Values above what the tile allows act as 0.
 *   selections_per_item  0 (the default, 64) or a multiple of 64 up to
 *                  1024: the selection range a warp claims at a time in a
 *                  CTA's home list.  Longer items mean fewer claims and
 *                  bound lookups but a longer tail for one call alone.
 * Rebuilds the schedule for the current tile (synchronous; not capturable;
 * no call with this plan may be running; recapture CUDA graphs
 * afterwards).  Results of ar_select_batched do not depend on either value.
 * Errors: AR_ERR_ARG for a NULL plan, a value outside those sets or another
 * current device; AR_ERR_CUDA when the upload fails.
 * ------------------------------------------------------------------- */
int ar_plan_set_grid(ar_plan *plan, int ctas_per_sm, int selections_per_item);
int ar_select_batched(const void *d_alpha_cat, int dtype, const int64_t *d_offsets,
                      const int64_t *d_out_offsets, int64_t B, uint64_t seed,
                      uint64_t sel_offset, uint32_t realization_base, int cmp,
                      uint64_t trial_cap, const ar_plan *plan, double *d_bound_sum,
                      int32_t *d_idx, ar_stats *d_stats, uint32_t *d_status,
                      void *d_work, size_t work_bytes, void *stream);

/* ---------------------------------------------------------------------
 * ar_select_paper -- the paper's own GPU selection rule, for comparison
 * (Sections "Election step" and "Selection step", the Results'
 * pseudo-code; its quality experiment, Table 1).  FP32, as the paper's
 * arrays are float.  For selection s (id sel_offset + i) every reaction j
 * draws u_j = floor(w / 2^8) 2^-24 (counter (j/2, s, realization, 3), word
 * 2(j mod 2) + 1) and is eligible when fl(u_j T) < D_j and D_j != 0, with
 * rate R_j = fl(fl(u_j T) / D_j); the selection is argmin R (lowest j on
 * ties), or the sentinel M when min R >= 1 (a rejection).  The rule's law
 * differs from D_j / sum D (the bias that Table 1 measures).
 *   d_D          [M] FP32, 0 <= M < 2^31.
 *   d_bound      device double; T = fl32(*d_bound) (the paper's T_w).
 *   K            selections, sel_offset + K <= 2^32.
 *   d_idx        [K] int32 out.
 *   d_rejections nullable device uint64 accumulator of rejections.
 * ------------------------------------------------------------------- */
int ar_select_paper(const float *d_D, int64_t M, const double *d_bound, int64_t K,
                    uint64_t seed, uint64_t sel_offset, uint32_t realization, int32_t *d_idx,
                    unsigned long long *d_rejections, void *stream);

/* ---------------------------------------------------------------------
 * ar_select_it -- the direct method's inverse transform, the comparator
 * the paper argues against (Section "The Stochastic Simulation
 * Algorithm": j is the smallest index with alpha_0 + ... + alpha_j >
 * u alpha_0).  The running sums S_j are the exact prefix sums rounded once
 * to FP64 (ties to even), so they do not depend on the order of the
 * additions: each propensity enters as a whole number of units U, rounded
 * down (FP32 data: U = 2^(E-223); FP64 data: U = 2^(E-1119); E the biased
 * exponent of the maximum, at least 1 resp. 97 -- a term loses less than
 * 2^-96 of the maximum), the units are summed exactly in 128-bit integers
 * by a parallel scan over tiles of 4096 propensities, and every S_j is
 * rounded once.  u = (w0 2^21 + floor(w1 / 2^11)) 2^-53 from counter
 * (0, s, realization, 2); the selection is the first S_j > fl(u S_{M-1})
 * (bisection); if rounding leaves none, the last index with a positive
 * propensity.  Invalid propensities (BAD_ALPHA) or S_{M-1} = 0 (ALL_ZERO,
 * including M = 0) give the sentinel M for every selection.  Five kernels
 * and one memset of the workspace header.
 *   d_alpha      [M] FP32/FP64 (dtype), M < 2^31.
 *   d_idx        [K] int32 out.
 *   d_status     OR-ed with BAD_ALPHA and ALL_ZERO.
 *   d_work       ar_select_it_workspace_size(M) bytes (48 + 8 M rounded up
 *                to 16, + 16 per tile), 16-byte aligned, rewritten by every
 *                call.  Calls sharing it must not overlap.
 * ------------------------------------------------------------------- */
size_t ar_select_it_workspace_size(int64_t M);
int ar_select_it(const void *d_alpha, int dtype, int64_t M, int64_t K, uint64_t seed,
                 uint64_t sel_offset, uint32_t realization, int32_t *d_idx, uint32_t *d_status,
                 void *d_work, size_t work_bytes, void *stream);

/* ---------------------------------------------------------------------
 * SSA step (Section "The Stochastic Simulation Algorithm": select j, draw
 * tau = ln(1/u)/a_0, X += v_j, t += tau; the selection is the AR trial
 * above with T = max_j a_j and selection id = the realization's step
 * number).  Mass-action propensities a_r = c_r * h_r(X) with one FP64
 * rounding of the exact integer count h_r:
 *   type 0 (source)  h = 1
 *   type 1 (A)       h = x_A (0 if x_A <= 0)
 *   type 2 (A + B)   h = x_A x_B (0 if either <= 0)
 *   type 3 (2A)      h = x_A (x_A - 1) / 2 (0 if x_A < 2)
 * After reaction j only the propensities of reactions that read a species
 * j changes are recomputed (dependency graph, Gibson & Bruck, cited in the
 * Introduction); a_0 is kept as an exact fixed-point sum.
 *
 * ssa_net_create -- uploads a network: h_rtype[M], h_reactants[M][2]
 *   (species A, B; -1 where unused), h_rate[M] (finite, >= 0), the net
 *   state change as CSR h_nu_ptr[M+1], h_nu_species[nnz], h_nu_delta[nnz]
 *   (each species at most once per reaction).  Builds the dependency graph.
 *   The handle owns device memory until ssa_net_destroy.  AR_ERR_ARG on an
 *   invalid network, AR_ERR_CUDA on allocation failure.
 * ------------------------------------------------------------------- */
typedef struct ssa_net ssa_net;
int ssa_net_create(int32_t N, int32_t M, const int32_t *h_rtype, const int32_t *h_reactants,
                   const double *h_rate, const int32_t *h_nu_ptr, const int32_t *h_nu_species,
                   const int32_t *h_nu_delta, ssa_net **out);
void ssa_net_destroy(ssa_net *net);

/* ---------------------------------------------------------------------
 * ssa_step_batched -- advances B realizations by up to nsteps steps each.
 *   d_X       [B][N] int32 molecule counts (in/out).
 *   d_a       [B][M] double scratch/out: the propensities of the final state
 *             (recomputed from d_X at the start of every call).
 *   d_t       [B] double time (in/out); d_step [B] uint64 step counters
 *             (in/out; the selection id of a step is its counter, so a run
 *             split over several calls draws the same random numbers as one
 *             call).
 *   seed, realization_base  random stream; realization b uses id
 *             realization_base + b; tau uses counter (0, step, id, 1).
 *   cmp, trial_cap  as in ar_select_k.
 *   d_last    nullable [B] int32: the last reaction fired.
 *   d_status  [B] uint32 (in/out): ABSORBED (a_0 = 0: the realization
 *             stops), TRIAL_CAP (stops), UNSUPPORTED (the fixed-point a_0
 *             left its range: propensities grew 2^40-fold within the call).
 *             Realizations whose status already holds ABSORBED, TRIAL_CAP,
 *             BAD_ALPHA or UNSUPPORTED are not advanced.
 *   d_trials  nullable [B] uint64: trials consumed are added.
 * ------------------------------------------------------------------- */
int ssa_step_batched(const ssa_net *net, int64_t B, int32_t *d_X, double *d_a, double *d_t,
                     uint64_t *d_step, int64_t nsteps, uint64_t seed, uint32_t realization_base,
                     int cmp, uint64_t trial_cap, int32_t *d_last, uint32_t *d_status,
                     uint64_t *d_trials, void *stream);

/* ---------------------------------------------------------------------
 * ssa_run_until -- advances B realizations to the time limit t_end (the
 * SSA loop of Section "The Stochastic Simulation Algorithm": repeat until
 * the simulated time passes the end), at most max_steps reactions per
 * realization and call, recording trajectory samples.  Each step first
 * draws its waiting time tau (same stream as ssa_step_batched); if
 * t + tau > t_end the reaction does not fire and AR_STATUS_T_END is set
 * (informational); t stays at the realization's last reaction, its state
 * holding on [t, t_end], so a later call with a larger t_end continues
 * exactly as a single call would.  An absorbed realization (a_0 = 0)
 * keeps its state to t_end.
 *   d_sample_times  [nsamp] ascending sample times (nullable when nsamp =
 *                   0).  d_traj[b][k][s] receives the count of species
 *                   d_sample_species[s] (nullable: species s) at time
 *                   t_k, i.e. after the last reaction at a time <= t_k, for
 *                   every t_k this call passes (t_k >= the realization's
 *                   time at the start of the call and <= where it stops).
 *   Other arguments as in ssa_step_batched.
 * ------------------------------------------------------------------- */
int ssa_run_until(const ssa_net *net, int64_t B, int32_t *d_X, double *d_a, double *d_t,
                  uint64_t *d_step, double t_end, int64_t max_steps, uint64_t seed,
                  uint32_t realization_base, int cmp, uint64_t trial_cap,
                  const double *d_sample_times, int32_t nsamp, const int32_t *d_sample_species,
                  int32_t nspec, int32_t *d_traj, int32_t *d_last, uint32_t *d_status,
                  uint64_t *d_trials, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GBAR_H */
