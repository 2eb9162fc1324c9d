/*
 * CPU oracle for the parallel acceptance-rejection (AR) selection of the next
 * reaction to occur in the Stochastic Simulation Algorithm (Neri & Mestivier,
 * "An efficient GPU acceptance-rejection algorithm for the selection of the
 * next reaction to occur for Stochastic Simulation Algorithms", 2014).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, obviously correct
 * restatement of what the GPU library computes.  Only the tests, the smoke
 * check and the benchmark's CPU-baseline leg load it.  It shares no code,
 * header, table or constant generator with the CUDA library: every definition
 * below is written out from the paper and from the published Philox
 * definition (Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC'11).
 *
 * Build with -O2 -ffp-contract=off and without fast-math, so that every
 * floating-point operation is one IEEE-754 round-to-nearest operation.
 *
 * Status bits (same numeric values as the library's public header, restated):
 *   1  BAD_ALPHA   a propensity is NaN, infinite or negative
 *   2  ALL_ZERO    every propensity is zero (the paper's rejection case)
 *   4  TRIAL_CAP   a selection exhausted its trial budget (sentinel written)
 *   8  BAD_BOUND   the bound passed to a selection is NaN, infinite or < 0
 *   16 ABSORBED    an SSA realization reached a state with a0 = 0
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ST_BAD_ALPHA 1u
#define ST_ALL_ZERO 2u
#define ST_TRIAL_CAP 4u
#define ST_BAD_BOUND 8u
#define ST_ABSORBED 16u

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11, Section 4.2).                        */
/* One round maps (x0,x1,x2,x3) with key (k0,k1) to                          */
/*   (hi(M1*x2) ^ x1 ^ k0,  lo(M1*x2),  hi(M0*x0) ^ x3 ^ k1,  lo(M0*x0))      */
/* with M0 = 0xD2511F53, M1 = 0xCD9E8D57; between rounds the key is bumped   */
/* by the Weyl constants (0x9E3779B9, 0xBB67AE85).  Ten rounds.              */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], uint64_t seed, uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = (uint32_t)(seed & 0xffffffffu);
    uint32_t k1 = (uint32_t)(seed >> 32);
    for (int round = 0; round < 10; round++) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* n counters (4 words each) -> n outputs (4 words each). */
void orc_philox_many(const uint32_t *ctrs, int64_t n, uint64_t seed, uint32_t *out)
{
    for (int64_t i = 0; i < n; i++)
        orc_philox4x32_10(ctrs + 4 * i, seed, out + 4 * i);
}

/* ------------------------------------------------------------------------ */
/* Propensity access: dtype 0 = float32, 1 = float64.                        */
/* ------------------------------------------------------------------------ */
static double alpha_at(const void *alpha, int dtype, int64_t j)
{
    if (dtype == 0) return (double)((const float *)alpha)[j];
    return ((const double *)alpha)[j];
}

/* ------------------------------------------------------------------------ */
/* Bound and total propensity.                                               */
/* The threshold is the largest propensity, T = max_j alpha_j (Section      */
/* "Election step" and the experiments' T_w = w * max_j alpha_j with w = 1). */
/* alpha_0 = sum_j alpha_j (Section "The Stochastic Simulation Algorithm"). */
/* Plain loops: max by comparison, sum in FP64 in index order.              */
/* ------------------------------------------------------------------------ */
uint32_t orc_bound(const void *alpha, int dtype, int64_t M, double out[2])
{
    uint32_t status = 0;
    double mx = 0.0, sum = 0.0;
    for (int64_t j = 0; j < M; j++) {
        double x = alpha_at(alpha, dtype, j);
        if (!(x >= 0.0) || isinf(x)) status |= ST_BAD_ALPHA;
        if (x > mx) mx = x;
        sum += x;
    }
    if (!(status & ST_BAD_ALPHA) && mx == 0.0) status |= ST_ALL_ZERO;
    out[0] = mx;
    out[1] = sum;
    return status;
}

/* ------------------------------------------------------------------------ */
/* One AR trial (Section "A GPU acceptance-rejection algorithm", the        */
/* sequential AR method: pick j uniformly in 1..M and u uniform in [0,T),   */
/* repeat until u < alpha_j).                                                */
/*                                                                          */
/* Random stream: trial t of selection s of realization b uses the Philox  */
/* block at counter (t/2, s, b, 0) and, within it, words 2(t mod 2) (for j) */
/* and 2(t mod 2)+1 (for u).                                                */
/* Candidate: j = floor(w_a * M / 2^32).                                    */
/* FP64 comparison: u = w_b * 2^-32, accept iff fl64(u * T) < alpha_j.       */
/* FP32 comparison: u = floor(w_b / 2^8) * 2^-24, accept iff                 */
/*   fl32(u * fl32(T)) < fl32(alpha_j).                                      */
/* ------------------------------------------------------------------------ */
static void trial_words(uint64_t seed, uint32_t s, uint32_t b, uint32_t tag,
                        uint64_t t, uint32_t *wa, uint32_t *wb)
{
    uint32_t ctr[4] = {(uint32_t)(t >> 1), s, b, tag};
    uint32_t w[4];
    orc_philox4x32_10(ctr, seed, w);
    int half = (int)(t & 1u);
    *wa = w[2 * half];
    *wb = w[2 * half + 1];
}

static int64_t candidate(uint32_t wa, int64_t M)
{
    return (int64_t)(((uint64_t)wa * (uint64_t)M) >> 32);
}

static int accept_f64(uint32_t wb, double T, double a)
{
    double u = (double)wb * 0x1p-32;
    double p = u * T;
    return p < a;
}

static int accept_f32(uint32_t wb, float T, float a)
{
    float u = (float)(wb >> 8) * 0x1p-24f;
    float p = u * T;
    return p < a;
}

/* Selection s: the candidate of the first accepted trial; sentinel M when
 * no trial t < trial_cap is accepted (the paper's rejection code M+1, here
 * 0-based).  Returns the number of trials consumed in *ntrials. */
static int64_t select_one(const void *alpha, int dtype, int64_t M, double T,
                          int cmp, uint64_t seed, uint32_t s, uint32_t b,
                          uint64_t trial_cap, uint64_t *ntrials)
{
    float Tf = (float)T;
    for (uint64_t t = 0; t < trial_cap; t++) {
        uint32_t wa, wb;
        trial_words(seed, s, b, 0u, t, &wa, &wb);
        int64_t j = candidate(wa, M);
        double a = alpha_at(alpha, dtype, j);
        int ok = (cmp == 0) ? accept_f32(wb, Tf, (float)a) : accept_f64(wb, T, a);
        if (ok) {
            *ntrials = t + 1;
            return j;
        }
    }
    *ntrials = trial_cap;
    return M;
}

/* The bound is usable when it is finite and non-negative (and, in FP32
 * comparison mode, finite after rounding to FP32). */
static uint32_t bound_check(double T, int cmp)
{
    if (!(T >= 0.0) || isinf(T)) return ST_BAD_BOUND;
    if (cmp == 0 && isinf((float)T)) return ST_BAD_BOUND;
    return 0;
}

/* K selections from one propensity vector.  Selection ids are
 * sel_offset + i.  stats = {trials, accepted, capped}. */
uint32_t orc_select_ar(const void *alpha, int dtype, int64_t M, double T,
                       int64_t K, uint64_t seed, uint64_t sel_offset,
                       uint32_t realization, int cmp, uint64_t trial_cap,
                       int32_t *idx, uint64_t stats[3], int nthreads)
{
    uint32_t status = bound_check(T, cmp);
    if (status || T == 0.0 || M == 0) {
        for (int64_t i = 0; i < K; i++) idx[i] = (int32_t)M;
        if (!status && K > 0) status = ST_ALL_ZERO;
        return status;
    }
    uint64_t trials = 0, accepted = 0, capped = 0;
    (void)nthreads;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads > 0 ? nthreads : 1) \
    reduction(+ : trials, accepted, capped)
#endif
    for (int64_t i = 0; i < K; i++) {
        uint64_t nt = 0;
        int64_t j = select_one(alpha, dtype, M, T, cmp, seed,
                               (uint32_t)(sel_offset + (uint64_t)i), realization,
                               trial_cap, &nt);
        idx[i] = (int32_t)j;
        trials += nt;
        if (j < M) accepted++; else capped++;
    }
    if (capped) status |= ST_TRIAL_CAP;
    if (stats) {
        stats[0] += trials;
        stats[1] += accepted;
        stats[2] += capped;
    }
    return status;
}

/* ------------------------------------------------------------------------ */
/* Runs: the classical AR loop (Section "A GPU acceptance-rejection         */
/* algorithm": draw a uniform candidate j and a uniform u, accept when      */
/* u T < alpha_j, otherwise draw again) applied to consecutive selections   */
/* on one random sequence.  Selections are grouped in runs of 64            */
/* consecutive selection numbers; run g of realization b draws its trials   */
/* n = 0, 1, 2, ... in order, and its decision r (selection 64 g + r) is    */
/* the first accepted trial after decision r - 1, or the sentinel M once    */
/* trial_cap trials in a row were rejected (the next decision then starts   */
/* at the following trial).                                                 */
/* Trial n of run g: with G = floor(n / 64), h = floor(n / 32) mod 2 and    */
/* i = n mod 32, Philox block q = 32 G + i of counter                       */
/* (q mod 2^32, g, b, 256 floor(q / 2^32)); words 2h and 2h+1 are (w_a,     */
/* w_b), candidate and comparison as above.                                 */
/* ------------------------------------------------------------------------ */
#define RUN_LEN 64u

static void run_trial_words(uint64_t seed, uint32_t g, uint32_t b, uint64_t n,
                            uint32_t *wa, uint32_t *wb)
{
    uint64_t q = 32u * (n / 64u) + n % 32u;
    int h = (int)((n / 32u) % 2u);
    uint32_t ctr[4] = {(uint32_t)q, g, b, (uint32_t)(q >> 32) << 8};
    uint32_t w[4];
    orc_philox4x32_10(ctr, seed, w);
    *wa = w[2 * h];
    *wb = w[2 * h + 1];
}

/* Decisions first .. last - 1 of run g into out[0 .. last - first); adds the
 * trials those decisions consumed and counts the capped ones. */
static void select_run(const void *alpha, int dtype, int64_t M, double T, int cmp,
                       uint64_t seed, uint32_t g, uint32_t b, uint32_t first,
                       uint32_t last, uint64_t trial_cap, int32_t *out,
                       uint64_t *trials, uint64_t *capped)
{
    float Tf = (float)T;
    uint64_t n = 0;      /* next trial of the run */
    for (uint32_t r = 0; r < last; r++) {
        int64_t sel = M;  /* decision r: the sentinel unless a trial accepts */
        uint64_t t;
        for (t = 0; t < trial_cap; t++, n++) {
            uint32_t wa, wb;
            run_trial_words(seed, g, b, n, &wa, &wb);
            int64_t j = candidate(wa, M);
            double a = alpha_at(alpha, dtype, j);
            int ok = (cmp == 0) ? accept_f32(wb, Tf, (float)a) : accept_f64(wb, T, a);
            if (ok) {
                sel = j;
                n++;
                t++;
                break;
            }
        }
        if (r >= first) {
            out[r - first] = (int32_t)sel;
            *trials += t;
            if (sel == M) (*capped)++;
        }
    }
}

/* K selections from one propensity vector, numbers sel_offset + i, drawn
 * from the runs that hold them.  stats = {trials, accepted, capped}. */
uint32_t orc_select_runs(const void *alpha, int dtype, int64_t M, double T,
                         int64_t K, uint64_t seed, uint64_t sel_offset,
                         uint32_t realization, int cmp, uint64_t trial_cap,
                         int32_t *idx, uint64_t stats[3])
{
    uint32_t status = bound_check(T, cmp);
    if (status || T == 0.0 || M == 0) {
        for (int64_t i = 0; i < K; i++) idx[i] = (int32_t)M;
        if (!status && K > 0) status = ST_ALL_ZERO;
        return status;
    }
    uint64_t trials = 0, capped = 0;
    int64_t i = 0;
    while (i < K) {
        uint64_t s = sel_offset + (uint64_t)i;
        uint32_t g = (uint32_t)(s / RUN_LEN), first = (uint32_t)(s % RUN_LEN);
        uint32_t last = RUN_LEN;
        if ((int64_t)(last - first) > K - i) last = first + (uint32_t)(K - i);
        select_run(alpha, dtype, M, T, cmp, seed, g, realization, first, last, trial_cap,
                   idx + i, &trials, &capped);
        i += last - first;
    }
    if (capped) status |= ST_TRIAL_CAP;
    if (stats) {
        stats[0] += trials;
        stats[1] += (uint64_t)K - capped;
        stats[2] += capped;
    }
    return status;
}

/* Batched form: realization b owns alpha[offsets[b] .. offsets[b+1]) and
 * writes K_b = out_offsets[b+1] - out_offsets[b] indices at out_offsets[b].
 * Its bound is its own maximum (orc_bound); bound_sum[2b..2b+1] = (max, sum).
 * Its Philox realization id is realization_base + b. */
uint32_t orc_select_batched(const void *alpha, int dtype, const int64_t *offsets,
                            const int64_t *out_offsets, int64_t B, uint64_t seed,
                            uint64_t sel_offset, uint32_t realization_base, int cmp,
                            uint64_t trial_cap, double *bound_sum, int32_t *idx,
                            uint64_t stats[3], int nthreads)
{
    uint32_t status = 0;
    uint64_t s0 = 0, s1 = 0, s2 = 0;
    int64_t esize = dtype == 0 ? 4 : 8;
    (void)nthreads;
    /* realizations are independent: one at a time per thread */
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 8) num_threads(nthreads > 0 ? nthreads : 1) \
    reduction(| : status) reduction(+ : s0, s1, s2)
#endif
    for (int64_t b = 0; b < B; b++) {
        const char *ab = (const char *)alpha + offsets[b] * esize;
        int64_t Mb = offsets[b + 1] - offsets[b];
        int64_t Kb = out_offsets[b + 1] - out_offsets[b];
        double bs[2];
        uint64_t st[3] = {0, 0, 0};
        uint32_t sb = orc_bound(ab, dtype, Mb, bs);
        if (sb & ST_BAD_ALPHA) {
            /* an invalid realization has no usable bound: (NaN, NaN), no
             * selections (every index is the sentinel M) */
            bound_sum[2 * b] = bound_sum[2 * b + 1] = NAN;
            for (int64_t i = 0; i < Kb; i++) idx[out_offsets[b] + i] = (int32_t)Mb;
            status |= ST_BAD_ALPHA;
            continue;
        }
        bound_sum[2 * b] = bs[0];
        bound_sum[2 * b + 1] = bs[1];
        status |= orc_select_runs(ab, dtype, Mb, bs[0], Kb, seed, sel_offset,
                                  realization_base + (uint32_t)b, cmp, trial_cap,
                                  idx + out_offsets[b], st);
        s0 += st[0];
        s1 += st[1];
        s2 += st[2];
    }
    if (stats) {
        stats[0] += s0;
        stats[1] += s1;
        stats[2] += s2;
    }
    return status;
}

/* Batched selection with the caller's bounds: realization b uses
 * T_b = bound[b * stride] (T_w = w * max_j alpha_j, the paper's threshold
 * experiment, keeps the law for w >= 1).  Each realization as
 * orc_select_runs. */
uint32_t orc_select_batched_bounded(const void *alpha, int dtype, const int64_t *offsets,
                                    const int64_t *out_offsets, int64_t B, const double *bound,
                                    int64_t stride, uint64_t seed, uint64_t sel_offset,
                                    uint32_t realization_base, int cmp, uint64_t trial_cap,
                                    int32_t *idx, uint64_t stats[3], int nthreads)
{
    uint32_t status = 0;
    uint64_t s0 = 0, s1 = 0, s2 = 0;
    int64_t esize = dtype == 0 ? 4 : 8;
    (void)nthreads;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 8) num_threads(nthreads > 0 ? nthreads : 1) \
    reduction(| : status) reduction(+ : s0, s1, s2)
#endif
    for (int64_t b = 0; b < B; b++) {
        const char *ab = (const char *)alpha + offsets[b] * esize;
        uint64_t st[3] = {0, 0, 0};
        status |= orc_select_runs(ab, dtype, offsets[b + 1] - offsets[b], bound[b * stride],
                                  out_offsets[b + 1] - out_offsets[b], seed, sel_offset,
                                  realization_base + (uint32_t)b, cmp, trial_cap,
                                  idx + out_offsets[b], st);
        s0 += st[0];
        s1 += st[1];
        s2 += st[2];
    }
    if (stats) {
        stats[0] += s0;
        stats[1] += s1;
        stats[2] += s2;
    }
    return status;
}

/* ------------------------------------------------------------------------ */
/* Inverse-transform (direct method) selection, Section "The Stochastic     */
/* Simulation Algorithm": j is the smallest index whose running sum exceeds */
/* u * alpha_0.  Random stream: counter (0, s, b, 2), words 0 and 1 form a  */
/* 53-bit u = (w0 * 2^21 + floor(w1 / 2^11)) * 2^-53 in [0, 1).             */
/* If rounding leaves no index past the target, the last nonzero index is   */
/* taken.  All-zero input gives the sentinel M.                             */
/* ------------------------------------------------------------------------ */
static double u53(uint32_t w0, uint32_t w1)
{
    uint64_t m = ((uint64_t)w0 << 21) | (uint64_t)(w1 >> 11);
    return (double)m * 0x1p-53;
}

/* ------------------------------------------------------------------------ */
/* Running sums of the inverse transform.  Reading: S_j is the exact sum    */
/* alpha_0 + ... + alpha_j rounded once to the nearest double (ties to     */
/* even), which is what the method's "running sum" denotes in exact        */
/* arithmetic; it does not depend on the order the terms are added in.     */
/* Each propensity enters as a whole number of units U, rounded down:      */
/*   FP32 data: U = 2^(E - 223), E = max(biased exponent of the max, 1);   */
/*   FP64 data: U = 2^(E - 1119), E = max(biased exponent of the max, 97). */
/* The maximum is then below 2^97 units (exact: its 24- or 53-bit          */
/* significand shifted by 73 or 44 places), so a term loses less than     */
/* 2^-96 of the maximum, M < 2^31 terms fit in 128 bits, and every nonzero */
/* S_j = RN(P_j U) is a normal double.                                     */
/* ------------------------------------------------------------------------ */
typedef unsigned __int128 orc_u128;

/* value = m 2^q (m the significand as an integer, q its exponent) */
static void split_value(const void *alpha, int dtype, int64_t j, uint64_t *m, int *q)
{
    if (dtype == 0) {
        uint32_t bits;
        memcpy(&bits, (const float *)alpha + j, 4);
        int e = (int)((bits >> 23) & 0xffu);
        uint64_t f = bits & 0x7fffffu;
        *m = e ? (f | 0x800000u) : f;
        *q = (e ? e : 1) - 150;
    } else {
        uint64_t bits;
        memcpy(&bits, (const double *)alpha + j, 8);
        int e = (int)((bits >> 52) & 0x7ffu);
        uint64_t f = bits & 0xfffffffffffffull;
        *m = e ? (f | 0x10000000000000ull) : f;
        *q = (e ? e : 1) - 1075;
    }
}

/* m 2^q in units of 2^uexp, rounded down */
static orc_u128 to_units(uint64_t m, int q, int uexp)
{
    int sh = q - uexp;
    if (sh >= 0) return (orc_u128)m << sh;
    if (sh <= -64) return 0;
    return (orc_u128)(m >> (-sh));
}

/* n 2^e rounded to the nearest double, ties to even */
static double u128_scaled(orc_u128 n, int e)
{
    if (n == 0) return 0.0;
    int nb = 0;
    for (orc_u128 t = n; t; t >>= 1) nb++;
    if (nb <= 53) return ldexp((double)(uint64_t)n, e);
    int drop = nb - 53;
    orc_u128 q = n >> drop;
    orc_u128 rem = n - (q << drop);
    orc_u128 half = (orc_u128)1 << (drop - 1);
    if (rem > half || (rem == half && (q & 1))) q += 1;  /* q <= 2^53: exact in a double */
    return ldexp((double)(uint64_t)q, e + drop);
}

/* S[0..M) as above; returns the status bits of orc_bound.  With BAD_ALPHA
 * set the sums are not defined and S is left untouched. */
uint32_t orc_it_prefix(const void *alpha, int dtype, int64_t M, double *S)
{
    double bs[2];
    uint32_t status = orc_bound(alpha, dtype, M, bs);
    if (status & ST_BAD_ALPHA) return status;
    uint64_t m;
    int q;
    int E;
    if (dtype == 0) {
        float mx = (float)bs[0];
        uint32_t bits;
        memcpy(&bits, &mx, 4);
        E = (int)((bits >> 23) & 0xffu);
        if (E < 1) E = 1;
    } else {
        uint64_t bits;
        memcpy(&bits, &bs[0], 8);
        E = (int)((bits >> 52) & 0x7ffu);
        if (E < 97) E = 97;
    }
    int uexp = dtype == 0 ? E - 223 : E - 1119;
    orc_u128 P = 0;
    for (int64_t j = 0; j < M; j++) {
        split_value(alpha, dtype, j, &m, &q);
        P += to_units(m, q, uexp);
        S[j] = u128_scaled(P, uexp);
    }
    return status;
}

/* Selection: the smallest j with S_j > u * a0, a0 = S_{M-1} (one FP64
 * multiply); if rounding leaves none, the last index with a nonzero
 * propensity.  All-zero input (a0 = 0) and invalid propensities
 * (BAD_ALPHA) give the sentinel M. */
uint32_t orc_select_it(const void *alpha, int dtype, int64_t M, int64_t K,
                       uint64_t seed, uint64_t sel_offset, uint32_t realization,
                       int32_t *idx, int nthreads)
{
    double *S = (double *)malloc(sizeof(double) * (size_t)(M > 0 ? M : 1));
    uint32_t status = orc_it_prefix(alpha, dtype, M, S);
    double a0 = (M > 0 && !(status & ST_BAD_ALPHA)) ? S[M - 1] : 0.0;
    int64_t last_nz = -1;
    for (int64_t j = 0; j < M; j++)
        if (alpha_at(alpha, dtype, j) > 0.0) last_nz = j;
    (void)nthreads;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int64_t i = 0; i < K; i++) {
        if (!(a0 > 0.0)) {
            idx[i] = (int32_t)M;
            continue;
        }
        uint32_t ctr[4] = {0u, (uint32_t)(sel_offset + (uint64_t)i), realization, 2u};
        uint32_t w[4];
        orc_philox4x32_10(ctr, seed, w);
        double target = u53(w[0], w[1]) * a0;
        int64_t pick = last_nz;
        for (int64_t j = 0; j < M; j++) {
            if (S[j] > target) {
                pick = j;
                break;
            }
        }
        idx[i] = (int32_t)pick;
    }
    free(S);
    return status;
}

/* ------------------------------------------------------------------------ */
/* The paper's own GPU rule (Section "Election step", "Selection step" and  */
/* the Results' pseudo-code), in FP32 as the paper's arrays are float:      */
/*   election: per j, u in [0,T); eligible iff u < D_j and D_j != 0; the    */
/*             rate is R_j = u / D_j, and an ineligible reaction gets +inf  */
/*             (reading: the printed sentinel T*10 can fall below 1).       */
/*   selection: j = argmin R (lowest j on ties); if min R >= 1 the election */
/*             failed and the sentinel M is returned.                       */
/* Random stream: reaction j of selection s uses counter (j/2, s, b, 3),    */
/* word 2(j mod 2)+1; u = floor(w / 2^8) * 2^-24 * T in FP32.               */
/* ------------------------------------------------------------------------ */
uint32_t orc_select_paper(const float *D, int64_t M, float T, int64_t K,
                          uint64_t seed, uint64_t sel_offset, uint32_t realization,
                          int32_t *idx, uint64_t *rejections, int nthreads)
{
    uint64_t rej = 0;
    (void)nthreads;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1) \
    reduction(+ : rej)
#endif
    for (int64_t i = 0; i < K; i++) {
        uint32_t s = (uint32_t)(sel_offset + (uint64_t)i);
        float best = INFINITY;
        int64_t arg = M;
        for (int64_t j = 0; j < M; j++) {
            uint32_t ctr[4] = {(uint32_t)(j >> 1), s, realization, 3u};
            uint32_t w[4];
            orc_philox4x32_10(ctr, seed, w);
            uint32_t wb = w[2 * (int)(j & 1) + 1];
            float u = (float)(wb >> 8) * 0x1p-24f;
            float uT = u * T;
            float R = INFINITY;
            if (uT < D[j] && D[j] != 0.0f) R = uT / D[j];
            if (R < best) {
                best = R;
                arg = j;
            }
        }
        if (best < 1.0f) {
            idx[i] = (int32_t)arg;
        } else {
            idx[i] = (int32_t)M;
            rej++;
        }
    }
    if (rejections) *rejections += rej;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* SSA direct method with AR selection (Section "The Stochastic Simulation  */
/* Algorithm"; the selection is the AR trial above with T = max_j a_j).     */
/*                                                                          */
/* Mass-action propensity a_r = c_r * h_r(X), one FP64 rounding of c_r      */
/* times the exact integer h_r:                                             */
/*   type 0 (source)  h = 1                                                 */
/*   type 1 (A)       h = x_A                      (0 if x_A <= 0)          */
/*   type 2 (A + B)   h = x_A * x_B                (0 if x_A or x_B <= 0)   */
/*   type 3 (2A)      h = x_A * (x_A - 1) / 2      (0 if x_A < 2)           */
/* Every propensity is recomputed from X at every step (no dependency       */
/* graph here: that is the library's optimization and this checks it).     */
/* Step n of realization b: T = max a, alpha_0 = sum a (index order);       */
/* T == 0 -> absorbed (the realization stops).  j = AR selection with       */
/* selection id n; tau = -ln(1 - u) / alpha_0 with u the 53-bit uniform of  */
/* counter (0, n, b, 1); X += v_j; t += tau; n += 1.                        */
/* ------------------------------------------------------------------------ */
static double propensity(int type, const int32_t *reac, double c, const int32_t *X)
{
    int64_t h = 0;
    if (type == 0) {
        h = 1;
    } else if (type == 1) {
        int64_t xa = X[reac[0]];
        h = xa > 0 ? xa : 0;
    } else if (type == 2) {
        int64_t xa = X[reac[0]], xb = X[reac[1]];
        h = (xa > 0 && xb > 0) ? xa * xb : 0;
    } else {
        int64_t xa = X[reac[0]];
        h = xa >= 2 ? xa * (xa - 1) / 2 : 0;
    }
    return c * (double)h;
}

void orc_ssa(int32_t N, int32_t M, const int32_t *rtype, const int32_t *reac,
             const double *rate, const int32_t *nu_ptr, const int32_t *nu_sp,
             const int32_t *nu_d, int64_t B, int32_t *X, double *t, uint64_t *step,
             int64_t nsteps, uint64_t seed, uint32_t realization_base, int cmp,
             uint64_t trial_cap, int32_t *last, uint32_t *status, double *a_out,
             uint64_t *trials_out, int nthreads)
{
    (void)nthreads;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int64_t b = 0; b < B; b++) {
        int32_t *Xb = X + b * (int64_t)N;
        double a[M > 0 ? M : 1];
        uint32_t bid = realization_base + (uint32_t)b;
        uint64_t ntr = 0;
        for (int64_t n = 0; n < nsteps; n++) {
            if (status[b] & (ST_ABSORBED | ST_TRIAL_CAP | ST_BAD_ALPHA)) break;
            double T = 0.0, a0 = 0.0;
            for (int32_t r = 0; r < M; r++) {
                a[r] = propensity(rtype[r], reac + 2 * r, rate[r], Xb);
                if (!(a[r] >= 0.0) || isinf(a[r])) status[b] |= ST_BAD_ALPHA;
                if (a[r] > T) T = a[r];
                a0 += a[r];
            }
            if (status[b] & ST_BAD_ALPHA) break;
            if (T == 0.0) {
                status[b] |= ST_ABSORBED;
                break;
            }
            uint32_t s = (uint32_t)step[b];
            uint64_t nt = 0;
            int64_t j = select_one(a, 1, M, T, cmp, seed, s, bid, trial_cap, &nt);
            ntr += nt;
            if (j >= M) {
                status[b] |= ST_TRIAL_CAP;
                break;
            }
            uint32_t ctr[4] = {0u, s, bid, 1u};
            uint32_t w[4];
            orc_philox4x32_10(ctr, seed, w);
            double u = u53(w[0], w[1]);
            double tau = -log(1.0 - u) / a0;
            for (int32_t q = nu_ptr[j]; q < nu_ptr[j + 1]; q++) Xb[nu_sp[q]] += nu_d[q];
            t[b] += tau;
            step[b] += 1;
            if (last) last[b] = (int32_t)j;
        }
        if (a_out) {
            for (int32_t r = 0; r < M; r++)
                a_out[b * (int64_t)M + r] = propensity(rtype[r], reac + 2 * r, rate[r], Xb);
        }
        if (trials_out) trials_out[b] += ntr;
    }
}

/* SSA to a time limit (the loop of Section "The Stochastic Simulation     */
/* Algorithm" run until the simulated time passes t_end), with trajectory   */
/* samples.  Each step draws its waiting time first; if t + tau > t_end the */
/* reaction does not fire and status T_END (128) is set; t stays at the     */
/* last reaction (the state holds on [t, t_end]), so a later call with a    */
/* larger limit continues exactly as one call would.                       */
/* Sample k (times ascending) records the state after the last reaction at  */
/* a time <= t_k, for the t_k this call passes; an absorbed realization     */
/* keeps its state to t_end.  At most max_steps reactions per realization.  */
void orc_ssa_until(int32_t N, int32_t M, const int32_t *rtype, const int32_t *reac,
                   const double *rate, const int32_t *nu_ptr, const int32_t *nu_sp,
                   const int32_t *nu_d, int64_t B, int32_t *X, double *t, uint64_t *step,
                   double t_end, int64_t max_steps, uint64_t seed, uint32_t realization_base,
                   int cmp, uint64_t trial_cap, const double *samp_t, int32_t nsamp,
                   const int32_t *samp_sp, int32_t nspec, int32_t *traj, int32_t *last,
                   uint32_t *status, uint64_t *trials_out, int nthreads)
{
    (void)nthreads;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int64_t b = 0; b < B; b++) {
        int32_t *Xb = X + b * (int64_t)N;
        double a[M > 0 ? M : 1];
        uint32_t bid = realization_base + (uint32_t)b;
        uint64_t ntr = 0;
        int32_t k = 0;
        while (k < nsamp && samp_t[k] < t[b]) k++;
        for (int64_t n = 0; n < max_steps; n++) {
            if (status[b] & (ST_ABSORBED | ST_TRIAL_CAP | ST_BAD_ALPHA)) break;
            double T = 0.0, a0 = 0.0;
            for (int32_t r = 0; r < M; r++) {
                a[r] = propensity(rtype[r], reac + 2 * r, rate[r], Xb);
                if (!(a[r] >= 0.0) || isinf(a[r])) status[b] |= ST_BAD_ALPHA;
                if (a[r] > T) T = a[r];
                a0 += a[r];
            }
            if (status[b] & ST_BAD_ALPHA) break;
            if (T == 0.0) {
                status[b] |= ST_ABSORBED;
                for (; k < nsamp && samp_t[k] <= t_end; k++)
                    for (int32_t q = 0; q < nspec; q++)
                        traj[(b * nsamp + k) * (int64_t)nspec + q] = Xb[samp_sp ? samp_sp[q] : q];
                break;
            }
            uint32_t s = (uint32_t)step[b];
            uint32_t ctr[4] = {0u, s, bid, 1u};
            uint32_t w[4];
            orc_philox4x32_10(ctr, seed, w);
            double t_next = t[b] + -log(1.0 - u53(w[0], w[1])) / a0;
            int over = t_next > t_end;
            for (; k < nsamp && (over ? samp_t[k] <= t_end : samp_t[k] < t_next); k++)
                for (int32_t q = 0; q < nspec; q++)
                    traj[(b * nsamp + k) * (int64_t)nspec + q] = Xb[samp_sp ? samp_sp[q] : q];
            if (over) {
                status[b] |= 128u;
                break;
            }
            uint64_t nt = 0;
            int64_t j = select_one(a, 1, M, T, cmp, seed, s, bid, trial_cap, &nt);
            ntr += nt;
            if (j >= M) {
                status[b] |= ST_TRIAL_CAP;
                break;
            }
            for (int32_t q = nu_ptr[j]; q < nu_ptr[j + 1]; q++) Xb[nu_sp[q]] += nu_d[q];
            t[b] = t_next;
            step[b] += 1;
            if (last) last[b] = (int32_t)j;
        }
        if (trials_out) trials_out[b] += ntr;
    }
}

int orc_num_threads_available(void)
{
#ifdef _OPENMP
    return omp_get_num_procs();
#else
    return 1;
#endif
}
