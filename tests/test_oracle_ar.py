"""Pins for the oracle's bound, AR selection and inverse-transform sampler.

What fixes each expected value (never the oracle itself):
* the exact law P(j) = alpha_j / sum(alpha) (chi-square, p > 0.001);
* the counting law of the implemented trial (``oracle.law.impl_law``), whose
  distance to the exact law is bounded analytically;
* closed forms: constant alpha accepts every trial, one non-zero entry is always
  chosen, an all-zero vector is the paper's rejection case, M = 2 separates the
  exact rule (2/3, 1/3) from the paper's election rule (3/4, 1/4);
* the acceptance probability per trial sum(alpha) / (M T);
* math.fsum for the total propensity, numpy for the maximum.
"""
import math

import numpy as np
import pytest

from oracle import law
from paper_1404_0027_gb300 import workloads as W


def test_bound_max_and_sum(orc):
    for a in (W.plain_uniform(), W.skewed(), W.wide_range(M=1 << 14),
              np.array([0.0], dtype=np.float32), np.zeros(0)):
        mx, sm, st = orc.bound(a)
        ref_max = float(a.max()) if a.size else 0.0
        assert mx == ref_max
        exact = math.fsum(a.astype(np.float64).tolist())
        assert abs(sm - exact) <= max(a.size, 1) * 2.0 ** -53 * exact
        assert st == (orc.ST_ALL_ZERO if ref_max == 0 else 0)


@pytest.mark.parametrize("bad", [np.nan, -1.0, np.inf, -np.inf])
def test_bound_flags_bad_alpha(orc, bad):
    a = W.plain_uniform(64)
    a[17] = bad
    assert orc.bound(a)[2] & orc.ST_BAD_ALPHA
    assert orc.bound(a.astype(np.float32))[2] & orc.ST_BAD_ALPHA


def test_negative_zero_is_zero(orc):
    a = np.array([-0.0, 0.5, -0.0], dtype=np.float32)
    mx, sm, st = orc.bound(a)
    assert (mx, sm, st) == (0.5, 0.5, 0)
    idx, _, _ = orc.select_ar(a, 1000, cmp=orc.CMP_F32)
    assert np.all(idx == 1)


@pytest.mark.parametrize("cmp", [0, 1])
@pytest.mark.parametrize("M", [1, 3, 1000, 1 << 16, 1029])
def test_constant_alpha_accepts_first_trial(orc, cmp, M):
    """Constant alpha: u*T < alpha for every u < 1, so trial 0 decides and the
    index is floor(w * M / 2^32) of word 0 of Philox block (0, s, b, 0)."""
    K, b, off = 512, 9, 1000
    a = np.full(M, 0.37, dtype=np.float64)
    idx, stats, st = orc.select_ar(a, K, seed=5, sel_offset=off, realization=b, cmp=cmp)
    ctr = np.zeros((K, 4), dtype=np.uint32)
    ctr[:, 1] = off + np.arange(K)
    ctr[:, 2] = b
    w = orc.philox(ctr, 5)
    expect = [(int(x) * M) >> 32 for x in w[:, 0]]
    np.testing.assert_array_equal(idx, expect)
    assert stats.tolist() == [K, K, 0] and st == 0


def test_single_nonzero_and_all_zero(orc):
    a = np.zeros(777, dtype=np.float32)
    a[123] = 3.5
    idx, stats, st = orc.select_ar(a, 2000, cmp=0)
    assert np.all(idx == 123) and st == 0 and stats[1] == 2000
    # acceptance per trial is 1/M exactly (u*T < T always)
    trials = int(stats[0])
    assert abs(trials / 2000 - 777) < 6 * math.sqrt(777 * 776 / 2000)
    z = np.zeros(50)
    idx, stats, st = orc.select_ar(z, 10)
    assert np.all(idx == 50) and st == orc.ST_ALL_ZERO and stats.tolist() == [0, 0, 0]
    idx, stats, st = orc.select_ar(np.zeros(0), 4)
    assert np.all(idx == 0) and st == orc.ST_ALL_ZERO


def test_bad_bound(orc):
    a = W.plain_uniform(16)
    for T in (np.nan, -1.0, np.inf):
        idx, _, st = orc.select_ar(a, 8, bound_value=T)
        assert st == orc.ST_BAD_BOUND and np.all(idx == 16)
    idx, _, st = orc.select_ar(a, 8, bound_value=1e300, cmp=0)   # inf in FP32
    assert st == orc.ST_BAD_BOUND


def test_m2_exact_rule_vs_paper_rule(orc):
    """D = (T, T/2): the AR trial gives (2/3, 1/3); the paper's election rule
    gives (3/4, 1/4) (closed form of its law)."""
    a = np.array([2.0, 1.0])
    K = 200_000
    idx, _, _ = orc.select_ar(a, K, cmp=1, nthreads=4)
    c = np.bincount(idx, minlength=2)
    assert law.chi_square(c, [2 / 3, 1 / 3]) > 1e-3
    assert law.chi_square(c, [3 / 4, 1 / 4]) < 1e-12
    P, rej = law.paper_law(a)
    np.testing.assert_allclose(P, [0.75, 0.25], rtol=0, atol=1e-12)
    pidx, prej = orc.select_paper(a.astype(np.float32), K, nthreads=4)
    assert prej == 0
    assert law.chi_square(np.bincount(pidx, minlength=2), [0.75, 0.25]) > 1e-3


@pytest.mark.parametrize("cmp", [0, 1])
def test_impl_law_close_to_exact(cmp):
    """The finite random words realise the exact law up to the candidate
    mapping's preimage imbalance (relative <= M / 2^32 per index) and the u
    lattice (a step of 2^-24 T or 2^-32 T in the accepted length of each
    index, relative to the acceptance probability per trial p):
    TV <= M / 2^32 + 1 / (p 2^bits)."""
    bits = 24 if cmp == 0 else 32
    for a in (W.plain_uniform(64), W.skewed(61, seed=3), np.array([1e-3, 1.0, 0.0, 7.0])):
        P, pacc = law.impl_law(a, cmp=cmp)
        ex = law.exact_law(a)
        assert law.tv(P, ex) <= a.size / 2.0 ** 32 + 1.0 / (pacc * 2.0 ** bits)
        a64 = a.astype(np.float64)
        np.testing.assert_allclose(pacc, a64.sum() / (a.size * a64.max()),
                                   rtol=2.0 / (pacc * 2.0 ** bits) + a.size / 2.0 ** 32)
        assert np.all(P[a == 0] == 0)


def test_candidate_preimages_balanced():
    for M in (1, 3, 1000, 1029, 1 << 20):
        pre = law.candidate_preimages(M) if M < 5000 else None
        if pre is not None:
            assert pre.sum() == 1 << 32
            assert set(np.unique(pre)) <= {(1 << 32) // M, -(-(1 << 32) // M)}


@pytest.mark.parametrize("cmp", [0, 1])
def test_chi_square_plain_uniform(orc, cmp):
    a = W.plain_uniform()
    K = 2_000_000
    idx, stats, st = orc.select_ar(a, K, cmp=cmp, nthreads=8)
    assert st == 0 and int(stats[1]) == K
    counts = np.bincount(idx, minlength=a.size)
    assert law.chi_square(counts, law.exact_law(a)) > 1e-3
    # acceptance per trial = sum / (M max)
    pacc = a.sum() / (a.size * a.max())
    rate = K / float(stats[0])
    sd = math.sqrt(pacc * (1 - pacc) / float(stats[0]))
    assert abs(rate - pacc) < 6 * sd


def test_chi_square_skewed_f32(orc):
    a = W.skewed()
    K = 300_000
    idx, stats, st = orc.select_ar(a, K, cmp=0, nthreads=8)
    counts = np.bincount(idx, minlength=a.size)
    assert counts[a == 0].sum() == 0
    assert law.chi_square(counts, law.exact_law(a)) > 1e-3


def test_f32_f64_paired_mismatch_small(orc):
    """Same random words, two comparison precisions: decisions differ only on
    the thin set where fl32 rounding crosses alpha_j."""
    a = W.skewed(seed=201).astype(np.float32)
    K = 100_000
    i32, _, _ = orc.select_ar(a, K, cmp=0, nthreads=8)
    i64, _, _ = orc.select_ar(a, K, cmp=1, nthreads=8)
    assert np.mean(i32 != i64) < 1e-3


def test_trial_cap(orc):
    a = W.plain_uniform(100)
    T = a.max() * 1e6
    idx, stats, st = orc.select_ar(a, 1000, bound_value=T, trial_cap=8)
    capped = idx == 100
    assert capped.sum() > 990 and st & orc.ST_TRIAL_CAP
    assert int(stats[2]) == capped.sum() and int(stats[1]) == 1000 - capped.sum()
    # capped selections consumed exactly trial_cap trials
    assert int(stats[0]) >= 8 * int(stats[2])
    # a larger cap extends the same streams: uncapped results are unchanged
    idx2, _, _ = orc.select_ar(a, 1000, bound_value=T, trial_cap=16)
    np.testing.assert_array_equal(idx2[~capped], idx[~capped])


def test_larger_bound_keeps_law(orc):
    """T_w = w max with w > 1 keeps the exact law (only acceptance drops)."""
    a = W.plain_uniform(256, seed=5)
    K = 400_000
    idx, stats, _ = orc.select_ar(a, K, bound_value=4 * a.max(), nthreads=8)
    assert law.chi_square(np.bincount(idx, minlength=256), law.exact_law(a)) > 1e-3
    assert K / float(stats[0]) < 0.2


def test_selection_ids_and_realizations_are_streams(orc):
    a = W.skewed(seed=9)
    full, _, _ = orc.select_ar(a, 3000, sel_offset=100, realization=4, cmp=0)
    part, _, _ = orc.select_ar(a, 1000, sel_offset=1100, realization=4, cmp=0)
    np.testing.assert_array_equal(full[1000:2000], part)
    other, _, _ = orc.select_ar(a, 3000, sel_offset=100, realization=5, cmp=0)
    assert np.mean(other == full) < 0.2


def test_inverse_transform(orc):
    a = W.skewed(seed=11)
    idx, st = orc.select_it(a, 300_000, nthreads=8)
    counts = np.bincount(idx, minlength=a.size)
    assert counts[a == 0].sum() == 0
    assert law.chi_square(counts, law.exact_law(a)) > 1e-3
    # tiny case: boundaries of the cumulative sum, u from counter (0, s, b, 2)
    a3 = np.array([1.0, 0.0, 3.0])
    idx3, _ = orc.select_it(a3, 64, seed=3)
    ctr = np.zeros((64, 4), dtype=np.uint32)
    ctr[:, 1] = np.arange(64)
    ctr[:, 3] = 2
    w = orc.philox(ctr, 3)
    u = [((int(x) << 21) | (int(y) >> 11)) / 2.0 ** 53 for x, y in w[:, :2]]
    np.testing.assert_array_equal(idx3, [0 if x * 4.0 < 1.0 else 2 for x in u])
    assert np.all(orc.select_it(np.zeros(5), 3)[0] == 5)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_it_prefix_is_fsum_of_each_prefix(orc, dtype):
    """Running sums of the inverse transform: the exact prefix sums rounded
    once (math.fsum returns the correctly rounded sum of its arguments), for
    data whose terms all lie within 2^73 (FP32) / 2^44 (FP64) of the
    maximum's binade, so that no term is rounded down to the unit."""
    rng = np.random.default_rng(5)
    a = rng.lognormal(0.0, 2.0, 1500).astype(dtype)
    a[rng.permutation(a.size)[:300]] = 0.0
    S, st = orc.it_prefix(a)
    assert st == 0
    want = [math.fsum(a[:j + 1].astype(np.float64)) for j in range(a.size)]
    np.testing.assert_array_equal(S, want)
    # a larger vector on sampled prefixes; index-order FP64 sums differ
    a = rng.lognormal(0.0, 3.0, 1 << 16).astype(dtype)
    S, _ = orc.it_prefix(a)
    for j in rng.integers(0, a.size, 40):
        assert S[j] == math.fsum(a[:j + 1].astype(np.float64))
    assert np.any(S != np.cumsum(a.astype(np.float64)))


def test_it_prefix_truncation_bound(orc):
    """Terms far below the maximum enter rounded down to the unit
    2^(E - 223) (FP32): the sums stay within j units (plus the final
    rounding) of the exact ones."""
    a = np.float32([3e20, 1e-10, 7.5, 2e-30, 4.0e10, 1e-25] * 50)
    S, st = orc.it_prefix(a)
    assert st == 0
    E = int(np.float32(3e20).view(np.uint32) >> 23)
    unit = 2.0 ** (E - 223)
    for j in range(a.size):
        exact = math.fsum(a[:j + 1].astype(np.float64))
        assert abs(S[j] - exact) <= (j + 1) * unit + 2.0 ** -53 * exact
    # the tiny terms (below one unit) do not move the sum
    assert S[1] == S[0] and S[3] == S[2]


def test_it_invalid_and_zero(orc):
    for a in (np.float32([1.0, np.nan, 2.0]), np.array([1.0, -1.0, 3.0]),
              np.float32([np.inf, 1.0])):
        idx, st = orc.select_it(a, 20)
        assert st & 1 and np.all(idx == a.size)        # reading: BAD_ALPHA -> sentinel
    idx, st = orc.select_it(np.zeros(4), 5)
    assert st == 2 and np.all(idx == 4)


def test_batched_oracle_matches_single(orc):
    bt = W.batched_uneven(B=6, seed=3, m_lo=4, m_hi=300, K=40)
    bs, idx, stats, st = orc.select_batched(bt, seed=2, sel_offset=7, realization_base=10)
    for b in range(bt.B):
        a = bt.alpha[bt.offsets[b]:bt.offsets[b + 1]]
        mx, sm, _ = orc.bound(a)
        assert bs[b, 0] == mx and bs[b, 1] == sm
        ib, _, _ = orc.select_runs(a, 40, seed=2, sel_offset=7, realization=10 + b, cmp=0)
        np.testing.assert_array_equal(idx[bt.out_offsets[b]:bt.out_offsets[b + 1]], ib)
    assert int(stats[1]) == 6 * 40


def test_batched_invalid_realization(orc):
    """A realization with an invalid propensity has no usable bound: (NaN, NaN),
    every index the sentinel M_b, BAD_ALPHA; the others are unaffected."""
    bt = W.batched_uneven(B=5, seed=4, m_lo=8, m_hi=200, K=30)
    bad = bt.alpha.copy()
    bad[bt.offsets[2] + 3] = np.nan
    bt2 = W.Batch(bad, bt.offsets, bt.out_offsets)
    bs, idx, _, st = orc.select_batched(bt)
    bs2, idx2, _, st2 = orc.select_batched(bt2)
    assert st2 & orc.ST_BAD_ALPHA and not st & orc.ST_BAD_ALPHA
    assert np.isnan(bs2[2]).all()
    M2 = bt.offsets[3] - bt.offsets[2]
    np.testing.assert_array_equal(idx2[bt.out_offsets[2]:bt.out_offsets[3]], M2)
    keep = np.ones(idx.size, bool)
    keep[bt.out_offsets[2]:bt.out_offsets[3]] = False
    np.testing.assert_array_equal(idx2[keep], idx[keep])


@pytest.mark.parametrize("w", [1.5, 2.0, 4.0])
def test_threshold_sweep_trials_and_law(orc, w):
    """T_w = w max (the paper's threshold experiment): the expected number of
    trials per selection is M T_w / sum(alpha) (geometric with success
    probability sum(alpha) / (M T_w)), and the law stays exact."""
    a = W.plain_uniform(200, seed=21)
    bt = W.batch_from_vectors([a], [60_000])
    T = w * float(a.max())
    idx, stats, st = orc.select_batched_bounded(bt, [T], nthreads=8)
    assert st == 0
    p = math.fsum(a.tolist()) / (a.size * T)
    mean_t = float(stats[0]) / 60_000
    sd = math.sqrt((1 - p) / p ** 2 / 60_000)
    assert abs(mean_t - 1 / p) < 4 * sd, (mean_t, 1 / p, sd)
    assert law.chi_square(np.bincount(idx, minlength=a.size), law.exact_law(a)) > 1e-3


def test_bounded_batched_with_own_maxima_equals_batched(orc):
    """Bounds equal to each realization's maximum reproduce ar_select_batched;
    stride 2 reads a bound_sum array; bad bounds give BAD_BOUND and M_b."""
    bt = W.batched_uneven(B=7, seed=8, m_lo=4, m_hi=500, K=25)
    bs, idx, stats, st = orc.select_batched(bt, seed=3, sel_offset=5, realization_base=2)
    idx2, stats2, st2 = orc.select_batched_bounded(bt, bs.ravel(), stride=2, seed=3, sel_offset=5,
                                                   realization_base=2)
    np.testing.assert_array_equal(idx2, idx)
    np.testing.assert_array_equal(stats2, stats)
    assert st2 == st
    T = bs[:, 0].copy()
    T[1], T[4] = np.nan, -1.0
    idx3, _, st3 = orc.select_batched_bounded(bt, T, seed=3, sel_offset=5, realization_base=2)
    assert st3 & orc.ST_BAD_BOUND
    for b in (1, 4):
        sl = slice(bt.out_offsets[b], bt.out_offsets[b + 1])
        assert (idx3[sl] == bt.offsets[b + 1] - bt.offsets[b]).all()
