"""CPU pins of the accuracy report's statistics (paper_1404_0027_gb300/accuracy.py):
exact samplers pass the chi-square and show the predicted TV noise floor, a
sampler biased by a few per cent fails, paired figures on hand-made arrays."""
import numpy as np
import pytest

from paper_1404_0027_gb300 import accuracy as A

pytest.importorskip("scipy")


def test_paired_hand_made():
    a = np.array([0, 1, 2, 2, 3])
    b = np.array([0, 1, 2, 3, 3])
    r = A.paired(a, b, 5)
    assert r["n"] == 5
    assert r["index_mismatch"] == pytest.approx(0.2)
    # histograms (1,1,2,1,0) and (1,1,1,2,0): TV = 0.5 * 2 / 5
    assert r["paired_tv"] == pytest.approx(0.2)
    # a permutation of the same multiset: every index differs, TV = 0
    r = A.paired(np.array([1, 2, 3]), np.array([3, 1, 2]), 4)
    assert r["index_mismatch"] == 1.0 and r["paired_tv"] == 0.0


def test_merged_bins_reach_five():
    rng = np.random.default_rng(3)
    e = rng.exponential(1.3, size=5000)
    bins = A.merged_bins(e)
    tot = np.bincount(bins, weights=e)
    assert (tot >= 5.0).all()
    assert (np.diff(bins) >= 0).all() and (np.diff(bins) <= 1).all()   # adjacent cells only


def _alpha(M, seed, zeros=0):
    rng = np.random.default_rng(seed)
    a = rng.lognormal(0.0, 2.0, size=M)
    a[rng.permutation(M)[:zeros]] = 0.0
    return a


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_exact_sampler_passes(seed):
    a = _alpha(1029, seed, zeros=309)
    p = a / a.sum()
    n = 1_000_000
    idx = np.random.default_rng(100 + seed).choice(a.size, size=n, p=p)
    r = A.law(idx, a)
    assert r["count_in_zero_bins"] == 0
    assert r["p_value"] > 1e-3, r
    # the noise floor formula predicts the TV of an exact sampler
    assert 0.85 * r["tv_exact_sampler_expected"] < r["tv_vs_exact"] < 1.15 * r[
        "tv_exact_sampler_expected"], r


def test_biased_sampler_fails():
    a = _alpha(1029, 7)
    p = a / a.sum()
    q = p * np.where(np.arange(a.size) % 2 == 0, 1.03, 0.97)   # +-3 % bias
    q /= q.sum()
    idx = np.random.default_rng(8).choice(a.size, size=2_000_000, p=q)
    assert A.law(idx, a)["p_value"] < 1e-6


def test_zero_bin_and_sentinel_counted():
    a = np.array([1.0, 0.0, 2.0])
    idx = np.array([0, 1, 2, 3, 2, 0])
    r = A.law(idx, a)
    assert r["count_in_zero_bins"] == 2     # one on the zero propensity, one sentinel
