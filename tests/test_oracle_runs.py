"""Pins for the oracle's run selection (the random sequence of the batched
entry points): selections in runs of 64 consecutive selection numbers, each
run one sequence of AR trials whose accepted trials are, in order, its
selections (the classical AR loop of Section "A GPU acceptance-rejection
algorithm" applied to consecutive selections).

What fixes each expected value (never the run oracle itself):
* constant alpha accepts every trial, so the selections are the candidate
  sequence floor(w_a M / 2^32) of the Philox words (Philox itself pinned
  against cuRAND's host generator), which pins the trial -> word mapping;
* one non-zero entry k: a trial accepts iff its candidate is k, so with a
  trial cap the decisions follow from the candidate sequence alone (a
  brute-force walk over it), which pins the cap rule and the trial counts;
* the exact law alpha_j / sum(alpha) (chi-square), and independence of
  consecutive selections of a run (chi-square of pairs against the product
  law);
* the expected number of trials per selection M T / sum(alpha);
* splitting a call's selections over two calls (sel_offset) changes nothing.
"""
import numpy as np
import pytest

from oracle import law


def run_words(orc, seed, g, b, n):
    """(w_a, w_b) of trials 0 .. n - 1 of run g of realization b: trial
    64 G + 32 h + i takes words 2h, 2h + 1 of block 32 G + i of counter
    (block, g, b, 0)."""
    nb = 32 * ((n + 63) // 64)
    ctr = np.zeros((nb, 4), dtype=np.uint32)
    ctr[:, 0] = np.arange(nb)
    ctr[:, 1] = g
    ctr[:, 2] = b
    w = orc.philox(ctr, seed).reshape(-1, 32, 4)
    wa = np.stack([w[:, :, 0], w[:, :, 2]], 1).reshape(-1)[:n]
    wb = np.stack([w[:, :, 1], w[:, :, 3]], 1).reshape(-1)[:n]
    return wa, wb


def candidates(orc, seed, g, b, n, M):
    wa, _ = run_words(orc, seed, g, b, n)
    return ((wa.astype(np.uint64) * np.uint64(M)) >> np.uint64(32)).astype(np.int64)


@pytest.mark.parametrize("cmp", [0, 1])
@pytest.mark.parametrize("M", [1, 7, 1000, 16384])
def test_constant_alpha_is_the_candidate_sequence(orc, cmp, M):
    a = np.full(M, 2.5, dtype=np.float32 if cmp == 0 else np.float64)
    K, off, b = 300, 50, 9          # selections 50 .. 349: runs 0 .. 5, partial at both ends
    idx, stats, st = orc.select_runs(a, K, seed=3, sel_offset=off, realization=b, cmp=cmp)
    assert st == 0
    want = []
    for s in range(off, off + K):
        g, r = divmod(s, 64)
        want.append(candidates(orc, 3, g, b, r + 1, M)[r])   # decision r = trial r
    np.testing.assert_array_equal(idx, want)
    assert list(stats) == [K, K, 0]   # one trial per selection


def walk(cands, k, M, first, last, cap):
    """Decisions first .. last - 1 of a run whose trial n accepts iff
    cands[n] == k: (decisions, trials consumed by them, capped count)."""
    n, out, trials, capped = 0, [], 0, 0
    for r in range(last):
        start = n
        sel = M
        while n - start < cap:
            n += 1
            if cands[n - 1] == k:
                sel = k
                break
        if r >= first:
            out.append(sel)
            trials += n - start
            capped += sel == M
    return out, trials, capped


@pytest.mark.parametrize("cap", [1, 2, 3, 7, 1 << 20])
@pytest.mark.parametrize("cmp", [0, 1])
def test_one_nonzero_entry_with_trial_cap(orc, cap, cmp):
    M, k = 5, 3
    a = np.zeros(M, dtype=np.float32 if cmp == 0 else np.float64)
    a[k] = 0.75
    K, off, b, seed = 150, 20, 4, 11   # decisions 20 .. 169: runs 0 .. 2
    idx, stats, st = orc.select_runs(a, K, seed=seed, sel_offset=off, realization=b, cmp=cmp,
                                     trial_cap=cap)
    want, trials, capped = [], 0, 0
    for g in range(off // 64, (off + K - 1) // 64 + 1):
        first = max(off, 64 * g) - 64 * g
        last = min(off + K, 64 * g + 64) - 64 * g
        c = candidates(orc, seed, g, b, 64 * 64 * 40, M)
        d, t, cp = walk(c, k, M, first, last, cap)
        want += d
        trials += t
        capped += cp
    np.testing.assert_array_equal(idx, want)
    assert list(stats) == [trials, K - capped, capped]
    assert bool(st & orc.ST_TRIAL_CAP) == (capped > 0)
    if cap <= 3:
        assert capped > 0            # the cap is reached for this seed


def test_law_of_the_selections(orc):
    a = np.array([3.0, 0.0, 1.0, 2.0, 4.0, 0.5])
    idx, stats, st = orc.select_runs(a, 400_000, seed=5, realization=2, cmp=1)
    assert st == 0
    counts = np.bincount(idx, minlength=a.size)
    assert counts[1] == 0
    assert law.chi_square(counts, law.exact_law(a)) > 1e-3
    # M = 2: the exact rule (2/3, 1/3)
    idx, _, _ = orc.select_runs(np.array([2.0, 1.0]), 300_000, seed=6, cmp=1)
    assert abs(np.mean(idx == 0) - 2.0 / 3.0) < 4 * np.sqrt(2.0 / 9.0 / 300_000)


def test_consecutive_selections_are_independent(orc):
    """Pairs (d_r, d_r+1) inside a run follow the product law."""
    a = np.array([1.0, 2.0, 3.0], dtype=np.float32)
    K = 64 * 4000
    idx, _, _ = orc.select_runs(a, K, seed=8, realization=1, cmp=0)
    d = idx.reshape(-1, 64)
    pairs = 3 * d[:, :-1] + d[:, 1:]
    counts = np.bincount(pairs.ravel(), minlength=9)
    p = law.exact_law(a)
    assert law.chi_square(counts, np.outer(p, p).ravel()) > 1e-3


@pytest.mark.parametrize("w", [1.0, 2.0])
def test_expected_trials_per_selection(orc, w):
    rng = np.random.default_rng(2)
    a = rng.exponential(1.0, 300)
    T = w * float(a.max())
    K = 100_000
    idx, stats, st = orc.select_runs(a, K, seed=9, cmp=1, bound_value=T)
    p = a.sum() / (a.size * T)                   # acceptance probability per trial
    mean, var = 1.0 / p, (1.0 - p) / p ** 2      # geometric trials per selection
    assert abs(stats[0] / K - mean) < 5 * np.sqrt(var / K)
    assert stats[1] == K and stats[2] == 0


def test_split_calls_equal_one_call(orc):
    a = np.random.default_rng(4).lognormal(0.0, 1.0, 777)
    full, sf, _ = orc.select_runs(a, 500, seed=12, sel_offset=30, realization=6, cmp=1)
    parts, st_sum = [], np.zeros(3, np.uint64)
    for lo, hi in ((30, 67), (67, 128), (128, 129), (129, 530)):
        i, s, _ = orc.select_runs(a, hi - lo, seed=12, sel_offset=lo, realization=6, cmp=1)
        parts.append(i)
        st_sum += s
    np.testing.assert_array_equal(np.concatenate(parts), full)
    np.testing.assert_array_equal(st_sum, sf)
    # another realization id is another sequence
    other, _, _ = orc.select_runs(a, 500, seed=12, sel_offset=30, realization=7, cmp=1)
    assert np.mean(other == full) < 0.2


def test_degenerate_inputs(orc):
    idx, stats, st = orc.select_runs(np.zeros(6), 70)
    assert st == orc.ST_ALL_ZERO and np.all(idx == 6) and list(stats) == [0, 0, 0]
    idx, _, st = orc.select_runs(np.zeros(0), 3)
    assert st == orc.ST_ALL_ZERO and np.all(idx == 0)
    idx, stats, st = orc.select_runs(np.ones(4), 0)
    assert st == 0 and idx.size == 0
    for T in (np.nan, -1.0, np.inf):
        idx, _, st = orc.select_runs(np.ones(4), 65, bound_value=T)
        assert st == orc.ST_BAD_BOUND and np.all(idx == 4)
