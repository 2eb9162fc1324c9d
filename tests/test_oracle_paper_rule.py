"""Pins the paper's own election/argmin rule to the paper's printed Table 1.

The law of the election rule (u_j uniform in [0,T), eligible iff u_j < D_j,
winner = argmin u_j / D_j) has the closed form ``oracle.law.paper_law``.  Its
predicted MSE on the paper's discrete Gaussian propensities (Section "Test and
validation of the algorithm") must reproduce Table 1 (Section "Quality of the
selection of the reaction indexes"; fixture tests/golden/table1_mse.txt): the
printed values must fall inside the sampling spread of one run and of the worst
of ten runs of 10^7 selections drawn from that law.  An exact sampler would give
MSEs a hundred times smaller at M = 64: the printed errors are the rule's bias.
"""
import os

import numpy as np
import pytest

from oracle import law
from paper_1404_0027_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_mse.txt")
N_SEL = 10_000_000


def _table():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            dist, K, M, t1, t2 = line.split()
            rows.append((dist, int(K), int(M), float(t1), float(t2)))
    return rows


def _mse_spread(P, p, rng, reps=150):
    single, worst = [], []
    for _ in range(reps):
        runs = [float(np.mean((p - rng.multinomial(N_SEL, P) / N_SEL) ** 2)) for _ in range(10)]
        single.append(runs[0])
        worst.append(max(runs))
    return np.array(single), np.array(worst)


@pytest.mark.parametrize("M", [64, 256, 1024])
def test_table1_gaussian_rows(M):
    rows = [r for r in _table() if r[0] == "gaussian" and r[2] == M]
    assert len(rows) == 5
    D = W.gaussian_paper(M)
    p = D / D.sum()
    P, p_rej = law.paper_law(D)
    assert p_rej == 0.0                       # T = max: never rejects (Section 3.3)
    assert abs(P.sum() - 1.0) < 1e-9
    rng = np.random.default_rng(1000 + M)
    single, worst = _mse_spread(P / P.sum(), p, rng)
    lo, hi = np.quantile(single, 0.0005), np.quantile(worst, 0.9995)
    printed = [v for r in rows for v in r[3:]]
    assert all(lo <= v <= hi for v in printed), (lo, hi, printed)
    if M == 64:
        # an exact sampler cannot produce the printed errors
        _, worst_exact = _mse_spread(p, p, rng, reps=40)
        assert worst_exact.max() < 0.05 * min(printed)


def test_paper_rule_threshold_has_no_effect():
    """Table 1's two thresholds give the same MSE; so does the law for w in [1, 2]."""
    D = W.gaussian_paper(64)
    p = D / D.sum()
    m1 = law.predicted_mse(law.paper_law(D)[0], p, N_SEL)
    P2, rej2 = law.paper_law(D, T=1.5 * D.max())
    m2 = law.predicted_mse(P2 / P2.sum(), p, N_SEL)
    assert abs(m1 - m2) < 1e-3 * m1 and rej2 < 1e-6


def test_oracle_paper_sampler_follows_paper_law(orc):
    D = W.gaussian_paper(64).astype(np.float32)
    P, _ = law.paper_law(D.astype(np.float64))
    idx, rej = orc.select_paper(D, 400_000, nthreads=8)
    assert rej == 0
    assert law.chi_square(np.bincount(idx, minlength=64), P) > 1e-3
    assert law.chi_square(np.bincount(idx, minlength=64), law.exact_law(D)) < 1e-6
