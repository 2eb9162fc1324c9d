"""Accuracy report of an FP32-comparison result against the FP64 comparison on
the same random streams, and against the exact law P(j) = alpha_j / sum(alpha)
(Section "A GPU acceptance-rejection algorithm"; the paper's quality
experiment draws 10^7 selections and compares their frequencies with the
normalised propensities, Results, "Quality of the selection of the reaction
indexes", Table 1).

Host-side statistics on index arrays the library returned; none of the
selection's arithmetic is here.

* paired index-mismatch rate: the fraction of selections whose FP32 and FP64
  results differ (both draw the same Philox words);
* paired TV: total-variation distance between the two empirical histograms,
  0.5 sum_j |h32_j - h64_j| / n, never above the mismatch rate;
* empirical TV against the exact law, reported with the TV an exact sampler
  shows at the same n (its noise floor, 0.5 sum_j sqrt(2 p_j (1 - p_j) / (pi n))
  from the normal approximation of each binomial count);
* chi-square goodness of fit against the exact law, adjacent bins merged in
  index order until each expected count is at least 5 (the merging uses the
  expected counts only), and the count in zero-propensity bins, which must be
  zero.
"""
from __future__ import annotations

import math

import numpy as np


def paired(idx32: np.ndarray, idx64: np.ndarray, ncells: int) -> dict:
    """Mismatch rate and paired TV of two index arrays over cells 0..ncells-1."""
    idx32 = np.asarray(idx32).astype(np.int64, copy=False)
    idx64 = np.asarray(idx64).astype(np.int64, copy=False)
    n = idx32.size
    h32 = np.bincount(idx32, minlength=ncells)
    h64 = np.bincount(idx64, minlength=ncells)
    return {"n": int(n), "index_mismatch": float(np.count_nonzero(idx32 != idx64)) / n,
            "paired_tv": 0.5 * float(np.abs(h32 - h64).sum()) / n}


def merged_bins(expected: np.ndarray, min_expected: float = 5.0) -> np.ndarray:
    """Bin id per cell: adjacent cells merged in index order until each bin's
    expected count reaches min_expected (a short last bin joins the one
    before).  Cells with zero expectation are left to the caller."""
    e = np.asarray(expected, dtype=np.float64)
    bins = np.empty(e.size, dtype=np.int64)
    b, acc = 0, 0.0
    for k in range(e.size):
        bins[k] = b
        acc += e[k]
        if acc >= min_expected:
            b += 1
            acc = 0.0
    if acc < min_expected and b > 0:
        bins[bins == b] = b - 1
    return bins


def law(idx: np.ndarray, alpha: np.ndarray) -> dict:
    """Chi-square and TV of the histogram of idx (values 0..M, M = the
    sentinel) against alpha_j / sum(alpha)."""
    from scipy.stats import chi2

    a = np.asarray(alpha, dtype=np.float64)
    M = a.size
    n = int(np.asarray(idx).size)
    h = np.bincount(np.asarray(idx).astype(np.int64), minlength=M + 1)
    p = a / a.sum()
    zero = p == 0.0
    in_zero = int(h[:M][zero].sum()) + int(h[M])   # zero-propensity bins and sentinels
    nz = np.flatnonzero(~zero)
    exp = n * p[nz]
    bins = merged_bins(exp)
    nb = int(bins.max()) + 1
    o_b = np.bincount(bins, weights=h[nz].astype(np.float64), minlength=nb)
    e_b = np.bincount(bins, weights=exp, minlength=nb)
    stat = float(((o_b - e_b) ** 2 / e_b).sum())
    dof = nb - 1
    tv = 0.5 * float(np.abs(h[:M] / n - p).sum() + h[M] / n)
    floor = 0.5 * float(np.sqrt(2.0 * p * (1.0 - p) / (math.pi * n)).sum())
    return {"n": n, "chi2": stat, "dof": dof, "p_value": float(chi2.sf(stat, dof)),
            "bins": nb, "count_in_zero_bins": in_zero, "tv_vs_exact": tv,
            "tv_exact_sampler_expected": floor}
