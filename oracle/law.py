"""Selection laws that pin the oracle (test infrastructure only).

* ``exact_law``      P(j) = alpha_j / sum_i alpha_i, the law every SSA next-reaction
                     selection must follow (Section "Assessing the qualities of
                     GPU/AR algorithm": the selection probability should match the
                     normalised propensity distribution).
* ``impl_law``       the law the AR trial realises with the finite random words it
                     is given: P(j) proportional to (number of 32-bit words that map
                     to candidate j) x (number of 32-bit words u for which the
                     comparison accepts j).  Counted exactly with integer arithmetic
                     and a binary search over the monotone acceptance predicate,
                     which is evaluated with numpy's IEEE float32/float64 scalars --
                     a different computation from the oracle's sampler.
* ``paper_law``      the law of the paper's election/argmin rule (u_j uniform in
                     [0,T), eligible iff u_j < D_j, winner = argmin u_j / D_j):
                     P(j) = int_0^{min(1,T/D_j)} (D_j/T) prod_{i!=j} max(0, 1 - r D_i/T) dr.
* ``predicted_mse``  expected MSE of the paper's quality experiment (Section "Test
                     and validation of the algorithm") for a sampler with law P and
                     N samples: (1/M) sum_j [(P_j - p_j)^2 + P_j (1 - P_j) / N].
* ``chi_square``     goodness-of-fit p-value with bins merged to expected count >= 5.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import stats as sps


def exact_law(alpha) -> np.ndarray:
    a = np.asarray(alpha, dtype=np.float64)
    return a / math.fsum(a.tolist())


def candidate_preimages(M: int) -> np.ndarray:
    """#{w in [0, 2^32): floor(w M / 2^32) = j} for j < M, exact."""
    j = np.arange(M + 1, dtype=object)
    first = [-(-(int(k) << 32) // M) for k in j]       # ceil(k 2^32 / M)
    return np.array([first[k + 1] - first[k] for k in range(M)], dtype=np.int64)


def _accept_count_f64(T: float, a: float) -> int:
    """#{w in [0,2^32): fl64(w 2^-32 * T) < a}; the predicate is monotone in w."""
    T64, a64 = np.float64(T), np.float64(a)
    lo, hi = 0, 1 << 32          # answer in [lo, hi]
    while lo < hi:
        mid = (lo + hi) // 2
        p = np.float64(mid) * np.float64(2.0 ** -32) * T64
        if p < a64:
            lo = mid + 1
        else:
            hi = mid
    return lo


def _accept_count_f32(T: float, a: float) -> int:
    """#{w in [0,2^32): fl32(floor(w/256) 2^-24 * fl32(T)) < fl32(a)} = 256 * #v."""
    T32, a32 = np.float32(T), np.float32(a)
    lo, hi = 0, 1 << 24
    while lo < hi:
        mid = (lo + hi) // 2
        u = np.float32(mid) * np.float32(2.0 ** -24)
        if np.float32(u * T32) < a32:
            lo = mid + 1
        else:
            hi = mid
    return 256 * lo


def impl_law(alpha, T=None, cmp: int = 1):
    """Exact law of one AR selection (conditioned on acceptance) for the given
    random-word mapping and comparison precision (cmp 0 = FP32, 1 = FP64).

    Returns (law, p_accept_per_trial)."""
    a = np.asarray(alpha, dtype=np.float64)
    M = a.size
    T = float(a.max()) if T is None else float(T)
    pre = candidate_preimages(M)
    cnt = np.array([(_accept_count_f32 if cmp == 0 else _accept_count_f64)(T, float(x))
                    for x in a], dtype=object)
    w = [int(pre[j]) * int(cnt[j]) for j in range(M)]
    tot = sum(w)
    law = np.array([x / tot for x in w], dtype=np.float64) if tot else np.zeros(M)
    return law, tot / float(1 << 64)


def tv(p, q) -> float:
    return 0.5 * float(np.abs(np.asarray(p, dtype=np.float64) - np.asarray(q)).sum())


def paper_law(D, T=None, n_nodes: int = 4096):
    """Law of the paper's election/argmin rule; returns (P[j], P(rejection)).

    Gauss-Legendre on each interval between the break points T/D_i < 1 of the
    piecewise-polynomial integrand (degree M-1 per piece; n_nodes >= M/2 makes
    the rule exact up to rounding)."""
    D = np.asarray(D, dtype=np.float64)
    T = float(D.max()) if T is None else float(T)
    d = D / T
    breaks = sorted({0.0, 1.0, *[1.0 / x for x in d if x > 1.0]})
    xg, wg = np.polynomial.legendre.leggauss(n_nodes)
    P = np.zeros(D.size)
    for lo, hi in zip(breaks[:-1], breaks[1:]):
        r = 0.5 * (hi - lo) * xg + 0.5 * (hi + lo)
        w = 0.5 * (hi - lo) * wg
        fac = 1.0 - np.outer(r, d)                 # [nodes, M]
        alive = fac > 0.0
        logf = np.where(alive, np.log(np.where(alive, fac, 1.0)), 0.0)
        nz_dead = (~alive).sum(axis=1)             # factors that are zero
        L = logf.sum(axis=1)
        for j in range(D.size):
            if d[j] == 0.0:
                continue
            # density of R_j on r < min(1, 1/d_j) is d_j; product over i != j
            dead_others = nz_dead - (~alive[:, j])
            prod = np.where(dead_others > 0, 0.0,
                            np.exp(L - logf[:, j]))
            inside = r < min(1.0, 1.0 / d[j])
            P[j] += float(np.sum(w * d[j] * prod * inside))
    p_rej = float(np.prod(np.maximum(0.0, 1.0 - d)))
    return P, p_rej


def predicted_mse(P, p, n_samples: int) -> float:
    P = np.asarray(P, dtype=np.float64)
    p = np.asarray(p, dtype=np.float64)
    return float(np.mean((P - p) ** 2 + P * (1.0 - P) / n_samples))


def empirical_mse(idx, p) -> float:
    p = np.asarray(p, dtype=np.float64)
    counts = np.bincount(np.asarray(idx), minlength=p.size)[: p.size]
    return float(np.mean((p - counts / len(idx)) ** 2))


def chi_square(counts, probs, min_expected: float = 5.0):
    """Pearson chi-square p-value of counts against probs.

    Zero-probability bins must be empty (returns p = 0 otherwise).  Adjacent
    bins are merged until every merged bin expects >= min_expected."""
    counts = np.asarray(counts, dtype=np.float64)
    probs = np.asarray(probs, dtype=np.float64)
    n = counts.sum()
    if np.any((probs == 0) & (counts > 0)):
        return 0.0
    keep = probs > 0
    c, e = counts[keep], probs[keep] * n
    mc, me = [], []
    acc_c = acc_e = 0.0
    for ci, ei in zip(c, e):
        acc_c += ci
        acc_e += ei
        if acc_e >= min_expected:
            mc.append(acc_c)
            me.append(acc_e)
            acc_c = acc_e = 0.0
    if acc_e > 0:
        if me:
            mc[-1] += acc_c
            me[-1] += acc_e
        else:
            mc.append(acc_c)
            me.append(acc_e)
    mc, me = np.array(mc), np.array(me)
    if len(me) < 2:
        return 1.0
    stat = float(((mc - me) ** 2 / me).sum())
    return float(sps.chi2.sf(stat, len(me) - 1))
