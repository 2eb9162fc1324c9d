"""Pins for the oracle's SSA (direct method with AR selection, Section "The
Stochastic Simulation Algorithm").

Expected values come from closed forms of small networks:
* pure decay A -> 0: extinction after exactly X0 steps; the extinction time has
  mean sum_k 1/(c k) and variance sum_k 1/(c k)^2;
* birth-death 0 -> A, A -> 0: the time-weighted occupancy is Poisson(c1/c2);
* first step of a mixed network (2A -> B, A + C -> D, A -> E): the reaction law
  is a_r / a_0 with the mass-action counts x(x-1)/2, x_A x_C, x_A, and the
  waiting time is Exp(a_0);
* A <-> B conserves A + B.
"""
import math

import numpy as np
from scipy import stats as sps

from oracle import law
from paper_1404_0027_gb300 import workloads as W


def test_pure_decay_extinction(orc):
    c, n0, B = 0.7, 25, 4000
    net = W.network_from_lists(1, [(W.RT_UNI, (0, -1), c, [(0, -1)])])
    X = np.full((B, 1), n0, dtype=np.int32)
    out = orc.ssa(net, X, nsteps=n0, seed=3)
    assert np.all(out["X"] == 0) and np.all(out["step"] == n0) and np.all(out["status"] == 0)
    mean = sum(1.0 / (c * k) for k in range(1, n0 + 1))
    var = sum(1.0 / (c * k) ** 2 for k in range(1, n0 + 1))
    assert abs(out["t"].mean() - mean) < 5 * math.sqrt(var / B)
    assert abs(out["t"].var() / var - 1.0) < 0.15
    out2 = orc.ssa(net, out["X"], t=out["t"], step=out["step"], nsteps=3, seed=3)
    assert np.all(out2["status"] == orc.ST_ABSORBED)
    np.testing.assert_array_equal(out2["t"], out["t"])


def test_birth_death_poisson(orc):
    c1, c2, B, burn, steps = 5.0, 0.5, 128, 200, 1200
    net = W.network_from_lists(1, [(W.RT_SOURCE, (-1, -1), c1, [(0, 1)]),
                                   (W.RT_UNI, (0, -1), c2, [(0, -1)])])
    X = np.zeros((B, 1), dtype=np.int32)
    t = np.zeros(B)
    step = np.zeros(B, dtype=np.uint64)
    occ = np.zeros(60)
    for n in range(steps):
        out = orc.ssa(net, X, t=t, step=step, nsteps=1, seed=11)
        if n >= burn:
            np.add.at(occ, np.minimum(X[:, 0], 59), out["t"] - t)
        X, t, step = out["X"], out["t"], out["step"]
    lam = c1 / c2
    pm = occ / occ.sum()
    k = np.arange(60)
    mean = float((pm * k).sum())
    varr = float((pm * (k - mean) ** 2).sum())
    assert abs(mean - lam) < 0.35 and abs(varr - lam) < 1.2
    assert law.tv(pm[:30], sps.poisson.pmf(k[:30], lam)) < 0.03


def test_first_step_law_and_waiting_time(orc):
    net = W.network_from_lists(5, [
        (W.RT_DIMER, (0, -1), 0.3, [(0, -2), (1, 1)]),
        (W.RT_BI, (0, 2), 0.02, [(0, -1), (2, -1), (3, 1)]),
        (W.RT_UNI, (0, -1), 1.1, [(0, -1), (4, 1)]),
    ])
    B = 30000
    X = np.zeros((B, 5), dtype=np.int32)
    X[:, 0], X[:, 2] = 10, 7
    a = np.array([0.3 * 45, 0.02 * 70, 1.1 * 10])
    for cmp in (0, 1):
        out = orc.ssa(net, X, nsteps=1, seed=21, cmp=cmp)
        assert law.chi_square(np.bincount(out["last"], minlength=3), a / a.sum()) > 1e-3
        assert sps.kstest(out["t"], "expon", args=(0, 1.0 / a.sum())).pvalue > 1e-3
        fired = out["last"]
        np.testing.assert_array_equal(out["X"][:, 1], (fired == 0).astype(np.int32))
        np.testing.assert_array_equal(out["X"][:, 0], 10 - np.where(fired == 0, 2, 1))
    out = orc.ssa(net, X[:4], nsteps=0, want_a=True)
    np.testing.assert_array_equal(out["a"], np.tile(a, (4, 1)))


def test_isomerization_conserves_total(orc):
    net = W.network_from_lists(2, [(W.RT_UNI, (0, -1), 1.0, [(0, -1), (1, 1)]),
                                   (W.RT_UNI, (1, -1), 2.0, [(1, -1), (0, 1)])])
    X = np.tile(np.array([[30, 5]], dtype=np.int32), (64, 1))
    out = orc.ssa(net, X, nsteps=500, seed=4)
    assert np.all(out["X"].sum(axis=1) == 35)
    # stationary Binomial(35, 2/3) for A; mean over realizations
    assert abs(out["X"][:, 0].mean() - 35 * 2 / 3) < 5 * math.sqrt(35 * 2 / 9 / 64)


def test_resume_is_bit_identical(orc):
    net = W.random_network(N=40, M=70, seed=8)
    X0 = W.initial_counts(40, 16, seed=9)
    full = orc.ssa(net, X0, nsteps=300, seed=2, cmp=0)
    half = orc.ssa(net, X0, nsteps=150, seed=2, cmp=0)
    rest = orc.ssa(net, half["X"], t=half["t"], step=half["step"], nsteps=150, seed=2, cmp=0)
    np.testing.assert_array_equal(rest["X"], full["X"])
    np.testing.assert_array_equal(rest["last"], full["last"])
    np.testing.assert_allclose(rest["t"], full["t"], rtol=1e-12)
    assert np.all(full["X"] >= 0)


def test_ssa_until_birth_death_poisson_at_sample_times(orc):
    """Birth-death from 0 (birth 5, death 0.5 per molecule): X(t) is Poisson
    with mean 10 (1 - exp(-t / 2)) at every sample time; every realization
    stops before the time limit with T_END."""
    from scipy import stats
    net = W.network_from_lists(1, [(W.RT_SOURCE, (-1, -1), 5.0, [(0, 1)]),
                                   (W.RT_UNI, (0, -1), 0.5, [(0, -1)])])
    X0 = np.zeros((6000, 1), dtype=np.int32)
    ts = np.array([0.0, 1.0, 5.0, 20.0])
    o = orc.ssa_until(net, X0, t_end=20.0, sample_times=ts, nthreads=8)
    assert (o["status"] == orc.ST_T_END).all() and (o["t"] <= 20.0).all()
    assert (o["traj"][:, 0, 0] == 0).all()
    for k, tk in enumerate(ts[1:], start=1):
        lam = 10.0 * (1.0 - np.exp(-0.5 * tk))
        x = o["traj"][:, k, 0]
        hi = int(x.max()) + 1
        obs = np.bincount(x, minlength=hi + 1).astype(float)
        exp = stats.poisson.pmf(np.arange(hi + 1), lam) * x.size
        exp[-1] += stats.poisson.sf(hi, lam) * x.size
        keep = exp >= 5
        obs_m = np.append(obs[keep], obs[~keep].sum())
        exp_m = np.append(exp[keep], exp[~keep].sum())
        assert stats.chisquare(obs_m, exp_m * obs_m.sum() / exp_m.sum()).pvalue > 1e-3


def test_ssa_until_absorption_holds_state_and_resumes(orc):
    """Pure decay: after absorption the remaining samples hold 0; a run split
    at an intermediate time limit equals one run (the time stays at the last
    reaction, so the waiting time that crossed the limit is redrawn from the
    same counter and the same time)."""
    net = W.network_from_lists(1, [(W.RT_UNI, (0, -1), 1.0, [(0, -1)])])
    X0 = np.full((300, 1), 5, dtype=np.int32)
    ts = np.linspace(0.0, 50.0, 11)
    o = orc.ssa_until(net, X0, t_end=50.0, sample_times=ts)
    assert (o["status"] & orc.ST_ABSORBED).all() and (o["X"] == 0).all()
    assert (o["traj"][:, -1, 0] == 0).all()
    assert (np.diff(o["traj"][:, :, 0], axis=1) <= 0).all()      # counts only fall
    net2 = W.random_network(N=30, M=50, seed=12)
    X1 = W.initial_counts(30, 20, seed=13)
    full = orc.ssa_until(net2, X1, t_end=0.05, sample_times=[0.01, 0.03, 0.05])
    h = orc.ssa_until(net2, X1, t_end=0.02, sample_times=[0.01, 0.03, 0.05])
    r = orc.ssa_until(net2, h["X"], t_end=0.05, t=h["t"], step=h["step"],
                      sample_times=[0.01, 0.03, 0.05])
    np.testing.assert_array_equal(r["X"], full["X"])
    np.testing.assert_array_equal(r["step"], full["step"])
    np.testing.assert_array_equal(r["t"], full["t"])
    np.testing.assert_array_equal(h["traj"][:, 0], full["traj"][:, 0])
    np.testing.assert_array_equal(r["traj"][:, 1:], full["traj"][:, 1:])
