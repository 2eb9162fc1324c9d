"""GPU parity of ssa_step_batched against the oracle's SSA.

Molecule counts, fired reactions, step counters, status and trial counts must
be bit-exact (they depend only on exact integer counts, exact FP64
propensities and the exact maximum); the final propensities too.  Time is
compared with a relative tolerance: the oracle adds tau = -ln(1-u)/a_0 with
libm's log and a naive FP64 a_0, the library with CUDA's log and an exact
fixed-point a_0, so each step's tau may differ by a few ulps (relative
1e-15); over n steps the relative gap stays below n * 4e-16 + 1e-13.
"""
import numpy as np
import pytest

from paper_1404_0027_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import torch
    from paper_1404_0027_gb300 import build
    build.build()
    from paper_1404_0027_gb300 import binding
    binding.lib()
    assert torch.cuda.is_available()
    return binding


def _compare(gb, orc, net, X0, nsteps, cmp, seed=1, base=0, t=None, step=None, status=None):
    gn = gb.SsaNet(net)
    g = gb.ssa_run(gn, X0, nsteps, seed=seed, realization_base=base, cmp=cmp, t=t, step=step,
                   status=status)
    o = orc.ssa(net, X0, t=t, step=step, nsteps=nsteps, seed=seed, realization_base=base, cmp=cmp,
                status=status, nthreads=8, want_a=True)
    gX = g["X"].cpu().numpy()
    bad = np.flatnonzero((gX != o["X"]).any(axis=1))
    assert bad.size == 0, f"X differs in realizations {bad[:5]}"
    np.testing.assert_array_equal(g["last"].cpu().numpy(), o["last"])
    np.testing.assert_array_equal(g["step"].cpu().numpy().astype(np.uint64), o["step"])
    np.testing.assert_array_equal(g["status"].cpu().numpy().astype(np.uint32), o["status"])
    np.testing.assert_array_equal(g["trials"].cpu().numpy().astype(np.uint64), o["trials"])
    np.testing.assert_array_equal(g["a"].cpu().numpy(), o["a"])
    steps = o["step"].astype(np.float64)
    rtol = steps.max() * 4e-16 + 1e-13
    np.testing.assert_allclose(g["t"].cpu().numpy(), o["t"], rtol=rtol, atol=0)
    gn.close()
    return g, o


@pytest.mark.parametrize("cmp", [0, 1])
def test_ssa_small_network(gb, orc, cmp):
    net = W.random_network(N=40, M=70, seed=8)
    X0 = W.initial_counts(40, 64, seed=9)
    _compare(gb, orc, net, X0, 3000, cmp)


def test_ssa_iron_sized_network(gb, orc):
    """The full SSA network (641 species, 1029 reactions), 64 realizations,
    10^4 steps: bit-exact trajectories."""
    net = W.random_network()
    X0 = W.initial_counts(641, 64, seed=501)
    _compare(gb, orc, net, X0, 10_000, 0, base=1000)


def test_ssa_absorption_and_resume(gb, orc):
    net = W.network_from_lists(2, [(W.RT_UNI, (0, -1), 0.7, [(0, -1), (1, 1)]),
                                   (W.RT_DIMER, (1, -1), 0.01, [(1, -2)])])
    X0 = np.tile(np.array([[30, 0]], dtype=np.int32), (96, 1))
    g, o = _compare(gb, orc, net, X0, 200, 0)
    assert (o["status"] & orc.ST_ABSORBED).all()
    # resume: two calls of 25 steps equal one call of 50 (random network)
    net2 = W.random_network(N=30, M=50, seed=12)
    X1 = W.initial_counts(30, 40, seed=13)
    full = gb.ssa_run(gb.SsaNet(net2), X1, 50, seed=5)
    half = gb.ssa_run(gb.SsaNet(net2), X1, 25, seed=5)
    rest = gb.ssa_run(gb.SsaNet(net2), half["X"].cpu().numpy(), 25, seed=5,
                      t=half["t"].cpu().numpy(), step=half["step"].cpu().numpy())
    np.testing.assert_array_equal(rest["X"].cpu().numpy(), full["X"].cpu().numpy())
    np.testing.assert_array_equal(rest["last"].cpu().numpy(), full["last"].cpu().numpy())
    np.testing.assert_allclose(rest["t"].cpu().numpy(), full["t"].cpu().numpy(), rtol=1e-13)


def test_ssa_birth_death_and_trial_cap(gb, orc):
    net = W.network_from_lists(1, [(W.RT_SOURCE, (-1, -1), 5.0, [(0, 1)]),
                                   (W.RT_UNI, (0, -1), 0.5, [(0, -1)])])
    X0 = np.zeros((128, 1), dtype=np.int32)
    _compare(gb, orc, net, X0, 500, 1)
    # a cap of 1 trial stops most realizations at their first rejection
    gn = gb.SsaNet(net)
    g = gb.ssa_run(gn, X0, 50, trial_cap=1)
    o = orc.ssa(net, X0, nsteps=50, trial_cap=1)
    np.testing.assert_array_equal(g["status"].cpu().numpy().astype(np.uint32), o["status"])
    np.testing.assert_array_equal(g["X"].cpu().numpy(), o["X"])


@pytest.mark.parametrize("cmp", [0, 1])
def test_ssa_until_parity(gb, orc, cmp):
    """Time-limited runs with trajectory samples: counts, samples, steps,
    status, last reaction and trials bit-exact against the oracle."""
    net = W.random_network(N=40, M=70, seed=8)
    X0 = W.initial_counts(40, 64, seed=9)
    ts = np.linspace(0.0, 0.02, 9)
    sp = np.array([0, 5, 17, 39], dtype=np.int32)
    gn = gb.SsaNet(net)
    g = gb.ssa_until(gn, X0, 0.02, sample_times=ts, species=sp, cmp=cmp, seed=4)
    o = orc.ssa_until(net, X0, 0.02, sample_times=ts, species=sp, cmp=cmp, seed=4, nthreads=8)
    np.testing.assert_array_equal(g["X"].cpu().numpy(), o["X"])
    np.testing.assert_array_equal(g["traj"].cpu().numpy(), o["traj"])
    np.testing.assert_array_equal(g["step"].cpu().numpy().astype(np.uint64), o["step"])
    np.testing.assert_array_equal(g["status"].cpu().numpy().astype(np.uint32), o["status"])
    np.testing.assert_array_equal(g["last"].cpu().numpy(), o["last"])
    np.testing.assert_array_equal(g["trials"].cpu().numpy().astype(np.uint64), o["trials"])
    assert (o["status"] == orc.ST_T_END).all()
    rtol = float(o["step"].max()) * 4e-16 + 1e-13
    np.testing.assert_allclose(g["t"].cpu().numpy(), o["t"], rtol=rtol, atol=0)
    gn.close()


def test_ssa_until_absorption_and_resume(gb, orc):
    """Absorbed realizations hold their state to the limit; two calls split
    at an intermediate limit give the single call's path."""
    net = W.network_from_lists(1, [(W.RT_UNI, (0, -1), 1.0, [(0, -1)])])
    X0 = np.full((96, 1), 5, dtype=np.int32)
    ts = np.linspace(0.0, 50.0, 11)
    gn = gb.SsaNet(net)
    g = gb.ssa_until(gn, X0, 50.0, sample_times=ts, cmp=1)
    o = orc.ssa_until(net, X0, 50.0, sample_times=ts, cmp=1)
    np.testing.assert_array_equal(g["traj"].cpu().numpy(), o["traj"])
    np.testing.assert_array_equal(g["status"].cpu().numpy().astype(np.uint32), o["status"])
    gn.close()
    net2 = W.random_network(N=30, M=50, seed=12)
    X1 = W.initial_counts(30, 40, seed=13)
    gn2 = gb.SsaNet(net2)
    full = gb.ssa_until(gn2, X1, 0.05, seed=5)
    h = gb.ssa_until(gn2, X1, 0.02, seed=5)
    r = gb.ssa_until(gn2, h["X"].cpu().numpy(), 0.05, seed=5, t=h["t"].cpu().numpy(),
                     step=h["step"].cpu().numpy())
    np.testing.assert_array_equal(r["X"].cpu().numpy(), full["X"].cpu().numpy())
    np.testing.assert_array_equal(r["step"].cpu().numpy(), full["step"].cpu().numpy())
    np.testing.assert_array_equal(r["t"].cpu().numpy(), full["t"].cpu().numpy())
    gn2.close()
