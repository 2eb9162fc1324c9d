"""GPU parity of the one-launch form of ar_select_batched (FP32 data with a
plan whose realizations all sit in CTA home lists, global share 0): each CTA
reduces the chunks of its own realizations, then selects them.  The results
must be exactly those of the oracle (and of the two-launch form): indices,
counters and maxima bit-exact, totals within the FP64 bound, status bits."""
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


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _check(gb, orc, bt, warps, cmp=0, seed=1, sel_offset=0, realization_base=0,
           trial_cap=1 << 20, status=None):
    plan = gb.Plan(bt.offsets, bt.out_offsets)
    gb.ar_plan_set_tile(plan, warps, 0)   # every realization in a home list: one launch
    bs, idx, stats, st = gb.select_batched(_t(bt.alpha), _t(bt.offsets), _t(bt.out_offsets),
                                           seed=seed, sel_offset=sel_offset,
                                           realization_base=realization_base, cmp=cmp,
                                           trial_cap=trial_cap, plan=plan)
    obs, oidx, ostats, ost = orc.select_batched(bt, seed=seed, sel_offset=sel_offset,
                                                realization_base=realization_base, cmp=cmp,
                                                trial_cap=trial_cap, nthreads=8)
    g = idx.cpu().numpy()
    mism = np.flatnonzero(g != oidx)
    assert mism.size == 0, f"{mism.size} mismatches of {g.size}, first at {mism[:5]}"
    np.testing.assert_array_equal(stats.cpu().numpy().astype(np.uint64), ostats)
    gbs = bs.cpu().numpy()
    np.testing.assert_array_equal(np.isnan(gbs), np.isnan(obs))
    ok = ~np.isnan(obs[:, 0])
    np.testing.assert_array_equal(gbs[ok, 0], obs[ok, 0])
    tol = 2.0 * (np.diff(bt.offsets) + 8) * 2.0 ** -53 * np.abs(obs[:, 1])
    bad = np.flatnonzero(ok & ~(np.abs(gbs[:, 1] - obs[:, 1]) <= tol))
    assert bad.size == 0, bad[:5]
    assert int(st.item()) == ost
    if status is not None:
        assert ost == status
    plan.close()


@pytest.mark.parametrize("warps", [8, 16, 32])
def test_fused_full_workload(gb, orc, warps):
    """The benchmark's batch: 4096 realizations, M_b log-uniform in [64, 16384]."""
    _check(gb, orc, W.batched_uneven(seed=302), warps)


@pytest.mark.parametrize("warps", [8, 32])
@pytest.mark.parametrize("cmp", [0, 1])
def test_fused_ragged(gb, orc, warps, cmp):
    """Empty realizations (M_b = 0), realizations without selections
    (K_b = 0), all-zero propensities, realizations of one chunk and of many,
    offsets not on 16-byte boundaries inside the batch."""
    vecs = [W.skewed(m, seed=m).astype(np.float32) for m in (1, 2, 3, 5, 7, 64, 1000, 4099,
                                                               16384, 20_000, 9, 1)]
    vecs.insert(4, np.zeros(0, dtype=np.float32))
    vecs.append(np.zeros(33, dtype=np.float32))
    ks = [5, 0, 17, 1, 7, 256, 300, 256, 1000, 64, 77, 3, 2, 9]
    _check(gb, orc, W.batch_from_vectors(vecs, ks), warps, cmp=cmp, seed=7, sel_offset=11,
           realization_base=100)


@pytest.mark.parametrize("warps", [8, 32])
def test_fused_invalid_realizations(gb, orc, warps):
    """NaN, negative and infinite propensities in three realizations:
    BAD_ALPHA, (NaN, NaN) bounds and the sentinel there, the others exact."""
    bt = W.batched_uneven(B=400, seed=308, m_lo=16, m_hi=5000, K=40)
    a = bt.alpha.copy()
    a[bt.offsets[5] + 2] = np.nan
    a[bt.offsets[17]] = -1.0
    a[bt.offsets[390] + 1] = np.inf
    _check(gb, orc, W.Batch(a, bt.offsets, bt.out_offsets), warps,
           status=gb.AR_STATUS_BAD_ALPHA)


@pytest.mark.parametrize("cap", [1, 2, 7])
def test_fused_trial_cap(gb, orc, cap):
    _check(gb, orc, W.batched_uneven(B=200, seed=309, K=64), 16, trial_cap=cap,
           status=gb.AR_STATUS_TRIAL_CAP)


def test_fused_graph_replays(gb, orc):
    """One launch per call replayed from a CUDA graph: every replay gives the
    same indices and the counters add up (the launch leaves no state behind)."""
    import torch
    bt = W.batched_uneven(B=1200, seed=310, K=96)
    plan = gb.Plan(bt.offsets, bt.out_offsets)
    gb.ar_plan_set_tile(plan, 32, 0)
    a, off, oo = _t(bt.alpha), _t(bt.offsets), _t(bt.out_offsets)
    bs = torch.empty((bt.B, 2), dtype=torch.float64, device="cuda")
    idx = torch.empty(int(bt.out_offsets[-1]), dtype=torch.int32, device="cuda")
    stats = torch.zeros(3, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        gb.ar_select_batched(a, off, oo, 1, 0, 0, 0, 1 << 20, plan, bs, idx, stats, st, None, s)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        gb.ar_select_batched(a, off, oo, 1, 0, 0, 0, 1 << 20, plan, bs, idx, stats, st, None, s)
    for _ in range(7):
        g.replay()
    torch.cuda.synchronize()
    obs, oidx, ostats, ost = orc.select_batched(bt, nthreads=8)
    np.testing.assert_array_equal(idx.cpu().numpy(), oidx)
    np.testing.assert_array_equal(stats.cpu().numpy().astype(np.uint64), 8 * ostats)
    assert int(st.item()) == ost
    plan.close()


def test_fused_falls_back_for_very_long_home_lists(gb, orc):
    """More home realizations per CTA than the one-launch form keeps counters
    for (1.6 M realizations of 1-3 propensities): the call takes the
    two-launch form and still gives the oracle's results."""
    rng = np.random.default_rng(11)
    B = 1_600_000
    sizes = rng.integers(1, 4, size=B)
    off = np.zeros(B + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    oo = np.arange(B + 1, dtype=np.int64)   # one selection per realization
    alpha = rng.exponential(1.0, size=int(off[-1])).astype(np.float32)
    _check(gb, orc, W.Batch(alpha, off, oo), 32)


def test_unaligned_fp32_takes_two_launches(gb, orc):
    """FP32 propensities whose base is not 16-byte aligned (a view one element
    into a buffer): the one-launch form needs 16-byte loads, so the call takes
    the two-launch form with the plan and gives the oracle's results."""
    import torch
    bt = W.batched_uneven(B=300, seed=311, K=64)
    buf = torch.zeros(bt.alpha.size + 1, dtype=torch.float32, device="cuda")
    buf[1:] = torch.from_numpy(bt.alpha).cuda()
    a = buf[1:]                                    # 4-byte aligned, not 16
    assert a.data_ptr() % 16 != 0
    plan = gb.Plan(bt.offsets, bt.out_offsets)
    gb.ar_plan_set_tile(plan, 32, 0)
    bs, idx, stats, st = gb.select_batched(a, _t(bt.offsets), _t(bt.out_offsets), plan=plan)
    obs, oidx, ostats, ost = orc.select_batched(bt, nthreads=8)
    np.testing.assert_array_equal(idx.cpu().numpy(), oidx)
    np.testing.assert_array_equal(stats.cpu().numpy().astype(np.uint64), ostats)
    np.testing.assert_array_equal(bs.cpu().numpy()[:, 0], obs[:, 0])
    assert int(st.item()) == ost
    plan.close()


@pytest.mark.parametrize("use_plan", [False, True])
def test_runs_split_over_calls(gb, orc, use_plan):
    """One call drawing selections 0 .. 199 of every realization equals four
    calls drawing 0 .. 36, 37 .. 74, 75 .. 127 and 128 .. 199 (runs of 64
    split inside and at their boundaries): the same indices, and the trial
    counters add up.  Both forms, with a plan (one launch) and without."""
    K = 200
    bt = W.batched_uneven(B=300, seed=312, K=K)
    off = _t(bt.offsets)
    a = _t(bt.alpha)

    def call(lo, hi):
        oo = np.arange(bt.B + 1, dtype=np.int64) * (hi - lo)
        plan = None
        if use_plan:
            plan = gb.Plan(bt.offsets, oo)
            gb.ar_plan_set_tile(plan, 32, 0)
        bs, idx, stats, st = gb.select_batched(a, off, _t(oo), seed=9, sel_offset=lo,
                                               realization_base=3, plan=plan)
        out = idx.cpu().numpy().reshape(bt.B, hi - lo), stats.cpu().numpy(), int(st.item())
        if plan is not None:
            plan.close()
        return out

    full, sfull, st = call(0, K)
    assert st == 0
    parts, ssum = [], np.zeros(3, np.int64)
    for lo, hi in ((0, 37), (37, 75), (75, 128), (128, K)):
        idx, s, st = call(lo, hi)
        assert st == 0
        parts.append(idx)
        ssum += s
    np.testing.assert_array_equal(np.concatenate(parts, axis=1), full)
    np.testing.assert_array_equal(ssum, sfull)
    # and the oracle agrees with the single call
    want_bs, want, _, _ = orc.select_batched(W.Batch(bt.alpha, bt.offsets,
                                                     np.arange(bt.B + 1, dtype=np.int64) * K),
                                             seed=9, realization_base=3, nthreads=8)
    np.testing.assert_array_equal(full.ravel(), want)


@pytest.mark.parametrize("cap", [300, 500, 1000])
def test_cap_with_fast_and_stepwise_rounds(gb, orc, cap):
    """Acceptance around 1 in 300 trials with caps of a few hundred trials:
    runs mix 192-trial rounds with trial-by-trial rounds near the cap, and
    many selections are capped.  Indices, trial counts and status equal the
    oracle's on the bounded path (T_w = 60 max) and on the one-launch path
    (one dominant propensity per realization)."""
    bt = W.batched_uneven(B=120, seed=313, m_lo=64, m_hi=2000, K=64)
    bw = 60.0 * np.array([bt.alpha[bt.offsets[b]:bt.offsets[b + 1]].max()
                          for b in range(bt.B)], dtype=np.float64)
    plan = gb.Plan(bt.offsets, bt.out_offsets)
    idx, stats, st = gb.select_batched_bounded(_t(bt.alpha), _t(bt.offsets), _t(bt.out_offsets),
                                               _t(bw), 1, seed=4, trial_cap=cap, plan=plan)
    oidx, ostats, ost = orc.select_batched_bounded(bt, bw, 1, seed=4, trial_cap=cap, nthreads=8)
    np.testing.assert_array_equal(idx.cpu().numpy(), oidx)
    np.testing.assert_array_equal(stats.cpu().numpy().astype(np.uint64), ostats)
    assert int(st.item()) == ost and ost & gb.AR_STATUS_TRIAL_CAP
    assert 0 < ostats[2] < ostats[1]          # capped and accepted selections both occur
    plan.close()
    # one dominant propensity: M T / sum close to M
    a = np.full(bt.alpha.size, 1e-3, dtype=np.float32)
    a[bt.offsets[:-1]] = 1.0
    _check(gb, orc, W.Batch(a, bt.offsets, bt.out_offsets), 16, seed=5, trial_cap=cap)


def test_grid_setting(gb, orc):
    """CTAs per SM 0 (as many as fit), 1, 2 and 4 and items of 64, 128, 256 and
    1024 selections with every tile: the same indices, counters and status
    as the oracle (K_b = 300: items cut inside and across runs, sel_offset
    not a multiple of 64); values outside the allowed sets are rejected and
    leave the plan usable."""
    bt = W.batched_uneven(B=700, seed=314, K=300)
    obs, oidx, ostats, ost = orc.select_batched(bt, seed=2, sel_offset=37, nthreads=8)
    plan = gb.Plan(bt.offsets, bt.out_offsets)
    a, off, oo = _t(bt.alpha), _t(bt.offsets), _t(bt.out_offsets)
    for warps in (8, 16, 32):
        gb.ar_plan_set_tile(plan, warps, 0)
        for cps, items in ((0, 0), (1, 128), (2, 256), (4, 1024), (1, 64)):
            gb.ar_plan_set_grid(plan, cps, items)
            bs, idx, stats, st = gb.select_batched(a, off, oo, seed=2, sel_offset=37, plan=plan)
            np.testing.assert_array_equal(idx.cpu().numpy(), oidx)
            np.testing.assert_array_equal(stats.cpu().numpy().astype(np.uint64), ostats)
            assert int(st.item()) == ost
    for bad in ((-1, 0), (5, 0), (1, 32), (1, 2048), (0, -64)):
        with pytest.raises(gb.GbarError):
            gb.ar_plan_set_grid(plan, *bad)
    bs, idx, _, _ = gb.select_batched(a, off, oo, seed=2, sel_offset=37, plan=plan)
    np.testing.assert_array_equal(idx.cpu().numpy(), oidx)
    plan.close()


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("cmp", [0, 1])
def test_grid_setting_two_launch_and_bounded(gb, orc, dtype, cmp):
    """The plan's grid and item settings on the paths other than the
    one-launch call: FP64 data (reduction, then selections), FP32 data with a
    global queue, and ar_select_batched_bounded with the caller's bounds
    T_w = 1.5 max.  Indices, counters and status equal the oracle's."""
    bt = W.batched_uneven(B=500, seed=315, m_lo=16, m_hi=6000, K=200, dtype=dtype)
    a, off, oo = _t(bt.alpha), _t(bt.offsets), _t(bt.out_offsets)
    plan = gb.Plan(bt.offsets, bt.out_offsets)
    obs, oidx, ostats, ost = orc.select_batched(bt, seed=6, sel_offset=64, cmp=cmp, nthreads=8)
    bw = 1.5 * obs[:, 0].copy()
    bidx, bstats, bst = orc.select_batched_bounded(bt, bw, 1, seed=7, cmp=cmp, nthreads=8)
    for tile, share, cps, items in ((16, 0, 1, 256), (8, 400, 2, 128), (32, 0, 0, 64)):
        gb.ar_plan_set_tile(plan, tile, share)
        gb.ar_plan_set_grid(plan, cps, items)
        bs, idx, stats, st = gb.select_batched(a, off, oo, seed=6, sel_offset=64, cmp=cmp,
                                               plan=plan)
        np.testing.assert_array_equal(idx.cpu().numpy(), oidx)
        np.testing.assert_array_equal(stats.cpu().numpy().astype(np.uint64), ostats)
        assert int(st.item()) == ost
        idx2, stats2, st2 = gb.select_batched_bounded(a, off, oo, _t(bw), 1, seed=7, cmp=cmp,
                                                      plan=plan)
        np.testing.assert_array_equal(idx2.cpu().numpy(), bidx)
        np.testing.assert_array_equal(stats2.cpu().numpy().astype(np.uint64), bstats)
        assert int(st2.item()) == bst
    plan.close()


@pytest.mark.parametrize("cps, items", [(1, 256), (2, 1024), (4, 64)])
def test_grid_setting_tiny_and_ragged_batches(gb, orc, cps, items):
    """Grid and item settings on batches far smaller than the grid (most CTAs
    have empty home lists) and with empty realizations, realizations without
    selections and K_b not a multiple of 64."""
    cases = [
        W.batch_from_vectors([W.skewed(50, seed=1).astype(np.float32)], [7]),
        W.batch_from_vectors([W.skewed(m, seed=m).astype(np.float32) for m in (3, 700, 1)],
                             [300, 0, 65]),
        W.batch_from_vectors([np.zeros(0, np.float32), W.skewed(2000, seed=9).astype(np.float32),
                              np.zeros(40, np.float32), W.skewed(10, seed=3).astype(np.float32)],
                             [5, 1000, 3, 129]),
    ]
    for bt in cases:
        obs, oidx, ostats, ost = orc.select_batched(bt, seed=8, sel_offset=5, nthreads=8)
        plan = gb.Plan(bt.offsets, bt.out_offsets)
        gb.ar_plan_set_tile(plan, 16, 0)
        gb.ar_plan_set_grid(plan, cps, items)
        bs, idx, stats, st = gb.select_batched(_t(bt.alpha), _t(bt.offsets), _t(bt.out_offsets),
                                               seed=8, sel_offset=5, plan=plan)
        np.testing.assert_array_equal(idx.cpu().numpy(), oidx)
        np.testing.assert_array_equal(stats.cpu().numpy().astype(np.uint64), ostats)
        np.testing.assert_array_equal(np.isnan(bs.cpu().numpy()), np.isnan(obs))
        assert int(st.item()) == ost
        plan.close()


def _bound_data(offsets, seed):
    """FP32 Exp(1) propensities for the offsets; realization 4 all zero and a
    NaN in realization 6 (BAD_ALPHA)."""
    a = np.random.default_rng(seed).exponential(1.0, int(offsets[-1])).astype(np.float32)
    a[offsets[4]:offsets[5]] = 0.0
    a[offsets[6] + 500] = np.nan
    return a


def _bound_exact(a, offsets):
    """{max, correctly rounded sum} per valid realization (NaN row otherwise)."""
    import math
    B = len(offsets) - 1
    out = np.zeros((B, 2))
    for b in range(B):
        seg = a[offsets[b]:offsets[b + 1]]
        if np.isnan(seg).any():
            out[b] = np.nan
        elif seg.size:
            out[b] = float(seg.max()), math.fsum(seg.astype(np.float64))
    return out


@pytest.mark.parametrize("full", [False, True])
def test_bound_batched_exact_paths_and_replays(gb, full):
    """ar_bound_batched: exact maxima and correctly rounded FP32 totals, bit
    for bit the same from the plan's vector path (16-byte aligned data), its
    register path (the same data at an address that is not 16-byte aligned)
    and the plan-less path, with the same status (ALL_ZERO, BAD_ALPHA).
    Repeated calls on new data with the same plan, and replays of a captured
    graph on new data in the same buffer, rewrite every output row."""
    import torch
    if full:   # the benchmark's batch shape: 4096 realizations, M_b in [64, 16384]
        ms = np.diff(W.batched_uneven(B=4096, seed=300, m_lo=64, m_hi=16384, K=1).offsets)
        ms[[4, 6]] = [1024, 3000]
        ms[0] = 0
    else:      # empty, single-element, one-chunk, chunk-edge, many-chunk realizations
        ms = np.array([0, 1, 3, 17, 1024, 1025, 4099, 20_000, 70_000] +
                      list(np.random.default_rng(7).integers(1, 5000, 200)))
    offsets = np.concatenate([[0], np.cumsum(ms)]).astype(np.int64)
    B = len(ms)
    plan = gb.Plan(offsets, np.arange(B + 1, dtype=np.int64))
    off_d = _t(offsets)
    stream = torch.cuda.Stream()
    want_st = gb.AR_STATUS_ALL_ZERO | gb.AR_STATUS_BAD_ALPHA

    def run(alpha, pl):
        bs = torch.full((B, 2), -7.0, dtype=torch.float64, device="cuda")
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        gb.ar_bound_batched(alpha, off_d, pl, bs, st, None if pl is not None else
                            torch.zeros(gb.ar_select_batched_workspace_size(B), dtype=torch.uint8,
                                        device="cuda"), stream)
        stream.synchronize()
        return bs.cpu().numpy(), int(st.item())

    for seed in (11, 12, 13):
        a = _bound_data(offsets, seed)
        alpha = _t(a)
        assert alpha.data_ptr() % 16 == 0
        got, st = run(alpha, plan)
        buf = torch.empty(alpha.numel() + 1, dtype=torch.float32, device="cuda")
        buf[1:].copy_(alpha)
        two, st2 = run(buf[1:], plan)        # not 16-byte aligned: two launches
        nop, st3 = run(alpha, None)
        exact = _bound_exact(a, offsets)
        np.testing.assert_array_equal(got, exact)
        np.testing.assert_array_equal(got.view(np.int64), two.view(np.int64))
        np.testing.assert_array_equal(got.view(np.int64), nop.view(np.int64))
        assert st == st2 == st3 == want_st

    # a captured call replayed on new data in the same buffer
    alpha_g = torch.empty(int(offsets[-1]), dtype=torch.float32, device="cuda")
    bs_g = torch.empty((B, 2), dtype=torch.float64, device="cuda")
    st_g = torch.zeros(1, dtype=torch.int32, device="cuda")
    alpha_g.copy_(_t(_bound_data(offsets, 20)))
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        gb.ar_bound_batched(alpha_g, off_d, plan, bs_g, st_g, None, stream)
    for seed in (21, 22, 23):
        a = _bound_data(offsets, seed)
        alpha_g.copy_(_t(a))
        bs_g.fill_(-7.0)
        st_g.zero_()
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(bs_g.cpu().numpy(), _bound_exact(a, offsets))
        assert int(st_g.item()) == want_st
    plan.close()
