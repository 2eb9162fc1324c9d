"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Indices, trial counts and maxima must be bit-exact; the total propensity must
lie within 2 (M + 8) 2^-53 sum of the oracle's FP64 index-order sum (the
oracle's own rounding is at most (M - 1) 2^-53 sum, the library's at most
(M + 8) 2^-53 sum of the exact value).
"""
import numpy as np
import pytest

from paper_1404_0027_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CAP = 1 << 20


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


def _sum_tol(a, total):
    return 2.0 * (a.size + 8) * 2.0 ** -53 * abs(total)


# ---------------------------------------------------------------- ar_bound
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("M", [0, 1, 7, 1024, 4095, 4096, 4097, 8191, 8192, 8193, 100_003, 1 << 20])
def test_bound_parity(gb, orc, dtype, M):
    a = W.wide_range(M, seed=M + 3).astype(dtype) if M else np.zeros(0, dtype=dtype)
    out, st = gb.bound(_t(a))
    mx, sm, ost = orc.bound(a)
    got = out.cpu().numpy()
    assert got[0] == mx
    assert abs(got[1] - sm) <= _sum_tol(a, sm)
    assert int(st.item()) == ost


@pytest.mark.parametrize("make", [W.plain_uniform, W.skewed, lambda: W.gaussian_paper(1024)])
def test_bound_workloads(gb, orc, make):
    a = make()
    out, st = gb.bound(_t(a))
    mx, sm, ost = orc.bound(a)
    got = out.cpu().numpy()
    assert got[0] == mx and abs(got[1] - sm) <= _sum_tol(a, sm) and int(st.item()) == ost


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("bad", [np.nan, -1.0, np.inf])
@pytest.mark.parametrize("M", [100, 50_000])
def test_bound_flags(gb, orc, dtype, bad, M):
    a = W.plain_uniform(M).astype(dtype)
    a[M // 3] = bad
    _, st = gb.bound(_t(a))
    assert int(st.item()) & gb.AR_STATUS_BAD_ALPHA
    z = np.zeros(M, dtype=dtype)
    z[5] = -0.0
    out, st = gb.bound(_t(z))
    assert int(st.item()) == gb.AR_STATUS_ALL_ZERO and out.cpu().numpy().tolist() == [0.0, 0.0]


# ------------------------------------------------------------- ar_select_k
def _check_select(gb, orc, a, K, cmp, fused, seed=1, sel_offset=0, realization=0,
                  bound_value=None, cap=CAP):
    import torch
    T = orc.bound(a)[0] if bound_value is None else bound_value
    bound = None if fused else torch.tensor([T], dtype=torch.float64, device="cuda")
    idx, stats, st = gb.select_k(_t(a), K, seed=seed, sel_offset=sel_offset,
                                 realization=realization, cmp=cmp, bound=bound, trial_cap=cap)
    oidx, ostats, ost = orc.select_ar(a, K, seed=seed, sel_offset=sel_offset,
                                      realization=realization, cmp=cmp, bound_value=T,
                                      trial_cap=cap, nthreads=8)
    g = idx.cpu().numpy()
    mism = np.flatnonzero(g != oidx)
    assert mism.size == 0, f"{mism.size} mismatches, first at {mism[:5]}: {g[mism[:5]]} vs {oidx[mism[:5]]}"
    np.testing.assert_array_equal(stats.cpu().numpy().astype(np.uint64), ostats)
    assert int(st.item()) == ost


@pytest.mark.parametrize("cmp", [0, 1])
@pytest.mark.parametrize("fused", [True, False])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_select_plain(gb, orc, cmp, fused, dtype):
    _check_select(gb, orc, W.plain_uniform().astype(dtype), 1000, cmp, fused)


def _prefilter_vector(dtype):
    """Propensities over six decades with zeros and values below FP32's normal
    range (subnormal in the data's own precision too)."""
    rng = np.random.default_rng(77)
    if dtype == np.float64:
        special = [5e-324, 1e-310, 2.0 ** -1022, 2.0 ** -130, 2.0 ** -126, 2.0 ** -125, 0.0, 0.0]
    else:
        special = [1e-45, 1e-40, 2.0 ** -127, 2.0 ** -126, 2.0 ** -125, 0.0, 0.0]
    body = rng.exponential(1.0, 1000) * 10.0 ** rng.uniform(-4, 2, 1000)
    a = np.concatenate([special, body]).astype(dtype)
    rng.shuffle(a)
    return a


@pytest.mark.parametrize("fused", [True, False])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_fp64_comparison_prefilter_edges(gb, orc, dtype, fused):
    """The FP64 comparison decides most trials in FP32 with proven margins and
    takes the FP64 product within a 2^-17 band of the threshold, for
    propensities outside FP32's normal range (zeros are rejected outright),
    and for every trial when the bound lies outside [2^-94, 2^127].  Indices,
    counters and status equal the oracle's FP64 comparison bit for bit."""
    a = _prefilter_vector(dtype)
    _check_select(gb, orc, a, 20_000, 1, fused)                     # T = max
    if not fused:                                                     # T just above max
        _check_select(gb, orc, a, 20_000, 1, False,
                      bound_value=float(a.max()) * (1.0 + 2.0 ** -40))
    # bounds outside the pre-filter's range: every trial takes the FP64 product
    scales = (2.0 ** 200, 2.0 ** -300) if dtype == np.float64 else (2.0 ** -110,)
    for sc in scales:
        b = (a.astype(np.float64) * sc).astype(dtype)
        _check_select(gb, orc, b, 5_000, 1, fused)


@pytest.mark.parametrize("cmp", [0, 1])
@pytest.mark.parametrize("K", [1, 33, 4097, 65536])
def test_select_skewed(gb, orc, cmp, K):
    _check_select(gb, orc, W.skewed(seed=200), K, cmp, fused=True, sel_offset=65536 * 3)


@pytest.mark.parametrize("M", [1, 2, 3, 31, 32, 33, 1029, 40_000])
@pytest.mark.parametrize("cmp", [0, 1])
def test_select_sizes(gb, orc, M, cmp):
    _check_select(gb, orc, W.skewed(M, seed=M), 3000, cmp, fused=(M <= 40_000),
                  realization=M % 7)


@pytest.mark.parametrize("cmp", [0, 1])
def test_select_wide_range_l2_path(gb, orc, cmp):
    """M = 2^20 does not fit shared memory: gathers from L2 with the bound
    from ar_bound (the wide-dynamic-range workload, 12 decades)."""
    a = W.wide_range(M=1 << 20)
    _check_select(gb, orc, a, 20_000, cmp, fused=False)


def test_select_trial_cap_and_bound_multiplier(gb, orc):
    a = W.plain_uniform(100)
    _check_select(gb, orc, a, 2000, 1, fused=False, bound_value=float(a.max()) * 1e6, cap=8)
    _check_select(gb, orc, a, 2000, 0, fused=False, bound_value=float(a.max()) * 3.0)
    _check_select(gb, orc, a, 2000, 0, fused=False, bound_value=float(a.max()) * 1e6,
                  cap=(1 << 32))


def test_select_degenerate(gb, orc):
    import torch
    z = np.zeros(40, dtype=np.float32)
    _check_select(gb, orc, z, 100, 0, fused=True)
    one = np.zeros(555, dtype=np.float32)
    one[321] = 2.5
    _check_select(gb, orc, one, 500, 0, fused=True)
    _check_select(gb, orc, np.full(64, 3.0), 256, 1, fused=False)
    for T in (float("nan"), -1.0, float("inf")):
        _check_select(gb, orc, W.plain_uniform(16), 8, 1, fused=False, bound_value=T)
    # K = 0 is a no-op; M = 0 returns the sentinel 0
    idx, stats, st = gb.select_k(_t(np.zeros(0, dtype=np.float32)), 5)
    assert idx.cpu().tolist() == [0] * 5 and int(st.item()) == gb.AR_STATUS_ALL_ZERO
    idx, _, _ = gb.select_k(_t(W.plain_uniform(8)), 0)
    assert idx.numel() == 0
    with pytest.raises(gb.GbarError):
        gb.select_k(_t(W.plain_uniform(8)), 4, sel_offset=(1 << 32) - 2)
    with pytest.raises(gb.GbarError):
        big = torch.zeros(60_000_000, dtype=torch.float32, device="cuda")
        gb.select_k(big, 4)   # no bound and too large for shared memory


# -------------------------------------------------------- ar_select_batched
def _check_batched(gb, orc, bt, cmp=0, seed=1, sel_offset=0, realization_base=0, plan=False,
                   trial_cap=1 << 20):
    pl = gb.Plan(bt.offsets, bt.out_offsets) if plan else None
    bs, idx, stats, st = gb.select_batched(_t(bt.alpha), _t(bt.offsets), _t(bt.out_offsets),
                                           seed=seed, sel_offset=sel_offset,
                                           realization_base=realization_base, cmp=cmp,
                                           trial_cap=trial_cap, plan=pl)
    obs, oidx, ostats, ost = orc.select_batched(bt, seed=seed, sel_offset=sel_offset,
                                                realization_base=realization_base, cmp=cmp,
                                                trial_cap=trial_cap, nthreads=8)
    g = idx.cpu().numpy()
    mism = np.flatnonzero(g != oidx)
    assert mism.size == 0, f"{mism.size} mismatches of {g.size}, first at {mism[:5]}"
    gbs = bs.cpu().numpy()
    np.testing.assert_array_equal(gbs[:, 0], obs[:, 0])
    for b in range(bt.B):
        a = bt.alpha[bt.offsets[b]:bt.offsets[b + 1]]
        assert abs(gbs[b, 1] - obs[b, 1]) <= _sum_tol(a, obs[b, 1]), b
    np.testing.assert_array_equal(stats.cpu().numpy().astype(np.uint64), ostats)
    assert int(st.item()) == ost


@pytest.mark.parametrize("plan", [False, True])
@pytest.mark.parametrize("cmp", [0, 1])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_batched_ragged(gb, orc, cmp, dtype, plan):
    vecs = [W.skewed(m, seed=m).astype(dtype) for m in (1, 2, 3, 5, 7, 64, 1000, 4099, 16384,
                                                          20_000, 9, 1)]
    vecs.append(np.zeros(33, dtype=dtype))
    ks = [5, 0, 17, 1, 256, 300, 256, 1000, 64, 77, 3, 2, 9]
    _check_batched(gb, orc, W.batch_from_vectors(vecs, ks), cmp=cmp, seed=7, sel_offset=11,
                   realization_base=100, plan=plan)


@pytest.mark.parametrize("plan", [False, True])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_batched_wide_range(gb, orc, dtype, plan):
    """Propensities spread over many binades, subnormal and -0 entries: the
    exact fixed-point totals take every window (and drop nothing that
    matters), the maxima stay exact."""
    rng = np.random.default_rng(77)
    pw = np.ldexp(1.0, rng.integers(-149, 31, size=3000)) * rng.uniform(1, 2, size=3000)
    pw[rng.integers(0, 3000, size=50)] = -0.0
    pw[rng.integers(0, 3000, size=50)] = 0.0
    vecs = [W.wide_range(5000, seed=1).astype(dtype), pw.astype(np.float32).astype(dtype),
            W.wide_range(1030, seed=2).astype(dtype), W.wide_range(70_000, seed=3).astype(dtype)]
    _check_batched(gb, orc, W.batch_from_vectors(vecs, [100, 300, 7, 50]), cmp=0, seed=3,
                   plan=plan)


@pytest.mark.parametrize("plan", [False, True])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_batched_fp64_comparison_prefilter_edges(gb, orc, dtype, plan):
    """The batched round's FP64 comparison (FP32 pre-filter, FP64 product near
    the threshold and outside FP32's range): realizations with subnormal and
    sub-FP32 propensities and zeros, with bounds inside the pre-filter's range
    and above 2^127 or below 2^-94 (the FP64 product for every trial), equal
    the oracle's FP64 comparison bit for bit."""
    a = _prefilter_vector(dtype)
    scales = (1.0, 2.0 ** 200, 2.0 ** -300) if dtype == np.float64 else (1.0, 2.0 ** -110)
    vecs = [(a.astype(np.float64) * sc).astype(dtype) for sc in scales]
    vecs.append(a[:300].copy())
    _check_batched(gb, orc, W.batch_from_vectors(vecs, [3000, 700, 450, 1000][:len(vecs)]),
                   cmp=1, seed=9, sel_offset=5, plan=plan)


@pytest.mark.parametrize("plan", [False, True])
@pytest.mark.parametrize("cmp", [0, 1])
def test_batched_uneven_small(gb, orc, cmp, plan):
    _check_batched(gb, orc, W.batched_uneven(B=300, seed=301, K=256), cmp=cmp, plan=plan)


@pytest.mark.parametrize("plan", [False, True])
@pytest.mark.parametrize("seed", [300, 301, 305])
def test_batched_uneven_full(gb, orc, seed, plan):
    """The full batched workload: 4096 realizations, M_b log-uniform in
    [64, 16384], K_b = 256, FP32 comparison (the benchmark's launch)."""
    _check_batched(gb, orc, W.batched_uneven(seed=seed), plan=plan)


def test_batched_repeated_launches_reuse_workspace(gb, orc):
    """Back-to-back launches on one workspace (the benchmark's pattern, also
    under graph replay) give identical results: the claim counter in the
    workspace's first 16 bytes returns to zero."""
    import torch
    bt = W.batched_uneven(B=1000, seed=302, K=64)
    a, off, oo = _t(bt.alpha), _t(bt.offsets), _t(bt.out_offsets)
    work = torch.zeros(gb.ar_select_batched_workspace_size(bt.B), dtype=torch.uint8,
                       device="cuda")
    bs = torch.empty((bt.B, 2), dtype=torch.float64, device="cuda")
    idx = torch.empty(int(bt.out_offsets[-1]), dtype=torch.int32, device="cuda")
    stats = torch.zeros(3, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    _, oidx, _, _ = orc.select_batched(bt, nthreads=8)
    s = torch.cuda.Stream()
    for plan in (None, gb.Plan(bt.offsets, bt.out_offsets)):
        with torch.cuda.stream(s):
            for _ in range(5):
                idx.fill_(-1)
                gb.ar_select_batched(a, off, oo, 1, 0, 0, 0, 1 << 20, plan, bs, idx, stats, st,
                                     work, s)
                s.synchronize()
                assert np.array_equal(idx.cpu().numpy(), oidx)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s):
                gb.ar_select_batched(a, off, oo, 1, 0, 0, 0, 1 << 20, plan, bs, idx, stats, st,
                                     work, s)
            for _ in range(3):
                idx.fill_(-1)
                g.replay()
                s.synchronize()
                assert np.array_equal(idx.cpu().numpy(), oidx)
        assert work[:16].cpu().numpy().tolist() == [0] * 16
    assert int(st.item()) == 0


# ------------------------------------------- ar_bound_batched / _bounded
@pytest.mark.parametrize("plan", [False, True])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_bound_batched(gb, orc, dtype, plan):
    """The reduction step alone: exact maxima, totals within the FP64 bound,
    ALL_ZERO for an all-zero realization and for M_b = 0."""
    vecs = [W.wide_range(m, seed=m).astype(dtype) for m in (1, 3, 1000, 1025, 4099, 20_000)]
    vecs += [np.zeros(17, dtype=dtype), np.zeros(0, dtype=dtype), W.skewed(3000).astype(dtype)]
    bt = W.batch_from_vectors(vecs, [1] * len(vecs))
    pl = gb.Plan(bt.offsets, bt.out_offsets) if plan else None
    bs, st = gb.bound_batched(_t(bt.alpha), _t(bt.offsets), plan=pl)
    got = bs.cpu().numpy()
    for b, a in enumerate(vecs):
        mx, sm, _ = orc.bound(a)
        assert got[b, 0] == mx, b
        assert abs(got[b, 1] - sm) <= _sum_tol(a, sm), b
    assert int(st.item()) == gb.AR_STATUS_ALL_ZERO


@pytest.mark.parametrize("plan", [False, True])
@pytest.mark.parametrize("w", [1.0, 1.5, 2.0, 4.0])
def test_select_batched_bounded_threshold_sweep(gb, orc, w, plan):
    """T_w = w max per realization (the paper's threshold experiment): indices
    and trial counts bit-exact against the oracle at every w."""
    bt = W.batched_uneven(B=300, seed=303, K=128)
    bs_o, _, _, _ = orc.select_batched(bt)
    T = w * bs_o[:, 0]
    pl = gb.Plan(bt.offsets, bt.out_offsets) if plan else None
    idx, stats, st = gb.select_batched_bounded(_t(bt.alpha), _t(bt.offsets), _t(bt.out_offsets),
                                               _t(T), seed=4, sel_offset=9, plan=pl)
    oidx, ostats, ost = orc.select_batched_bounded(bt, T, seed=4, sel_offset=9, nthreads=8)
    np.testing.assert_array_equal(idx.cpu().numpy(), oidx)
    np.testing.assert_array_equal(stats.cpu().numpy().astype(np.uint64), ostats)
    assert int(st.item()) == ost


def test_select_batched_bounded_stride_and_bad_bounds(gb, orc):
    """Stride 2 over a bound_sum array; NaN, negative and infinite bounds give
    BAD_BOUND and the sentinel; a zero bound gives ALL_ZERO."""
    bt = W.batched_uneven(B=40, seed=304, m_lo=8, m_hi=3000, K=50)
    bs, _ = gb.bound_batched(_t(bt.alpha), _t(bt.offsets))
    idx, stats, st = gb.select_batched_bounded(_t(bt.alpha), _t(bt.offsets), _t(bt.out_offsets),
                                               bs, bound_stride=2)
    _, oidx, ostats, ost = orc.select_batched(bt)
    np.testing.assert_array_equal(idx.cpu().numpy(), oidx)
    assert int(st.item()) == ost
    T = bs[:, 0].cpu().numpy().copy()
    T[3], T[7], T[11], T[20] = np.nan, -2.0, np.inf, 0.0
    for cmp in (0, 1):
        idx, _, st = gb.select_batched_bounded(_t(bt.alpha), _t(bt.offsets), _t(bt.out_offsets),
                                               _t(T), cmp=cmp)
        oidx, _, ost = orc.select_batched_bounded(bt, T, cmp=cmp)
        np.testing.assert_array_equal(idx.cpu().numpy(), oidx)
        assert int(st.item()) == ost == gb.AR_STATUS_BAD_BOUND | gb.AR_STATUS_ALL_ZERO


@pytest.mark.parametrize("plan", [False, True])
def test_batched_invalid_realization(gb, orc, plan):
    """A realization holding NaN / -1 / inf: BAD_ALPHA, (NaN, NaN) bound, the
    sentinel for its indices; the other realizations are unaffected."""
    bt = W.batched_uneven(B=64, seed=305, m_lo=16, m_hi=5000, K=40)
    a = bt.alpha.copy()
    a[bt.offsets[5] + 2] = np.nan
    a[bt.offsets[17]] = -1.0
    a[bt.offsets[40] + 1] = np.inf
    bt2 = W.Batch(a, bt.offsets, bt.out_offsets)
    pl = gb.Plan(bt.offsets, bt.out_offsets) if plan else None
    bs, idx, stats, st = gb.select_batched(_t(a), _t(bt.offsets), _t(bt.out_offsets), plan=pl)
    obs, oidx, ostats, ost = orc.select_batched(bt2, nthreads=8)
    np.testing.assert_array_equal(idx.cpu().numpy(), oidx)
    np.testing.assert_array_equal(stats.cpu().numpy().astype(np.uint64), ostats)
    g = bs.cpu().numpy()
    np.testing.assert_array_equal(np.isnan(g), np.isnan(obs))
    np.testing.assert_array_equal(g[~np.isnan(g[:, 0]), 0], obs[~np.isnan(obs[:, 0]), 0])
    assert int(st.item()) == ost == gb.AR_STATUS_BAD_ALPHA


def test_plan_autotune(gb, orc):
    """The autotuner times the tile candidates on the data and keeps one;
    results do not depend on the schedule."""
    import torch
    bt = W.batched_uneven(B=600, seed=306, K=64)
    a, off, oo = _t(bt.alpha), _t(bt.offsets), _t(bt.out_offsets)
    plan = gb.Plan(bt.offsets, bt.out_offsets)
    bs = torch.empty((bt.B, 2), dtype=torch.float64, device="cuda")
    idx = torch.empty(int(bt.out_offsets[-1]), dtype=torch.int32, device="cuda")
    stats = torch.zeros(3, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    warps, share, ns = gb.ar_plan_autotune(plan, a, off, oo, 1, 0, bs, idx, stats, st, reps=3)
    assert warps in (8, 16, 32) and share in (0, 300, 600) and ns > 0
    _, oidx, ostats, _ = orc.select_batched(bt, nthreads=8)
    _, idx2, stats2, st2 = gb.select_batched(a, off, oo, plan=plan)
    np.testing.assert_array_equal(idx2.cpu().numpy(), oidx)
    np.testing.assert_array_equal(stats2.cpu().numpy().astype(np.uint64), ostats)


@pytest.mark.parametrize("warps,share", [(8, 0), (16, 1000), (32, 250)])
def test_plan_set_tile(gb, orc, warps, share):
    """Any tile the plan is set to gives the oracle's results; bad tiles are
    rejected."""
    bt = W.batched_uneven(B=300, seed=307, K=48)
    a, off, oo = _t(bt.alpha), _t(bt.offsets), _t(bt.out_offsets)
    plan = gb.Plan(bt.offsets, bt.out_offsets)
    gb.ar_plan_set_tile(plan, warps, share)
    _, oidx, ostats, _ = orc.select_batched(bt, nthreads=8)
    _, idx, stats, st = gb.select_batched(a, off, oo, plan=plan)
    np.testing.assert_array_equal(idx.cpu().numpy(), oidx)
    np.testing.assert_array_equal(stats.cpu().numpy().astype(np.uint64), ostats)
    for bad in ((12, 0), (16, -1), (16, 1001)):
        with pytest.raises(gb.GbarError):
            gb.ar_plan_set_tile(plan, *bad)


@pytest.mark.parametrize("tile", [(8, 300), (16, 0), (32, 0)])
def test_batched_two_calls_in_flight(gb, orc, tile):
    """Two independent batches, each with its own plan, alternating on two
    streams (the benchmark's headline pattern): both match the oracle after
    many overlapping calls."""
    import torch
    bts = [W.batched_uneven(B=1500, seed=320 + k, K=128) for k in range(2)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    bufs = []
    for bt in bts:
        plan = gb.Plan(bt.offsets, bt.out_offsets)
        gb.ar_plan_set_tile(plan, *tile)
        bufs.append(dict(
            a=_t(bt.alpha), off=_t(bt.offsets), oo=_t(bt.out_offsets), plan=plan,
            bs=torch.empty((bt.B, 2), dtype=torch.float64, device="cuda"),
            idx=torch.empty(int(bt.out_offsets[-1]), dtype=torch.int32, device="cuda"),
            stats=torch.zeros(3, dtype=torch.int64, device="cuda"),
            st=torch.zeros(1, dtype=torch.int32, device="cuda")))
    torch.cuda.synchronize()
    for i in range(20):  # ten calls per batch; the counters add up
        b = bufs[i % 2]
        gb.ar_select_batched(b["a"], b["off"], b["oo"], 1, 0, 0, 0, 1 << 20, b["plan"], b["bs"],
                             b["idx"], b["stats"], b["st"], None, streams[i % 2])
    torch.cuda.synchronize()
    for bt, b in zip(bts, bufs):
        obs, oidx, ostats, ost = orc.select_batched(bt, nthreads=8)
        np.testing.assert_array_equal(b["idx"].cpu().numpy(), oidx)
        np.testing.assert_array_equal(b["bs"].cpu().numpy()[:, 0], obs[:, 0])
        np.testing.assert_array_equal(b["stats"].cpu().numpy().astype(np.uint64), 10 * ostats)
        assert int(b["st"].item()) == ost


@pytest.mark.parametrize("plan", [False, True])
@pytest.mark.parametrize("cap", [1, 2, 3, 5, 6, 7, 13, 64])
def test_batched_trial_cap(gb, orc, cap, plan):
    """Small trial caps, odd and even, below, at and above the trials of one
    round: capped selections get the sentinel M_b and count cap trials, in
    steady rounds and in the tail where lanes share selections."""
    bt = W.batched_uneven(B=200, seed=330, m_lo=16, m_hi=3000, K=96)
    _check_batched(gb, orc, bt, cmp=0, seed=4, plan=plan, trial_cap=cap)


@pytest.mark.parametrize("plan", [False, True])
@pytest.mark.parametrize("cmp", [0, 1])
def test_batched_tiny_bounds(gb, orc, cmp, plan):
    """Realizations whose maximum lies near and below 2^-102 (where the FP32
    bound can no longer be pre-scaled by 2^-24 exactly) and in the subnormal
    range: the same indices as the oracle."""
    rng = np.random.default_rng(331)
    vecs = []
    for e in (-100, -102, -103, -110, -126, -140, -149):
        v = np.ldexp(rng.uniform(0.5, 1.0, size=300), e).astype(np.float32)
        v[rng.integers(0, 300, size=20)] = 0.0
        vecs.append(v)
    vecs.append(W.skewed(500, seed=9).astype(np.float32))
    _check_batched(gb, orc, W.batch_from_vectors(vecs, [200] * len(vecs)), cmp=cmp, seed=5,
                   plan=plan)
