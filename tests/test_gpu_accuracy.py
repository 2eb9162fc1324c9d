"""GPU: accuracy of the FP32 comparison at 10^7 selections (the paper's
quality experiment draws 10^7 selections, Results, "Quality of the selection
of the reaction indexes").

For the plain vector (M = 1024 FP64 Uniform(0,1]), the skewed vector
(M = 1029, lognormal, 309 zeros), the wide-range vector (M = 2^20 over 12
decades) and the batched workload, the FP32 and FP64
comparisons run on identical Philox streams.  Asserted:
* the paired index-mismatch rate and the paired TV are <= 1e-3;
* the FP32 histogram fits alpha_j / sum(alpha) (chi-square, bins merged to an
  expected count >= 5, p > 0.001), and no selection lands on a zero
  propensity;
* the first selections of both precisions equal the CPU oracle's, so the
  FP64 side of the pair is the oracle's stream.
"""
import numpy as np
import pytest

from paper_1404_0027_gb300 import accuracy as A
from paper_1404_0027_gb300 import workloads as W

pytestmark = pytest.mark.gpu

N = 10_000_000
GATE = 1e-3


@pytest.fixture(scope="module")
def gb():
    import torch
    from paper_1404_0027_gb300 import build
    build.build()
    from paper_1404_0027_gb300 import binding
    binding.lib()
    assert torch.cuda.is_available()
    return binding


def _single(gb, alpha):
    import torch
    t = torch.from_numpy(alpha).cuda()
    bs, st = gb.bound(t)
    out = {}
    for cmp in (gb.AR_CMP_F32, gb.AR_CMP_F64):
        idx, stats, st2 = gb.select_k(t, N, seed=1, cmp=cmp, bound=bs[:1])
        torch.cuda.synchronize()
        assert int(st.item()) == 0 and int(st2.item()) == 0
        assert int(stats[1].item()) == N          # every selection accepted
        out[cmp] = idx.cpu().numpy()
    return out[gb.AR_CMP_F32], out[gb.AR_CMP_F64]


@pytest.mark.parametrize("name", ["plain", "skewed", "wide_range"])
def test_fp32_accuracy_at_1e7(gb, orc, name):
    alpha = {"plain": lambda: W.plain_uniform(1024, seed=101),
             "skewed": lambda: W.skewed(1029, seed=200),
             "wide_range": lambda: W.wide_range(1 << 20, seed=400)}[name]()
    i32, i64 = _single(gb, alpha)
    # the first selections of each precision are the oracle's
    for cmp, got in ((0, i32), (1, i64)):
        want, _, _ = orc.select_ar(alpha, 20_000, seed=1, cmp=cmp)
        np.testing.assert_array_equal(got[:20_000], want)
    pr = A.paired(i32, i64, alpha.size + 1)
    assert pr["index_mismatch"] <= GATE, pr
    assert pr["paired_tv"] <= pr["index_mismatch"] + 1e-12
    for idx in (i32, i64):
        lw = A.law(idx, alpha)
        assert lw["count_in_zero_bins"] == 0, lw
        assert lw["p_value"] > 1e-3, lw
        # the empirical TV is that of an exact sampler (within 10 %)
        assert lw["tv_vs_exact"] < 1.1 * lw["tv_exact_sampler_expected"], lw


def test_batched_fp32_accuracy_at_1e7(gb):
    import torch
    bt = W.batched_uneven(B=4096, seed=300, m_lo=64, m_hi=16384, K=256)
    dev = torch.device("cuda")
    alpha = torch.from_numpy(bt.alpha).to(dev)
    off = torch.from_numpy(bt.offsets).to(dev)
    oo = torch.from_numpy(bt.out_offsets).to(dev)
    plan = gb.Plan(bt.offsets, bt.out_offsets)
    B, K = 4096, 256
    b_of = np.repeat(np.arange(B, dtype=np.int64), np.diff(bt.out_offsets))
    cell0 = (bt.offsets[:-1] + np.arange(B))[b_of]
    ncells = int(bt.offsets[-1]) + B
    calls = N // (B * K) + 1
    keys = {0: [], 1: []}
    bs = torch.empty((B, 2), dtype=torch.float64, device=dev)
    idx = torch.empty(B * K, dtype=torch.int32, device=dev)
    stats = torch.zeros(3, dtype=torch.int64, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    for c in range(calls):
        for cmp in (0, 1):
            gb.ar_select_batched(alpha, off, oo, 1, c * K, 0, cmp, 1 << 20, plan, bs, idx, stats,
                                 st, None)
            torch.cuda.synchronize()
            keys[cmp].append(cell0 + idx.cpu().numpy())
    assert int(st.item()) == 0
    assert int(stats[1].item()) == 2 * calls * B * K
    pr = A.paired(np.concatenate(keys[0]), np.concatenate(keys[1]), ncells)
    assert pr["n"] >= N
    assert pr["index_mismatch"] <= GATE, pr
    assert pr["paired_tv"] <= pr["index_mismatch"] + 1e-12
    plan.close()
