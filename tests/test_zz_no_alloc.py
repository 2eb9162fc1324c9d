"""ar_bound_noalloc against ar_bound (GPU).

ar_bound_noalloc serves callers that cannot allocate device memory -- a
plug-in handed only its input and output buffers, a component whose host
application owns all device allocations, a stepping loop that must not meet
cudaMalloc's implicit synchronisation.  Its scratch lives in one static
device array shared by every call, so two calls in a row must each give the
result of the workspace-taking entry point (the second call starts from
whatever the first left in the array).  This file is collected last so that
a run stopping at its first failure has already run every other test.
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


def _tol(a, total):
    # the parity tolerance of the bound tests: 2 (M + 8) 2^-53 |sum|
    return 2.0 * (a.size + 8) * 2.0 ** -53 * abs(total)


def _both(gb, a):
    import torch
    t = torch.from_numpy(a).cuda()
    ref, ref_st = gb.bound(t)                       # workspace-taking entry point
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    gb.ar_bound_noalloc(t, out, st)                 # the allocation-free one
    torch.cuda.synchronize()
    return ref.cpu().numpy(), int(ref_st.item()), out.cpu().numpy(), int(st.item())


@pytest.mark.parametrize("dtype,M", [(np.float32, 1 << 20), (np.float32, 5000),
                                     (np.float64, 300_001)])
def test_noalloc_matches_ar_bound_twice(gb, dtype, M):
    for call, seed in enumerate((11, 12)):        # two calls in a row
        a = W.wide_range(M, seed=seed + M).astype(dtype)
        ref, ref_st, out, st = _both(gb, a)
        assert out[0] == ref[0], (call, out, ref)
        assert abs(out[1] - ref[1]) <= _tol(a, ref[1]), (call, out, ref)
        assert st == ref_st == 0


def test_noalloc_status_and_limit(gb):
    import torch
    a = W.plain_uniform(70_000).astype(np.float32)
    a[123] = np.nan
    _, ref_st, _, st = _both(gb, a)
    assert st == ref_st == gb.AR_STATUS_BAD_ALPHA
    # the next call after a flagged one is clean again
    a[123] = 0.5
    ref, ref_st, out, st = _both(gb, a)
    assert st == ref_st == 0 and out[0] == ref[0]
    # sizes beyond the static array are rejected before any launch
    limit = 33554432
    big = torch.zeros(limit + 1, dtype=torch.float32, device="cuda")
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(gb.GbarError, match="AR_ERR_UNSUPPORTED"):
        gb.ar_bound_noalloc(big, out, st)
    gb.ar_bound_noalloc(big[:limit], out, st)     # exactly at the limit works
    torch.cuda.synchronize()
    assert int(st.item()) == gb.AR_STATUS_ALL_ZERO
