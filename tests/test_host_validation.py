"""Host-side argument checks of the C ABI, without a GPU.

Every case below is rejected (or accepted as a no-op) before the library
touches the CUDA runtime, so it runs on a machine without a GPU: pointers are
plain integers that are never dereferenced.  The codes are the ones
include/gbar.h documents for each entry point."""
import ctypes

import pytest

AR_OK, AR_ERR_ARG, AR_ERR_ALIGN, AR_ERR_WORKSPACE = 0, -1, -2, -4
F32, F64 = 0, 1
CMP_F32, CMP_F64 = 0, 1
P = 0x10000          # a 256-byte aligned fake device address
CAP = 1 << 20


@pytest.fixture(scope="module")
def L():
    from paper_1404_0027_gb300 import binding, build
    try:
        build.build()
    except RuntimeError as e:
        pytest.skip(f"nvcc unavailable: {e}")
    return binding.lib()


def vp(x):
    return ctypes.c_void_p(x)


# ------------------------------------------------------------- ar_select_k
def _select_k(L, alpha=P, dtype=F32, M=1000, bound=P + 0x1000, K=100, sel_offset=0, cmp=CMP_F32,
              cap=CAP, idx=P + 0x2000, stats=P + 0x3000, status=P + 0x4000):
    return L.ar_select_k(vp(alpha), dtype, M, vp(bound), K, 1, sel_offset, 0, cmp, cap, vp(idx),
                         vp(stats), vp(status), None)


@pytest.mark.parametrize("kw,code", [
    (dict(dtype=7), AR_ERR_ARG), (dict(cmp=5), AR_ERR_ARG), (dict(M=-1), AR_ERR_ARG),
    (dict(M=1 << 31), AR_ERR_ARG), (dict(K=-1), AR_ERR_ARG), (dict(cap=0), AR_ERR_ARG),
    (dict(cap=(1 << 32) + 1), AR_ERR_ARG), (dict(sel_offset=(1 << 32) - 10, K=11), AR_ERR_ARG),
    (dict(idx=0), AR_ERR_ARG), (dict(status=0), AR_ERR_ARG), (dict(alpha=0), AR_ERR_ARG),
    (dict(alpha=P + 2), AR_ERR_ALIGN), (dict(dtype=F64, alpha=P + 4), AR_ERR_ALIGN),
    (dict(idx=P + 0x2002), AR_ERR_ALIGN), (dict(stats=P + 0x3004), AR_ERR_ALIGN),
    (dict(bound=P + 0x1004), AR_ERR_ALIGN), (dict(status=P + 0x4001), AR_ERR_ALIGN),
    (dict(K=0), AR_OK), (dict(K=0, idx=0, alpha=0), AR_OK),
])
def test_select_k_arguments(L, kw, code):
    assert _select_k(L, **kw) == code


# ------------------------------------------------------------------ ar_bound
def test_bound_arguments(L):
    wsz = L.ar_bound_workspace_size(1 << 22, F32)
    assert wsz > 16
    args = lambda **k: (vp(k.get("alpha", P)), k.get("dtype", F32), k.get("M", 1 << 22),
                        vp(k.get("bs", P + 0x100)), vp(k.get("st", P + 0x200)),
                        vp(k.get("work", P + 0x1000)), k.get("wb", wsz), None)
    assert L.ar_bound(*args(M=-1)) == AR_ERR_ARG
    assert L.ar_bound(*args(dtype=3)) == AR_ERR_ARG
    assert L.ar_bound(*args(bs=0)) == AR_ERR_ARG
    assert L.ar_bound(*args(alpha=0)) == AR_ERR_ARG
    assert L.ar_bound(*args(alpha=P + 1)) == AR_ERR_ALIGN
    assert L.ar_bound(*args(bs=P + 0x104)) == AR_ERR_ALIGN
    # a multi-CTA reduction needs its zero-filled workspace
    assert L.ar_bound(*args(work=0)) == AR_ERR_WORKSPACE
    assert L.ar_bound(*args(wb=wsz - 1)) == AR_ERR_WORKSPACE
    assert L.ar_bound(*args(work=P + 0x1008)) == AR_ERR_ALIGN


# ---------------------------------------------------------- ar_bound_noalloc
LIMIT_F32, LIMIT_F64 = 33554432, 16777216   # AR_BOUND_NOALLOC_MAX_M_F32 / _F64


def test_bound_noalloc_arguments(L):
    """Every rejection comes back before the CUDA runtime is touched: on a
    machine without a GPU, a call that reached cudaGetSymbolAddress or a
    launch would return AR_ERR_CUDA instead of these codes."""
    AR_ERR_UNSUPPORTED = -5
    args = lambda **k: (vp(k.get("alpha", P)), k.get("dtype", F32), k.get("M", 1 << 22),
                        vp(k.get("bs", P + 0x100)), vp(k.get("st", P + 0x200)), None)
    assert L.ar_bound_noalloc(*args(M=-1)) == AR_ERR_ARG
    assert L.ar_bound_noalloc(*args(dtype=3)) == AR_ERR_ARG
    assert L.ar_bound_noalloc(*args(st=0)) == AR_ERR_ARG
    assert L.ar_bound_noalloc(*args(bs=0)) == AR_ERR_ARG
    assert L.ar_bound_noalloc(*args(alpha=0)) == AR_ERR_ARG
    # sizes beyond the static scratch array, for each dtype
    assert L.ar_bound_noalloc(*args(M=LIMIT_F32 + 1)) == AR_ERR_UNSUPPORTED
    assert L.ar_bound_noalloc(*args(dtype=F64, M=LIMIT_F64 + 1)) == AR_ERR_UNSUPPORTED
    # alignment is checked before the scratch header is cleared
    assert L.ar_bound_noalloc(*args(alpha=P + 2)) == AR_ERR_ALIGN
    assert L.ar_bound_noalloc(*args(dtype=F64, alpha=P + 4)) == AR_ERR_ALIGN
    assert L.ar_bound_noalloc(*args(bs=P + 0x104)) == AR_ERR_ALIGN
    assert L.ar_bound_noalloc(*args(st=P + 0x201)) == AR_ERR_ALIGN


# --------------------------------------------------- batched entry points
B = 100


def _batched(L, fn, **k):
    alpha = vp(k.get("alpha", P))
    dtype = k.get("dtype", F32)
    off, oo = vp(k.get("off", P + 0x1000)), vp(k.get("oo", P + 0x2000))
    nb = k.get("B", B)
    bs, idx = vp(k.get("bs", P + 0x3000)), vp(k.get("idx", P + 0x4000))
    stats, st = vp(k.get("stats", P + 0x5000)), vp(k.get("st", P + 0x6000))
    work = vp(k.get("work", P + 0x10000))
    wb = k.get("wb", L.ar_select_batched_workspace_size(nb))
    cmp, cap = k.get("cmp", CMP_F32), k.get("cap", CAP)
    base, sel = k.get("base", 0), k.get("sel", 0)
    if fn == "select":
        return L.ar_select_batched(alpha, dtype, off, oo, nb, 1, sel, base, cmp, cap, None, bs,
                                   idx, stats, st, work, wb, None)
    if fn == "bounded":
        return L.ar_select_batched_bounded(alpha, dtype, off, oo, nb, bs, k.get("stride", 2), 1,
                                           sel, base, cmp, cap, None, idx, stats, st, work, wb,
                                           None)
    return L.ar_bound_batched(alpha, dtype, off, nb, None, bs, st, work, wb, None)


@pytest.mark.parametrize("fn", ["select", "bounded", "bound"])
def test_batched_common_arguments(L, fn):
    assert _batched(L, fn, dtype=9) == AR_ERR_ARG
    assert _batched(L, fn, B=-1) == AR_ERR_ARG
    assert _batched(L, fn, B=1 << 31) == AR_ERR_ARG
    assert _batched(L, fn, alpha=0) == AR_ERR_ARG
    assert _batched(L, fn, off=0) == AR_ERR_ARG
    assert _batched(L, fn, st=0) == AR_ERR_ARG
    assert _batched(L, fn, alpha=P + 2) == AR_ERR_ALIGN
    assert _batched(L, fn, off=P + 0x1004) == AR_ERR_ALIGN
    assert _batched(L, fn, st=P + 0x6002) == AR_ERR_ALIGN
    # without a plan the workspace is required, large enough and 16-byte aligned
    assert _batched(L, fn, work=0) == AR_ERR_WORKSPACE
    assert _batched(L, fn, wb=L.ar_select_batched_workspace_size(B) - 1) == AR_ERR_WORKSPACE
    assert _batched(L, fn, work=P + 0x10008) == AR_ERR_ALIGN
    assert _batched(L, fn, bs=0) == AR_ERR_ARG
    if fn != "bounded":
        assert _batched(L, fn, bs=P + 0x3004) == AR_ERR_ALIGN


@pytest.mark.parametrize("fn", ["select", "bounded"])
def test_batched_selection_arguments(L, fn):
    assert _batched(L, fn, B=0) == AR_OK                     # nothing to do
    assert _batched(L, fn, cmp=4) == AR_ERR_ARG
    assert _batched(L, fn, cap=0) == AR_ERR_ARG
    assert _batched(L, fn, cap=(1 << 32) + 1) == AR_ERR_ARG
    assert _batched(L, fn, base=(1 << 32) - B + 1) == AR_ERR_ARG   # realization ids past 2^32
    assert _batched(L, fn, sel=1 << 32) == AR_ERR_ARG
    assert _batched(L, fn, oo=0) == AR_ERR_ARG
    assert _batched(L, fn, idx=0) == AR_ERR_ARG
    assert _batched(L, fn, idx=P + 0x4002) == AR_ERR_ALIGN
    assert _batched(L, fn, stats=P + 0x5004) == AR_ERR_ALIGN
    if fn == "bounded":
        assert _batched(L, fn, stride=0) == AR_ERR_ARG


def test_plan_set_tile_needs_a_plan(L):
    assert L.ar_plan_set_tile(None, 16, 0) == AR_ERR_ARG
    assert L.ar_plan_set_grid(None, 1, 0) == AR_ERR_ARG
    assert L.ar_plan_set_grid(None, 0, 128) == AR_ERR_ARG


# ------------------------------------------------------------- comparators
def test_select_paper_arguments(L):
    args = lambda **k: (vp(k.get("D", P)), k.get("M", 64), vp(k.get("bd", P + 0x100)),
                        k.get("K", 10), 1, k.get("sel", 0), 0, vp(k.get("idx", P + 0x200)),
                        vp(k.get("rej", P + 0x300)), None)
    assert L.ar_select_paper(*args(M=-1)) == AR_ERR_ARG
    assert L.ar_select_paper(*args(K=-1)) == AR_ERR_ARG
    assert L.ar_select_paper(*args(sel=(1 << 32) - 5)) == AR_ERR_ARG
    assert L.ar_select_paper(*args(K=0)) == AR_OK
    assert L.ar_select_paper(*args(bd=0)) == AR_ERR_ARG
    assert L.ar_select_paper(*args(idx=0)) == AR_ERR_ARG
    assert L.ar_select_paper(*args(D=P + 2)) == AR_ERR_ALIGN
    assert L.ar_select_paper(*args(rej=P + 0x304)) == AR_ERR_ALIGN


def test_select_it_arguments(L):
    M = 1000
    wsz = L.ar_select_it_workspace_size(M)
    assert wsz >= 8 * M
    args = lambda **k: (vp(k.get("a", P)), k.get("dtype", F32), M, k.get("K", 10), 1, 0, 0,
                        vp(k.get("idx", P + 0x1000)), vp(k.get("st", P + 0x2000)),
                        vp(k.get("work", P + 0x10000)), k.get("wb", wsz), None)
    assert L.ar_select_it(*args(dtype=5)) == AR_ERR_ARG
    assert L.ar_select_it(*args(K=-1)) == AR_ERR_ARG
    assert L.ar_select_it(*args(st=0)) == AR_ERR_ARG
    assert L.ar_select_it(*args(work=0)) == AR_ERR_WORKSPACE
    assert L.ar_select_it(*args(wb=wsz - 1)) == AR_ERR_WORKSPACE
    assert L.ar_select_it(*args(a=P + 2)) == AR_ERR_ALIGN
    assert L.ar_select_it(*args(work=P + 0x10008)) == AR_ERR_ALIGN


# ------------------------------------------------------------------- probe
def test_probe_arguments():
    """The benchmark's probe library (not part of libgbar's ABI) rejects bad
    arguments before any CUDA call."""
    from paper_1404_0027_gb300 import build, probe
    try:
        build.build()
    except RuntimeError as e:
        pytest.skip(f"nvcc unavailable: {e}")
    f = probe.lib().gbar_probe_throughput
    out = vp(P)
    assert f(2, None, 0, 4, 256, out, 1 << 20, None) == -1
    assert f(0, None, 0, 3, 256, out, 1 << 20, None) == -1
    assert f(0, None, 0, 0, 256, out, 1 << 20, None) == -1
    assert f(0, None, 0, 4, 100, out, 1 << 20, None) == -1
    assert f(0, None, 0, 4, 256, None, 1 << 20, None) == -1
    assert f(1, None, 1000, 4, 256, out, 1 << 20, None) == -1
    assert f(1, vp(P + 0x100), 0, 4, 256, out, 1 << 20, None) == -1
    assert f(0, None, 0, 4, 256, vp(P + 2), 1 << 20, None) == -2


def test_probe_not_in_product_abi(L):
    assert not hasattr(L, "ar_probe_throughput")


# --------------------------------------------------------------------- SSA
def test_ssa_arguments(L):
    n = None
    assert L.ssa_step_batched(n, 10, vp(P), vp(P), vp(P), vp(P), 5, 1, 0, 0, CAP, None,
                              vp(P), None, None) == AR_ERR_ARG
    # ssa_run_until: a negative or NaN time limit, negative counts
    for t_end, nsamp, nspec in ((-1.0, 0, 0), (float("nan"), 0, 0), (1.0, -1, 0), (1.0, 0, -1)):
        assert L.ssa_run_until(n, 10, vp(P), vp(P), vp(P), vp(P), t_end, 5, 1, 0, 0, CAP, None,
                               nsamp, None, nspec, None, None, vp(P), None, None) == AR_ERR_ARG
