"""Thin Python binding of libgbar.so (the C ABI declared in include/gbar.h).

Functions keep the C names and argument order; device buffers are passed as
CUDA torch tensors (PyTorch is only the device-memory and stream provider).
Every step of the selection runs in the library's kernels: there is no
Python or CPU fallback, and calling anything here without the built library
raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgbar.so")

AR_OK = 0
AR_ERR_ARG = -1
AR_ERR_ALIGN = -2
AR_ERR_CUDA = -3
AR_ERR_WORKSPACE = -4
AR_ERR_UNSUPPORTED = -5
_ERR_NAMES = {AR_ERR_ARG: "AR_ERR_ARG", AR_ERR_ALIGN: "AR_ERR_ALIGN", AR_ERR_CUDA: "AR_ERR_CUDA",
              AR_ERR_WORKSPACE: "AR_ERR_WORKSPACE", AR_ERR_UNSUPPORTED: "AR_ERR_UNSUPPORTED"}

AR_STATUS_BAD_ALPHA = 1
AR_STATUS_ALL_ZERO = 2
AR_STATUS_TRIAL_CAP = 4
AR_STATUS_BAD_BOUND = 8
AR_STATUS_ABSORBED = 16
AR_STATUS_WAIT_LIMIT = 32
AR_STATUS_UNSUPPORTED = 64

AR_F32 = 0
AR_F64 = 1
AR_CMP_F32 = 0
AR_CMP_F64 = 1

_lock = threading.Lock()
_lib = None

_vp, _i64, _u64, _u32, _int, _sz = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64,
                                     ctypes.c_uint32, ctypes.c_int, ctypes.c_size_t)

# name -> (restype, argtypes); mirrors include/gbar.h
SIGNATURES = {
    "ar_version": (_int, []),
    "ar_last_cuda_error": (_int, []),
    "ar_bound_workspace_size": (_sz, [_i64, _int]),
    "ar_bound": (_int, [_vp, _int, _i64, _vp, _vp, _vp, _sz, _vp]),
    "ar_bound_noalloc": (_int, [_vp, _int, _i64, _vp, _vp, _vp]),
    "ar_select_k_smem_limit": (_sz, []),
    "ar_select_k": (_int, [_vp, _int, _i64, _vp, _i64, _u64, _u64, _u32, _int, _u64, _vp, _vp,
                           _vp, _vp]),
    "ar_select_batched_workspace_size": (_sz, [_i64]),
    "ar_plan_create": (_int, [_vp, _vp, _i64, ctypes.POINTER(ctypes.c_void_p)]),
    "ssa_net_create": (_int, [ctypes.c_int32, ctypes.c_int32, _vp, _vp, _vp, _vp, _vp, _vp,
                              ctypes.POINTER(ctypes.c_void_p)]),
    "ssa_net_destroy": (None, [_vp]),
    "ssa_step_batched": (_int, [_vp, _i64, _vp, _vp, _vp, _vp, _i64, _u64, _u32, _int, _u64,
                                _vp, _vp, _vp, _vp]),
    "ar_plan_destroy": (None, [_vp]),
    "ssa_run_until": (_int, [_vp, _i64, _vp, _vp, _vp, _vp, ctypes.c_double, _i64, _u64, _u32,
                             _int, _u64, _vp, ctypes.c_int32, _vp, ctypes.c_int32, _vp, _vp,
                             _vp, _vp, _vp]),
    "ar_select_batched": (_int, [_vp, _int, _vp, _vp, _i64, _u64, _u64, _u32, _int, _u64, _vp,
                                 _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "ar_bound_batched": (_int, [_vp, _int, _vp, _i64, _vp, _vp, _vp, _vp, _sz, _vp]),
    "ar_select_paper": (_int, [_vp, _i64, _vp, _i64, _u64, _u64, _u32, _vp, _vp, _vp]),
    "ar_plan_autotune": (_int, [_vp, _vp, _int, _vp, _vp, _u64, _int, _vp, _vp, _vp, _vp, _int,
                                _vp, _vp]),
    "ar_select_it_workspace_size": (_sz, [_i64]),
    "ar_select_it": (_int, [_vp, _int, _i64, _i64, _u64, _u64, _u32, _vp, _vp, _vp, _sz, _vp]),
    "ar_select_batched_bounded": (_int, [_vp, _int, _vp, _vp, _i64, _vp, _i64, _u64, _u64, _u32,
                                         _int, _u64, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "ar_plan_set_tile": (_int, [_vp, _int, _int]),
    "ar_plan_set_grid": (_int, [_vp, _int, _int]),
}


class GbarError(RuntimeError):
    pass


def lib():
    """Load libgbar.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        with _lock:
            if _lib is None:
                if not os.path.exists(LIB_PATH):
                    raise GbarError(f"{LIB_PATH} is missing: build it with "
                                    "paper_1404_0027_gb300.build.build() (needs nvcc)")
                L = ctypes.CDLL(LIB_PATH)
                for name, (res, args) in SIGNATURES.items():
                    f = getattr(L, name)
                    f.restype = res
                    f.argtypes = args
                _lib = L
    return _lib


def _check(rc: int, what: str):
    if rc != AR_OK:
        extra = ""
        if rc == AR_ERR_CUDA:
            extra = f" (cudaError {lib().ar_last_cuda_error()})"
        raise GbarError(f"{what} returned {_ERR_NAMES.get(rc, rc)}{extra}")


def _dev(t, dtype=None, name="tensor"):
    """Device pointer of a contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise GbarError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise GbarError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise GbarError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return AR_F32
    if t.dtype == torch.float64:
        return AR_F64
    raise GbarError("propensities must be float32 or float64")


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


# --------------------------------------------------------------------------
# C-ABI mirrors
# --------------------------------------------------------------------------
def ar_bound_workspace_size(M: int, dtype: int) -> int:
    return int(lib().ar_bound_workspace_size(M, dtype))


def ar_bound(alpha, bound_sum, status, work=None, stream=None):
    """alpha [M] f32/f64 -> bound_sum [2] f64 (max, sum); status u32[1] |= bits."""
    nbytes = 0 if work is None else work.numel() * work.element_size()
    _check(lib().ar_bound(_dev(alpha, name="alpha"), _dtype_code(alpha), alpha.numel(),
                          _dev(bound_sum, torch.float64, "bound_sum"),
                          _dev(status, torch.int32, "status"), _dev(work, name="work"), nbytes,
                          _stream(stream)), "ar_bound")


def ar_bound_noalloc(alpha, bound_sum, status, stream=None):
    """ar_bound without a workspace (scratch in a static device array shared
    by all calls; see include/gbar.h)."""
    _check(lib().ar_bound_noalloc(_dev(alpha, name="alpha"), _dtype_code(alpha), alpha.numel(),
                                  _dev(bound_sum, torch.float64, "bound_sum"),
                                  _dev(status, torch.int32, "status"), _stream(stream)),
           "ar_bound_noalloc")


def ar_select_k_smem_limit() -> int:
    return int(lib().ar_select_k_smem_limit())


def ar_select_k(alpha, bound, K, seed, sel_offset, realization, cmp, trial_cap, idx, stats,
                status, stream=None):
    """K selections from alpha into idx int32[K]; bound f64[>=1] tensor or None."""
    _check(lib().ar_select_k(_dev(alpha, name="alpha"), _dtype_code(alpha), alpha.numel(),
                             _dev(bound, torch.float64, "bound"), K, seed, sel_offset,
                             realization, cmp, trial_cap, _dev(idx, torch.int32, "idx"),
                             _dev(stats, torch.int64, "stats"), _dev(status, torch.int32, "status"),
                             _stream(stream)), "ar_select_k")


def ar_select_batched_workspace_size(B: int) -> int:
    return int(lib().ar_select_batched_workspace_size(B))


class Plan:
    """Owner of an ar_plan handle (see ar_plan_create in include/gbar.h)."""

    def __init__(self, h_offsets, h_out_offsets):
        import numpy as np
        self._off = np.ascontiguousarray(h_offsets, dtype=np.int64)
        self._oo = np.ascontiguousarray(h_out_offsets, dtype=np.int64)
        h = ctypes.c_void_p()
        _check(lib().ar_plan_create(self._off.ctypes.data_as(ctypes.c_void_p),
                                    self._oo.ctypes.data_as(ctypes.c_void_p),
                                    len(self._off) - 1, ctypes.byref(h)), "ar_plan_create")
        self.handle = h.value

    def close(self):
        if self.handle:
            lib().ar_plan_destroy(ctypes.c_void_p(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ar_plan_create(h_offsets, h_out_offsets) -> Plan:
    return Plan(h_offsets, h_out_offsets)


def ar_plan_destroy(plan: Plan):
    plan.close()


def ar_select_batched(alpha_cat, offsets, out_offsets, seed, sel_offset, realization_base, cmp,
                      trial_cap, plan, bound_sum, idx, stats, status, work, stream=None):
    B = offsets.numel() - 1
    nbytes = 0 if work is None else work.numel() * work.element_size()
    _check(lib().ar_select_batched(
        _dev(alpha_cat, name="alpha_cat"), _dtype_code(alpha_cat),
        _dev(offsets, torch.int64, "offsets"), _dev(out_offsets, torch.int64, "out_offsets"), B,
        seed, sel_offset, realization_base, cmp, trial_cap,
        _plan_ptr(plan), _dev(bound_sum, torch.float64, "bound_sum"), _dev(idx, torch.int32, "idx"),
        _dev(stats, torch.int64, "stats"), _dev(status, torch.int32, "status"),
        _dev(work, name="work"), nbytes, _stream(stream)), "ar_select_batched")


def _plan_ptr(plan):
    if plan is None:
        return None
    return ctypes.c_void_p(plan.handle if isinstance(plan, Plan) else plan)


def ar_bound_batched(alpha_cat, offsets, plan, bound_sum, status, work, stream=None):
    B = offsets.numel() - 1
    nbytes = 0 if work is None else work.numel() * work.element_size()
    _check(lib().ar_bound_batched(
        _dev(alpha_cat, name="alpha_cat"), _dtype_code(alpha_cat),
        _dev(offsets, torch.int64, "offsets"), B, _plan_ptr(plan),
        _dev(bound_sum, torch.float64, "bound_sum"), _dev(status, torch.int32, "status"),
        _dev(work, name="work"), nbytes, _stream(stream)), "ar_bound_batched")


def ar_select_batched_bounded(alpha_cat, offsets, out_offsets, bound, bound_stride, seed,
                              sel_offset, realization_base, cmp, trial_cap, plan, idx, stats,
                              status, work, stream=None):
    B = offsets.numel() - 1
    nbytes = 0 if work is None else work.numel() * work.element_size()
    _check(lib().ar_select_batched_bounded(
        _dev(alpha_cat, name="alpha_cat"), _dtype_code(alpha_cat),
        _dev(offsets, torch.int64, "offsets"), _dev(out_offsets, torch.int64, "out_offsets"), B,
        _dev(bound, torch.float64, "bound"), bound_stride, seed, sel_offset, realization_base,
        cmp, trial_cap, _plan_ptr(plan), _dev(idx, torch.int32, "idx"),
        _dev(stats, torch.int64, "stats"), _dev(status, torch.int32, "status"),
        _dev(work, name="work"), nbytes, _stream(stream)), "ar_select_batched_bounded")


# --------------------------------------------------------------------------
# Convenience wrappers that allocate their outputs
# --------------------------------------------------------------------------
def bound(alpha, stream=None):
    """-> (bound_sum f64[2] tensor, status i32[1] tensor)."""
    dev = alpha.device
    out = torch.empty(2, dtype=torch.float64, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    ws = ar_bound_workspace_size(alpha.numel(), _dtype_code(alpha))
    work = torch.zeros(max(ws, 16), dtype=torch.uint8, device=dev) if ws else None
    ar_bound(alpha, out, st, work, stream)
    return out, st


def select_k(alpha, K, seed=1, sel_offset=0, realization=0, cmp=AR_CMP_F32, bound=None,
             trial_cap=1 << 20, stream=None):
    """-> (idx int32[K], stats int64[3] = trials/accepted/capped, status int32[1])."""
    dev = alpha.device
    idx = torch.empty(K, dtype=torch.int32, device=dev)
    stats = torch.zeros(3, dtype=torch.int64, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    ar_select_k(alpha, bound, K, seed, sel_offset, realization, cmp, trial_cap, idx, stats, st,
                stream)
    return idx, stats, st


def select_batched(alpha_cat, offsets, out_offsets, seed=1, sel_offset=0, realization_base=0,
                   cmp=AR_CMP_F32, trial_cap=1 << 20, plan=None, stream=None):
    """-> (bound_sum f64[B,2], idx int32[sum K], stats int64[3], status int32[1])."""
    dev = alpha_cat.device
    B = offsets.numel() - 1
    bs = torch.empty((B, 2), dtype=torch.float64, device=dev)
    idx = torch.empty(int(out_offsets[-1].item()), dtype=torch.int32, device=dev)
    stats = torch.zeros(3, dtype=torch.int64, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    work = torch.zeros(max(ar_select_batched_workspace_size(B), 16), dtype=torch.uint8,
                       device=dev)
    ar_select_batched(alpha_cat, offsets, out_offsets, seed, sel_offset, realization_base, cmp,
                      trial_cap, plan, bs, idx, stats, st, work, stream)
    return bs, idx, stats, st


def ar_plan_autotune(plan, alpha_cat, offsets, out_offsets, seed, cmp, bound_sum, idx, stats,
                     status, reps=20, stream=None):
    """Times the plan's selection tile candidates on this data and keeps the
    fastest -> (warps per CTA, global share per mille, ns per call)."""
    choice = (ctypes.c_int32 * 3)()
    _check(lib().ar_plan_autotune(
        _plan_ptr(plan), _dev(alpha_cat, name="alpha_cat"), _dtype_code(alpha_cat),
        _dev(offsets, torch.int64, "offsets"), _dev(out_offsets, torch.int64, "out_offsets"),
        seed, cmp, _dev(bound_sum, torch.float64, "bound_sum"), _dev(idx, torch.int32, "idx"),
        _dev(stats, torch.int64, "stats"), _dev(status, torch.int32, "status"), reps, choice,
        _stream(stream)), "ar_plan_autotune")
    return tuple(int(x) for x in choice)


def ar_plan_set_tile(plan, warps_per_cta, global_share_pm):
    """Sets the plan's selection tile (warps per CTA, global share per mille)."""
    _check(lib().ar_plan_set_tile(_plan_ptr(plan), warps_per_cta, global_share_pm),
           "ar_plan_set_tile")


def ar_plan_set_grid(plan, ctas_per_sm, selections_per_item=0):
    """CTAs per SM (0: as many as fit) and selections per home work item
    (0: 64) of the plan's schedule."""
    _check(lib().ar_plan_set_grid(_plan_ptr(plan), ctas_per_sm, selections_per_item),
           "ar_plan_set_grid")


def ar_select_paper(D, bound, K, seed, sel_offset, realization, idx, rejections, stream=None):
    _check(lib().ar_select_paper(
        _dev(D, torch.float32, "D"), D.numel(), _dev(bound, torch.float64, "bound"), K, seed,
        sel_offset, realization, _dev(idx, torch.int32, "idx"),
        _dev(rejections, torch.int64, "rejections"), _stream(stream)), "ar_select_paper")


def ar_select_it_workspace_size(M: int) -> int:
    return int(lib().ar_select_it_workspace_size(M))


def ar_select_it(alpha, K, seed, sel_offset, realization, idx, status, work, stream=None):
    nbytes = 0 if work is None else work.numel() * work.element_size()
    _check(lib().ar_select_it(
        _dev(alpha, name="alpha"), _dtype_code(alpha), alpha.numel(), K, seed, sel_offset,
        realization, _dev(idx, torch.int32, "idx"), _dev(status, torch.int32, "status"),
        _dev(work, name="work"), nbytes, _stream(stream)), "ar_select_it")


def select_paper(D, K, T, seed=1, sel_offset=0, realization=0, stream=None):
    """The paper's election rule -> (idx int32[K], rejections int64[1])."""
    dev = D.device
    idx = torch.empty(K, dtype=torch.int32, device=dev)
    rej = torch.zeros(1, dtype=torch.int64, device=dev)
    bound = torch.tensor([float(T)], dtype=torch.float64, device=dev)
    ar_select_paper(D, bound, K, seed, sel_offset, realization, idx, rej, stream)
    return idx, rej


def select_it(alpha, K, seed=1, sel_offset=0, realization=0, stream=None):
    """Inverse transform -> (idx int32[K], status int32[1])."""
    dev = alpha.device
    idx = torch.empty(K, dtype=torch.int32, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    work = torch.empty(ar_select_it_workspace_size(alpha.numel()), dtype=torch.uint8, device=dev)
    ar_select_it(alpha, K, seed, sel_offset, realization, idx, st, work, stream)
    return idx, st


def bound_batched(alpha_cat, offsets, plan=None, stream=None):
    """-> (bound_sum f64[B,2], status int32[1])."""
    dev = alpha_cat.device
    B = offsets.numel() - 1
    bs = torch.empty((B, 2), dtype=torch.float64, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    work = torch.zeros(max(ar_select_batched_workspace_size(B), 16), dtype=torch.uint8,
                       device=dev)
    ar_bound_batched(alpha_cat, offsets, plan, bs, st, work, stream)
    return bs, st


def select_batched_bounded(alpha_cat, offsets, out_offsets, bound, bound_stride=1, seed=1,
                           sel_offset=0, realization_base=0, cmp=AR_CMP_F32, trial_cap=1 << 20,
                           plan=None, stream=None):
    """-> (idx int32[sum K], stats int64[3], status int32[1])."""
    dev = alpha_cat.device
    B = offsets.numel() - 1
    idx = torch.empty(int(out_offsets[-1].item()), dtype=torch.int32, device=dev)
    stats = torch.zeros(3, dtype=torch.int64, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    work = torch.zeros(max(ar_select_batched_workspace_size(B), 16), dtype=torch.uint8,
                       device=dev)
    ar_select_batched_bounded(alpha_cat, offsets, out_offsets, bound, bound_stride, seed,
                              sel_offset, realization_base, cmp, trial_cap, plan, idx, stats, st,
                              work, stream)
    return idx, stats, st


# --------------------------------------------------------------------------
# SSA
# --------------------------------------------------------------------------
class SsaNet:
    """Owner of an ssa_net handle built from a workloads.Network."""

    def __init__(self, net):
        import numpy as np
        self._arrs = [np.ascontiguousarray(x, dtype=dt) for x, dt in (
            (net.rtype, np.int32), (net.reactants, np.int32), (net.rate, np.float64),
            (net.nu_ptr, np.int32), (net.nu_species, np.int32), (net.nu_delta, np.int32))]
        h = ctypes.c_void_p()
        _check(lib().ssa_net_create(net.n_species, net.M,
                                    *[x.ctypes.data_as(ctypes.c_void_p) for x in self._arrs],
                                    ctypes.byref(h)), "ssa_net_create")
        self.handle = h.value
        self.N, self.M = net.n_species, net.M

    def close(self):
        if self.handle:
            lib().ssa_net_destroy(ctypes.c_void_p(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ssa_net_create(net) -> SsaNet:
    return SsaNet(net)


def ssa_net_destroy(net: SsaNet):
    net.close()


def ssa_step_batched(net, X, a, t, step, nsteps, seed, realization_base, cmp, trial_cap, last,
                     status, trials, stream=None):
    """X int32 [B,N], a f64 [B,M], t f64 [B], step int64 [B], last int32 [B] or None,
    status int32 [B], trials int64 [B] or None (all CUDA tensors)."""
    B = X.shape[0]
    _check(lib().ssa_step_batched(ctypes.c_void_p(net.handle), B, _dev(X, torch.int32, "X"),
                                  _dev(a, torch.float64, "a"), _dev(t, torch.float64, "t"),
                                  _dev(step, torch.int64, "step"), nsteps, seed, realization_base,
                                  cmp, trial_cap, _dev(last, torch.int32, "last"),
                                  _dev(status, torch.int32, "status"),
                                  _dev(trials, torch.int64, "trials"), _stream(stream)),
           "ssa_step_batched")


def ssa_run(net, X0, nsteps, seed=1, realization_base=0, cmp=AR_CMP_F32, trial_cap=1 << 20,
            t=None, step=None, status=None, stream=None):
    """Convenience: copies X0 (numpy or tensor) to the device and runs nsteps.
    -> dict of CUDA tensors X, a, t, step, last, status, trials."""
    import numpy as np
    dev = torch.device("cuda")
    Xd = torch.as_tensor(np.ascontiguousarray(X0, dtype=np.int32)).to(dev).contiguous()
    B = Xd.shape[0]
    out = dict(
        X=Xd,
        a=torch.zeros((B, net.M), dtype=torch.float64, device=dev),
        t=(torch.zeros(B, dtype=torch.float64, device=dev) if t is None
           else torch.as_tensor(t, dtype=torch.float64).to(dev).contiguous()),
        step=(torch.zeros(B, dtype=torch.int64, device=dev) if step is None
              else torch.as_tensor(np.asarray(step).astype(np.int64)).to(dev).contiguous()),
        last=-torch.ones(B, dtype=torch.int32, device=dev),
        status=(torch.zeros(B, dtype=torch.int32, device=dev) if status is None
                else torch.as_tensor(np.asarray(status).astype(np.int32)).to(dev).contiguous()),
        trials=torch.zeros(B, dtype=torch.int64, device=dev))
    ssa_step_batched(net, out["X"], out["a"], out["t"], out["step"], nsteps, seed,
                     realization_base, cmp, trial_cap, out["last"], out["status"],
                     out["trials"], stream)
    return out


def ssa_run_until(net, X, a, t, step, t_end, max_steps, seed, realization_base, cmp, trial_cap,
                  sample_times, species, traj, last, status, trials, stream=None):
    """As ssa_step_batched, to the time limit t_end, recording traj[b, k, s] =
    count of species[s] at sample_times[k] (CUDA tensors; sample_times and
    traj may be None)."""
    B = X.shape[0]
    nsamp = 0 if sample_times is None else sample_times.numel()
    nspec = 0 if nsamp == 0 else (net.N if species is None else species.numel())
    _check(lib().ssa_run_until(
        ctypes.c_void_p(net.handle), B, _dev(X, torch.int32, "X"), _dev(a, torch.float64, "a"),
        _dev(t, torch.float64, "t"), _dev(step, torch.int64, "step"), float(t_end), max_steps,
        seed, realization_base, cmp, trial_cap, _dev(sample_times, torch.float64, "sample_times"),
        nsamp, _dev(species, torch.int32, "species"), nspec, _dev(traj, torch.int32, "traj"),
        _dev(last, torch.int32, "last"), _dev(status, torch.int32, "status"),
        _dev(trials, torch.int64, "trials"), _stream(stream)), "ssa_run_until")


def ssa_until(net, X0, t_end, sample_times=None, species=None, max_steps=1 << 40, seed=1,
              realization_base=0, cmp=AR_CMP_F32, trial_cap=1 << 20, t=None, step=None,
              stream=None):
    """Convenience: runs to t_end with samples -> dict of CUDA tensors
    X, a, t, step, last, status, trials, traj [B, nsamp, nspec]."""
    import numpy as np
    dev = torch.device("cuda")
    Xd = torch.as_tensor(np.ascontiguousarray(X0, dtype=np.int32)).to(dev).contiguous()
    B = Xd.shape[0]
    ts = None if sample_times is None else torch.as_tensor(
        np.asarray(sample_times, dtype=np.float64)).to(dev).contiguous()
    sp = None if species is None else torch.as_tensor(
        np.asarray(species, dtype=np.int32)).to(dev).contiguous()
    nspec = net.N if sp is None else sp.numel()
    nsamp = 0 if ts is None else ts.numel()
    out = dict(
        X=Xd, a=torch.zeros((B, net.M), dtype=torch.float64, device=dev),
        t=(torch.zeros(B, dtype=torch.float64, device=dev) if t is None
           else torch.as_tensor(t, dtype=torch.float64).to(dev).contiguous()),
        step=(torch.zeros(B, dtype=torch.int64, device=dev) if step is None
              else torch.as_tensor(np.asarray(step).astype(np.int64)).to(dev).contiguous()),
        last=-torch.ones(B, dtype=torch.int32, device=dev),
        status=torch.zeros(B, dtype=torch.int32, device=dev),
        trials=torch.zeros(B, dtype=torch.int64, device=dev),
        traj=torch.full((B, nsamp, nspec), -1, dtype=torch.int32, device=dev))
    ssa_run_until(net, out["X"], out["a"], out["t"], out["step"], t_end, max_steps, seed,
                  realization_base, cmp, trial_cap, ts, sp, out["traj"] if nsamp else None,
                  out["last"], out["status"], out["trials"], stream)
    return out
