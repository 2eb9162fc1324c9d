"""CPU oracle for parallel acceptance-rejection next-reaction selection.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The oracle shares no code
with the CUDA library (``oracle.c`` is compiled on its own with gcc) and never
imports it.  ``law.py`` holds the closed-form and counting laws that pin it.

Python wrappers here only marshal numpy arrays into ``liboracle.so``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
          "-std=gnu11", "-fopenmp", "-Wall", "-Wno-unknown-pragmas"]

ST_BAD_ALPHA = 1
ST_ALL_ZERO = 2
ST_TRIAL_CAP = 4
ST_BAD_BOUND = 8
ST_ABSORBED = 16

CMP_F32 = 0
CMP_F64 = 1


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, no FMA contraction)."""
    with _lock:
        if (force or not os.path.exists(_LIB)
                or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)):
            tmp = _LIB + ".tmp%d" % os.getpid()
            subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        vp, i64, u64, u32, i32, dbl = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64,
                                       ctypes.c_uint32, ctypes.c_int, ctypes.c_double)
        L.orc_philox4x32_10.argtypes = [vp, u64, vp]
        L.orc_philox_many.argtypes = [vp, i64, u64, vp]
        L.orc_bound.argtypes = [vp, i32, i64, vp]
        L.orc_bound.restype = u32
        L.orc_select_ar.argtypes = [vp, i32, i64, dbl, i64, u64, u64, u32, i32, u64, vp, vp, i32]
        L.orc_select_ar.restype = u32
        L.orc_select_runs.argtypes = [vp, i32, i64, dbl, i64, u64, u64, u32, i32, u64, vp, vp]
        L.orc_select_runs.restype = u32
        L.orc_select_batched.argtypes = [vp, i32, vp, vp, i64, u64, u64, u32, i32, u64,
                                         vp, vp, vp, i32]
        L.orc_select_batched.restype = u32
        L.orc_select_batched_bounded.argtypes = [vp, i32, vp, vp, i64, vp, i64, u64, u64, u32,
                                                 i32, u64, vp, vp, i32]
        L.orc_select_batched_bounded.restype = u32
        L.orc_select_it.argtypes = [vp, i32, i64, i64, u64, u64, u32, vp, i32]
        L.orc_select_it.restype = u32
        L.orc_it_prefix.argtypes = [vp, i32, i64, vp]
        L.orc_it_prefix.restype = u32
        L.orc_select_paper.argtypes = [vp, i64, ctypes.c_float, i64, u64, u64, u32, vp, vp, i32]
        L.orc_select_paper.restype = u32
        L.orc_ssa.argtypes = [ctypes.c_int32, ctypes.c_int32, vp, vp, vp, vp, vp, vp, i64,
                              vp, vp, vp, i64, u64, u32, i32, u64, vp, vp, vp, vp, i32]
        L.orc_ssa.restype = None
        L.orc_ssa_until.argtypes = [ctypes.c_int32, ctypes.c_int32, vp, vp, vp, vp, vp, vp, i64,
                                    vp, vp, vp, ctypes.c_double, i64, u64, u32, i32, u64, vp,
                                    i32, vp, i32, vp, vp, vp, vp, i32]
        L.orc_ssa_until.restype = None
        L.orc_num_threads_available.restype = i32
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _dtype_code(a: np.ndarray) -> int:
    if a.dtype == np.float32:
        return 0
    if a.dtype == np.float64:
        return 1
    raise TypeError("alpha must be float32 or float64")


def num_threads_available() -> int:
    return int(lib().orc_num_threads_available())


def philox(counters: np.ndarray, seed: int) -> np.ndarray:
    """Philox4x32-10 of an [n, 4] uint32 counter array -> [n, 4] uint32."""
    c = np.ascontiguousarray(counters, dtype=np.uint32).reshape(-1, 4)
    out = np.zeros_like(c)
    lib().orc_philox_many(_ptr(c), c.shape[0], ctypes.c_uint64(seed), _ptr(out))
    return out


def bound(alpha: np.ndarray):
    """-> (max, sum, status) of one propensity vector."""
    a = np.ascontiguousarray(alpha)
    out = np.zeros(2, dtype=np.float64)
    st = lib().orc_bound(_ptr(a), _dtype_code(a), a.size, _ptr(out))
    return float(out[0]), float(out[1]), int(st)


def select_ar(alpha, K, seed=1, sel_offset=0, realization=0, cmp=CMP_F64,
              bound_value=None, trial_cap=1 << 20, nthreads=1):
    """-> (idx int32[K], stats uint64[3] = trials/accepted/capped, status)."""
    a = np.ascontiguousarray(alpha)
    T = bound(a)[0] if bound_value is None else float(bound_value)
    idx = np.zeros(K, dtype=np.int32)
    stats = np.zeros(3, dtype=np.uint64)
    st = lib().orc_select_ar(_ptr(a), _dtype_code(a), a.size, T, K, ctypes.c_uint64(seed),
                             ctypes.c_uint64(sel_offset), realization, cmp,
                             ctypes.c_uint64(trial_cap), _ptr(idx), _ptr(stats), nthreads)
    return idx, stats, int(st)


def select_runs(alpha, K, seed=1, sel_offset=0, realization=0, cmp=CMP_F64,
                bound_value=None, trial_cap=1 << 20):
    """Selections sel_offset .. sel_offset + K - 1 drawn from runs of 64 (the
    batched entry points' stream) -> (idx int32[K], stats uint64[3], status)."""
    a = np.ascontiguousarray(alpha)
    T = bound(a)[0] if bound_value is None else float(bound_value)
    idx = np.zeros(K, dtype=np.int32)
    stats = np.zeros(3, dtype=np.uint64)
    st = lib().orc_select_runs(_ptr(a), _dtype_code(a), a.size, T, K, ctypes.c_uint64(seed),
                               ctypes.c_uint64(sel_offset), realization, cmp,
                               ctypes.c_uint64(trial_cap), _ptr(idx), _ptr(stats))
    return idx, stats, int(st)


def select_batched(batch, seed=1, sel_offset=0, realization_base=0, cmp=CMP_F32,
                   trial_cap=1 << 20, nthreads=1):
    """-> (bound_sum float64[B,2], idx int32[sum K], stats uint64[3], status)."""
    a = np.ascontiguousarray(batch.alpha)
    off = np.ascontiguousarray(batch.offsets, dtype=np.int64)
    oo = np.ascontiguousarray(batch.out_offsets, dtype=np.int64)
    B = len(off) - 1
    bs = np.zeros((B, 2), dtype=np.float64)
    idx = np.zeros(int(oo[-1]), dtype=np.int32)
    stats = np.zeros(3, dtype=np.uint64)
    st = lib().orc_select_batched(_ptr(a), _dtype_code(a), _ptr(off), _ptr(oo), B,
                                  ctypes.c_uint64(seed), ctypes.c_uint64(sel_offset),
                                  realization_base, cmp, ctypes.c_uint64(trial_cap),
                                  _ptr(bs), _ptr(idx), _ptr(stats), nthreads)
    return bs, idx, stats, int(st)


def select_batched_bounded(batch, bound, stride=1, seed=1, sel_offset=0, realization_base=0,
                           cmp=CMP_F32, trial_cap=1 << 20, nthreads=1):
    """Batched selection with the caller's bounds T_b = bound[b * stride]
    -> (idx int32[sum K], stats uint64[3], status)."""
    a = np.ascontiguousarray(batch.alpha)
    off = np.ascontiguousarray(batch.offsets, dtype=np.int64)
    oo = np.ascontiguousarray(batch.out_offsets, dtype=np.int64)
    bd = np.ascontiguousarray(bound, dtype=np.float64)
    B = len(off) - 1
    idx = np.zeros(int(oo[-1]), dtype=np.int32)
    stats = np.zeros(3, dtype=np.uint64)
    st = lib().orc_select_batched_bounded(_ptr(a), _dtype_code(a), _ptr(off), _ptr(oo), B,
                                          _ptr(bd), stride, ctypes.c_uint64(seed),
                                          ctypes.c_uint64(sel_offset), realization_base, cmp,
                                          ctypes.c_uint64(trial_cap), _ptr(idx), _ptr(stats),
                                          nthreads)
    return idx, stats, int(st)


def select_it(alpha, K, seed=1, sel_offset=0, realization=0, nthreads=1):
    a = np.ascontiguousarray(alpha)
    idx = np.zeros(K, dtype=np.int32)
    st = lib().orc_select_it(_ptr(a), _dtype_code(a), a.size, K, ctypes.c_uint64(seed),
                             ctypes.c_uint64(sel_offset), realization, _ptr(idx), nthreads)
    return idx, int(st)


def it_prefix(alpha):
    """Running sums of the inverse transform: S_j = the exact sum of
    alpha_0..alpha_j (each term rounded down to 2^-96 of the maximum's
    binade), rounded once to FP64 -> (S float64[M], status)."""
    a = np.ascontiguousarray(alpha)
    S = np.zeros(a.size, dtype=np.float64)
    st = lib().orc_it_prefix(_ptr(a), _dtype_code(a), a.size, _ptr(S))
    return S, int(st)


def select_paper(D, K, T=None, seed=1, sel_offset=0, realization=0, nthreads=1):
    """The paper's election/argmin rule in FP32 -> (idx, rejections)."""
    d = np.ascontiguousarray(D, dtype=np.float32)
    T = float(d.max()) if T is None else float(T)
    idx = np.zeros(K, dtype=np.int32)
    rej = np.zeros(1, dtype=np.uint64)
    lib().orc_select_paper(_ptr(d), d.size, ctypes.c_float(T), K, ctypes.c_uint64(seed),
                           ctypes.c_uint64(sel_offset), realization, _ptr(idx), _ptr(rej),
                           nthreads)
    return idx, int(rej[0])


def ssa(net, X, t=None, step=None, nsteps=1, seed=1, realization_base=0, cmp=CMP_F64,
        trial_cap=1 << 20, status=None, nthreads=1, want_a=False):
    """Advance B realizations by nsteps SSA steps (in place on copies).

    -> dict(X, t, step, last, status, a (optional), trials)."""
    X = np.array(X, dtype=np.int32, order="C", copy=True)
    B = X.shape[0]
    t = np.zeros(B, dtype=np.float64) if t is None else np.array(t, dtype=np.float64)
    step = (np.zeros(B, dtype=np.uint64) if step is None
            else np.array(step, dtype=np.uint64))
    status = (np.zeros(B, dtype=np.uint32) if status is None
              else np.array(status, dtype=np.uint32))
    last = -np.ones(B, dtype=np.int32)
    trials = np.zeros(B, dtype=np.uint64)
    a_out = np.zeros((B, net.M), dtype=np.float64) if want_a else None
    arrs = [np.ascontiguousarray(x) for x in (net.rtype, net.reactants, net.rate, net.nu_ptr,
                                              net.nu_species, net.nu_delta)]
    lib().orc_ssa(net.n_species, net.M, *[_ptr(x) for x in arrs], B, _ptr(X), _ptr(t),
                  _ptr(step), nsteps, ctypes.c_uint64(seed), realization_base, cmp,
                  ctypes.c_uint64(trial_cap), _ptr(last), _ptr(status), _ptr(a_out),
                  _ptr(trials), nthreads)
    out = dict(X=X, t=t, step=step, last=last, status=status, trials=trials)
    if want_a:
        out["a"] = a_out
    return out


ST_T_END = 128


def ssa_until(net, X, t_end, t=None, step=None, max_steps=1 << 40, seed=1, realization_base=0,
              cmp=CMP_F64, trial_cap=1 << 20, status=None, sample_times=None, species=None,
              nthreads=1):
    """Run B realizations to the time limit t_end with trajectory samples.

    -> dict(X, t, step, last, status, trials, traj [B, nsamp, nspec])."""
    X = np.array(X, dtype=np.int32, order="C", copy=True)
    B = X.shape[0]
    t = np.zeros(B, dtype=np.float64) if t is None else np.array(t, dtype=np.float64)
    step = (np.zeros(B, dtype=np.uint64) if step is None
            else np.array(step, dtype=np.uint64))
    status = (np.zeros(B, dtype=np.uint32) if status is None
              else np.array(status, dtype=np.uint32))
    last = -np.ones(B, dtype=np.int32)
    trials = np.zeros(B, dtype=np.uint64)
    st_times = (np.zeros(0) if sample_times is None
                else np.ascontiguousarray(sample_times, dtype=np.float64))
    sp = None if species is None else np.ascontiguousarray(species, dtype=np.int32)
    nspec = net.n_species if sp is None else sp.size
    traj = np.full((B, st_times.size, nspec), -1, dtype=np.int32)
    arrs = [np.ascontiguousarray(x) for x in (net.rtype, net.reactants, net.rate, net.nu_ptr,
                                              net.nu_species, net.nu_delta)]
    lib().orc_ssa_until(net.n_species, net.M, *[_ptr(x) for x in arrs], B, _ptr(X), _ptr(t),
                        _ptr(step), float(t_end), max_steps, ctypes.c_uint64(seed),
                        realization_base, cmp, ctypes.c_uint64(trial_cap), _ptr(st_times),
                        st_times.size, _ptr(sp), nspec, _ptr(traj), _ptr(last), _ptr(status),
                        _ptr(trials), nthreads)
    return dict(X=X, t=t, step=step, last=last, status=status, trials=trials, traj=traj)
