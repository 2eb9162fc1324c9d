"""Binding of libgbar_probe.so, the benchmark's throughput probes (the
practical ceilings of Philox trial generation, alone and with random gathers).

A measurement aid, kept out of libgbar's C ABI: only the benchmark and its
test use it.  Built by ``paper_1404_0027_gb300.build.build()`` next to this
file.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgbar_probe.so")

PHILOX = 0
PHILOX_GATHER = 1

_lock = threading.Lock()
_lib = None


def lib():
    """Load libgbar_probe.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        with _lock:
            if _lib is None:
                if not os.path.exists(LIB_PATH):
                    raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                       "paper_1404_0027_gb300.build.build() (needs nvcc)")
                L = ctypes.CDLL(LIB_PATH)
                f = L.gbar_probe_throughput
                f.restype = ctypes.c_int
                f.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32,
                              ctypes.c_uint32, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
                _lib = L
    return _lib


def throughput(mode, table, blocks_per_thread, threads_per_sm, out, stream=None):
    """Launches the probe on `stream` (timed by the caller).  table: CUDA
    float32 tensor or None; out: CUDA int32 tensor, one word per thread."""
    import torch
    M = 0 if table is None else table.numel()
    tp = None if table is None else ctypes.c_void_p(table.data_ptr())
    if table is not None and (table.dtype != torch.float32 or not table.is_cuda):
        raise RuntimeError("table must be a CUDA float32 tensor")
    if out.dtype != torch.int32 or not out.is_cuda:
        raise RuntimeError("out must be a CUDA int32 tensor")
    s = torch.cuda.current_stream() if stream is None else stream
    rc = lib().gbar_probe_throughput(mode, tp, M, blocks_per_thread, threads_per_sm,
                                     ctypes.c_void_p(out.data_ptr()), out.numel(),
                                     ctypes.c_void_p(s.cuda_stream))
    if rc != 0:
        raise RuntimeError(f"gbar_probe_throughput returned {rc}")
