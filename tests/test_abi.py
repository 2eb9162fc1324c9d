"""The C-ABI library builds, loads and exports every symbol include/gbar.h
declares; the Python binding mirrors exactly those names.  No compute call is
made (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b([A-Za-z_][A-Za-z0-9_ \*]*?)\b([a-z][a-z0-9_]*)\s*\(", src):
            name = m.group(2)
            if name.startswith(("ar_", "ssa_")):
                names.add(name)
    return names


@pytest.fixture(scope="module")
def libgbar():
    from paper_1404_0027_gb300 import build
    try:
        path = build.build()
    except RuntimeError as e:
        pytest.skip(f"nvcc unavailable: {e}")
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(libgbar):
    names = _declared()
    assert {"ar_bound", "ar_select_k", "ar_select_batched"} <= names
    missing = [n for n in names if not hasattr(libgbar, n)]
    assert not missing, missing


def test_binding_mirrors_header(libgbar):
    from paper_1404_0027_gb300 import binding
    assert set(binding.SIGNATURES) == _declared()


def test_version_and_sizes_without_gpu(libgbar):
    from paper_1404_0027_gb300 import binding
    assert binding.lib().ar_version() >= 100
    assert binding.ar_bound_workspace_size(1024, binding.AR_F32) == 0
    assert binding.ar_bound_workspace_size(1 << 20, binding.AR_F32) > 0
    assert binding.ar_select_batched_workspace_size(4096) == 16 + 32 * 4096
