"""CPU checks of the benchmark's bookkeeping: the algorithmic bytes that the
roofline divides by (counted here from the buffers a call reads and writes),
and the kernel-source hash that decides whether a committed ncu summary
still describes the current kernels."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1404_0027_gb300 import workloads as W  # noqa: E402


def _buffers(bt):
    """The arrays of one ar_select_batched call, as the caller holds them."""
    B = bt.B
    K = int(bt.out_offsets[-1])
    return {"alpha": bt.alpha, "offsets": bt.offsets, "out_offsets": bt.out_offsets,
            "idx": np.empty(K, np.int32), "bound_sum": np.empty((B, 2), np.float64)}


def test_algorithmic_bytes_are_the_call_buffers():
    """alpha, both offset arrays read once; indices and {max, sum} written once."""
    for bt in (W.batched_uneven(B=37, seed=3, m_lo=1, m_hi=5000, K=100),
               W.batch_from_vectors([np.ones(5, np.float32), np.zeros(0, np.float32)], [3, 0])):
        buf = _buffers(bt)
        assert bench.algorithmic_bytes(bt) == sum(a.nbytes for a in buf.values())
        # the reduction alone: alpha and the offsets read, {max, sum} written
        assert bench.reduction_bytes(bt) == (buf["alpha"].nbytes + buf["offsets"].nbytes
                                             + buf["bound_sum"].nbytes)


def test_algorithmic_bytes_of_the_benchmark_batches():
    """The figures the roofline uses: the mean over the benchmark's rotating
    4096-realization batches (rank 0's slots)."""
    bts = [W.batched_uneven(B=bench.B_REAL, seed=bench.slot_seed(0, i), m_lo=bench.M_LO,
                            m_hi=bench.M_HI, K=bench.K_B) for i in range(bench.N_SLOTS)]
    assert round(np.mean([bench.algorithmic_bytes(b) for b in bts]) / 1e6, 2) == 52.19
    assert round(np.mean([bench.reduction_bytes(b) for b in bts]) / 1e6, 2) == 47.96
    # together the rotating batches' propensities exceed the 129 MB L2
    assert sum(b.alpha.nbytes for b in bts) > 129e6


def test_code_only_ignores_comments_and_whitespace():
    src = "int f(int x) {\n  return x + 1;  // one more\n}\n/* block\n comment */\n"
    same = "int   f(int x) {\n\treturn x + 1; }  // other words\n\n\n"
    other = "int f(int x) { return x + 2; }"
    assert bench._code_only(src) == bench._code_only(same)
    assert bench._code_only(src) != bench._code_only(other)
    assert "one more" not in bench._code_only(src)


def test_profiled_traffic_follows_the_source_hash(tmp_path, monkeypatch):
    """A summary's traffic is used only when its source hash is the current one."""
    h = bench.kernel_source_hash()
    assert len(h) == 16 and int(h, 16) >= 0
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "cur.md").write_text(f"x\nsource_hash: `{h}`\ntraffic_bytes_per_launch: 1234\n")
    (prof / "old.md").write_text("source_hash: `0000000000000000`\n"
                                 "traffic_bytes_per_launch: 99\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # the hash is taken over the sources under ROOT: keep the repository's
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: h)
    assert bench.profiled_traffic("cur.md") == 1234
    assert bench.profiled_traffic("old.md") is None
    assert bench.profiled_traffic("missing.md") is None
