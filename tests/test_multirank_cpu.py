"""The N > 1 path on CPU: two gloo ranks (world size 2).

The batched path shards by realization: rank r takes realizations
[r B, (r + 1) B) with ``realization_base = r B`` (bench.rank_realization_base)
and no data-path collective.  Because the Philox counters are global, the
union of the ranks' results must equal one run over all 2 B realizations
(checked with the oracle, which the GPU path matches bit for bit); the
timing and count reductions (bench.reduce_max / reduce_sum) must give the
slowest rank's time and the job's total.
"""
import os
import socket

import numpy as np
import pytest

from paper_1404_0027_gb300 import workloads as W

B = 12


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    import bench
    import oracle

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    full = W.batched_uneven(B=world * B, seed=77, m_lo=8, m_hi=600, K=20)
    lo, hi = rank * B, (rank + 1) * B
    mine = W.batch_from_vectors([full.alpha[full.offsets[b]:full.offsets[b + 1]]
                                 for b in range(lo, hi)], [20] * B)
    base = bench.rank_realization_base(rank, B)
    bs, idx, stats, st = oracle.select_batched(mine, seed=5, realization_base=base)
    t_max = bench.reduce_max(float(rank + 1), dist, "cpu")
    n_all = bench.reduce_sum(float(stats[1]), dist, "cpu")
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), idx=idx, bs=bs, t_max=t_max,
             n_all=n_all, accepted=int(stats[1]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_realizations(tmp_path, orc):
    mp = pytest.importorskip("torch.multiprocessing")
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, str(tmp_path)))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=240)
        assert p.exitcode == 0
    res = [np.load(tmp_path / f"rank{r}.npz") for r in range(world)]
    full = W.batched_uneven(B=world * B, seed=77, m_lo=8, m_hi=600, K=20)
    bs, idx, stats, _ = orc.select_batched(full, seed=5, realization_base=0)
    np.testing.assert_array_equal(np.concatenate([r["idx"] for r in res]), idx)
    np.testing.assert_array_equal(np.concatenate([r["bs"] for r in res]), bs)
    for r in res:
        assert float(r["t_max"]) == 2.0                        # the slowest rank
        assert float(r["n_all"]) == float(stats[1]) == world * B * 20
