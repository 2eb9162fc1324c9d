"""GPU: the benchmark's throughput probe (libgbar_probe.so, outside the
product ABI) computes what it claims (Philox words of the selection's counter
layout; candidates, gathers and the FP32 acceptance test), checked against
the oracle's Philox on every launched thread."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pr():
    import torch
    from paper_1404_0027_gb300 import build
    build.build()
    from paper_1404_0027_gb300 import probe
    probe.lib()
    assert torch.cuda.is_available()
    return probe


def _words(orc, n, nthreads):
    tid = np.arange(nthreads, dtype=np.uint32)
    i = np.arange(n, dtype=np.uint32)
    c = np.zeros((nthreads, n, 4), dtype=np.uint32)
    c[:, :, 0] = i[None, :]
    c[:, :, 1] = tid[:, None]
    c[:, :, 2] = 7
    w = orc.philox(c.reshape(-1, 4), 1 | (2 << 32))
    return w.reshape(nthreads, n, 4)


def test_probe_philox_words(pr, orc):
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    nthreads = sms * 256
    out = torch.zeros(nthreads, dtype=torch.int32, device="cuda")
    pr.throughput(pr.PHILOX, None, 4, 256, out)
    torch.cuda.synchronize()
    w = _words(orc, 4, nthreads)
    want = np.bitwise_xor.reduce(w.reshape(nthreads, -1), axis=1)
    np.testing.assert_array_equal(out.cpu().numpy().view(np.uint32), want)


@pytest.mark.parametrize("M", [1000, 4096])
def test_probe_gather_accepts(pr, orc, M):
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    nthreads = sms * 256
    rng = np.random.default_rng(M)
    table = rng.random(M, dtype=np.float32)
    out = torch.zeros(nthreads, dtype=torch.int32, device="cuda")
    pr.throughput(pr.PHILOX_GATHER, torch.from_numpy(table).cuda(), 4, 256, out)
    torch.cuda.synchronize()
    w = _words(orc, 4, nthreads).astype(np.uint64)
    acc = np.zeros(nthreads, dtype=np.int64)
    for a, b in ((0, 1), (2, 3)):  # (candidate word, uniform word) of the two trials
        j = (w[:, :, a] * M) >> 32
        u = (w[:, :, b] >> 8).astype(np.float32) * np.float32(2.0 ** -24)
        acc += (u * np.float32(1.0) < table[j]).sum(axis=1)
    np.testing.assert_array_equal(out.cpu().numpy().astype(np.int64), acc)


def test_probe_rejects_bad_arguments(pr):
    import torch
    out = torch.zeros(16, dtype=torch.int32, device="cuda")
    with pytest.raises(RuntimeError):
        pr.throughput(pr.PHILOX, None, 3, 256, out)   # odd block count
    with pytest.raises(RuntimeError):
        pr.throughput(pr.PHILOX, None, 4, 256, out)   # output too small
    with pytest.raises(RuntimeError):
        pr.throughput(pr.PHILOX_GATHER, None, 4, 256, out)  # no table
