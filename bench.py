#!/usr/bin/env python3
"""Benchmark of the batched AR selection hot path on GB300.

One step = one ``ar_select_batched`` call (bound/sum reduction, Philox
trials, gathers, ballot compaction and output for every realization; one
kernel when the batch's plan keeps every realization in a CTA home list,
else two) on the batched-uneven workload: B = 4096 realizations, M_b log-uniform in
[64, 16384], alpha FP32 Exponential(1), K_b = 256 selections each, FP32
comparison.  The launch is replayed from a captured CUDA graph.  Inputs are
rotated over several independently drawn batches whose total size exceeds
the 129 MB L2, so every step streams its propensities from HBM.  The
headline throughput keeps several independent batches in flight
(consecutive steps rotate over 2-4 streams, each batch with its own plan;
the launch pattern -- tile, CTAs per SM, calls in flight -- is picked by
timing): one call's tail and reduction overlap another call's selections.
The rate with one call at a time is reported beside it.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle on
the host cores instead (the comparison arm).
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import re
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1404_0027_gb300 import accuracy as A  # noqa: E402
from paper_1404_0027_gb300 import workloads as W  # noqa: E402



def launches_per_call(global_share_pm: int) -> int:
    """Kernels one ar_select_batched call on aligned FP32 data enqueues: one
    when the plan leaves no realization to the global queue (each CTA reduces
    its own realizations, then selects them), else two (the reduction, then
    the selections)."""
    return 1 if global_share_pm == 0 else 2


METRIC = "accepted selections/sec and HBM-roofline fraction, FP32-batched vs FP64-plain at TV<=1e-3"
UNIT = "selections/s"
B_REAL, K_B, M_LO, M_HI = 4096, 256, 64, 16384
N_SLOTS = 6                      # 6 x ~52 MB > 129 MB L2
SEED = 1
ACC_SAMPLES = 10_000_000         # selections per accuracy comparison (FP32 vs FP64)
PHILOX_IMAD_PER_BLOCK = 40       # 10 rounds x 2 multiplies x (hi + lo)
IMAD_PER_SM_CLK = 64             # 32-bit integer multiply-add issue rate per SM per clock


def workload_config():
    return {"workload": f"batched-uneven: B={B_REAL} realizations, M_b log-uniform "
                        f"[{M_LO},{M_HI}], alpha FP32 Exponential(1), K_b={K_B}, FP32 comparison, "
                        "one ar_select_batched call per step from a CUDA graph (one kernel: "
                        "each CTA reduces then selects its own realizations), "
                        "selection tiles picked per batch by ar_plan_autotune; consecutive "
                        "steps rotate over several streams (independent batches, one plan "
                        "each), so several calls are in flight (batches_in_flight)",
            "B": B_REAL, "K_b": K_B, "M_range": [M_LO, M_HI], "cmp": "f32", "seed": SEED,
            "l2": f"inputs rotated over {N_SLOTS} independently drawn batches "
                  f"(~{N_SLOTS * 52} MB > 129 MB L2)"}


def slot_seed(rank: int, slot: int) -> int:
    return 300 + 1000 * rank + slot


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured", d
    except Exception:
        return 6800.0, "fallback", {}


def _code_only(text: str) -> str:
    """C/C++/CUDA source without comments and with whitespace collapsed, so
    that the hash follows the code, not its documentation.  (Comment markers
    inside string literals would be stripped too; the kernel sources have
    none that matter.)"""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_source_hash() -> str:
    """Hash of the kernel sources' code (comments and whitespace ignored)."""
    h = hashlib.sha256()
    for f in sorted(glob.glob(os.path.join(ROOT, "paper_1404_0027_gb300", "csrc", "*"))):
        with open(f, encoding="utf-8") as fh:
            h.update(os.path.basename(f).encode())
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def profiled_traffic(name: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", name)
    try:
        txt = open(path).read()
    except OSError:
        return None
    vals = {}
    for line in txt.splitlines():
        if ":" in line and line.strip().startswith(("traffic_bytes_per_launch", "source_hash")):
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("source_hash") != kernel_source_hash():
        return None
    try:
        return float(vals["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.samples = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50", "-i", gpu_id], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                text=True)
        except OSError:
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == 9:
                self.samples.append((time.time(), parts))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0, t1):
        inside = [s for t, s in self.samples if t0 <= t <= t1]
        if not inside and self.samples:
            inside = [min(self.samples, key=lambda x: min(abs(x[0] - t0), abs(x[0] - t1)))[1]]
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(s[1]) for s in inside if num(s[1]) is not None]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in inside:
            for n, v in zip(names, s[5:9]):
                if v.strip().lower() in ("active", "1"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": num(inside[0][2]), "reasons": sorted(reasons),
                "samples": len(inside), "power_w_max": max((num(s[3]) or 0) for s in inside)}


def gpu_id_for(torch, dev) -> str:
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        return vis.split(",")[dev.index or 0] if vis else str(dev.index or 0)


# --------------------------------------------------------------------------
# Multi-rank helpers (one process per GPU; realizations shard by rank, no
# data-path collective -- only the timing and count reductions below)
# --------------------------------------------------------------------------
def rank_realization_base(rank: int, B: int) -> int:
    """Philox realization ids of rank r: [r B, (r + 1) B), disjoint across ranks,
    so every rank's streams equal those of one run over all realizations."""
    return rank * B


def reduce_max(value: float, dist, device) -> float:
    """Max over ranks (the slowest rank's time defines the job's time)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(value: float, dist, device) -> float:
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t)
    return float(t.item())


def algorithmic_bytes(bt) -> int:
    """alpha read once + both offset arrays read + indices and (max, sum) written."""
    return 4 * int(bt.offsets[-1]) + 16 * (bt.B + 1) + 4 * int(bt.out_offsets[-1]) + 16 * bt.B


def reduction_bytes(bt) -> int:
    """The reduction step: alpha and the offsets read once, (max, sum) written."""
    return 4 * int(bt.offsets[-1]) + 8 * (bt.B + 1) + 16 * bt.B


def probe_peaks(dev, stream):
    """Practical ceilings of trial generation on this GPU (Philox4x32-10
    blocks/s): Philox alone, and Philox with both trials' gathers and the
    FP32 test from a 48 MB table (L2-resident) and a 16 KB table (L1).
    Each probe launch is timed with CUDA events on `stream`, median of 5."""
    import torch
    from paper_1404_0027_gb300 import probe
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    tps, n = 1024, 2048
    out = torch.empty(sms * tps, dtype=torch.int32, device=dev)
    big = torch.rand(12 << 20, dtype=torch.float32, device=dev)
    small = torch.rand(4096, dtype=torch.float32, device=dev)
    res = {}
    for name, mode, table in (("philox_only", probe.PHILOX, None),
                              ("philox_gather_l2_48MB", probe.PHILOX_GATHER, big),
                              ("philox_gather_l1_16KB", probe.PHILOX_GATHER, small)):
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            for _ in range(2):
                probe.throughput(mode, table, n, tps, out, stream)
            ms = []
            for _ in range(5):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                probe.throughput(mode, table, n, tps, out, stream)
                e1.record(stream)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
        res[name] = sms * tps * n / (float(np.median(ms)) * 1e-3)
    res["unit"] = "Philox4x32-10 blocks/s"
    res["probe"] = f"gbar_probe_throughput, {tps} threads/SM x {n} blocks per thread"
    return res


# --------------------------------------------------------------------------
# CPU oracle arm
# --------------------------------------------------------------------------
def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    bt = W.batched_uneven(B=B_REAL, seed=slot_seed(0, 0), m_lo=M_LO, m_hi=M_HI, K=K_B)
    # size one step so that warmup + steps finish within about two minutes
    t = time.perf_counter()
    probe = W.batch_from_vectors([bt.alpha[bt.offsets[b]:bt.offsets[b + 1]] for b in range(64)],
                                 [K_B] * 64)
    oracle.select_batched(probe, seed=SEED, nthreads=cores)
    per_real = (time.perf_counter() - t) / 64
    budget = 120.0 / max(1, args.steps + args.warmup)
    nb = int(max(16, min(B_REAL, budget / max(per_real, 1e-9))))
    sub = W.batch_from_vectors([bt.alpha[bt.offsets[b]:bt.offsets[b + 1]] for b in range(nb)],
                               [K_B] * nb)
    for _ in range(args.warmup):
        oracle.select_batched(sub, seed=SEED, nthreads=cores)
    t0 = time.perf_counter()
    acc = 0
    for _ in range(args.steps):
        _, _, st, _ = oracle.select_batched(sub, seed=SEED, nthreads=cores)
        acc += int(st[1])
    dt = time.perf_counter() - t0
    value = acc / dt
    sample = (f"first {nb} of the {B_REAL} realizations of the batched workload per step "
              f"({nb * K_B} selections, oracle C, FP32 comparison, OpenMP over realizations)")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic", "config": workload_config(),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def cpu_baseline_leg():
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    bt = W.batched_uneven(B=B_REAL, seed=slot_seed(0, 0), m_lo=M_LO, m_hi=M_HI, K=K_B)
    t0 = time.perf_counter()
    reps = 0
    acc = 0
    while True:
        _, _, st, _ = oracle.select_batched(bt, seed=SEED, nthreads=cores)
        acc += int(st[1])
        reps += 1
        if time.perf_counter() - t0 > 10.0:
            break
    dt = time.perf_counter() - t0
    # one host thread, about 3 s
    t1 = time.perf_counter()
    reps1 = acc1 = 0
    while True:
        _, _, st, _ = oracle.select_batched(bt, seed=SEED, nthreads=1)
        acc1 += int(st[1])
        reps1 += 1
        if time.perf_counter() - t1 > 3.0:
            break
    dt1 = time.perf_counter() - t1
    return {"value": acc / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{reps} pass(es) over the full batched workload (slot 0: {B_REAL} "
                      f"realizations, {B_REAL * K_B} selections), oracle C, FP32 comparison, "
                      f"OpenMP over realizations, {dt:.1f} s",
            "single_thread_value": acc1 / dt1,
            "single_thread_sample": f"{reps1} pass(es) over the same workload on one host "
                                    f"thread, {dt1:.1f} s"}


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ssa", action="store_true")
    ap.add_argument("--ssa-steps", type=int, default=10_000)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    from paper_1404_0027_gb300 import build
    build.build()
    from paper_1404_0027_gb300 import binding as gb

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    # ---- data: N_SLOTS batches, resident in HBM --------------------------
    slots = []
    for i in range(N_SLOTS):
        bt = W.batched_uneven(B=B_REAL, seed=slot_seed(rank, i), m_lo=M_LO, m_hi=M_HI, K=K_B)
        s = {"bt": bt,
             "alpha": torch.from_numpy(bt.alpha).to(dev),
             "off": torch.from_numpy(bt.offsets).to(dev),
             "oo": torch.from_numpy(bt.out_offsets).to(dev),
             "bs": torch.empty((B_REAL, 2), dtype=torch.float64, device=dev),
             "idx": torch.empty(int(bt.out_offsets[-1]), dtype=torch.int32, device=dev),
             "stats": torch.zeros(3, dtype=torch.int64, device=dev),
             "st": torch.zeros(1, dtype=torch.int32, device=dev),
             "work": torch.zeros(max(gb.ar_select_batched_workspace_size(B_REAL), 16),
                                 dtype=torch.uint8, device=dev),
             # schedule built once per batch shape (host LPT over the CTAs)
             "plan": gb.Plan(bt.offsets, bt.out_offsets)}
        slots.append(s)
    b_base = rank_realization_base(rank, B_REAL)
    stream = torch.cuda.Stream(dev)

    def launch(s, cmp=gb.AR_CMP_F32, idx=None):
        gb.ar_select_batched(s["alpha"], s["off"], s["oo"], SEED, 0, b_base, cmp, 1 << 20,
                             s["plan"],
                             s["bs"], s["idx"] if idx is None else idx, s["stats"], s["st"],
                             s["work"], stream)

    # tile shape of the selection kernel per batch, picked by the autotuner
    tuned = []
    for s in slots:
        tuned.append(gb.ar_plan_autotune(s["plan"], s["alpha"], s["off"], s["oo"], SEED,
                                         gb.AR_CMP_F32, s["bs"], s["idx"], s["stats"], s["st"],
                                         reps=10, stream=stream))
    with torch.cuda.stream(stream):
        launch(slots[0])
    stream.synchronize()
    bt0 = slots[0]["bt"]
    g_idx = slots[0]["idx"].cpu().numpy()
    # FP32 vs FP64 comparison on identical streams (paired mismatch >= paired
    # TV), over N_ACC_CALLS calls with disjoint selection ids (>= 10^7
    # selections); cell of a result = (realization b, index j), the sentinel
    # M_b included
    n_acc = ACC_SAMPLES // (B_REAL * K_B) + 1
    b_of = np.repeat(np.arange(B_REAL, dtype=np.int64), np.diff(bt0.out_offsets))
    cell0 = (bt0.offsets[:-1] + np.arange(B_REAL))[b_of]
    ncells = int(bt0.offsets[-1]) + B_REAL
    keys = {gb.AR_CMP_F32: [], gb.AR_CMP_F64: []}
    acc_idx = torch.empty_like(slots[0]["idx"])
    for c in range(n_acc):
        for cmp in keys:
            with torch.cuda.stream(stream):
                gb.ar_select_batched(slots[0]["alpha"], slots[0]["off"], slots[0]["oo"], SEED,
                                     c * K_B, b_base, cmp, 1 << 20, slots[0]["plan"],
                                     slots[0]["bs"], acc_idx, slots[0]["stats"], slots[0]["st"],
                                     slots[0]["work"], stream)
            stream.synchronize()
            keys[cmp].append(cell0 + acc_idx.cpu().numpy())
    acc_batched = dict(A.paired(np.concatenate(keys[gb.AR_CMP_F32]),
                                np.concatenate(keys[gb.AR_CMP_F64]), ncells),
                       sample=f"{n_acc} ar_select_batched calls on one batch, selection ids "
                              f"c*{K_B} .. c*{K_B}+{K_B - 1}, FP32 and FP64 comparison")
    del keys

    # ---- CUDA graphs, one per slot (recaptured whenever a plan's tile
    # changes: the launch shape is part of the graph) ----------------------
    def capture():
        gs = []
        for s in slots:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream):
                launch(s)
            gs.append(g)
        torch.cuda.synchronize()
        return gs

    graphs = capture()
    K = args.steps
    pipe = [stream] + [torch.cuda.Stream(dev) for _ in range(3)]  # up to 4 calls in flight

    def replay(gs, nstreams, n, evs=None):
        """n steps, step i on stream i % nstreams after the events e[0]."""
        for i in range(n):
            st = pipe[i % nstreams]
            with torch.cuda.stream(st):
                if evs:
                    evs[i][0].record(st)
                gs[i % N_SLOTS].replay()
                if evs:
                    evs[i][1].record(st)

    def join(nstreams):
        for st in pipe[1:nstreams]:
            j = torch.cuda.Event()
            j.record(st)
            pipe[0].wait_event(j)

    def rate_us(gs, nstreams, n):
        """Microseconds per step of n steps (after a short warm-up)."""
        replay(gs, nstreams, 2 * N_SLOTS)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(pipe[0])
        for st in pipe[1:nstreams]:
            st.wait_event(e0)
        replay(gs, nstreams, n)
        join(nstreams)
        e1.record(pipe[0])
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n * 1e3

    def timed_run(gs, nstreams, nvtx):
        """K steps, step i on stream i % nstreams (batches are independent and
        each slot has its own plan, so two calls may overlap); per-step
        events only on one stream.  -> (ms, per-step ms, accepted, trials,
        status)"""
        # the warm-up replays run on the pipe streams: let every one of them
        # finish before the counters are cleared on torch's current stream,
        # so that no warm-up CTA adds to the timed region's counts
        torch.cuda.synchronize()
        for s in slots:
            s["stats"].zero_()
            s["st"].zero_()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(K if nstreams == 1 else 0)]
        ev_all = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        if nvtx:
            torch.cuda.nvtx.range_push("timed")  # lets a profiler select the timed launches
        ev_all[0].record(pipe[0])
        for st in pipe[1:nstreams]:
            st.wait_event(ev_all[0])
        replay(gs, nstreams, K, ev)
        join(nstreams)
        ev_all[1].record(pipe[0])
        torch.cuda.synchronize()
        if nvtx:
            torch.cuda.nvtx.range_pop()
        if dist:
            dist.barrier()
        acc = sum(int(s["stats"][1].item()) for s in slots)
        tri = sum(int(s["stats"][0].item()) for s in slots)
        stt = 0
        for s in slots:
            stt |= int(s["st"].item())
        return (ev_all[0].elapsed_time(ev_all[1]),
                np.array([a.elapsed_time(b) for a, b in ev]), acc, tri, stt)

    sampler = ClockSampler(gpu_id_for(torch, dev))
    time.sleep(0.3)
    t_wall0 = time.time()
    # one call at a time (per-step latency), with the autotuned tiles
    replay(graphs, 1, args.warmup)
    ms1, kern_ms, acc1, trials1, st1 = timed_run(graphs, 1, nvtx=True)
    # several batches in flight: the launch pattern is picked again by
    # timing -- smaller CTAs, or fewer CTAs per SM (ar_plan_set_grid), let a
    # call's kernel share the SMs with the other calls' kernels
    pipe_tiles = []
    best = None
    n_try = max(1, min(K, 600))
    # (tile, CTAs per SM, selections per item, calls in flight)
    for cand in (("autotuned", 0, 0, 2), ((16, 0), 0, 0, 2), ((8, 300), 0, 0, 2),
                 ((8, 0), 0, 0, 2), ((32, 0), 0, 0, 2), ((16, 0), 1, 0, 3), ((16, 0), 1, 0, 4),
                 ((8, 0), 2, 0, 4), ((16, 0), 0, 256, 2), ((16, 0), 1, 128, 4),
                 ((16, 0), 1, 256, 3), ((16, 0), 1, 256, 4), ((8, 0), 2, 256, 4)):
        tile, grid, items, nst = cand
        for s, t in zip(slots, tuned):
            gb.ar_plan_set_tile(s["plan"], *(t[:2] if tile == "autotuned" else tile))
            gb.ar_plan_set_grid(s["plan"], grid, items)
        us = rate_us(capture(), nst, n_try)
        pipe_tiles.append({"tile": tile if tile == "autotuned" else list(tile),
                           "ctas_per_sm": grid if grid else "as many as fit",
                           "selections_per_item": items if items else 64,
                           "in_flight": nst, "us_per_step": us})
        if best is None or us < best[1]:
            best = (cand, us)
    best_tile, best_grid, best_items, in_flight = best[0]
    for s, t in zip(slots, tuned):
        gb.ar_plan_set_tile(s["plan"], *(t[:2] if best_tile == "autotuned" else best_tile))
        gb.ar_plan_set_grid(s["plan"], best_grid, best_items)
    # kernels the headline's K steps launch (step i replays slot i % N_SLOTS)
    shares = [(t[1] if best_tile == "autotuned" else best_tile[1]) for t in tuned]
    launches_timed = sum(launches_per_call(shares[i % N_SLOTS]) for i in range(K))
    graphs = capture()
    replay(graphs, in_flight, args.warmup)
    elapsed_ms, _, accepted, trials, status = timed_run(graphs, in_flight, nvtx=False)
    status |= st1
    t_wall1 = time.time()
    # the rest (kernels timed alone, end to end) runs one call at a time:
    # back to the autotuned tiles
    for s, t in zip(slots, tuned):
        gb.ar_plan_set_tile(s["plan"], *t[:2])
        gb.ar_plan_set_grid(s["plan"], 0, 0)
    time.sleep(0.2)
    sampler.stop()
    # every step selects B x K_b indices; the counters of the timed region
    # must say exactly that (no selection hits the trial cap on this data)
    sel_per_step = B_REAL * K_B
    for name, acc in (("one call at a time", acc1), ("several in flight", accepted)):
        if acc != K * sel_per_step:
            raise RuntimeError(f"{name}: {acc} accepted selections counted in the timed "
                               f"region, expected {K} steps x {sel_per_step}")
    ms1 = reduce_max(ms1, dist, dev)
    elapsed_ms = reduce_max(elapsed_ms, dist, dev)
    sel_all = world * K * sel_per_step
    value = sel_all / (elapsed_ms * 1e-3)
    value_one_stream = sel_all / (ms1 * 1e-3)

    # ---- per-kernel durations: the two steps of the call, each replayed
    # alone from its own graphs (CUDA events on the launching stream) -----
    for s in slots:
        s["st2"] = torch.zeros(1, dtype=torch.int32, device=dev)
        s["stats2"] = torch.zeros(3, dtype=torch.int64, device=dev)

    def bound_only(s):
        gb.ar_bound_batched(s["alpha"], s["off"], s["plan"], s["bs"], s["st2"], s["work"], stream)

    def select_only(s):  # bounds from the last full step on this batch
        gb.ar_select_batched_bounded(s["alpha"], s["off"], s["oo"], s["bs"], 2, SEED, 0, b_base,
                                     gb.AR_CMP_F32, 1 << 20, s["plan"], s["idx"], s["stats2"],
                                     s["st2"], s["work"], stream)

    def time_alone(fn, reps):
        gs = []
        for s in slots:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream):
                fn(s)
            gs.append(g)
        for i in range(3 * N_SLOTS):
            gs[i % N_SLOTS].replay()
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(reps)]
        with torch.cuda.stream(stream):
            for i in range(reps):
                evs[i][0].record(stream)
                gs[i % N_SLOTS].replay()
                evs[i][1].record(stream)
        torch.cuda.synchronize()
        return np.array([x.elapsed_time(y) for x, y in evs])

    reps = min(K, 3000)
    red_ms = time_alone(bound_only, reps)
    sel_ms = time_alone(select_only, reps)

    def call_fp64(s):  # the whole call with the FP64 comparison (same plans and tiles)
        gb.ar_select_batched(s["alpha"], s["off"], s["oo"], SEED, 0, b_base, gb.AR_CMP_F64,
                             1 << 20, s["plan"], s["bs"], s["idx"], s["stats2"], s["st2"],
                             s["work"], stream)
    f64_ms = time_alone(call_fp64, min(reps, 1000))
    probes = probe_peaks(dev, stream)

    # ---- rooflines ---------------------------------------------------------
    peak, peak_kind, peaks = measured_peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    clk = float(peaks.get("sm_max_mhz", 2070.0))
    alu_peak = IMAD_PER_SM_CLK * sm_count * clk * 1e6 / PHILOX_IMAD_PER_BLOCK
    blocks_per_launch = trials / K / 2.0      # the timed region's own trials
    sel_s = float(sel_ms.mean()) * 1e-3
    red_s = float(red_ms.mean()) * 1e-3
    alg_bytes = float(np.mean([algorithmic_bytes(s["bt"]) for s in slots]))
    call_s = elapsed_ms / K * 1e-3               # per batch, several calls in flight
    step_s = float(kern_ms.mean()) * 1e-3        # per call, one call at a time
    # the headline: the whole call against the HBM roofline (algorithmic
    # bytes: alpha and the offsets read once, indices and {T, sum} written)
    roofline = {"bound": "hbm", "achieved": alg_bytes / call_s / 1e9, "peak": peak,
                "unit": "GB/s", "frac": alg_bytes / call_s / 1e9 / peak,
                "peak_kind": f"{peak_kind} (MEASURED_PEAKS hbm_gbs)" if peak_kind == "measured"
                else peak_kind,
                "traffic": profiled_traffic("ar_select_batched_call_batched_uneven.md"),
                "kernel": "ar_select_batched (one launch of k_batched_select<float, AR_CMP_F32, "
                          "NW, fused> per call when the tile's global share is 0, else "
                          "k_bound_reg + k_batched_select), "
                          f"{in_flight} independent calls in flight",
                "algorithmic_bytes_per_launch": alg_bytes, "us_per_call": call_s * 1e6,
                "one_call_at_a_time": {"achieved": alg_bytes / step_s / 1e9,
                                       "frac": alg_bytes / step_s / 1e9 / peak,
                                       "us_per_call": step_s * 1e6},
                "share_reduction": red_s / (red_s + sel_s),
                "share_selection": sel_s / (red_s + sel_s)}
    # the selection kernel alone: bound by 32-bit integer multiply issue
    # (Philox) with random gathers; work = the Philox blocks the accepted
    # trials consume
    roofline_alu = {"bound": "alu", "achieved": blocks_per_launch / sel_s, "peak": alu_peak,
                    "unit": "Philox4x32-10 blocks/s",
                    "frac": blocks_per_launch / sel_s / alu_peak,
                    # this kernel's own live traffic was not captured on these
                    # sources (the capture covers the one-launch call)
                    "traffic": None,
                    "kernel": "k_batched_select<float, AR_CMP_F32> (ar_select_batched_bounded)",
                    "peak_from": f"{IMAD_PER_SM_CLK} IMAD/clk/SM x {sm_count} SMs x "
                                 f"{clk:.0f} MHz / {PHILOX_IMAD_PER_BLOCK} IMAD per block",
                    "work_per_launch": blocks_per_launch, "trials_per_launch": trials / K,
                    "kernel_ms_mean": sel_s * 1e3, "kernel_ms_median": float(np.median(sel_ms)),
                    "microbench": probes,
                    "frac_of_microbench_philox": blocks_per_launch / sel_s / probes["philox_only"]}
    red_bytes = float(np.mean([reduction_bytes(s["bt"]) for s in slots]))
    roofline_reduction = {
        "bound": "hbm", "achieved": red_bytes / red_s / 1e9, "peak": peak, "unit": "GB/s",
        "frac": red_bytes / red_s / 1e9 / peak, "peak_kind": peak_kind,
        "traffic": profiled_traffic("k_bound_reg_batched_uneven.md"),
        "kernel": "k_bound_reg + k_batched_combine (ar_bound_batched; in ar_select_batched "
                  "the combine is folded into the selection kernel)",
        "algorithmic_bytes_per_launch": red_bytes, "kernel_ms_mean": red_s * 1e3,
        "kernel_ms_median": float(np.median(red_ms))}
    # inside ar_select_batched the reduction runs without the combine kernel:
    # its share of the step is the step less the selection timed alone
    in_step_s = step_s - sel_s
    if in_step_s > 0:
        # (with the one-launch form this is what folding the reduction into
        # the call costs beyond the selections alone)
        roofline_reduction["in_step_ms_derived"] = in_step_s * 1e3
        roofline_reduction["in_step_frac_derived"] = red_bytes / in_step_s / 1e9 / peak

    # ---- end to end through the C ABI with host buffers ------------------
    # Every step copies its inputs from pinned host memory, runs the call and
    # reads its indices, bounds and counters back.  Steps are pipelined over
    # three streams with two buffer sets: the copies of step i + 1 and the
    # read-back of step i - 1 overlap the kernels of step i (the kernels
    # themselves stay in order on one stream: they share the plan).
    ke = min(K, 100)
    s0 = slots[0]
    h_alpha = torch.from_numpy(s0["bt"].alpha).pin_memory()
    h_off = torch.from_numpy(s0["bt"].offsets).pin_memory()
    h_oo = torch.from_numpy(s0["bt"].out_offsets).pin_memory()
    nbuf = 2
    bufs = []
    for _ in range(nbuf):
        bufs.append({
            "alpha": torch.empty_like(h_alpha, device=dev),
            "off": torch.empty_like(h_off, device=dev),
            "oo": torch.empty_like(h_oo, device=dev),
            "bs": torch.empty((B_REAL, 2), dtype=torch.float64, device=dev),
            "idx": torch.empty(s0["idx"].numel(), dtype=torch.int32, device=dev),
            "stats": torch.zeros(3, dtype=torch.int64, device=dev),
            "st": torch.zeros(1, dtype=torch.int32, device=dev),
            "h_idx": torch.empty(s0["idx"].numel(), dtype=torch.int32).pin_memory(),
            "h_bs": torch.empty((B_REAL, 2), dtype=torch.float64).pin_memory(),
            "h_stats": torch.empty(3, dtype=torch.int64).pin_memory(),
            "in_done": torch.cuda.Event(), "comp_done": torch.cuda.Event(),
            "out_done": torch.cuda.Event()})
    s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    h2d = h_alpha.numel() * 4 + h_off.numel() * 8 + h_oo.numel() * 8
    d2h = s0["idx"].numel() * 4 + B_REAL * 2 * 8 + 24
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reduce_max(0.0, dist, dev)  # align the ranks before the timed region
    torch.cuda.synchronize()
    e0.record(s_in)
    stream.wait_event(e0)
    s_out.wait_event(e0)
    for i in range(ke):
        u = bufs[i % nbuf]
        if i >= nbuf:
            s_in.wait_event(u["comp_done"])       # buffer set free again
            stream.wait_event(u["out_done"])      # its results were read back
        with torch.cuda.stream(s_in):
            u["alpha"].copy_(h_alpha, non_blocking=True)
            u["off"].copy_(h_off, non_blocking=True)
            u["oo"].copy_(h_oo, non_blocking=True)
            u["in_done"].record(s_in)
        stream.wait_event(u["in_done"])
        with torch.cuda.stream(stream):
            gb.ar_select_batched(u["alpha"], u["off"], u["oo"], SEED, 0, b_base, gb.AR_CMP_F32,
                                 1 << 20, s0["plan"], u["bs"], u["idx"], u["stats"], u["st"],
                                 s0["work"], stream)
            u["comp_done"].record(stream)
        s_out.wait_event(u["comp_done"])
        with torch.cuda.stream(s_out):
            u["h_idx"].copy_(u["idx"], non_blocking=True)
            u["h_bs"].copy_(u["bs"], non_blocking=True)
            u["h_stats"].copy_(u["stats"], non_blocking=True)
            u["out_done"].record(s_out)
    s_in.wait_stream(stream)
    s_in.wait_stream(s_out)
    e1.record(s_in)
    torch.cuda.synchronize()
    e2e_ms = reduce_max(e0.elapsed_time(e1), dist, dev)
    e2e_value = world * ke * B_REAL * K_B / (e2e_ms * 1e-3)
    e2e_ok = all(bool(np.array_equal(u["h_idx"].numpy(), g_idx)) for u in bufs)

    # ---- FP64-plain: one M=1024 FP64 vector, K=1000, FP64 comparison ------
    a1 = W.plain_uniform(1024, seed=101)
    d_a1 = torch.from_numpy(a1).to(dev)
    p_bs = torch.empty(2, dtype=torch.float64, device=dev)
    p_st = torch.zeros(1, dtype=torch.int32, device=dev)
    p_idx = torch.empty(1000, dtype=torch.int32, device=dev)
    p_stats = torch.zeros(3, dtype=torch.int64, device=dev)

    def plain():
        gb.ar_bound(d_a1, p_bs, p_st, None, stream)
        gb.ar_select_k(d_a1, p_bs, 1000, SEED, 0, 0, gb.AR_CMP_F64, 1 << 20, p_idx, p_stats,
                       p_st, stream)
    with torch.cuda.stream(stream):
        plain()
    stream.synchronize()
    gp = torch.cuda.CUDAGraph()
    with torch.cuda.graph(gp, stream=stream):
        plain()
    for _ in range(20):
        gp.replay()
    torch.cuda.synchronize()
    npl = 2000
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        f0.record(stream)
        for _ in range(npl):
            gp.replay()
        f1.record(stream)
    torch.cuda.synchronize()
    plain_ms = f0.elapsed_time(f1) / npl
    # the same pair captured 50 times in one graph: the device time per call
    # without the host's cost of one graph launch per call
    gp50 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(gp50, stream=stream):
        for _ in range(50):
            plain()
    for _ in range(3):
        gp50.replay()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        f0.record(stream)
        for _ in range(npl // 50):
            gp50.replay()
        f1.record(stream)
    torch.cuda.synchronize()
    plain_dev_ms = f0.elapsed_time(f1) / npl
    fp64_plain = {"value": 1000 / (plain_ms * 1e-3), "unit": UNIT, "ms_per_call": plain_ms,
                  "device_ms_per_call": plain_dev_ms,
                  "device_value": 1000 / (plain_dev_ms * 1e-3),
                  "workload": "one FP64 vector M=1024 alpha~U(0,1], K=1000 selections, "
                              "ar_bound + ar_select_k, FP64 comparison, CUDA graph: one "
                              "graph launch per call (value), 50 calls per graph launch "
                              "(device_value)"}

    # ---- the single-vector workloads: skewed (M = 1029 lognormal with 30 %
    # zeros, K = 65536) and wide range (M = 2^20 spread over 12 decades,
    # K = 2^20), one ar_bound + ar_select_k per call, FP32 comparison -------
    def single_leg(alpha_np, K, reps):
        d_al = torch.from_numpy(alpha_np).to(dev)
        bs1 = torch.empty(2, dtype=torch.float64, device=dev)
        st1 = torch.zeros(1, dtype=torch.int32, device=dev)
        dt = gb.AR_F64 if d_al.dtype == torch.float64 else gb.AR_F32
        wk = torch.zeros(max(gb.ar_bound_workspace_size(d_al.numel(), dt), 16),
                         dtype=torch.uint8, device=dev)  # zero-filled before first use
        ix = torch.empty(K, dtype=torch.int32, device=dev)
        sts = torch.zeros(3, dtype=torch.int64, device=dev)

        def call(c, k, out, stats):
            gb.ar_bound(d_al, bs1, st1, wk, stream)
            gb.ar_select_k(d_al, bs1, k, SEED, 0, 0, c, 1 << 20, out, stats, st1, stream)
        # accuracy: ACC_SAMPLES selections in one call per comparison precision
        big = {c: torch.empty(ACC_SAMPLES, dtype=torch.int32, device=dev) for c in (0, 1)}
        with torch.cuda.stream(stream):
            call(gb.AR_CMP_F64, ACC_SAMPLES, big[1], None)
            call(gb.AR_CMP_F32, ACC_SAMPLES, big[0], None)
        stream.synchronize()
        i32, i64 = big[0].cpu().numpy(), big[1].cpu().numpy()
        del big
        accuracy = dict(A.paired(i32, i64, alpha_np.size + 1),
                        fp32_law=A.law(i32, alpha_np), fp64_law=A.law(i64, alpha_np))
        with torch.cuda.stream(stream):
            call(gb.AR_CMP_F32, K, ix, sts)
        stream.synchronize()
        trials = int(sts[0].item())
        g1 = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g1, stream=stream):
            call(gb.AR_CMP_F32, K, ix, None)
        for _ in range(5):
            g1.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            for _ in range(reps):
                g1.replay()
            e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        # the FP64 comparison on the same vector and K
        g1d = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g1d, stream=stream):
            call(gb.AR_CMP_F64, K, ix, None)
        for _ in range(5):
            g1d.replay()
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            e0.record(stream)
            for _ in range(reps):
                g1d.replay()
            e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1) / reps
        # the inverse transform on the same vector and K (the comparator the
        # paper argues against): exact running sums by a parallel scan, then a
        # bisection per selection
        it_ix = torch.empty(K, dtype=torch.int32, device=dev)
        it_st = torch.zeros(1, dtype=torch.int32, device=dev)
        it_wk = torch.empty(gb.ar_select_it_workspace_size(d_al.numel()), dtype=torch.uint8,
                            device=dev)
        g2 = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g2, stream=stream):
            gb.ar_select_it(d_al, K, SEED, 0, 0, it_ix, it_st, it_wk, stream)
        for _ in range(5):
            g2.replay()
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            e0.record(stream)
            for _ in range(reps):
                g2.replay()
            e1.record(stream)
        torch.cuda.synchronize()
        it_ms = e0.elapsed_time(e1) / reps
        blocks = trials / 2.0
        return {"value": K / (ms * 1e-3), "unit": UNIT, "ms_per_call": ms,
                "fp64_comparison": {"value": K / (ms64 * 1e-3), "unit": UNIT,
                                    "ms_per_call": ms64},
                "inverse_transform": {"value": K / (it_ms * 1e-3), "unit": UNIT,
                                      "ms_per_call": it_ms, "status": int(it_st.item()),
                                      "call": "ar_select_it (5 kernels + header memset)"},
                "trials_per_selection": trials / K,
                "alu": {"achieved": blocks / (ms * 1e-3), "peak": alu_peak,
                        "unit": "Philox4x32-10 blocks/s", "frac": blocks / (ms * 1e-3) / alu_peak},
                "accuracy": accuracy, "status": int(st1.item())}

    single = {
        # the plain vector with the FP32 comparison (the FP64 one is fp64_plain)
        "plain": dict(single_leg(W.plain_uniform(1024, seed=101), 1000, 2000),
                      workload="M=1024 FP64 alpha~U(0,1] (seed 101), K=1000, FP32 comparison"),
        "skewed": dict(single_leg(W.skewed(1029, seed=200), 65536, 400),
                       workload="M=1029 FP32 lognormal(0,2), 309 zeros (seed 200), K=65536"),
        "wide_range": dict(single_leg(W.wide_range(1 << 20, seed=400), 1 << 20, 40),
                           workload="M=2^20 FP32 10^U(-6,6) (seed 400), K=2^20")}

    # ---- the paper's timing workload: M = 1024 (Table 1's Gaussian
    # propensities), 62 500 selections per launch, 10^7 in all; the paper's
    # own election rule and the classical AR trial on the same data ---------
    def paper_workload():
        D = W.gaussian_paper(1024).astype(np.float32)
        d_D = torch.from_numpy(D).to(dev)
        T = torch.tensor([float(D.max())], dtype=torch.float64, device=dev)
        Kp, calls = 62_500, 160
        ix = torch.empty(Kp, dtype=torch.int32, device=dev)
        rej = torch.zeros(1, dtype=torch.int64, device=dev)
        stp = torch.zeros(1, dtype=torch.int32, device=dev)
        out = {}
        for name, fn in (
                ("paper_rule", lambda c: gb.ar_select_paper(d_D, T, Kp, SEED, c * Kp, 0, ix, rej,
                                                             stream)),
                ("classical_ar", lambda c: gb.ar_select_k(d_D, T, Kp, SEED, c * Kp, 0,
                                                          gb.AR_CMP_F32, 1 << 20, ix, None, stp,
                                                          stream))):
            with torch.cuda.stream(stream):
                fn(0)
            stream.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream):
                for c in range(calls):
                    fn(c)
            g.replay()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                e0.record(stream)
                g.replay()
                e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            out[name] = {"value": Kp * calls / (ms * 1e-3), "unit": UNIT, "ms_for_1e7": ms}
        out["workload"] = ("M=1024 FP32 Gaussian (Table 1's propensities), 160 launches of "
                           "62 500 selections = 10^7 selections in one CUDA graph")
        out["paper_context"] = ("the paper's own rule took 2277.18 ms (Tesla M2075) and 1326.78 ms "
                                "(Tesla K20) for this workload: context, not a target")
        out["status"] = int(stp.item())
        return out

    paper_wl = paper_workload()

    # ---- full batched SSA: 10^4 realizations x 10^4 steps ------------------
    ssa = None
    if not args.no_ssa:
        net = W.random_network(N=641, M=1029, seed=500)
        gnet = gb.SsaNet(net)
        B_ssa, n_ssa = 10_000, args.ssa_steps
        X0 = torch.from_numpy(W.initial_counts(641, B_ssa, seed=501 + rank)).to(dev)
        sx = {"X": torch.empty_like(X0), "a": torch.empty((B_ssa, 1029), dtype=torch.float64,
                                                          device=dev),
              "t": torch.zeros(B_ssa, dtype=torch.float64, device=dev),
              "step": torch.zeros(B_ssa, dtype=torch.int64, device=dev),
              "last": torch.zeros(B_ssa, dtype=torch.int32, device=dev),
              "status": torch.zeros(B_ssa, dtype=torch.int32, device=dev),
              "trials": torch.zeros(B_ssa, dtype=torch.int64, device=dev)}

        def ssa_run():
            sx["X"].copy_(X0)
            sx["t"].zero_()
            sx["step"].zero_()
            sx["status"].zero_()
            sx["trials"].zero_()
            gb.ssa_step_batched(gnet, sx["X"], sx["a"], sx["t"], sx["step"], n_ssa, SEED,
                                rank * B_ssa, gb.AR_CMP_F32, 1 << 20, sx["last"], sx["status"],
                                sx["trials"], stream)
        with torch.cuda.stream(stream):
            ssa_run()
        torch.cuda.synchronize()
        times = []
        for _ in range(3):
            s0e, s1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                sx["X"].copy_(X0)
                sx["t"].zero_()
                sx["step"].zero_()
                sx["status"].zero_()
                sx["trials"].zero_()
                s0e.record(stream)
                gb.ssa_step_batched(gnet, sx["X"], sx["a"], sx["t"], sx["step"], n_ssa, SEED,
                                    rank * B_ssa, gb.AR_CMP_F32, 1 << 20, sx["last"],
                                    sx["status"], sx["trials"], stream)
                s1e.record(stream)
            torch.cuda.synchronize()
            times.append(s0e.elapsed_time(s1e))
        steps_done = int(sx["step"].sum().item())
        ms = float(np.median(times))
        trials_ssa = float(sx["trials"].sum().item())
        sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
        clk = float(measured_peaks()[2].get("sm_max_mhz", 2070.0))
        alu_peak = IMAD_PER_SM_CLK * sm_count * clk * 1e6 / PHILOX_IMAD_PER_BLOCK
        ssa = {"value": steps_done / (ms * 1e-3), "unit": "SSA steps/s",
               "selections_per_s": steps_done / (ms * 1e-3), "kernel_ms": ms,
               "trials_per_step": trials_ssa / max(steps_done, 1),
               "roofline": {"bound": "alu", "kernel": "k_ssa<AR_CMP_F32>",
                            "achieved": trials_ssa / 2.0 / (ms * 1e-3), "peak": alu_peak,
                            "unit": "Philox4x32-10 blocks/s",
                            "frac": trials_ssa / 2.0 / (ms * 1e-3) / alu_peak,
                            "traffic": profiled_traffic("k_ssa_network_641x1029.md"),
                            "note": "sequential per realization; issue-bound (see profile)"},
               "status_or": int(np.bitwise_or.reduce(sx["status"].cpu().numpy())),
               "workload": f"{B_ssa} realizations of a random mass-action network "
                           f"(641 species, 1029 uni/bi/dimer reactions, seed 500), "
                           f"{n_ssa} steps each, FP32 comparison, FP64 propensities"}
        gnet.close()

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_leg()
    clocks = sampler.summary(t_wall0, t_wall1)
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
           "warmup": args.warmup, "ms_per_step": elapsed_ms / K, "higher_is_better": True,
           "one_call_at_a_time": {"value": value_one_stream, "ms_per_step": ms1 / K,
                                  "step_ms_mean": float(kern_ms.mean())},
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": dict(workload_config(),
                          autotuned_tiles=[{"warps_per_cta": t[0], "global_share_pm": t[1],
                                            "ns_per_call": t[2]} for t in tuned],
                          batches_in_flight=in_flight,
                          tile_in_flight=(best_tile if best_tile == "autotuned"
                                          else list(best_tile)),
                          ctas_per_sm_in_flight=best_grid if best_grid else "as many as fit",
                          selections_per_item_in_flight=best_items if best_items else 64,
                          in_flight_candidates=pipe_tiles),
           "clocks": clocks,
           "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                   "d2h_bytes_per_step": d2h, "steps": ke, "ms_per_step": e2e_ms / ke,
                   "indices_match_device_run": e2e_ok,
                   "pipelining": "copies of step i+1 and read-back of step i-1 overlap step i "
                                 "(3 streams, 2 buffer sets)"},
           "gpu_launches": launches_timed,
           "roofline": roofline,
           "roofline_alu": roofline_alu,
           "roofline_reduction": roofline_reduction,
           "cpu_baseline": cpu,
           # the metric's comparison: the FP32 batched rate over the plain FP64
           # single-vector form's (one graph launch per call; device time)
           "fp64_plain": dict(fp64_plain, fp32_batched_over_fp64_plain=value / fp64_plain["value"],
                              fp32_batched_over_fp64_plain_device=value
                              / fp64_plain["device_value"]),
           "single_vector": single,
           # the batched call with the FP64 comparison, one call at a time
           # (the FP32 figure beside it: one_call_at_a_time.step_ms_mean)
           "batched_fp64_comparison": {"value": sel_per_step / (float(f64_ms.mean()) * 1e-3),
                                       "unit": UNIT, "ms_per_call": float(f64_ms.mean()),
                                       "fp32_ms_per_call": float(kern_ms.mean())},
           "paper_workload": paper_wl,
           "ssa": ssa,
           "accuracy": {"batched_fp32_vs_fp64": acc_batched,
                        "plain_fp32_vs_fp64": single["plain"]["accuracy"],
                        "skewed_fp32_vs_fp64": single["skewed"]["accuracy"],
                        "wide_range_fp32_vs_fp64": single["wide_range"]["accuracy"],
                        "note": "FP64 indices of the library are bit-exact with the FP64 oracle "
                                "(parity tests), so the paired figures are against the oracle",
                        "status": status, "accepted_per_step": accepted / K},
           "kernel_source_hash": kernel_source_hash()}
    print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
