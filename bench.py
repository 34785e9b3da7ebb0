#!/usr/bin/env python
"""Benchmark: all-pairs Smith-Waterman read distances at paper scale on GB300.

Workload (default): 100,000 synthetic reads, lengths U[250,450], 200 ancestors from a
3-level tree (section "A sample from Lake Geneva" gives ~1e5 reads per sample; section
2.2 computes ~5e9 pairwise values).  One step = the whole path for one read set:
ingest/pack from device-resident bytes, then the all-pairs triangle (4,999,950,000
uint16 distances, ~10 GB, larger than L2).  The metric is GCUPS: DP cells
(sum over pairs of len_i * len_j) per second of device time; pairs/s is reported beside.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gbd|reference]

Under torchrun each rank runs an independent replica of the workload on its own GPU
(the path is computed on one GPU; there is no data-path collective), the time is the
maximum over ranks, and value counts the cells of every rank.

Besides the timed steps, rank 0 measures: the end-to-end figure (the last warm-up step,
run through host buffers), the oracle on a bounded sample of the same pairs (the
cpu_baseline, whose sample is grown to 2e6 pairs to check the timed triangle), and, while
the --time-budget allows, the batched form against per-sample launches (64 uneven
samples), the served form against per-request launches (a burst of requests against the
resident 1e5-read set), and the served-batch latency under Poisson arrivals.  The run
exits 1 when a checked distance differs from the oracle's.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

T_START = time.perf_counter()        # the time guard of the optional phases counts from here
METRIC = "GCUPS, all-pairs n=1e5 (bit-exact)"
UNIT = "GCUPS"
L2_FLUSH_BYTES = 512 << 20


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gbd", "reference"], default="gbd")
    ap.add_argument("--n", type=int, default=100_000, help="reads (default: paper scale)")
    ap.add_argument("--len-lo", type=int, default=250, help="shortest read (default 250)")
    ap.add_argument("--len-hi", type=int, default=450, help="longest read (default 450)")
    ap.add_argument("--kernel", choices=["auto", "general", "systolic"], default="auto")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--check-pairs", type=int, default=2_000_000,
                    help="uniformly sampled pairs of the timed triangle compared with the oracle")
    ap.add_argument("--mode", choices=["allpairs", "batch", "serve", "mds", "components", "affine", "annotate"],
                    default="allpairs")
    ap.add_argument("--serve-requests", type=int, default=200,
                    help="requests in the serving phase of the all-pairs run (0 = skip); fewer (at "
                         "least 40) when the time budget leaves less room")
    ap.add_argument("--time-budget", type=float, default=1700.0,
                    help="seconds from start within which the all-pairs run schedules its optional "
                         "phases (batched and served comparisons, serving latency)")
    ap.add_argument("--no-batch", action="store_true", help="all-pairs run: skip the batched comparison")
    ap.add_argument("--compare-requests", type=int, default=24,
                    help="requests of the served-vs-plain burst comparison (0 = skip)")
    ap.add_argument("--serve-load", type=float, default=0.8,
                    help="offered load of that phase, as a fraction of measured pairs/s")
    ap.add_argument("--samples", type=int, default=64, help="batch mode: samples")
    ap.add_argument("--small-requests", type=int, default=400,
                    help="requests of 1-16 reads in the small-request served-vs-plain comparison (0 = skip)")
    ap.add_argument("--mds-k", type=int, default=64, help="mds mode: sketch columns k")
    ap.add_argument("--mds-r", type=int, default=50, help="mds mode: coordinates r (paper: 50)")
    ap.add_argument("--mds-q", type=int, default=2, help="mds mode: subspace-iteration rounds")
    ap.add_argument("--gap-open", type=int, default=2, help="affine mode: gap opening penalty")
    ap.add_argument("--th", type=str, default="25/100",
                    help="components mode: hit rule num/den (97 %% homology = 3/100) or an absolute d")
    return ap.parse_args(argv)


# ------------------------------------------------------------------ distributed plumbing

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def init_dist(world: int, backend: str):
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend)


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int, device=None) -> float:
    """Maximum of a per-rank float over all ranks (identity on one rank)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def combine(units_per_rank: float, seconds_this_rank: float, world: int, device=None):
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    t = max_over_ranks(seconds_this_rank, world, device)
    return units_per_rank * world / t, t


# ------------------------------------------------------------------ clocks sampling

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------ CPU oracle baseline

# ------------------------------------------------------------------ the cpu_baseline leg
# Every call into oracle/ that bench.py makes is in the functions below: each times the
# oracle on a bounded sample of its mode's workload (the cpu_baseline figure) and, when
# given the GPU's values for the same sample, compares them (the spot check).

def _oracle_cores():
    return os.cpu_count() or 1


def cpu_oracle_sample(rs, seconds: float, seed: int = 7, gpu_pairs=None, min_check: int = 0):
    """Time the CPU oracle on a bounded uniform sample of the workload's pairs; with
    gpu_pairs (a function (i, j) -> the GPU's distances) also compare the last sample,
    grown with further uniformly drawn pairs (untimed) to at least min_check pairs."""
    import oracle
    n = rs.n
    L = rs.lengths.astype(np.float64)
    cores = _oracle_cores()

    def sample(k, s):
        st_rng = np.random.default_rng(s)
        i = st_rng.integers(0, n - 1, size=k)
        j = i + 1 + (st_rng.random(k) * (n - 1 - i)).astype(np.int64)
        return i, j

    k = 4 * cores
    for attempt in range(6):           # grow the sample until it takes about `seconds`
        i, j = sample(k, seed + attempt)
        t0 = time.perf_counter()
        want = oracle.pairs(rs, i, j, nthreads=cores)
        dt = time.perf_counter() - t0
        if dt >= 0.5 * seconds or k >= 4_000_000:
            break
        k = int(min(4_000_000, max(2 * k, k * seconds / max(dt, 1e-6))))
    cells = float(np.sum(L[i] * L[j]))
    out = {"value": cells / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{k} uniformly sampled pairs of the same {n}-read workload, "
                     f"{cells:.3e} cells in {dt:.1f} s on {cores} host threads"}
    if gpu_pairs is not None:
        if k < min_check:
            xi, xj = sample(min_check - k, seed + 1000)
            want = np.concatenate([want, oracle.pairs(rs, xi, xj, nthreads=cores)])
            i, j = np.concatenate([i, xi]), np.concatenate([j, xj])
        got = np.asarray(gpu_pairs(i, j), dtype=np.uint16)
        out["check"] = {"pairs_checked": int(len(i)), "mismatches": int(np.count_nonzero(got != want))}
    return out


def cpu_baseline_pairs(qs, i, j, ref=None, got=None, gap_open: int = 0, what: str = "pairs"):
    """The oracle on given pairs (qs[i[t]], ref[j[t]]) (ref = qs if None), timed; compared
    with the GPU's values `got` when given."""
    import oracle
    cores = _oracle_cores()
    i = np.asarray(i, dtype=np.int64)
    j = np.asarray(j, dtype=np.int64)
    t0 = time.perf_counter()
    want = oracle.pairs(qs, i, j, ref, nthreads=cores, gap_open=gap_open)
    dt = max(time.perf_counter() - t0, 1e-9)
    La = qs.lengths.astype(np.float64)[i]
    Lb = (ref if ref is not None else qs).lengths.astype(np.float64)[j]
    cells = float(np.sum(La * Lb))
    out = {"value": cells / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{len(i)} sampled {what}, {cells:.3e} cells in {dt:.2f} s on {cores} host threads"}
    if got is not None:
        got = np.asarray(got, dtype=np.uint16)
        out["check"] = {"pairs_checked": int(len(i)), "mismatches": int(np.count_nonzero(got != want))}
    return out


def cpu_baseline_batch(samples, got_fn, all_pairs_upto: int = 600, per_sample: int = 3000, seed: int = 44):
    """The oracle on the batched workload: every pair of the samples of at most
    all_pairs_upto reads, per_sample uniformly drawn pairs of each larger one; compared with
    the GPU's triangles (got_fn(s, i, j) -> distances of sample s)."""
    import oracle
    cores = _oracle_cores()
    rng = np.random.default_rng(seed)
    checked = mism = 0
    cells = 0.0
    t0 = time.perf_counter()
    n_all = 0
    for s, rs in enumerate(samples):
        n = rs.n
        if n < 2:
            continue
        if n <= all_pairs_upto:
            i, j = np.triu_indices(n, 1)
            n_all += 1
        else:
            i = rng.integers(0, n - 1, size=per_sample)
            j = i + 1 + (rng.random(per_sample) * (n - 1 - i)).astype(np.int64)
        i = i.astype(np.int64)
        j = j.astype(np.int64)
        want = oracle.pairs(rs, i, j, nthreads=cores)
        got = np.asarray(got_fn(s, i, j), dtype=np.uint16)
        checked += len(i)
        mism += int(np.count_nonzero(got != want))
        L = rs.lengths.astype(np.float64)
        cells += float(np.sum(L[i] * L[j]))
    dt = max(time.perf_counter() - t0, 1e-9)
    return {"value": cells / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"all pairs of the {n_all} samples of <= {all_pairs_upto} reads, {per_sample} uniformly "
                      f"drawn pairs of each other sample: {checked} pairs, {dt:.1f} s on {cores} host threads",
            "check": {"pairs_checked": checked, "mismatches": mism}}


def cpu_baseline_components(rs, i, j, th, labels):
    """The oracle's distances and hit rule on sampled pairs, timed; every sampled hit pair
    must share a component of the GPU's labels, and every label must be a root."""
    import oracle
    from oracle import threshold as oth
    cores = _oracle_cores()
    t0 = time.perf_counter()
    d = oracle.pairs(rs, i, j, nthreads=cores)
    L = rs.lengths
    hit = oth.is_hit(d, L[i], L[j], th.num, th.den, th.abs_max)
    dt = max(time.perf_counter() - t0, 1e-9)
    cells = float(np.sum(L[i].astype(np.float64) * L[j]))
    n = len(labels)
    return {"value": cells / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{len(i)} uniformly sampled pairs with the hit rule, {dt:.2f} s on {cores} host threads",
            "check": {"pairs_checked": int(len(i)), "hits": int(hit.sum()),
                      "hit_pairs_split": int(np.count_nonzero(hit & (labels[i] != labels[j]))),
                      "labels_are_roots": bool(np.all(labels[labels] == labels) and np.all(labels <= np.arange(n)))}}


def cpu_baseline_annotate(qs, ref, ref_lab, th, got_rows):
    """The oracle's rectangle and annotation rule for sample reads qs against ref, timed;
    compared with the GPU's row labels for the same reads."""
    import oracle
    from oracle import threshold as oth
    cores = _oracle_cores()
    t0 = time.perf_counter()
    D = oracle.rect(qs, 0, qs.n, ref, 0, ref.n, nthreads=cores)
    want = oth.annotate(D, qs.lengths, ref.lengths, ref_lab, th.num, th.den, th.abs_max)
    dt = max(time.perf_counter() - t0, 1e-9)
    cells = float(qs.lengths.sum()) * float(ref.lengths.sum())
    return {"value": cells / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{qs.n} sample reads against all {ref.n} references, annotated, {dt:.1f} s "
                      f"on {cores} host threads",
            "check": {"rows_checked": int(qs.n), "mismatches": int(np.count_nonzero(np.asarray(got_rows) != want))}}


def cpu_baseline_mds(n_full: int, k: int, r: int, q: int, n_sample: int = 2000):
    """Time the oracle's randomized MDS on an n_sample-read synthetic triangle; the
    oracle forms G with two dense n x n products (O(n^3)), so the full-size figure is
    extrapolated as n^3."""
    from oracle import mds as omds
    from paper_1803_02272_gb300 import synth
    m = n_sample * (n_sample - 1) // 2
    tri = synth.Stream(91, 0).integers(0, 450, (m,)).astype(np.uint16)
    omega = synth.Stream(92, 0).normal((n_sample, k))
    t0 = time.perf_counter()
    omds.mds_randomized(omds.tri_to_square(tri, n_sample), r, omega, q)
    dt = time.perf_counter() - t0
    scale = (n_full / n_sample) ** 3
    return {"value": dt * scale, "unit": "s", "cores": os.cpu_count() or 1, "kind": "oracle",
            "sample": f"oracle randomized MDS of a {n_sample}-read triangle (k={k}, r={r}, q={q}) "
                      f"in {dt:.2f} s, extrapolated by (n/{n_sample})^3 to n={n_full}"}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_1803_02272_gb300 import synth
    rs = synth.workload_paper_scale(n=args.n, len_lo=args.len_lo, len_hi=args.len_hi)
    per_step = max(1.0, min(args.cpu_seconds, 60.0 / max(1, args.steps + args.warmup)))
    for w in range(args.warmup):
        cpu_oracle_sample(rs, per_step / 4, seed=100 + w)
    vals = [cpu_oracle_sample(rs, per_step, seed=200 + s) for s in range(args.steps)]
    v = float(np.mean([x["value"] for x in vals]))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": workload_config(rs),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": vals[0]["cores"],
                             "kind": "oracle", "sample": vals[0]["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def workload_config(rs):
    n = rs.n
    L = rs.lengths
    return {"workload": f"paper-scale all-pairs: {n} synthetic reads, lengths "
                        f"U[{L.min()},{L.max()}], "
                        "200 tree ancestors (2-8 % divergence per level), 5 % sub / 1.5 % indel",
            "n_reads": n, "pairs": n * (n - 1) // 2, "cells": rs.total_cells(),
            "output": f"uint16 strict upper triangle, {n * (n - 1) // 2 * 2 / 1e9:.2f} GB",
            "l2": "output larger than L2 every step; 512 MiB L2 flush between timed steps",
            "scores": "match +1, mismatch -1, gap -1; d = max(la,lb) - S"}


# ------------------------------------------------------------------ GPU arm

# DP ALU ops per int16x2 pair of cells in the kernel's recurrence: one add-max (diagonal
# plus score against the floor), one 3-way max, and half a 3-way max for the running
# maximum.  The textbook count is 4 ops per cell (add score, max with gap, 3-way max with
# 0, running max) on 2 cells per int16x2 op.
OPS_PER_CELL_PAIR = 2.5
TEXTBOOK_OPS_PER_CELL = 4.0
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "sw_systolic_traffic.md")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_1803_02272_gb300", "csrc", f)
                  for f in ("sw_systolic.cu", "sw_systolic.cuh")]


def measured_peak_gcups(gbd, stream) -> dict:
    """Integer-DP roofline from the measured issue rate of the int16x2 DPX max class
    (the ALU pipe every max/min form shares)."""
    rates = {}
    for name in ("VIMAX3_S16X2", "VIADDMAX_S16X2"):
        op = gbd.PROBE_OPS.index(name)
        rates[name] = gbd.gbd_probe_op_rate(op, 20000, stream)
    best = max(rates.values())
    return {"peak_gcups": best * 2 / OPS_PER_CELL_PAIR / 1e9,
            "textbook_gcups": best * 2 / TEXTBOOK_OPS_PER_CELL / 1e9,
            "rates": rates}


def kernel_sha() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def traffic_value(key: str):
    """A per-pair DRAM figure from the committed ncu summary of the distance kernel, or
    None once the kernel source differs from the profiled one."""
    try:
        kv = {}
        for line in open(TRAFFIC_FILE):
            if ":" in line and line.startswith("- "):
                k, v = line[2:].split(":", 1)
                kv[k.strip()] = v.strip().strip("`")
        if kv.get("kernel_sha") != kernel_sha():
            return None
        return float(kv[key])
    except (OSError, KeyError, ValueError):
        return None


def traffic_per_launch(pairs: int):
    """DRAM bytes (read + write) per all-pairs launch: the per-pair figure of the committed
    ncu summary (traffic is dominated by the uint16 output, so it grows with the pair
    count) times the pairs; None once the kernel source differs from the profiled one."""
    per_pair = traffic_value("dram_bytes_per_pair")
    return None if per_pair is None else per_pair * pairs


def triangle_write(pairs: int, seconds: float):
    """HBM write rate of the triangle: the algorithmic 2 bytes per pair, and the DRAM
    bytes written per pair in the committed ncu summary, over the kernel time."""
    per_pair = traffic_value("dram_write_bytes_per_pair")
    return {"algorithmic_gbs": 2.0 * pairs / seconds / 1e9,
            "dram_gbs": None if per_pair is None else per_pair * pairs / seconds / 1e9,
            "dram_bytes_per_pair": per_pair}


def run_gbd(args):
    import torch
    world, rank, local = dist_env()
    init_dist(world, "nccl")
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    from paper_1803_02272_gb300 import gbd, synth

    rs = synth.workload_paper_scale(n=args.n, len_lo=args.len_lo, len_hi=args.len_hi)
    n = rs.n
    m = n * (n - 1) // 2
    cells = float(rs.total_cells())
    kernel = {"auto": gbd.GBD_KERNEL_AUTO, "general": gbd.GBD_KERNEL_GENERAL,
              "systolic": gbd.GBD_KERNEL_SYSTOLIC}[args.kernel]
    ctx = gbd.Context(local, kernel=kernel)
    stream = torch.cuda.current_stream()
    seq_d = torch.from_numpy(rs.seq).to(dev)
    off_d = torch.from_numpy(rs.offsets.view(np.int64)).to(dev)
    tri = torch.empty(m, dtype=torch.int16, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def step(ev=None):
        s = gbd.gbd_load_reads(ctx.handle, seq_d, off_d, n, stream)
        if ev is not None:
            ev[0].record(stream)
        gbd.gbd_all_pairs(ctx.handle, s, tri, m, stream)
        if ev is not None:
            ev[1].record(stream)
        return s

    # the last warm-up step is the end-to-end one: the same step through host buffers (reads
    # copied in from pinned host memory, the triangle copied back), timed as e2e
    e2e = None
    for w in range(args.warmup):
        if w == args.warmup - 1 and not args.no_e2e and rank == 0:
            e2e = run_e2e(gbd, ctx, rs, dev, stream)
            e2e["note"] = "measured on the last warm-up step"
        else:
            gbd.gbd_free_set(step())
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    barrier(world)
    torch.cuda.synchronize()
    launches0 = gbd.gbd_kernel_launches()
    step_ms, kern_ms, sets = [], [], []
    for _ in range(args.steps):
        flush.zero_()                                  # evict L2 between steps (untimed)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        k0 = torch.cuda.Event(enable_timing=True)
        k1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sets.append(step((k0, k1)))
        e1.record(stream)
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        kern_ms.append(k0.elapsed_time(k1))
    torch.cuda.synchronize()
    barrier(world)
    launches = gbd.gbd_kernel_launches() - launches0
    clocks = sampler.stop()
    for s in sets:
        gbd.gbd_free_set(s)

    total_s = sum(step_ms) / 1e3
    value_cps, t_max = combine(cells * args.steps, total_s, world, dev)
    gcups = value_cps / 1e9
    pairs_per_s = m * args.steps * world / t_max

    def gpu_pairs(i, j):
        """The GPU triangle's distances of pairs (i, j), i < j."""
        idx = i * n - i * (i + 1) // 2 + (j - i - 1)
        return tri[torch.from_numpy(idx).to(dev)].cpu().numpy().view(np.uint16)

    line = None
    if rank == 0:
        peak = measured_peak_gcups(gbd, stream)
        kern_s = float(np.mean(kern_ms)) / 1e3
        achieved = cells / kern_s / 1e9
        line = {
            "metric": METRIC, "value": gcups, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": float(np.mean(step_ms)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "int32" if args.kernel == "general" else "int16x2",
            "data": "synthetic", "config": workload_config(rs),
            "pairs_per_s": pairs_per_s,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak["peak_gcups"],
                         "unit": UNIT, "frac": achieved / peak["peak_gcups"],
                         "traffic": traffic_per_launch(m),
                         "peak_source": "of measured: ALU-pipe issue rate of int16x2 DPX max "
                                        "(probe in libgbd) x 2 cells / 2.5 ops per cell pair",
                         "textbook_peak": peak["textbook_gcups"],
                         "textbook_frac": achieved / peak["textbook_gcups"],
                         "probe_lane_ops_per_s": peak["rates"]},
            "triangle_write": triangle_write(m, kern_s),
            "clocks": clocks, "gpu_launches": int(launches), "spot_check": None,
        }
    if rank == 0:
        if e2e is None and not args.no_e2e:
            e2e = run_e2e(gbd, ctx, rs, dev, stream)
        line["e2e"] = e2e
    if rank == 0:
        if not args.no_cpu_baseline and world == 1:
            # the oracle's sample doubles as an exactness check of this very triangle
            line["cpu_baseline"] = cpu_oracle_sample(rs, args.cpu_seconds, gpu_pairs=gpu_pairs,
                                                     min_check=args.check_pairs)
            line["spot_check"] = line["cpu_baseline"].pop("check")
        else:
            # no timed baseline: still compare a fixed uniform sample of this very triangle
            rng = np.random.default_rng(17)
            ci = rng.integers(0, n - 1, size=20000)
            cj = ci + 1 + (rng.random(20000) * (n - 1 - ci)).astype(np.int64)
            chk = cpu_baseline_pairs(rs, ci, cj, got=gpu_pairs(ci, cj),
                                     what="uniformly sampled pairs (exactness check only, untimed)")
            line["spot_check"] = chk.pop("check")
        line["exact"] = line["spot_check"]["mismatches"] == 0
    if rank == 0:
        del tri
        line.update(optional_phases(args, gbd, ctx, rs, dev, pairs_per_s, gcups))
        line["wall_s"] = time.perf_counter() - T_START
    if rank == 0:
        print(json.dumps(line), flush=True)
    barrier(world)
    if rank == 0 and not line["exact"]:
        print(f"bench: {line['spot_check']['mismatches']} of {line['spot_check']['pairs_checked']} "
              "checked distances differ from the oracle", file=sys.stderr)
        return 1
    return 0


def optional_phases(args, gbd, ctx, rs, dev, pairs_per_s: float, gcups: float) -> dict:
    """After the timed all-pairs steps: the batched comparison (64 uneven samples), the
    served-vs-plain comparison (a burst of requests against the resident paper-scale set)
    and the served-batch latency (Poisson arrivals), in that order.  Each runs only when
    its duration, estimated from the rates measured so far, fits what is left of
    --time-budget; the serving phase takes fewer requests (at least 40) to fit."""
    from paper_1803_02272_gb300 import synth
    out = {}

    def left():
        return args.time_budget - (time.perf_counter() - T_START)

    if not args.no_batch:
        samples = synth.workload_batched(n_samples=args.samples)
        t_call = sum(x.total_cells() for x in samples) / (gcups * 1e9)
        est = 2 * 1.1 * t_call + 6 * t_call + 40          # plain 1 + 1, batched 5 + 1, loads and check
        if est < left():
            out["batch"] = batch_phase(gbd, ctx, samples, dev, 1, check=not args.no_cpu_baseline)
        else:
            out["batch"] = {"skipped": f"time budget: needs about {est:.0f} s, {left():.0f} s left"}
        del samples
    ref = ctx.load(rs) if (args.compare_requests > 0 or args.small_requests > 0 or args.serve_requests > 0) else None
    capacity = pairs_per_s
    if args.compare_requests > 0:
        reqs = synth.workload_served_queries(args.compare_requests, 1.0, seed=1006)
        est = 2 * sum(r.reads.n for r in reqs) * rs.n / pairs_per_s + 20
        if est < left():
            out["serve_vs_plain"] = serve_compare(gbd, ctx, ref, rs, dev, args.compare_requests, seed=1006)
            capacity = out["serve_vs_plain"]["server_burst"]["pairs_per_s"]
        else:
            out["serve_vs_plain"] = {"skipped": f"time budget: needs about {est:.0f} s, {left():.0f} s left"}
    if args.small_requests > 0:
        # many small requests (1-16 reads each): a plain loop pays its per-request launch and
        # set-up costs, the server folds concurrent requests into shared launches
        reqs = synth.workload_served_queries(args.small_requests, 1.0, seed=1007, nq_hi=16)
        est = 0.01 * len(reqs) + 2 * sum(r.reads.n for r in reqs) * rs.n / (0.8 * pairs_per_s) + 15
        if est < left():
            out["serve_vs_plain_small"] = serve_compare(gbd, ctx, ref, rs, dev, args.small_requests, seed=1007,
                                                        nq_hi=16)
        else:
            out["serve_vs_plain_small"] = {"skipped": f"time budget: needs about {est:.0f} s, {left():.0f} s left"}
    if args.serve_requests > 0:
        n_req, est = args.serve_requests, None
        while True:
            reqs = synth.workload_served_queries(n_req, 1.0, seed=1005)
            sizes = [r.reads.n for r in reqs]
            # Poisson arrivals: the last one comes about 1 +- 1/sqrt(n) of the mean span late
            est = (1.0 + 2.0 / np.sqrt(n_req)) * sum(sizes) * rs.n / (args.serve_load * capacity) + \
                max(sizes) * rs.n / capacity + 15
            if est < left() or n_req <= 40:
                break
            n_req = max(40, n_req - 40)
        if est < left():
            out["serving"] = serve_phase(gbd, ctx, ref, rs, dev, n_req, load=args.serve_load, capacity_pps=capacity,
                                         seed=1005)
            out["serving"]["capacity_basis"] = ("server burst pairs/s of serve_vs_plain" if "server_burst" in
                                                out.get("serve_vs_plain", {}) else "all-pairs pairs/s")
        else:
            out["serving"] = {"skipped": f"time budget: needs about {est:.0f} s, {left():.0f} s left"}
    del ref
    return out


def run_e2e(gbd, ctx, rs, dev, stream):
    """The same metric through the C ABI with host buffers: reads copied in from pinned
    host memory by gbd_load_reads, the triangle written to pinned host memory by
    gbd_all_pairs_to_host (band by band, each band's copy overlapping the next band)."""
    import torch
    n = rs.n
    m = n * (n - 1) // 2
    seq_h = torch.from_numpy(rs.seq).pin_memory()
    off_h = torch.from_numpy(rs.offsets.view(np.int64)).pin_memory()
    host = torch.empty(m, dtype=torch.int16, pin_memory=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s = gbd.gbd_load_reads(ctx.handle, seq_h, off_h, n, stream)
    gbd.gbd_all_pairs_to_host(ctx.handle, s, host, m, 0, stream)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    gbd.gbd_free_set(s)
    return {"value": rs.total_cells() / dt / 1e9, "unit": UNIT,
            "h2d_bytes_per_step": int(rs.seq.nbytes + rs.offsets.nbytes),
            "d2h_bytes_per_step": int(m * 2), "seconds": dt}


# ------------------------------------------------------------------ serving and batching

def percentile(xs, p):
    return float(np.percentile(np.asarray(xs, dtype=np.float64), p)) if len(xs) else None


def serve_phase(gbd, ctx, ref_handle, ref_rs, dev, n_requests, load=1.0, capacity_pps=1.0,
                seed=1005, check=True, burst=False, nq_hi=4096):
    """Poisson arrivals of query batches against a resident reference set; returns
    latency percentiles (submit -> rows complete) and served pairs/s.  The arrival rate
    makes the offered pairs/s of this very request sample `load` x `capacity_pps`."""
    import torch
    from paper_1803_02272_gb300 import synth
    reqs = synth.workload_served_queries(n_requests, 1.0, seed=seed, nq_hi=nq_hi)   # arrivals at rate 1/s
    n_ref = ref_rs.n
    mean_pairs = float(np.mean([r.reads.n for r in reqs])) * n_ref
    rate_per_s = load * capacity_pps / mean_pairs
    for r in reqs:                     # Poisson gaps scale as 1/rate
        r.arrival_s = r.arrival_s / rate_per_s
    srv = gbd.Server(ctx, ref_handle)
    pending, lat, outs = {}, [], []
    # every request's output rows are allocated before the clock starts (the plain
    # per-request loop it is compared with reuses one preallocated buffer)
    req_out = [torch.empty((r.reads.n, n_ref), dtype=torch.int16, device=dev) for r in reqs]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    i = 0
    total_pairs = sum(r.reads.n for r in reqs) * n_ref
    while i < len(reqs) or pending:
        now = time.perf_counter() - t0
        while i < len(reqs) and (burst or reqs[i].arrival_s <= now):
            out = req_out[i]
            t, _ = srv.submit(reqs[i].reads, out)
            pending[t] = (time.perf_counter(), i, out)
            i += 1
        for t in list(pending):
            if srv.poll(t):
                ts, k, out = pending.pop(t)
                lat.append(time.perf_counter() - ts)
                outs.append((k, out))
        time.sleep(0.0005)
    wall = time.perf_counter() - t0
    srv.close()
    torch.cuda.synchronize()
    mism, base = None, None
    if check:
        # four sampled (row, reference) entries of every request, against the oracle
        rng = np.random.default_rng(seed)
        pj, got, q_all = [], [], []
        for k, out in outs:
            q = reqs[k].reads
            rows = rng.integers(0, q.n, size=4)
            cols = rng.integers(0, n_ref, size=4)
            vals = out[torch.from_numpy(rows).to(dev), torch.from_numpy(cols).to(dev)]
            vals = vals.cpu().numpy().view(np.uint16)
            for r_, c_, v_ in zip(rows, cols, vals):
                q_all.append(q.read(int(r_)))
                pj.append(int(c_))
                got.append(int(v_))
        qs = synth.from_strings(q_all)
        base = cpu_baseline_pairs(qs, np.arange(len(q_all)), np.array(pj), ref_rs, got,
                                  what="served (query, reference) pairs")
        mism = base.pop("check")["mismatches"]
    del outs, req_out
    nq = [r.reads.n for r in reqs]
    return {"requests": len(reqs), "mean_queries": float(np.mean(nq)),
            "offered_load": None if burst else load, "rate_per_s": None if burst else rate_per_s,
            "p50_ms": percentile(lat, 50) * 1e3, "p99_ms": percentile(lat, 99) * 1e3,
            "pairs_per_s": total_pairs / wall, "wall_s": wall,
            "spot_check_mismatches": mism, "cpu_baseline": base}


def batch_phase(gbd, ctx, samples, dev, steps: int, check: bool = True):
    """The batched workload: one gbd_batch call against one gbd_all_pairs call per sample,
    timed after warm-up (the batch autotuner's five timed candidates and its pick run as
    warm-up calls); outputs compared with each other in full and with the oracle on a
    sample (the cpu_baseline leg)."""
    import torch
    sets = [ctx.load(s) for s in samples]
    outs_b = [torch.empty(max(s.n * (s.n - 1) // 2, 1), dtype=torch.int16, device=dev) for s in samples]
    outs_p = [torch.empty_like(o) for o in outs_b]
    pairs = sum(s.n * (s.n - 1) // 2 for s in samples)
    cells = sum(s.total_cells() for s in samples)

    def plain():
        for st, o in zip(sets, outs_p):
            ctx.all_pairs(st, out=o)

    def batched():
        ctx.batch(sets, outs=outs_b)

    res = {}
    for name, fn, warm in (("plain_per_sample", plain, 1), ("batched", batched, 5)):
        for _ in range(warm):                  # batched: the autotuner's five timed candidates;
            fn()                               # the first timed call records and runs its pick
        torch.cuda.synchronize()
        ts = []
        for _ in range(steps):
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        t = float(np.median(ts))
        res[name] = {"seconds": t, "pairs_per_s": pairs / t, "gcups": cells / t / 1e9}
    same = all(torch.equal(a, b) for a, b in zip(outs_b, outs_p))
    tuning = gbd.gbd_batch_tuning(ctx.handle)
    out = {"workload": f"{len(samples)} samples, read counts {min(s.n for s in samples)}-"
                       f"{max(s.n for s in samples)}, lengths U[150,500]",
           "pairs": pairs, "cells": cells, "identical_outputs": bool(same), **res,
           "speedup": res["plain_per_sample"]["seconds"] / res["batched"]["seconds"], "autotuner": tuning}
    if check:
        def got(s, i, j):
            idx = i * samples[s].n - i * (i + 1) // 2 + (j - i - 1)
            return outs_b[s][torch.from_numpy(idx).to(dev)].cpu().numpy().view(np.uint16)
        base = cpu_baseline_batch(samples, got)
        out["spot_check"] = base.pop("check")
        out["cpu_baseline"] = base
    del outs_b, outs_p, sets
    return out


def run_batch_mode(args):
    """64 uneven samples: one gbd_batch call against one gbd_all_pairs call per sample."""
    import torch
    from paper_1803_02272_gb300 import gbd, synth
    dev = torch.device("cuda:0")
    torch.cuda.set_device(0)
    samples = synth.workload_batched(n_samples=args.samples)
    ctx = gbd.Context(0)
    line = {"mode": "batch", **batch_phase(gbd, ctx, samples, dev, args.steps, check=not args.no_cpu_baseline)}
    print(json.dumps(line), flush=True)
    return 0 if line.get("spot_check", {"mismatches": 0})["mismatches"] == 0 and line["identical_outputs"] else 1


def serve_compare(gbd, ctx, ref, ref_rs, dev, n_requests: int, seed: int = 1006, nq_hi: int = 4096):
    """Served against plain: the same requests as one gbd_tile per request back to back
    (each after its own gbd_load_reads), then all at once through a server."""
    import torch
    from paper_1803_02272_gb300 import synth
    reqs = synth.workload_served_queries(n_requests, 1.0, seed=seed, nq_hi=nq_hi)
    total_pairs = sum(r.reads.n for r in reqs) * ref_rs.n
    out = torch.empty((max(r.reads.n for r in reqs), ref_rs.n), dtype=torch.int16, device=dev)
    q0 = ctx.load(reqs[0].reads)
    ctx.tile(q0, 0, q0.n, ref, 0, ref.n, out=out.view(-1))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for r in reqs:
        qh = ctx.load(r.reads)
        ctx.tile(qh, 0, qh.n, ref, 0, ref.n, out=out.view(-1))
    torch.cuda.synchronize()
    plain_pps = total_pairs / (time.perf_counter() - t0)
    del out
    burst = serve_phase(gbd, ctx, ref, ref_rs, dev, n_requests, seed=seed, check=True, burst=True, nq_hi=nq_hi)
    return {"requests": len(reqs), "queries_per_request": f"log-U[1,{nq_hi}]",
            "plain_sequential_pairs_per_s": plain_pps, "server_burst": burst,
            "server_vs_plain": burst["pairs_per_s"] / plain_pps}


def run_serve_mode(args):
    """Served queries against a resident paper-scale reference: burst throughput of the
    server against plain sequential per-request rectangles, then latency under load."""
    import torch
    from paper_1803_02272_gb300 import gbd, synth
    dev = torch.device("cuda:0")
    torch.cuda.set_device(0)
    ref_rs = synth.workload_paper_scale(n=args.n)
    ctx = gbd.Context(0)
    ref = ctx.load(ref_rs)
    cmp_big = serve_compare(gbd, ctx, ref, ref_rs, dev, args.compare_requests, seed=1006)
    burst = cmp_big["server_burst"]
    loads = {}
    for load in (0.5, 0.8, 0.95):
        loads[str(load)] = serve_phase(gbd, ctx, ref, ref_rs, dev, args.serve_requests, load=load,
                                       capacity_pps=burst["pairs_per_s"], seed=1005)
    # many small requests (1-16 reads each): per-request launch and set-up costs dominate a
    # plain loop, and the server folds concurrent requests into shared launches
    cmp_small = serve_compare(gbd, ctx, ref, ref_rs, dev, args.small_requests, seed=1007, nq_hi=16)
    line = {"mode": "serve", "reference_reads": ref_rs.n, "requests": args.serve_requests,
            "plain_sequential_pairs_per_s": cmp_big["plain_sequential_pairs_per_s"], "server_burst": burst,
            "server_under_load": loads, "server_vs_plain": cmp_big["server_vs_plain"],
            "small_requests": cmp_small}
    print(json.dumps(line), flush=True)
    return 0


def run_mds_mode(args):
    """Classical MDS (sections 3 and 6.2) of the paper-scale distance triangle: gbd_mds timed per
    call, the tensor-core G X product timed alone for its HBM roofline."""
    import torch
    from paper_1803_02272_gb300 import gbd, synth
    dev = torch.device("cuda:0")
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    n, k, r, q = args.n, args.mds_k, args.mds_r, args.mds_q
    rs = synth.workload_paper_scale(n=n, len_lo=args.len_lo, len_hi=args.len_hi)
    ctx = gbd.Context(0)
    s_h = ctx.load(rs)
    t0 = time.perf_counter()
    tri = ctx.all_pairs(s_h)
    torch.cuda.synchronize()
    allpairs_s = time.perf_counter() - t0
    omega = torch.from_numpy(synth.Stream(1003, 9).normal((n, k)).astype(np.float32)).to(dev)
    lam = torch.empty(r, dtype=torch.float32, device=dev)
    X = torch.empty((n, r), dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def ev():
        return torch.cuda.Event(enable_timing=True)

    for _ in range(args.warmup):
        gbd.gbd_mds(ctx.handle, tri, n, omega, k, r, q, lam, X, stream)
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    launches0 = gbd.gbd_kernel_launches()
    times = []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = ev(), ev()
        e0.record(stream)
        gbd.gbd_mds(ctx.handle, tri, n, omega, k, r, q, lam, X, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    launches = gbd.gbd_kernel_launches() - launches0

    # the dominant kernel alone: W X on the tensor cores (inside gbd_gram_apply)
    ld = (n + 127) // 128 * 128
    W = torch.empty(ld * ld, dtype=torch.int16, device=dev)
    e0, e1 = ev(), ev()
    e0.record(stream)
    shift = gbd.gbd_sqdist_square(ctx.handle, tri, n, W, ld, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    square_s = e0.elapsed_time(e1) / 1e3
    Y = torch.empty((n, k), dtype=torch.float32, device=dev)
    for _ in range(3):
        gbd.gbd_gram_apply(ctx.handle, W, n, ld, shift, omega, k, Y, stream)
    prod = []
    for _ in range(5):
        flush.zero_()
        e0, e1 = ev(), ev()
        e0.record(stream)
        gbd.gbd_gram_apply(ctx.handle, W, n, ld, shift, omega, k, Y, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        prod.append(e0.elapsed_time(e1) / 1e3)
    clocks = sampler.stop()
    prod_s = float(np.mean(prod))
    prod_bytes = ld * ld * 2 + k * ld * 2 + n * k * 4 * 2
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    hbm = float(peaks["hbm_gbs"])

    # properties of this very output (any size): sorted eigenvalues, centred and
    # mutually orthogonal coordinate columns with squared norms equal to the eigenvalues
    lam_h = lam.cpu().numpy().astype(np.float64)
    Xh = X.cpu().numpy().astype(np.float64)
    xtx = Xh.T @ Xh
    pos = lam_h > 1e-6 * lam_h[0]
    props = {"sorted": bool(np.all(np.diff(lam_h) <= 0)),
             "max_rel_norm_err": float(np.max(np.abs(np.diag(xtx)[pos] - lam_h[pos]) / lam_h[pos])),
             "max_rel_offdiag": float(np.abs(xtx - np.diag(np.diag(xtx))).max() / lam_h[0]),
             "max_rel_colsum": float(np.abs(Xh.sum(0)).max() / np.sqrt(lam_h[0] * n))}
    del W, Y

    # end to end through the C ABI with host buffers: triangle in from pinned host memory,
    # eigenvalues and coordinates back
    tri_h = torch.empty(tri.numel(), dtype=torch.int16, pin_memory=True)
    tri_h.copy_(tri)
    tri_d = torch.empty_like(tri)
    X_h = torch.empty((n, r), dtype=torch.float32, pin_memory=True)
    lam_hh = torch.empty(r, dtype=torch.float32, pin_memory=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tri_d.copy_(tri_h, non_blocking=True)
    gbd.gbd_mds(ctx.handle, tri_d, n, omega, k, r, q, lam, X, stream)
    X_h.copy_(X, non_blocking=True)
    lam_hh.copy_(lam, non_blocking=True)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0

    t_mds = float(np.mean(times))
    line = {
        "metric": f"classical MDS time, n={n} reads, r={r} (randomized SVD, k={k}, q={q})",
        "value": t_mds, "unit": "s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_mds * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "fp16 products, f32/f64 accumulation", "data": "synthetic",
        "config": {"workload": f"classical MDS (sections 3, 6.2) of the all-pairs SW distance triangle "
                               f"of {n} paper-scale synthetic reads", "n_reads": n, "k": k, "r": r,
                   "q": q, "square_bytes": ld * ld * 2,
                   "l2": "fp16 square (20 GB at n=1e5) far larger than L2; 512 MiB flush between steps"},
        "roofline": {"bound": "hbm", "achieved": prod_bytes / prod_s / 1e9, "peak": hbm, "unit": "GB/s",
                     "frac": prod_bytes / prod_s / 1e9 / hbm, "traffic": None,
                     "kernel": "w_times_x_kernel (tcgen05 + TMA), timed with the rest of one G X call",
                     "peak_source": "of measured: MEASURED_PEAKS hbm_gbs (copy)"},
        "g_times_x_ms": prod_s * 1e3, "sqdist_square_ms": square_s * 1e3,
        "sqdist_square_gbs": (n * (n - 1) + ld * ld * 2) / square_s / 1e9,
        "allpairs_input_s": allpairs_s, "clocks": clocks, "gpu_launches": int(launches // max(args.steps, 1)),
        "properties": props,
        "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": int(tri.numel() * 2),
                "d2h_bytes_per_step": int(n * r * 4 + r * 4)},
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_mds(n, k, r, q)
    print(json.dumps(line), flush=True)
    return 0


def run_components_mode(args):
    """Threshold-graph components (section 5) of the paper-scale triangle: the streaming
    pass over a computed triangle timed alone (HBM roofline), then the whole pipeline from
    host reads to host labels."""
    import torch
    from paper_1803_02272_gb300 import gbd, synth
    dev = torch.device("cuda:0")
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    if "/" in args.th:
        num, den = (int(x) for x in args.th.split("/"))
        th = gbd.threshold(num, den, 65535)
    else:
        th = gbd.threshold(1, 1, int(args.th))
    rs = synth.workload_paper_scale(n=args.n, len_lo=args.len_lo, len_hi=args.len_hi)
    n = rs.n
    m = n * (n - 1) // 2
    ctx = gbd.Context(0)
    s_h = ctx.load(rs)
    tri = ctx.all_pairs(s_h)
    labels = torch.empty(n, dtype=torch.int32, device=dev)
    edges = torch.empty(1, dtype=torch.int64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        gbd.gbd_tri_components(ctx.handle, s_h.handle, tri, th, labels, edges, stream)
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    launches0 = gbd.gbd_kernel_launches()
    times = []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        gbd.gbd_tri_components(ctx.handle, s_h.handle, tri, th, labels, edges, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    launches = (gbd.gbd_kernel_launches() - launches0) // max(args.steps, 1)
    clocks = sampler.stop()
    t = float(np.mean(times))
    lab = labels.cpu().numpy().astype(np.int64)
    ne = int(edges.cpu().numpy()[0])
    # sampled check against the oracle (the cpu_baseline leg): every sampled hit pair
    # shares a component; labels are roots (label[label[i]] == label[i] <= i)
    rng = np.random.default_rng(5)
    i = rng.integers(0, n - 1, size=3000)
    j = i + 1 + (rng.random(3000) * (n - 1 - i)).astype(np.int64)
    base = cpu_baseline_components(rs, i, j, th, lab)
    check = base.pop("check")
    # whole pipeline through the C ABI with host buffers: reads in, labels out
    seq_h = torch.from_numpy(rs.seq).pin_memory()
    off_h = torch.from_numpy(rs.offsets.view(np.int64)).pin_memory()
    lab_h = torch.empty(n, dtype=torch.int32, pin_memory=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sh = gbd.gbd_load_reads(ctx.handle, seq_h, off_h, n, stream)
    gbd.gbd_threshold_components(ctx.handle, sh, th, labels, edges, None, stream)
    lab_h.copy_(labels, non_blocking=True)
    torch.cuda.synchronize()
    e2e = time.perf_counter() - t0
    gbd.gbd_free_set(sh)
    bytes_alg = m * 2 + n * 2 + n * 4 * 3
    hbm = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    line = {"metric": f"threshold-graph components of the n={n} triangle, rule {args.th}",
            "value": t, "unit": "s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "u16 distances, u32 labels", "data": "synthetic",
            "config": {"workload": f"threshold graph (section 5) over the all-pairs triangle of {n} "
                                   "paper-scale synthetic reads", "n_reads": n, "pairs": m,
                       "rule": "d*den <= num*max(la,lb)" if "/" in args.th else "d <= theta",
                       "l2": "10 GB triangle, larger than L2; 512 MiB flush between steps"},
            "roofline": {"bound": "hbm", "achieved": bytes_alg / t / 1e9, "peak": hbm, "unit": "GB/s",
                         "frac": bytes_alg / t / 1e9 / hbm, "traffic": None,
                         "kernel": "span_epilogue_kernel, triangle layout, with hit_bound, hook, union and flatten (one gbd_tri_components call)",
                         "peak_source": "of measured: MEASURED_PEAKS hbm_gbs (copy)"},
            "components": int(len(np.unique(lab))), "edges": ne, "clocks": clocks,
            "gpu_launches": int(launches), "spot_check": check, "cpu_baseline": base,
            "e2e": {"value": e2e, "unit": "s", "h2d_bytes_per_step": int(rs.seq.nbytes + rs.offsets.nbytes),
                    "d2h_bytes_per_step": int(n * 4), "note": "load + all-pairs + components, host labels"}}
    print(json.dumps(line), flush=True)
    return 0


# Affine recurrence (gap extension 1) on the systolic kernel, per int16x2 pair of cells:
# the horizontal and vertical gap states (one add-max each), the cell (an add-max against
# the floor and a 3-way max) and half a 3-way max for the running maximum.
AFFINE_OPS_PER_CELL_PAIR = 4.5


def run_affine_mode(args):
    """Affine-gap scoring (Gotoh; open --gap-open, extend 1) on the systolic kernel: all
    pairs of a read set, exact against the oracle on sampled pairs."""
    import torch
    from paper_1803_02272_gb300 import gbd, synth
    dev = torch.device("cuda:0")
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    n = args.n
    rs = synth.workload_paper_scale(n=n, len_lo=args.len_lo, len_hi=args.len_hi)
    m = n * (n - 1) // 2
    cells = float(rs.total_cells())
    ctx = gbd.Context(0, gap_open=args.gap_open)
    s_h = ctx.load(rs)
    tri = torch.empty(m, dtype=torch.int16, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        gbd.gbd_all_pairs(ctx.handle, s_h.handle, tri, m, stream)
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    launches0 = gbd.gbd_kernel_launches()
    times = []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        gbd.gbd_all_pairs(ctx.handle, s_h.handle, tri, m, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    launches = (gbd.gbd_kernel_launches() - launches0) // max(args.steps, 1)
    clocks = sampler.stop()
    # 400 sampled pairs against the oracle's Gotoh mode (the cpu_baseline leg)
    rng = np.random.default_rng(11)
    i = rng.integers(0, n - 1, size=400)
    j = i + 1 + (rng.random(400) * (n - 1 - i)).astype(np.int64)
    idx = i * n - i * (i + 1) // 2 + (j - i - 1)
    got = tri[torch.from_numpy(idx).to(dev)].cpu().numpy().view(np.uint16)
    base = cpu_baseline_pairs(rs, i, j, got=got, gap_open=args.gap_open, what="pairs with affine gaps")
    check = base.pop("check")
    t = float(np.mean(times))
    rate = max(gbd.gbd_probe_op_rate(gbd.PROBE_OPS.index(nm), 20000, stream)
               for nm in ("VIMAX3_S16X2", "VIADDMAX_S16X2"))
    peak = rate * 2 / AFFINE_OPS_PER_CELL_PAIR / 1e9
    line = {"metric": f"GCUPS, all-pairs n={n}, affine gaps (open {args.gap_open}, extend 1), exact",
            "value": cells / t / 1e9, "unit": "GCUPS", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int16x2", "data": "synthetic", "config": workload_config(rs),
            "roofline": {"bound": "alu", "achieved": cells / t / 1e9, "peak": peak, "unit": "GCUPS",
                         "frac": cells / t / 1e9 / peak, "traffic": None,
                         "peak_source": "of measured: ALU-pipe issue rate (probe) x 2 cells / 4.5 ops "
                                        "(E, F and H add-max, 3-way max, half a 3-way max for the running max)"},
            "clocks": clocks, "gpu_launches": int(launches),
            "spot_check": check, "cpu_baseline": base,
            "e2e": None}
    print(json.dumps(line), flush=True)
    return 0


def run_annotate_mode(args):
    """Section 4.3 annotation: 4,096 sample reads against the 10^5-read reference with a
    species label per reference read (its ancestor); the rectangle is computed, then the
    homology-gap epilogue streams over it (hit list and row labels), timed alone."""
    import torch
    from paper_1803_02272_gb300 import gbd, synth
    dev = torch.device("cuda:0")
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    anc = synth.paper_scale_ancestors()
    ref, ref_lab = synth.reads_from_ancestors(synth.Stream(1003, 77), anc, args.n, args.len_lo, args.len_hi,
                                              0.05, 0.015, return_parents=True)
    qs = synth.reads_from_ancestors(synth.Stream(1003, 78), anc, 4096, args.len_lo, args.len_hi, 0.05, 0.015)
    th = gbd.threshold(*(int(x) for x in args.th.split("/")), 65535) if "/" in args.th else gbd.threshold(1, 1, int(args.th))
    ctx = gbd.Context(0)
    A, B = ctx.load(qs), ctx.load(ref)
    nq, nr = qs.n, ref.n
    rect = torch.empty(nq * nr, dtype=torch.int16, device=dev)
    ctx.tile(A, 0, nq, B, 0, nr, out=rect)
    cap = 1 << 24
    hits = torch.empty(3 * cap, dtype=torch.int32, device=dev)
    count = torch.empty(1, dtype=torch.int64, device=dev)
    labels = torch.from_numpy(ref_lab).to(dev)
    rows = torch.empty(nq, dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    # the epilogue alone, over the computed rectangle (gbd_rect_hits)
    def call():
        gbd.gbd_rect_hits(ctx.handle, A.handle, 0, nq, B.handle, 0, nr, rect, nr, th, hits, cap, count,
                          labels, rows, stream)
    for _ in range(args.warmup):
        call()
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    t_call = []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        call()
        e1.record(stream)
        torch.cuda.synchronize()
        t_call.append(e0.elapsed_time(e1) / 1e3)
    clocks = sampler.stop()
    tc = float(np.mean(t_call))
    t_ep = tc
    # the whole annotation from host reads: rectangle + epilogue, labels back to the host
    lab_h = torch.empty(nq, dtype=torch.int32, pin_memory=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    gbd.gbd_tile_hits(ctx.handle, A.handle, 0, nq, B.handle, 0, nr, th, None, 0, hits, cap, count, labels, rows,
                      stream)
    lab_h.copy_(rows, non_blocking=True)
    torch.cuda.synchronize()
    tt = time.perf_counter() - t0
    n_hits = int(count.cpu().numpy()[0])
    lab = rows.cpu().numpy()
    # sampled rows against the oracle's annotation (the cpu_baseline leg)
    sel = np.arange(0, nq, 256)
    base = cpu_baseline_annotate(qs.subset(sel), ref, ref_lab, th, lab[sel])
    check = base.pop("check")
    bytes_alg = nq * nr * 2 + nr * 6
    hbm = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    line = {"metric": f"homology-gap annotation of {nq} reads against {nr} labelled references, rule {args.th}",
            "value": tc, "unit": "s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": tc * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "u16 distances", "data": "synthetic",
            "config": {"workload": f"section 4.3 annotation: {nq} sample reads vs {nr} references labelled by "
                                   "ancestor (200 species)", "pairs": nq * nr},
            "roofline": {"bound": "hbm", "achieved": bytes_alg / t_ep / 1e9, "peak": hbm, "unit": "GB/s",
                         "frac": bytes_alg / t_ep / 1e9 / hbm, "traffic": None,
                         "kernel": "span_epilogue_kernel, rectangle layout (one gbd_rect_hits call)",
                         "peak_source": "of measured: MEASURED_PEAKS hbm_gbs (copy)"},
            "epilogue_ms": t_ep * 1e3, "hits": n_hits,
            "assigned": int((lab >= 0).sum()), "ambiguous": int((lab == -2).sum()), "unassigned": int((lab == -1).sum()),
            "spot_check": check, "cpu_baseline": base,
            "clocks": clocks,
            "e2e": {"value": tt, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": int(nq * 4),
                    "note": "gbd_tile_hits: rectangle + epilogue on resident sets, labels to pinned host memory"}}
    print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "batch":
        return run_batch_mode(args)
    if args.mode == "serve":
        return run_serve_mode(args)
    if args.mode == "mds":
        return run_mds_mode(args)
    if args.mode == "components":
        return run_components_mode(args)
    if args.mode == "affine":
        return run_affine_mode(args)
    if args.mode == "annotate":
        return run_annotate_mode(args)
    return run_gbd(args)


if __name__ == "__main__":
    sys.exit(main())
