#!/usr/bin/env python3
"""Benchmark of the AMR dual-mesh + iso-surface hot path on one B300.

One step = the whole path over one data set resident in HBM:
  amr_upload (device arrays) -> amr_build_locator -> amr_dual_cells -> amr_iso
(--fused-iso uses amr_dual_cells_iso, the one-pass form, instead).
Prints one JSON line (rank 0). `value` = dual cells per second of step time;
triangles/s, per-stage rates, the dominant kernel's roofline (live CUDA
events, algorithmic bytes / launch time / measured HBM copy peak), an
end-to-end figure through the C ABI with host buffers, SM clocks sampled
during the timed region and the CPU oracle timed on a bounded sample are
added to the same line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload wing|octree|block|sphere]
  python bench.py --impl reference ...   (the CPU oracle as the reference arm)
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2004_08475_b300 import synth  # noqa: E402

METRIC = "dual cells/s + triangles/s (1 B300, % HBM roofline); served p50/p99 latency"

WORKLOADS = {
    "wing": ("wing_bands: Exajet-sized AMR, widths 1-8 in distance bands around a swept wing, "
             "holes in the solid, log-normal scalar (sigma 2)", lambda dev: synth.wing_bands(device=dev)),
    "octree": ("octree_gaussians: 512^3 octree AMR, widths 1-16, |grad f| w refinement, "
               "iso = 60th percentile", lambda dev: synth.octree_gaussians(device=dev)),
    "block": ("block_vortex: 8^3-cell blocks, widths 1-8, 4096x2048x2048, 5% holes, |curl| of "
              "vortex rings", lambda dev: synth.block_vortex(device=dev)),
    "sphere": ("sphere_tiny: 32^3, 2 levels, distance field, iso 8", lambda dev: synth.sphere_tiny(device=dev)),
    # an eighth of the wing workload (inputs still far larger than L2): the
    # stand-in on which ncu captures of the wing's kernels are taken
    "wing_eighth": ("wing_bands at half the root grid per axis (profiling stand-in)",
                    lambda dev: synth.wing_bands(device=dev, dims=(224, 224, 48), scale=0.5)),
    # 9.5M cells (80 % finest level, like the full wing's 86 %), about 1 GB
    # on the device: the stand-in for multi-pass ncu captures
    "wing_small": ("wing_bands at a quarter of the root grid per axis (profiling stand-in)",
                   lambda dev: synth.wing_bands(device=dev, dims=(112, 112, 24), scale=0.25)),
}


def algorithmic_bytes(kernel: str, n: int, n_slots: int, nd: int, nt: int, placement: int = 0,
                      log2_brick: int = 3) -> float:
    """Compulsory bytes per launch of each kernel under the library's data
    layout: what the kernel must read and write at least once. placement 1
    (binned): the insert pass records each cell's 4-byte table code and the
    coarse binning reads it instead of the cell's corner and level."""
    coded = placement == 1
    b3 = 512.0 if log2_brick == 3 else 64.0
    return {
        "k_insert_bricks": 13.0 * n + (4.0 * n if coded else 0.0),   # xyz + level (+ code)
        "k_scatter_cells": 17.0 * n + 8.0 * n,       # read the cell, write id + scalar
        "k_bin_coarse": 8.0 * n + 12.0 * n,          # read code + scalar, write a 12-byte entry
        "k_bin_fine": 12.0 * n + 12.0 * n,           # re-split the entries by window
        "k_place_windows": 12.0 * n + 16.0 * n_slots,  # read the entries, write record + view + scalar per slot
        "k_resolve_views": 16.0 * n_slots,           # read the record, write view + scalar
        "k_resolve_empty": 4.0 * (n_slots - n),      # the empty slots' views (at least)
        "k_order_count": 16.0 * n_slots / b3,        # read each brick's record
        "k_order_scan": 8.0 * 32768,                 # read and write the bucket counters
        "k_order_scatter": 20.0 * n_slots / b3,      # read each brick's record, write its position
        "k_dual_cells": 4.0 * n_slots + 32.0 * nd,   # read views once, write 8 slots / dual
        "k_mc": 32.0 * nd + 4.0 * n + 36.0 * nt,     # read tuples + scalars, write triangles
        # read views + scalars once, write the dual list and the triangles
        "k_dual_cells_iso": 8.0 * n_slots + 32.0 * nd + 36.0 * nt,
    }.get(kernel, 0.0)


def paper_bytes(stage: str, n: int, nd: int, nt: int) -> float:
    """The method's irreducible bytes per stage (the scope table's byte
    model, independent of this implementation's layout): locator 13 B per
    cell read (corner, level) + 12 B written (key, ID); dual pass 13 + 12 B
    per cell + 32 B per dual; Marching Cubes 32 B per dual + 17 B per cell
    (corner, level, scalar once) + 36 B per triangle. Staging passes, table
    slack and re-reads are implementation overhead and not counted."""
    return {
        "locator": 25.0 * n,
        "dual": 25.0 * n + 32.0 * nd,
        "mc": 32.0 * nd + 17.0 * n + 36.0 * nt,
        "step": 67.0 * n + 64.0 * nd + 36.0 * nt,
    }[stage]


# kernels whose work is exactly one stage of the method
PAPER_STAGE = {"k_mc": "mc", "k_dual_cells": "dual"}
LOCATOR_KERNELS = ("k_insert_bricks", "k_scatter_cells", "k_bin_coarse", "k_bin_fine", "k_place_windows",
                   "k_resolve_views", "k_resolve_empty", "k_brick_neighbors", "k_order_count", "k_order_scan",
                   "k_order_scatter")


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in ("kernels.cu", "kernels.h", "order.cu", "order.h"):
        with open(os.path.join(ROOT, "paper_2004_08475_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, workload: str, units: float):
    """DRAM bytes per launch from the committed ncu summary, scaled by units
    processed; None when absent or taken on another version of the kernels."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(f"{kernel}:{workload}")
    if not e or e.get("source_hash") != kernel_source_hash():
        return None
    return float(e["dram_bytes_per_unit"]) * units


class ClockSampler:
    """nvidia-smi SM clock / throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows]
        mx = max(float(r[2]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows)}


def reduce_over_ranks(ms: float, nd: int, nt: int, dist, device) -> tuple:
    """Max step time over ranks and summed dual / triangle counts (the
    replicas share no data; only the timing and totals are combined)."""
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    tot = torch.tensor([float(nd), float(nt)], dtype=torch.float64, device=device)
    dist.all_reduce(tot)
    nd_all, nt_all = tot.tolist()
    return float(t.item()), nd_all, nt_all


# ---------------------------------------------------------------------------
# CPU oracle leg (bounded sample)
# ---------------------------------------------------------------------------

def _in_box(xyz, c, half):
    """Indices (increasing) of the rows of int32 xyz with |xyz - c| <= half on
    every axis, one axis at a time on the surviving rows (no int64 copy of
    the whole array)."""
    idx = None
    for a in range(3):
        lo_a = max(int(np.ceil(c[a] - half[a])), -2 ** 31)
        hi_a = min(int(np.floor(c[a] + half[a])), 2 ** 31 - 1)
        col = xyz[:, a] if idx is None else xyz[idx, a]
        sel = (col >= lo_a) & (col <= hi_a)
        idx = np.flatnonzero(sel) if idx is None else idx[sel]
    return idx


def oracle_window(xyz, lv, s, target_cells: int, seed: int = 0, sub_max: int = 4_000_000):
    """Cells inside a box around a finest-level cell holding about
    `target_cells` cells (numpy arrays in, numpy arrays out, input order).
    The box is sized on a random subsample of at most `sub_max` cells, then
    cut from all cells in one pass (corrected if the estimate missed)."""
    n = xyz.shape[0]
    if n == 0:
        return xyz, lv, s
    rng = np.random.default_rng(seed)
    # drawn with replacement: count / f estimates the box's cell count
    xs = xyz[rng.integers(0, n, size=sub_max)] if n > sub_max else xyz
    lo, hi = xs.min(0).astype(np.int64), xs.max(0).astype(np.int64) + 1
    lmin = lv.min()
    c = None
    for _ in range(1000):            # a random finest-level cell (rejection sampling)
        i = int(rng.integers(0, n))
        if lv[i] == lmin:
            c = xyz[i].astype(np.int64)
            break
    if c is None:
        fine = np.flatnonzero(lv == lmin)
        c = xyz[fine[rng.integers(0, fine.shape[0])]].astype(np.int64)
    t = float(target_cells)
    half = np.maximum((hi - lo) * min(1.0, t / n) ** (1 / 3) / 2, 1)
    if n > sub_max:
        f = xs.shape[0] / n
        for _ in range(40):
            k = _in_box(xs, c, half).shape[0] / f
            if 0.8 * t <= k <= 1.25 * t:
                break
            half = half * (t / max(k, 1.0)) ** (1 / 3)
    idx = _in_box(xyz, c, half)
    for _ in range(40):
        k = int(idx.shape[0])
        if 0.8 * t <= k <= 1.25 * t or k == n:
            break
        half = half * (t / max(k, 1)) ** (1 / 3)
        idx = _in_box(xyz, c, half)
    return xyz[idx], lv[idx], s[idx]


def _pool_warmup(_):
    time.sleep(0.2)
    import oracle  # noqa: F401  (loads the oracle's library in the worker)
    return os.getpid()


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def oracle_pool(processes: int):
    """A started spawn pool of `processes` workers for the sharded oracle, or
    None (one process) when processes <= 1 or a pool cannot be had."""
    if processes <= 1:
        return None
    try:
        from oracle import shard
        pool = shard.spawn_pool(processes)
        list(pool.map(_pool_warmup, range(2 * processes)))   # workers up before any timing
        return pool
    except Exception as e:  # the one-process oracle is still the oracle
        print(f"[bench] oracle process pool unavailable ({e}); timing one process", file=sys.stderr)
        return None


def run_oracle_once(wx, wl, ws, iso, pool=None, processes: int = 1):
    """One run of the oracle (cell set + duals + MC) over a sample of cells.
    With a pool the sample is cut into `processes` x slabs of equal cell
    counts, each with a halo of the widest cell, run side by side
    (oracle.shard: the same duals and triangles as one process). Returns
    counts, wall seconds, summed per-process oracle seconds and cores; a pool
    failure raises."""
    import oracle
    from oracle import shard
    t0 = time.perf_counter()
    if pool is not None and processes > 1:
        o = shard.run_sharded(wx, wl, ws, iso, n_slabs=processes, executor=pool, balance="count",
                              want_keys=False)
        nd, nt, cpu_s, cores = int(o["duals"].shape[0]), int(o["tris"].shape[0]), o["cpu_seconds"], processes
    else:
        m = oracle.OracleMesh(wx, wl)
        d = m.duals()
        r = m.iso(ws, d, iso, want_keys=False)
        nd, nt, cpu_s, cores = int(d.shape[0]), int(r["tris"].shape[0]), None, 1
    dt = time.perf_counter() - t0
    return {"duals": nd, "tris": nt, "cells": int(wx.shape[0]), "seconds": dt,
            "cpu_seconds": dt if cpu_s is None else cpu_s, "cores": cores}


def time_oracle(xyz, lv, s, iso, seconds: float = 15.0, pool=None, processes: int = 1):
    """The oracle on a box of cells grown until one run takes about
    `seconds` / 4 to `seconds` of wall time (on `processes` processes when a
    pool is given); returns the last run (run_oracle_once) plus "window",
    the sample, for further timed runs. A pool that fails is dropped and
    the one-process oracle timed instead ("pool": the pool still in use)."""
    par = pool is not None and processes > 1
    target = 20000 * (processes if par else 1)
    while True:
        win = oracle_window(xyz, lv, s, target)
        try:
            r = run_oracle_once(*win, iso, pool if par else None, processes if par else 1)
        except Exception as e:   # a broken pool: time the one-process oracle instead
            if not par:
                raise
            print(f"[bench] oracle process pool failed ({e}); timing one process", file=sys.stderr)
            par = False
            target = max(20000, target // processes)
            continue
        if r["seconds"] > seconds / 4 or target > 2e7 * (processes if par else 1) or target >= xyz.shape[0]:
            break
        target = int(target * min(8.0, seconds / max(r["seconds"], 1e-3)))
    r["window"] = win
    r["pool"] = pool if par else None
    return r


def oracle_sample_text(r, workload):
    how = (f"cut into {r['cores']} x slabs (halo of the widest cell) on {r['cores']} processes"
           if r["cores"] > 1 else "one process")
    return (f"{r['cells']} cells in a box of the {workload} workload, {how}: {r['duals']} duals, "
            f"{r['tris']} triangles, {r['seconds']:.1f} s wall, {r['cpu_seconds']:.1f} s oracle time summed")


# ---------------------------------------------------------------------------

def run_reference(args, workload_desc, gen):
    """Reference arm: the CPU oracle as it stands, on this run's workload
    (bounded samples), rank 0 only."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = args.cpu_cores or host_cores()
    pool = oracle_pool(cores)
    dev = "cuda" if (torch.cuda.is_available() and args.workload in ("wing", "block")) else "cpu"
    xyz, lv, s, iso, info = gen(dev)
    x, l, v = xyz.cpu().numpy(), lv.cpu().numpy(), s.cpu().numpy()
    # one sample of the workload sized once (untimed), then every step runs it
    per = max(1.0, 60.0 / max(1, args.steps + args.warmup))
    use = pool
    while True:
        cal = time_oracle(x, l, v, iso, seconds=per, pool=use, processes=cores)
        win, use = cal["window"], cal["pool"]
        try:
            for _ in range(args.warmup):
                run_oracle_once(*win, iso, use, cores)
            duals = tris = 0
            secs = 0.0
            r = cal
            for _ in range(args.steps):
                r = run_oracle_once(*win, iso, use, cores)
                duals += r["duals"]
                tris += r["tris"]
                secs += r["seconds"]
            break
        except Exception as e:   # the pool broke after sizing: size and time one process
            if use is None:
                raise
            print(f"[bench] oracle process pool failed ({e}); timing one process", file=sys.stderr)
            use = None
    if pool is not None:
        pool.shutdown()
    cells = r["cells"]
    value = duals / secs
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "dual cells/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * secs / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "description": workload_desc, "n_cells": info["n"],
                   "sample_cells": cells},
        "triangles_per_s": tris / secs,
        "cpu_baseline": {"value": value, "unit": "dual cells/s", "cores": r["cores"], "kind": "oracle",
                         "sample": "per step, the same sample: " + oracle_sample_text(r, args.workload)},
        "e2e": {"value": value, "unit": "dual cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


class ServeBench:
    """The serving workload: 24 data sets of 50k..50M cells cut from the
    octree and block generators, Zipf(1) popularity (unrelated to size),
    requests of 1-16 iso-values (40th-95th percentile of the data set's
    scalar) arriving as a Poisson stream; the continuous-batching server
    against per-request plain extraction (FIFO). The plain path's capacity
    (requests/s, back to back) sets the arrival rates."""

    def __init__(self, slots: int, sample: int, seed: int = 5):
        from paper_2004_08475_b300 import serve
        self.serve = serve
        self.slots = slots
        sets = synth.serving_set(device="cuda")
        self.host = {name: (x.cpu().pin_memory(), l.cpu().pin_memory(), v.cpu().pin_memory())
                     for name, x, l, v, _ in sets}
        self.iso_rng = {name: r for name, _, _, _, r in sets}
        self.names = [t[0] for t in sets]
        self.cells = sum(int(v[0].shape[0]) for v in self.host.values())
        del sets
        torch.cuda.empty_cache()
        self.rng = np.random.default_rng(seed)
        pop = 1.0 / np.arange(1, len(self.names) + 1)
        perm = self.rng.permutation(len(self.names))
        self.prob = np.empty(len(self.names))
        self.prob[perm] = pop / pop.sum()
        reqs = self.make(sample, np.zeros(sample))   # plain capacity: back-to-back service of a sample
        t0 = time.perf_counter()
        for r in reqs:
            r.t_arrival = t0
        serve.serve_plain(self.host, reqs)
        self.cap_plain = len(reqs) / (max(r.t_done for r in reqs) - t0)

    def make(self, nreq, arrivals):
        reqs = []
        for i in range(nreq):
            name = self.names[self.rng.choice(len(self.names), p=self.prob)]
            a, b = self.iso_rng[name]
            isos = list(self.rng.uniform(a, b, size=int(self.rng.integers(1, 17))))
            reqs.append(self.serve.Request(i, name, [float(v) for v in isos], float(arrivals[i])))
        return reqs

    def poisson(self, nreq, load):
        return self.make(nreq, np.cumsum(self.rng.exponential(1.0 / (load * self.cap_plain), size=nreq)))

    def clone(self, reqs):
        return [self.serve.Request(r.rid, r.dataset, list(r.isos), r.t_arrival) for r in reqs]

    def run_server(self, reqs, budget):
        """The server, its data sets preloaded (most popular first) up to the
        budget before the stream starts; requests beyond it evict LRU."""
        srv = self.serve.Server(budget_bytes=budget, slots=self.slots)
        for name, (x, l, v) in self.host.items():
            srv.datasets[name] = self.serve._Dataset(name, x, l, v, {})
        srv.preload([self.names[i] for i in np.argsort(-self.prob)])
        srv.start()
        t_base = time.perf_counter() + 0.05
        for r in reqs:
            r.t_arrival += t_base
        for r in reqs:
            now = time.perf_counter()
            if r.t_arrival > now:
                time.sleep(r.t_arrival - now)
            with srv.cv:
                srv.queue.append(r)
                srv.cv.notify_all()
        for r in reqs:
            r.done.wait()
        stats = dict(srv.stats)
        srv.stop()
        return {**self.serve.latency_summary(reqs), "stats": stats}

    def run_plain(self, reqs):
        t_base = time.perf_counter() + 0.05
        for r in reqs:
            r.t_arrival += t_base
        self.serve.serve_plain(self.host, reqs)
        return self.serve.latency_summary(reqs)

    def config(self):
        return {"workload": "serving: 24 data sets 50k-50M cells (octree / block crops), Zipf(1), Poisson "
                            "arrivals, 1-16 iso-values per request",
                "cells": self.cells, "slots": self.slots, "budget_gb": 120}


def serve_leg(args, gpu_index):
    """The serving measurement carried by the default line: server and plain
    p50/p99 latency and triangles/s at 0.8 of the plain path's capacity, and
    both at saturation (every request waiting at t = 0; throughput =
    triangles / makespan), with the SM clocks sampled meanwhile."""
    sb = ServeBench(args.serve_slots, args.serve_sample)
    with ClockSampler(gpu_index) as clk:
        reqs = sb.poisson(args.serve_line_requests, 0.8)
        at08 = {"requests": len(reqs), "rate_per_s": 0.8 * sb.cap_plain,
                "server": sb.run_server(sb.clone(reqs), 120 << 30), "plain": sb.run_plain(reqs)}
        sat = sb.make(args.serve_saturation_requests, np.zeros(args.serve_saturation_requests))
        satr = {"requests": len(sat), "server": sb.run_server(sb.clone(sat), 120 << 30), "plain": sb.run_plain(sat)}
    return {"config": sb.config(), "plain_capacity_req_per_s": sb.cap_plain, "load_0.8": at08, "saturation": satr,
            "clocks": clk.summary()}


def run_serve(args):
    """--mode serve: the serving workload at 0.5/0.8/0.95 of the plain path's
    capacity, one run under an 8 GB budget (LRU evictions), and saturation."""
    torch.cuda.set_device(0)
    sb = ServeBench(args.serve_slots, args.serve_sample)
    results = {}
    with ClockSampler(0) as clk:
        for load in (0.5, 0.8, 0.95):
            reqs = sb.poisson(args.serve_requests, load)
            results[str(load)] = {"rate_per_s": load * sb.cap_plain,
                                  "server": sb.run_server(sb.clone(reqs), 120 << 30), "plain": sb.run_plain(reqs)}
        results["0.8_budget_8GB"] = {"server": sb.run_server(sb.poisson(args.serve_requests, 0.8), 8 << 30)}
        reqs = sb.make(args.serve_requests, np.zeros(args.serve_requests))
        results["saturation"] = {"server": sb.run_server(sb.clone(reqs), 120 << 30), "plain": sb.run_plain(reqs)}
    line = {"mode": "serve", "metric": METRIC, "unit": "ms (p50/p99 latency), triangles/s",
            "n_gpus": 1, "data": "synthetic", "config": {**sb.config(), "requests_per_load": args.serve_requests},
            "plain_capacity_req_per_s": sb.cap_plain, "loads": results, "clocks": clk.summary(),
            "gpu": torch.cuda.get_device_name(0)}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="wing", choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--log2-brick", type=int, default=3)
    ap.add_argument("--load-factor", type=float, default=0.5)
    ap.add_argument("--partitioned", type=int, default=0)
    ap.add_argument("--fused-iso", action="store_true",
                    help="amr_dual_cells_iso (one pass) instead of amr_dual_cells then amr_iso")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-cores", type=int, default=0,
                    help="processes for the CPU oracle (x slabs side by side); 0 = every core this "
                         "process may use, 1 = the single-process oracle")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-indexed", action="store_true", help="skip the indexed face set measurement")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--batch-isos", type=int, default=16)
    ap.add_argument("--mode", default="step", choices=["step", "serve"])
    ap.add_argument("--serve-requests", type=int, default=600)
    ap.add_argument("--serve-line-requests", type=int, default=2000,
                    help="requests at 0.8 load in the serving object of the default line")
    ap.add_argument("--serve-saturation-requests", type=int, default=1000)
    ap.add_argument("--no-serve", action="store_true", help="leave the serving object out of the default line")
    ap.add_argument("--serve-sample", type=int, default=80)
    ap.add_argument("--serve-slots", type=int, default=3)
    args = ap.parse_args()
    if args.mode == "serve":
        run_serve(args)
        return
    args.warmup = max(args.warmup, 3)
    desc, gen = WORKLOADS[args.workload]

    if args.impl == "reference":
        run_reference(args, desc, gen)
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    from paper_2004_08475_b300 import amriso

    xyz, lv, s, iso, info = gen("cuda")
    n = info["n"]
    stream = torch.cuda.current_stream()
    ctx = amriso.AmrContext(local, stream)
    opts = dict(log2_brick=args.log2_brick, load_factor=args.load_factor, partitioned=args.partitioned)

    def step(tri_buf):
        ctx.upload(xyz, lv, s)
        ctx.build_locator(**opts)
        if not args.fused_iso:
            nd = ctx.dual_cells()
            nt = ctx.iso_count(iso, tri_buf)
        else:
            nd, nt = ctx.dual_cells_iso(iso, tri_buf)
        return nd, nt

    # size the triangle buffer once (exact count), then warm up
    ctx.upload(xyz, lv, s)
    ctx.build_locator(**opts)
    ctx.dual_cells()
    nt0 = ctx.iso_count(iso, torch.empty((1, 3, 3), dtype=torch.float32, device="cuda"))
    tri_buf = torch.empty((max(nt0, 1), 3, 3), dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        step(tri_buf)
    torch.cuda.synchronize()
    ctx.kernel_times()          # discard warm-up timings
    ctx.enable_timing(True)

    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        start.record(stream)
        for _ in range(args.steps):
            nd, nt = step(tri_buf)
        stop.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = start.elapsed_time(stop) / args.steps
    ktimes = ctx.kernel_times()
    ctx.enable_timing(False)
    inf = ctx.info()
    if dist:
        ms, nd_all, nt_all = reduce_over_ranks(ms, nd, nt, dist, "cuda")
    else:
        nd_all, nt_all = float(nd), float(nt)

    kt = {k: v for k, v in ktimes.items() if v[1] > 0}
    t_dual = (kt.get("k_dual_cells", (0, 1))[0] + kt.get("k_dual_cells_iso", (0, 1))[0]) / args.steps
    t_iso = kt.get("k_mc", (0, 1))[0] / args.steps
    # the locator build's share of the step: what the dual and MC kernels leave
    # (its kernels' own event times overlap: neighbours and brick order run on
    # a second stream beside the placement)
    t_loc_kernels = sum(kt.get(k, (0, 0))[0] for k in LOCATOR_KERNELS) / args.steps
    t_loc = max(ms - t_dual - t_iso, 0.0)
    launches = int(sum(v[1] for v in kt.values()))

    # roofline of the dominant kernel
    peak, peak_src = load_peaks()
    total_kms = max(1e-9, sum(v[0] for v in kt.values()))
    kernels = {}
    for k, (tot_ms, cnt) in kt.items():
        per = tot_ms / cnt
        b = algorithmic_bytes(k, n, inf.n_slots, nd, nt, inf.placement, inf.log2_brick)
        kernels[k] = {"ms_per_launch": per, "launches": cnt, "share": tot_ms / total_kms,
                      "algorithmic_bytes": b, "gbs": b / per / 1e6 if per > 0 else 0.0}
    for k, rec in kernels.items():
        if k in PAPER_STAGE:
            pb = paper_bytes(PAPER_STAGE[k], n, nd, nt)
            rec["paper_bytes"] = pb
            rec["paper_gbs"] = pb / rec["ms_per_launch"] / 1e6 if rec["ms_per_launch"] > 0 else 0.0
    # the dominant kernel among those that are one stage of the method each
    # (the locator's stage spans several kernels: reported under "rates")
    staged = [k for k in kernels if k in PAPER_STAGE] or list(kernels)
    dom = max(staged, key=lambda k: kernels[k]["ms_per_launch"] * kernels[k]["launches"])
    dk = kernels[dom]
    units = {"k_insert_bricks": n, "k_scatter_cells": n, "k_bin_coarse": n, "k_bin_fine": n,
             "k_place_windows": inf.n_slots, "k_resolve_views": inf.n_slots,
             "k_dual_cells": inf.n_slots, "k_dual_cells_iso": inf.n_slots, "k_mc": nd}.get(dom, n)
    ach = dk.get("paper_gbs", dk["gbs"])
    roofline = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": ach / peak, "peak_source": peak_src,
                "traffic": ncu_traffic(dom, args.workload, units),
                "algorithmic_bytes_per_launch": dk.get("paper_bytes", dk["algorithmic_bytes"]),
                "bytes_model": "method (32 B/dual + 17 B/cell + 36 B/triangle for k_mc; 25 B/cell + 32 B/dual "
                               "for k_dual_cells)" if dom in PAPER_STAGE else "implementation",
                "impl_model_bytes_per_launch": dk["algorithmic_bytes"],
                "frac_impl_model": dk["gbs"] / peak}
    step_bytes_impl = sum(algorithmic_bytes(k, n, inf.n_slots, nd, nt, inf.placement, inf.log2_brick) * v[1]
                          for k, v in kt.items()) / args.steps
    step_bytes = paper_bytes("step", n, nd, nt)

    # batched multi-iso over the resident dual cells
    batch = None
    if args.batch_isos > 0 and rank == 0:
        # the workload's iso-value times 2^((k-8)/4), k = 0..15: quarter-octave steps around it
        isos = [float(iso * 2.0 ** ((k - args.batch_isos // 2) / 4)) for k in range(args.batch_isos)]
        _, offs = ctx.iso_batch(isos, torch.empty((0, 3, 3), dtype=torch.float32, device="cuda"))
        need = int(offs[-1])
        torch.cuda.empty_cache()
        buf = torch.empty((max(need, 1), 3, 3), dtype=torch.float32, device="cuda")
        ctx.iso_batch(isos, buf)
        torch.cuda.synchronize()
        ctx.kernel_times()
        ctx.enable_timing(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 3
        e0.record(stream)
        for _ in range(reps):
            ctx.iso_batch(isos, buf)
        e1.record(stream)
        torch.cuda.synchronize()
        bt = ctx.kernel_times()
        ctx.enable_timing(False)
        bms = e0.elapsed_time(e1) / reps
        bb = 32.0 * nd + 17.0 * n + 36.0 * need   # method bytes of k iso-values batched
        batch = {"n_iso": len(isos), "isos": "iso * 2^((k-8)/4), k = 0..15", "ms": bms, "triangles": need,
                 "triangles_per_s": need / (bms / 1e3), "ms_per_iso": bms / len(isos),
                 "single_iso_kernel_ms": t_iso, "paper_bytes": bb,
                 "frac_of_peak": bb / (bms / 1e3) / 1e9 / peak,
                 "kernels_ms": {k: v[0] / reps for k, v in bt.items() if v[1]}}
        del buf
        torch.cuda.empty_cache()

    # indexed face set of the step's iso-value (vertices welded by edge key)
    indexed = None
    if not args.no_indexed and rank == 0:
        vtx, tri, _ = ctx.iso_indexed(iso, with_keys=False)   # sizes the library's and our buffers
        nv, ntr = int(vtx.shape[0]), int(tri.shape[0])
        torch.cuda.synchronize()
        ctx.kernel_times()
        ctx.enable_timing(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 3
        vb = torch.empty((nv, 3), dtype=torch.float32, device="cuda")
        tb = torch.empty((ntr, 3), dtype=torch.int32, device="cuda")
        cnv, cnt_ = ctypes.c_int64(0), ctypes.c_int64(0)
        e0.record(stream)
        for _ in range(reps):
            rc = amriso.lib().amr_iso_indexed(ctx._h, ctypes.c_float(iso), vb.data_ptr(), nv, tb.data_ptr(), ntr,
                                              None, ctypes.byref(cnv), ctypes.byref(cnt_), amriso.DEVICE_PTRS)
            assert rc == 0 and cnv.value == nv and cnt_.value == ntr
        e1.record(stream)
        torch.cuda.synchronize()
        it = ctx.kernel_times()
        ctx.enable_timing(False)
        ims = e0.elapsed_time(e1) / reps
        indexed = {"ms": ims, "vertices": nv, "triangles": ntr, "triangles_per_s": ntr / (ims / 1e3),
                   "bytes_fat": 36 * ntr, "bytes_indexed": 12 * nv + 12 * ntr,
                   "kernels_ms": {k: v[0] / reps for k, v in it.items() if v[1]}}
        del vtx, tri, vb, tb
        # a second per-cell field at those vertices (here the scalar itself)
        _, _, vkeys = ctx.iso_indexed(iso, with_keys=True)
        ctx.interpolate(iso, s, vkeys)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            ctx.interpolate(iso, s, vkeys)
        e1.record(stream)
        torch.cuda.synchronize()
        indexed["interpolate_ms"] = e0.elapsed_time(e1) / reps
        del vkeys
        # shapes of the dual cells (distinct cells among the 8 vertices)
        _, hist = ctx.dual_shapes()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            ctx.dual_shapes()
        e1.record(stream)
        torch.cuda.synchronize()
        indexed["dual_shapes"] = {"ms": e0.elapsed_time(e1) / reps,
                                  "histogram_by_distinct_cells": [int(v) for v in hist]}
        torch.cuda.empty_cache()

    # end to end through the C ABI with host buffers (pinned)
    e2e = None
    if not args.no_e2e:
        hx, hl, hs = xyz.cpu().pin_memory(), lv.cpu().pin_memory(), s.cpu().pin_memory()
        hout = torch.empty((max(nt, 1), 3, 3), dtype=torch.float32).pin_memory()
        ectx = amriso.AmrContext(local, stream)

        def e2e_step():
            ectx.upload(hx, hl, hs)
            ectx.build_locator(**opts)
            if not args.fused_iso:
                d = ectx.dual_cells()
                t = ectx.iso_count(iso, hout)
            else:
                d, t = ectx.dual_cells_iso(iso, hout)
            return d, t
        e2e_step()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            d2, t2 = e2e_step()
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / args.e2e_steps
        if dist:
            t = torch.tensor([e2e_s], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_s = float(t.item())
        assert d2 == nd and t2 == nt
        e2e = {"value": nd_all / e2e_s, "unit": "dual cells/s", "h2d_bytes_per_step": int(17 * n),
               "d2h_bytes_per_step": int(36 * nt), "ms_per_step": 1000.0 * e2e_s,
               "triangles_per_s": nt_all / e2e_s}
        ectx.close()
        del hx, hl, hs, hout

    serve_obj = None
    if rank == 0 and world == 1 and not args.no_serve:
        ctx.trim()
        torch.cuda.empty_cache()
        serve_obj = serve_leg(args, local)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        x, l, v = xyz.cpu().numpy(), lv.cpu().numpy(), s.cpu().numpy()
        cores = args.cpu_cores or host_cores()
        pool = oracle_pool(cores)
        r = time_oracle(x, l, v, iso, seconds=15.0, pool=pool, processes=cores)
        if pool is not None:
            pool.shutdown()
        cpu = {"value": r["duals"] / r["seconds"], "unit": "dual cells/s", "cores": r["cores"], "kind": "oracle",
               "sample": oracle_sample_text(r, args.workload)}

    if rank == 0:
        line = {
            "metric": METRIC,
            "value": nd_all / (ms / 1e3),
            "unit": "dual cells/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "description": desc, "n_cells": n,
                       "step": "fused" if args.fused_iso else "dual_cells+iso",
                       "n_dual": nd, "n_triangles": nt, "iso": iso, "n_bricks": inf.n_bricks,
                       "placement": ["direct", "binned"][inf.placement],
                       "n_slots": inf.n_slots, "levels": inf.n_levels, "log2_brick": args.log2_brick,
                       "load_factor": args.load_factor, "parallelism": f"replicas{world}",
                       "l2": f"inputs larger than L2 ({(17 * n) / 1e6:.0f} MB of cells)"},
            "triangles_per_s": nt_all / (ms / 1e3),
            "rates": {"dual_cells_per_s_locator_plus_dual": nd / ((t_loc + t_dual) / 1e3) if t_loc + t_dual else None,
                      "triangles_per_s_iso_kernel": nt / (t_iso / 1e3) if t_iso else None,
                      "step_bytes": step_bytes,
                      "step_algorithmic_gbs": step_bytes / (ms / 1e3) / 1e9,
                      "step_frac_of_peak": step_bytes / (ms / 1e3) / 1e9 / peak,
                      "locator_ms": t_loc, "locator_kernels_ms": t_loc_kernels, "dual_ms": t_dual, "mc_ms": t_iso,
                      "locator_frac_of_peak": (paper_bytes("locator", n, nd, nt) / (t_loc / 1e3) / 1e9 / peak
                                               if t_loc else None),
                      "step_bytes_impl_model": step_bytes_impl,
                      "step_frac_impl_model": step_bytes_impl / (ms / 1e3) / 1e9 / peak},
            "roofline": roofline,
            "kernels": kernels,
            "batched_iso": batch,
            "indexed_face_set": indexed,
            "serve": serve_obj,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clk.summary(),
            "gpu_launches": launches,
            "gpu": torch.cuda.get_device_name(local),
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
