"""Autotuner for the locator and kernel launch options.

Sweeps the brick edge (4 or 8 cells), the brick-hash load factor and the
block size of the cell-parallel kernels on a data set, timing one full
extraction (locator, dual cells, one iso-value) with CUDA events, and caches
the fastest choice per (GPU name, log2 of the cell count, number of levels)
in a JSON file. The level probe order of Sec. 3.2 ("test the likely level
first") needs no tuning here: the locator resolves every brick's neighbour
levels once, so each snap is a single read.
"""
from __future__ import annotations

import itertools
import json
import math
import os

import torch

from . import amriso

DEFAULT = {"log2_brick": 3, "load_factor": 0.5, "block_size": 256}
SPACE = {"log2_brick": (2, 3), "load_factor": (0.25, 0.5, 0.7), "block_size": (128, 256, 512)}
CACHE_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tune_cache.json")


def bucket_key(n_cells: int, levels: int, gpu: str) -> str:
    return f"{gpu}|n2^{int(math.log2(max(n_cells, 1)))}|L{int(levels)}"


def load_cache(path: str = CACHE_PATH) -> dict:
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {}


def save_cache(cache: dict, path: str = CACHE_PATH):
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def best_options(n_cells: int, levels: int, gpu: str | None = None, path: str = CACHE_PATH) -> dict:
    """Cached choice for this size bucket (nearest bucket on the same GPU and
    level count), else the defaults."""
    gpu = gpu or (torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu")
    cache = load_cache(path)
    key = bucket_key(n_cells, levels, gpu)
    if key in cache:
        return dict(cache[key]["best"])
    same = [(abs(int(k.split("|")[1][3:]) - int(math.log2(max(n_cells, 1)))), v)
            for k, v in cache.items() if k.startswith(gpu + "|") and k.endswith(f"|L{int(levels)}")]
    if same:
        return dict(min(same, key=lambda t: t[0])[1]["best"])
    return dict(DEFAULT)


def time_options(xyz, lvl, s, iso: float, opts: dict, reps: int = 3) -> float:
    """Median ms of upload + locator + dual cells + one iso-value."""
    ctx = amriso.AmrContext()
    try:
        out = torch.empty((1, 3, 3), dtype=torch.float32, device="cuda")
        ctx.upload(xyz, lvl, s)
        ctx.build_locator(**opts)
        ctx.dual_cells()
        n = ctx.iso_count(iso, out)
        out = torch.empty((max(n, 1), 3, 3), dtype=torch.float32, device="cuda")
        times = []
        st = torch.cuda.current_stream()
        for _ in range(reps + 1):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            ctx.upload(xyz, lvl, s)
            ctx.build_locator(**opts)
            ctx.dual_cells()
            ctx.iso_count(iso, out)
            b.record(st)
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b))
    finally:
        ctx.close()
    times = sorted(times[1:])
    return times[len(times) // 2]


def tune(xyz, lvl, s, iso: float, space: dict | None = None, reps: int = 3, path: str | None = CACHE_PATH,
         levels: int | None = None) -> dict:
    """Sweep the option space on this data set; returns {"best", "table"} and
    records the result in the cache (path=None: do not record)."""
    space = space or SPACE
    names = list(space)
    table = []
    for combo in itertools.product(*(space[k] for k in names)):
        opts = dict(zip(names, combo))
        try:
            ms = time_options(xyz, lvl, s, iso, opts, reps)
        except amriso.AmrError as e:   # e.g. a slot count past the limits at small bricks
            table.append({**opts, "ms": None, "error": str(e)})
            continue
        table.append({**opts, "ms": ms})
    ok = [r for r in table if r["ms"] is not None]
    if not ok:
        raise RuntimeError(f"tune: no option set could run on this data set ({table[0]['error']})")
    best = min(ok, key=lambda r: r["ms"])
    result = {"best": {k: best[k] for k in names}, "best_ms": best["ms"], "table": table}
    if path is not None:
        lv = int(levels if levels is not None else int(lvl.max()) + 1)
        cache = load_cache(path)
        cache[bucket_key(int(xyz.shape[0]), lv, torch.cuda.get_device_name())] = result
        save_cache(cache, path)
    return result


def _main():
    import argparse
    from . import synth
    ap = argparse.ArgumentParser(description="tune the locator options on a synthetic workload")
    ap.add_argument("--workload", default="octree", choices=["octree", "block", "wing", "sphere"])
    ap.add_argument("--reps", type=int, default=3)
    args = ap.parse_args()
    gen = {"octree": synth.octree_gaussians, "block": synth.block_vortex, "wing": synth.wing_bands,
           "sphere": synth.sphere_tiny}[args.workload]
    x, l, s, iso, info = gen(device="cuda")
    r = tune(x, l, s, iso, reps=args.reps)
    print(json.dumps({"workload": args.workload, "n": info["n"], **r}))


if __name__ == "__main__":
    _main()
