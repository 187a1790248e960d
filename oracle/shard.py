"""Slab + halo sharding of the oracle, and an order-independent fingerprint.

TEST INFRASTRUCTURE ONLY, like the rest of this package: it lets the plain
single-threaded oracle cover data sets of 10^7 cells and more by running
independent x slabs in separate processes, and it compares outputs too large
to sort side by side through a multiset fingerprint.

Why the sharded result is exact (Sec. 4.2-4.4). A dual cell is emitted by
one cell S = (p, l) of width w = 2^l: its 8 query points are q = p + d * w
with d in {-1, 0, 1}^3, and every cell snap() can return for q contains q.
If S's lower corner lies in the slab [x0, x1), every such q has
x0 - w <= q_x < x1 + w, so every cell that contains one of them overlaps
[x0 - w_max, x1 + w_max), w_max the widest cell. A shard that holds every
cell overlapping that interval therefore snaps exactly as the whole data set
does for the owners in its slab, applies rules 1-3 to the same cells and
emits the same tuples; Marching Cubes on those tuples (Sec. 5) reads only
their vertex cells. Keeping the duals whose owner lies in the slab gives each
dual exactly once: the owner is the unique emitting cell (rule 3).

Pins (``tests/test_oracle_shard.py``): the sharded result equals the
unsharded oracle bit for bit for 1 to 13 slabs of either balance, a shard
planted without its halo does not, and the fingerprint's mixing function
reproduces the published splitmix64 outputs.
"""
from __future__ import annotations

import multiprocessing
import os
import time
from concurrent.futures import ProcessPoolExecutor

import numpy as np

GAMMA = 0x9E3779B97F4A7C15


def slab_windows(xyz, level, n_slabs, balance="width"):
    """Partition the cells into ``n_slabs`` x slabs by the x of their lower
    corner: slabs of (almost) equal width, or with ``balance="count"`` of
    (almost) equal cell counts. Returns a list of (owners, window): global
    indices, in increasing order, of the cells whose lower corner lies in
    the slab, and of every cell overlapping the slab grown by the widest cell
    on both sides (owners included). Increasing order keeps the order of
    cell IDs within a shard, so edge keys and the lower-ID-first vertex
    formula come out the same as on the whole data set."""
    x = np.asarray(xyz, dtype=np.int64).reshape(-1, 3)[:, 0]
    w = np.left_shift(np.int64(1), np.asarray(level, dtype=np.int64).reshape(-1))
    if x.shape[0] == 0:
        return [(np.zeros(0, np.int64), np.zeros(0, np.int64)) for _ in range(n_slabs)]
    wmax = int(w.max())
    lo, hi = int(x.min()), int((x + w).max())
    if balance == "count":
        xs = np.sort(x)
        bounds = [lo] + [int(xs[k * x.shape[0] // n_slabs]) for k in range(1, n_slabs)] + [hi]
    else:
        bounds = [lo + (hi - lo) * k // n_slabs for k in range(n_slabs + 1)]
    bounds[-1] = hi
    out = []
    for k in range(n_slabs):
        x0, x1 = bounds[k], bounds[k + 1]
        owners = np.nonzero((x >= x0) & (x < x1))[0]
        window = np.nonzero((x < x1 + wmax) & (x + w > x0 - wmax))[0]
        out.append((owners, window))
    return out


def _one_slab(args):
    """One shard: the oracle on the window's cells, duals kept for the
    slab's owners, Marching Cubes on them. Indices are mapped back to the
    whole data set's cell IDs; "seconds" is the shard's own oracle time."""
    from oracle import OracleMesh
    xw, lw, sw, owners_local, window, iso = args[:6]
    want_keys = args[6] if len(args) > 6 else True
    t0 = time.perf_counter()
    m = OracleMesh(xw, lw)
    d = m.duals(owners=owners_local)
    res = {"duals": window[d] if d.shape[0] else np.zeros((0, 8), np.int64)}
    if iso is not None:
        r = m.iso(sw, d, iso, want_keys=want_keys)
        res.update(cases=r["cases"], ntri=r["ntri"], tris=r["tris"], max_err=r["max_err"])
        if want_keys:
            res["keys"] = window[r["keys"]] if r["keys"].shape[0] else np.zeros((0, 3, 2), np.int64)
    res["seconds"] = time.perf_counter() - t0
    return res


def shard_jobs(xyz, level, scalar, iso, n_slabs, balance="width", want_keys=True):
    """The per-slab arguments of ``_one_slab`` (window arrays copied out)."""
    xyz = np.asarray(xyz, dtype=np.int32).reshape(-1, 3)
    level = np.asarray(level, dtype=np.uint8).reshape(-1)
    s = None if scalar is None else np.asarray(scalar, dtype=np.float32).reshape(-1)
    jobs = []
    for owners, window in slab_windows(xyz, level, n_slabs, balance):
        local = np.searchsorted(window, owners)
        jobs.append((xyz[window], level[window], None if s is None else s[window], local, window,
                     None if iso is None else float(iso), want_keys))
    return jobs


def spawn_pool(processes):
    """A process pool for ``run_sharded`` (``spawn``: safe in a process that
    already holds a CUDA context); an executor, unlike multiprocessing.Pool,
    raises when a worker dies instead of waiting for it."""
    return ProcessPoolExecutor(processes, mp_context=multiprocessing.get_context("spawn"))


def run_sharded(xyz, level, scalar=None, iso=None, n_slabs=8, processes=None, balance="width",
                executor=None, want_keys=True):
    """Dual cells (and, given ``scalar`` and ``iso``, the Marching Cubes
    output) of the whole data set, computed slab by slab in a ``spawn``
    process pool (``executor``, or one made for the call). Returns the
    concatenation over slabs, in slab order: duals [D, 8] (global cell IDs),
    and cases, ntri, tris, keys, max_err; "cpu_seconds" sums the shards'
    oracle times."""
    jobs = shard_jobs(xyz, level, scalar, iso, n_slabs, balance, want_keys)
    processes = processes or min(n_slabs, os.cpu_count() or 1)
    if executor is not None:
        parts = list(executor.map(_one_slab, jobs))
    elif processes <= 1:
        parts = [_one_slab(j) for j in jobs]
    else:
        with spawn_pool(processes) as ex:
            parts = list(ex.map(_one_slab, jobs))
    out = {"duals": np.concatenate([p["duals"] for p in parts]).reshape(-1, 8),
           "cpu_seconds": float(sum(p["seconds"] for p in parts))}
    if iso is not None:
        out["cases"] = np.concatenate([p["cases"] for p in parts])
        out["ntri"] = np.concatenate([p["ntri"] for p in parts])
        out["tris"] = np.concatenate([p["tris"] for p in parts]).reshape(-1, 3, 3)
        if want_keys:
            out["keys"] = np.concatenate([p["keys"] for p in parts]).reshape(-1, 3, 2)
        out["max_err"] = max([p["max_err"] for p in parts], default=0.0)
    return out


def _mix(z):
    """The splitmix64 output function on uint64 arrays (Steele, Lea and
    Flood, OOPSLA 2014): add the golden-ratio increment, then two
    xor-shift-multiply rounds and a final xor-shift."""
    with np.errstate(over="ignore"):
        z = z + np.uint64(GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def row_hashes(rows):
    """One 64-bit hash per row: h <- mix(h xor v) over the row's values
    (integers, or the bit patterns of fp32 values), h starting at 0."""
    a = np.asarray(rows)
    a = a.reshape(a.shape[0], -1) if a.ndim else a.reshape(1, 1)
    if a.dtype == np.float32:
        a = a.view(np.int32)
    v = a.astype(np.int64).view(np.uint64)
    h = np.zeros(a.shape[0], dtype=np.uint64)
    for c in range(v.shape[1]):
        h = _mix(h ^ v[:, c])
    return h


def fingerprint(rows):
    """(count, sum of row hashes, sum of their squares), sums mod 2^64: the
    same for any order of the same rows, and different, but for a 2^-64
    chance, when a row is added, dropped or changed."""
    h = row_hashes(rows)
    with np.errstate(over="ignore"):
        return (int(h.shape[0]), int(h.sum(dtype=np.uint64)), int((h * h).sum(dtype=np.uint64)))
