"""Serving: iso-surface requests against many resident AMR data sets.

A request is (data set, 1..64 iso-values). The server keeps each data set's
locator and dual-cell list resident on the device (an `AmrContext`), so a new
iso-value skips the dual-mesh pass; data sets are evicted least-recently-used
when the device-memory budget is exceeded. Requests are batched continuously:
``slots`` worker threads, each with its own CUDA stream, take the oldest
waiting request and every other waiting request for the same data set (up to
64 iso-values in total) and serve them with one batched launch
(`amr_iso_batch_async`, replayed from a captured CUDA graph once warm); one
worker's dual-mesh pass ("prefill") overlaps another worker's iso work on the
device. Latency = arrival -> triangles complete on the device and counts on
the host.

The per-request plain extraction (FIFO; upload, locator, dual cells and one
`amr_iso` per iso-value, no residency, no batching) is `serve_plain`.
"""
from __future__ import annotations

import collections
import threading
import time
import traceback
from dataclasses import dataclass, field

import numpy as np
import torch

from . import amriso

MAX_ISOS = 64
BYTES_PER_CELL_ESTIMATE = 110   # input copy + slots + dual list, before the real size is known


@dataclass
class Request:
    rid: int
    dataset: str
    isos: list
    t_arrival: float
    t_start: float = 0.0
    t_done: float = 0.0
    counts: list = None
    tris: list = None           # per iso, host tensors when the server keeps results
    batched_with: int = 1
    error: str = None
    done: threading.Event = field(default_factory=threading.Event)

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival


@dataclass
class _Dataset:
    name: str
    xyz: torch.Tensor     # host (pinned) arrays
    lvl: torch.Tensor
    s: torch.Tensor
    opts: dict


class _Resident:
    def __init__(self, name, ctx, nbytes):
        self.name = name
        self.ctx = ctx
        self.bytes = nbytes
        self.lock = threading.Lock()
        self.users = 0
        self.graphs = {}       # (worker, bucket) -> (graph, d_isos, out, d_offs)


class Server:
    """Continuous-batching iso-surface server on one GPU."""

    def __init__(self, budget_bytes: int, slots: int = 3, device: int = 0, keep_results: bool = False,
                 use_graphs: bool = True, out_capacity: int = 1 << 22):
        self.budget = int(budget_bytes)
        self.slots = int(slots)
        self.device = device
        self.keep_results = keep_results
        self.use_graphs = use_graphs
        self.out_capacity = int(out_capacity)
        self.datasets: dict[str, _Dataset] = {}
        self.resident: "collections.OrderedDict[str, _Resident]" = collections.OrderedDict()
        self.queue: list[Request] = []
        self.cv = threading.Condition()
        self.used = 0
        self.stop_flag = False
        self.workers = []
        self.stats = collections.Counter()
        self._rid = 0
        # Graph capture must not overlap device allocation or release in other
        # threads (context creation, locator buffers, eviction, buffer growth);
        # kernel work and graph replays run outside this lock.
        self.cuda_lock = threading.Lock()

    # -- registry ------------------------------------------------------------
    def add_dataset(self, name: str, xyz, lvl, s, **opts):
        """Register a data set (host tensors; pinned for fast prefill)."""
        pin = lambda t: t.cpu().contiguous().pin_memory()
        self.datasets[name] = _Dataset(name, pin(xyz), pin(lvl), pin(s), opts)

    # -- client side -----------------------------------------------------------
    def submit(self, dataset: str, isos, t_arrival: float | None = None) -> Request:
        isos = [float(v) for v in isos]
        assert 1 <= len(isos) <= MAX_ISOS and dataset in self.datasets
        with self.cv:
            self._rid += 1
            r = Request(self._rid, dataset, isos, time.perf_counter() if t_arrival is None else t_arrival)
            self.queue.append(r)
            self.cv.notify_all()
        return r

    def start(self):
        for w in range(self.slots):
            th = threading.Thread(target=self._worker, args=(w,), daemon=True)
            th.start()
            self.workers.append(th)

    def stop(self):
        with self.cv:
            self.stop_flag = True
            self.cv.notify_all()
        for th in self.workers:
            th.join()
        self.workers = []
        for r in list(self.resident.values()):
            if r.ctx is not None:
                r.ctx.close()
        self.resident.clear()
        self.used = 0

    # -- scheduling ------------------------------------------------------------
    def _take_batch(self):
        """Oldest request plus every waiting request for the same data set whose
        data set is not busy, up to MAX_ISOS iso-values. Caller holds cv."""
        for i, head in enumerate(self.queue):
            res = self.resident.get(head.dataset)
            if res is not None and res.users > 0:
                continue   # another worker serves this data set; it will pick these up
            batch = [head]
            n = len(head.isos)
            for r in self.queue[i + 1:]:
                if r.dataset == head.dataset and n + len(r.isos) <= MAX_ISOS:
                    batch.append(r)
                    n += len(r.isos)
            for r in batch:
                self.queue.remove(r)
            return batch
        return None

    def _admit(self, name: str):
        """Make room for `name` (LRU eviction of idle data sets) and mark it in
        use. Caller holds cv; may wait until memory frees up. Returns the
        resident entry, whether it still needs its dual-mesh pass, and the
        evicted contexts (to be closed by the caller outside cv)."""
        evicted = []
        while True:
            res = self.resident.get(name)
            if res is not None:
                if res.users > 0:          # another worker holds it (a context is
                    self.cv.wait(0.005)    # single-threaded); its prefill may be running
                    continue
                res.users += 1
                self.resident.move_to_end(name)
                return res, False, evicted
            need = self.datasets[name].xyz.shape[0] * BYTES_PER_CELL_ESTIMATE
            while self.used + need > self.budget:
                victim = next((r for r in self.resident.values() if r.users == 0), None)
                if victim is None:
                    break
                self.resident.pop(victim.name)
                if victim.ctx is not None:
                    evicted.append(victim.ctx)
                self.used -= victim.bytes
                self.stats["evictions"] += 1
            if self.used + need <= self.budget or not self.resident:
                res = _Resident(name, None, need)
                res.users = 1
                self.resident[name] = res
                self.used += need
                return res, True, evicted
            self.cv.wait(0.01)

    def _release(self, res: _Resident):
        with self.cv:
            res.users -= 1
            self.cv.notify_all()

    # -- worker ----------------------------------------------------------------
    def _worker(self, w: int):
        torch.cuda.set_device(self.device)
        with self.cuda_lock:
            stream = torch.cuda.Stream(self.device)
            out = torch.empty((self.out_capacity, 3, 3), dtype=torch.float32, device=self.device)
            d_isos = torch.empty(MAX_ISOS, dtype=torch.float32, device=self.device)
            d_offs = torch.zeros(MAX_ISOS + 1, dtype=torch.int64, device=self.device)
        h_offs = torch.zeros(MAX_ISOS + 1, dtype=torch.int64).pin_memory()
        h_isos = torch.empty(MAX_ISOS, dtype=torch.float32).pin_memory()
        while True:
            with self.cv:
                batch = None
                while not self.stop_flag:
                    batch = self._take_batch()
                    if batch:
                        break
                    self.cv.wait(0.005)
                if self.stop_flag and not batch:
                    return
                res, fresh, evicted = self._admit(batch[0].dataset)
            if evicted:
                with self.cuda_lock:
                    for ctx in evicted:
                        ctx.close()
            t0 = time.perf_counter()
            for r in batch:
                r.t_start = t0
            try:
                with torch.cuda.stream(stream):
                    if fresh:
                        self._prefill(res, stream)
                    out = self._serve(w, res, batch, stream, out, d_isos, d_offs, h_offs, h_isos)
            except Exception:  # report per request, keep serving
                err = traceback.format_exc()
                for r in batch:
                    r.error = err
                if res.ctx is None:                 # failed dual-mesh pass: forget the entry
                    with self.cv:
                        if self.resident.get(res.name) is res:
                            self.resident.pop(res.name)
                            self.used -= res.bytes
            t1 = time.perf_counter()
            for r in batch:
                r.t_done = t1
                r.batched_with = len(batch)
                r.done.set()
            self.stats["batches"] += 1
            self.stats["requests"] += len(batch)
            self._release(res)

    def _prefill(self, res: _Resident, stream):
        ds = self.datasets[res.name]
        with self.cuda_lock:   # allocates device buffers
            ctx = amriso.AmrContext(self.device, stream)
            try:
                ctx.upload(ds.xyz, ds.lvl, ds.s)
                ctx.build_locator(**ds.opts)
                ctx.dual_cells()
                ctx.trim()   # resident data sets keep no placement workspace
            except Exception:
                ctx.close()
                raise
        real = ctx.info().device_bytes
        with self.cv:
            self.used += real - res.bytes
            res.bytes = real
            res.ctx = ctx
        self.stats["prefills"] += 1

    def _serve(self, w, res, batch, stream, out, d_isos, d_offs, h_offs, h_isos):
        ctx = res.ctx
        ctx.set_stream(stream)
        isos = [v for r in batch for v in r.isos]
        k = len(isos)
        bucket = 1
        while bucket < k:
            bucket *= 2
        padded = isos + [float("inf")] * (bucket - k)   # +inf: no corner is above it, no triangles
        h_isos[:bucket] = torch.tensor(padded, dtype=torch.float32)
        d_isos[:bucket].copy_(h_isos[:bucket], non_blocking=True)
        # the graph bakes in the buffer's address and capacity: both are in the key
        key = (w, bucket, out.data_ptr(), int(out.shape[0]))
        g = res.graphs.get(key) if self.use_graphs else None
        if g is not None:
            g.replay()
            self.stats["graph_replays"] += 1
        else:
            ctx.iso_batch_async(d_isos[:bucket], out, d_offs[:bucket + 1])
            if self.use_graphs:
                res.graphs[key] = self._capture(ctx, stream, d_isos[:bucket], out, d_offs[:bucket + 1])
        h_offs[:bucket + 1].copy_(d_offs[:bucket + 1], non_blocking=True)
        stream.synchronize()
        offs = h_offs[:bucket + 1].tolist()
        if offs[bucket] > out.shape[0]:     # buffer too small: grow, drop stale graphs, rerun
            with self.cuda_lock:
                out = torch.empty((int(offs[bucket] * 1.25) + 1, 3, 3), dtype=torch.float32,
                                  device=self.device)
            with self.cv:   # this worker's graphs on every resident data set point at the old buffer
                for other in self.resident.values():
                    for gk in [gk for gk in other.graphs if gk[0] == w]:
                        del other.graphs[gk]
            ctx.iso_batch_async(d_isos[:bucket], out, d_offs[:bucket + 1])
            h_offs[:bucket + 1].copy_(d_offs[:bucket + 1], non_blocking=True)
            stream.synchronize()
            offs = h_offs[:bucket + 1].tolist()
        j = 0
        for r in batch:
            r.counts = [offs[j + q + 1] - offs[j + q] for q in range(len(r.isos))]
            if self.keep_results:
                r.tris = [out[offs[j + q]:offs[j + q + 1]].cpu() for q in range(len(r.isos))]
            j += len(r.isos)
        return out

    def _capture(self, ctx, stream, d_isos, out, d_offs):
        """CUDA graph of the batched step (count, device offsets, emit)."""
        stream.synchronize()
        g = torch.cuda.CUDAGraph()
        with self.cuda_lock:
            with torch.cuda.graph(g, stream=stream, capture_error_mode="thread_local"):
                ctx.iso_batch_async(d_isos, out, d_offs)
        return g


def serve_plain(datasets: dict, requests: list, device: int = 0, keep_results: bool = False):
    """Baseline: FIFO, one request at a time; upload, locator, dual cells and
    one amr_iso per iso-value; nothing kept between requests. `requests` are
    Request objects (arrival times honoured: a request does not start before
    it arrives)."""
    torch.cuda.set_device(device)
    stream = torch.cuda.current_stream(device)
    out = torch.empty((1 << 22, 3, 3), dtype=torch.float32, device=device)
    for r in sorted(requests, key=lambda q: q.t_arrival):
        now = time.perf_counter()
        if now < r.t_arrival:
            time.sleep(r.t_arrival - now)
        r.t_start = time.perf_counter()
        xyz, lvl, s = datasets[r.dataset]
        ctx = amriso.AmrContext(device, stream)
        ctx.upload(xyz, lvl, s)
        ctx.build_locator()
        ctx.dual_cells()
        r.counts, r.tris = [], [] if keep_results else None
        for v in r.isos:
            n = ctx.iso_count(v, out)
            if n > out.shape[0]:
                out = torch.empty((int(n * 1.25), 3, 3), dtype=torch.float32, device=device)
                n = ctx.iso_count(v, out)
            r.counts.append(n)
            if keep_results:
                r.tris.append(out[:n].cpu())
        ctx.close()
        r.t_done = time.perf_counter()
        r.done.set()
    return requests


def poisson_arrivals(n: int, rate: float, seed: int, t0: float):
    rng = np.random.default_rng(seed)
    return t0 + np.cumsum(rng.exponential(1.0 / rate, size=n))


def latency_summary(requests: list) -> dict:
    lat = np.array([r.latency for r in requests if r.error is None])
    tris = sum(sum(r.counts) for r in requests if r.counts)
    span = max(r.t_done for r in requests) - min(r.t_arrival for r in requests)
    return {"requests": len(requests), "errors": sum(r.error is not None for r in requests),
            "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3), "triangles": int(tris),
            "triangles_per_s": tris / span, "span_s": span}
