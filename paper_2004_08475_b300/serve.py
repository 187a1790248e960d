"""Serving: iso-surface requests against many resident AMR data sets.

A request is (data set, 1..64 iso-values). The server keeps each data set's
locator and dual-cell list resident on the device (an `AmrContext`), so a new
iso-value skips the dual-mesh pass; data sets are evicted least-recently-used
when the device-memory budget is exceeded. Requests are batched continuously:
``slots`` worker threads, each with its own CUDA stream, take the oldest
waiting request plus every other waiting request whose data set is resident
and ready - whatever the data set, up to 64 iso-values and 32 data sets - and
serve them with one batched launch over all their dual lists
(`amr_iso_multi_async`, replayed from a captured CUDA graph when the same
combination comes again); one worker's dual-mesh pass ("prefill") overlaps
another worker's iso work on the device. Latency = arrival -> triangles
complete on the device and counts on the host.

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
MAX_JOBS = 32                   # data sets in one batched launch
MAX_GRAPHS = 64                 # captured batch graphs kept per worker
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
        self.ctx = ctx          # None while its dual-mesh pass runs
        self.bytes = nbytes
        self.users = 0          # batches (in any worker) that read it now


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
        # captured batch graphs per worker: key (data sets, iso counts, buffers) -> graph;
        # a combination is captured the second time it comes (seen: keys met once)
        self.graphs: dict[int, "collections.OrderedDict"] = collections.defaultdict(collections.OrderedDict)
        self.seen: dict[int, "collections.OrderedDict"] = collections.defaultdict(collections.OrderedDict)
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

    def preload(self, names=None):
        """Run the dual-mesh pass of data sets before serving starts (in the
        given order, all registered ones by default) while their estimated
        size fits the budget: a server starts with its data sets resident.
        Call before start()."""
        torch.cuda.set_device(self.device)
        stream = torch.cuda.Stream(self.device)
        for name in (names if names is not None else list(self.datasets)):
            with self.cv:
                if name in self.resident:
                    continue
                if self.used + self.datasets[name].xyz.shape[0] * BYTES_PER_CELL_ESTIMATE > self.budget:
                    break
                res = _Resident(name, None, 0)
                res.users = 1
                self.resident[name] = res
                self._reserve(res)
            with torch.cuda.stream(stream):
                self._prefill(res, stream)
            self._release([res])
        torch.cuda.synchronize()

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
    def _ready(self, name: str) -> bool:
        res = self.resident.get(name)
        return res is not None and res.ctx is not None

    def _pin(self, name: str) -> _Resident:
        res = self.resident[name]
        res.users += 1
        self.resident.move_to_end(name)
        return res

    def _take_batch(self):
        """The next batch, or None. Caller holds cv. Scans the queue oldest
        first for a request that can start now:
          - its data set is resident and ready: the batch takes it and every
            later waiting request whose data set is resident and ready (any
            data set), up to MAX_ISOS iso-values and MAX_JOBS data sets;
          - its data set is not resident: the batch takes it and the later
            requests for the same data set only, and a placeholder entry
            (no context yet) marks the data set as being prepared;
          - its data set is being prepared by another worker: skipped.
        Every data set of the batch is pinned (users + 1) before cv is
        released, so nothing the batch reads can be evicted, and a batch that
        must wait for memory holds nothing else: no hold-and-wait. Returns
        (requests, [(resident entry, needs its dual-mesh pass)])."""
        for i, head in enumerate(self.queue):
            res = self.resident.get(head.dataset)
            if res is not None and res.ctx is None:
                continue   # another worker prepares it; it will pick these up
            fresh = res is None
            batch = [head]
            names = [head.dataset]
            n = len(head.isos)
            for r in self.queue[i + 1:]:
                if n + len(r.isos) > MAX_ISOS:
                    continue
                if r.dataset in names or (not fresh and len(names) < MAX_JOBS and self._ready(r.dataset)):
                    batch.append(r)
                    if r.dataset not in names:
                        names.append(r.dataset)
                    n += len(r.isos)
            for r in batch:
                self.queue.remove(r)
            if fresh:
                res = _Resident(head.dataset, None, 0)
                res.users = 1
                self.resident[head.dataset] = res
                return batch, [(res, True)]
            return batch, [(self._pin(name), False) for name in names]
        return None

    def _reserve(self, res: _Resident):
        """Device memory for a placeholder entry's dual-mesh pass: evict idle
        data sets least-recently-used first until the estimate fits (or
        nothing else is resident). Caller holds cv; waits while other
        batches hold what would have to go. Returns the evicted contexts (the
        caller closes them outside cv)."""
        need = self.datasets[res.name].xyz.shape[0] * BYTES_PER_CELL_ESTIMATE
        evicted = []
        while True:
            while self.used + need > self.budget:
                victim = next((r for r in self.resident.values() if r.users == 0), None)
                if victim is None:
                    break
                self.resident.pop(victim.name)
                if victim.ctx is not None:
                    evicted.append(victim.ctx)
                self.used -= victim.bytes
                self.stats["evictions"] += 1
                self._drop_graphs(victim.name)
            if self.used + need <= self.budget or all(r is res for r in self.resident.values()):
                self.used += need
                res.bytes = need
                return evicted
            self.cv.wait(0.01)

    def _drop_graphs(self, name: str):
        """Forget every captured graph that reads data set `name` (its device
        buffers are about to go). Caller holds cv."""
        for g in self.graphs.values():
            for key in [k for k in g if name in k[0]]:
                del g[key]

    def _release(self, residents):
        with self.cv:
            for res in residents:
                res.users -= 1
            self.cv.notify_all()

    # -- worker ----------------------------------------------------------------
    def _worker(self, w: int):
        torch.cuda.set_device(self.device)
        with self.cuda_lock:
            stream = torch.cuda.Stream(self.device)
            bufs = {"out": torch.empty((self.out_capacity, 3, 3), dtype=torch.float32, device=self.device),
                    "ws": torch.empty(1 << 20, dtype=torch.uint8, device=self.device),
                    "d_isos": torch.empty(MAX_ISOS, dtype=torch.float32, device=self.device),
                    "d_offs": torch.zeros(MAX_ISOS + 1, dtype=torch.int64, device=self.device)}
        bufs["h_offs"] = torch.zeros(MAX_ISOS + 1, dtype=torch.int64).pin_memory()
        bufs["h_isos"] = torch.empty(MAX_ISOS, dtype=torch.float32).pin_memory()
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
                batch, admitted = batch
                evicted = []
                for res, fresh in admitted:
                    if fresh:
                        evicted += self._reserve(res)
            if evicted:
                with self.cuda_lock:
                    for ctx in evicted:
                        ctx.close()
            t0 = time.perf_counter()
            for r in batch:
                r.t_start = t0
            try:
                with torch.cuda.stream(stream):
                    for res, fresh in admitted:
                        if fresh:
                            self._prefill(res, stream)
                    self._serve(w, [res for res, _ in admitted], batch, stream, bufs)
            except Exception:  # report per request, keep serving
                err = traceback.format_exc()
                for r in batch:
                    r.error = err
                with self.cv:
                    for res, fresh in admitted:
                        if fresh and res.ctx is None and self.resident.get(res.name) is res:   # failed prefill
                            self.resident.pop(res.name)
                            self.used -= res.bytes
            t1 = time.perf_counter()
            for r in batch:
                r.t_done = t1
                r.batched_with = len(batch)
                r.done.set()
            self.stats["batches"] += 1
            self.stats["requests"] += len(batch)
            if len(admitted) > 1:
                self.stats["multi_dataset_batches"] += 1
            self._release([res for res, _ in admitted])

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

    def _serve(self, w, residents, batch, stream, bufs):
        """One batched launch over the batch's data sets: job j = residents[j]
        at the iso-values of its requests (in batch order), each job's count
        padded with +inf up to a power of two when the padded total fits
        (+inf: no corner lies above it, so no triangles), so that recurring
        combinations replay one captured graph."""
        per = {res.name: [] for res in residents}
        for r in batch:
            per[r.dataset].extend(r.isos)
        counts = [len(per[res.name]) for res in residents]
        padded = [1 << (k - 1).bit_length() for k in counts]
        if sum(padded) > MAX_ISOS:
            padded = counts
        isos = []
        for res, k, p in zip(residents, counts, padded):
            isos += per[res.name] + [float("inf")] * (p - k)
        nq = len(isos)
        ctxs = [res.ctx for res in residents]
        bufs["h_isos"][:nq] = torch.tensor(isos, dtype=torch.float32)
        bufs["d_isos"][:nq].copy_(bufs["h_isos"][:nq], non_blocking=True)
        need_ws = amriso.iso_multi_workspace(ctxs, padded)
        if need_ws > bufs["ws"].numel():
            with self.cuda_lock:
                bufs["ws"] = torch.empty(int(need_ws * 1.5), dtype=torch.uint8, device=self.device)
            with self.cv:
                self.graphs[w].clear()
        out, ws = bufs["out"], bufs["ws"]
        d_isos, d_offs = bufs["d_isos"][:nq], bufs["d_offs"][:nq + 1]
        # a graph bakes in the data sets' buffers, the iso counts and the
        # worker's buffers (address and capacity): all are in the key
        key = (tuple(res.name for res in residents), tuple(padded), tuple(id(c) for c in ctxs),
               out.data_ptr(), int(out.shape[0]), ws.data_ptr())
        graphs = self.graphs[w]
        with self.cv:   # other workers drop graphs of evicted data sets under cv
            g = graphs.get(key) if self.use_graphs else None
            if g is not None:
                graphs.move_to_end(key)

        def launch():
            amriso.iso_multi_async(ctxs, padded, d_isos, out, d_offs, ws, stream)

        if g is not None:
            g.replay()
            self.stats["graph_replays"] += 1
        else:
            launch()
            seen = self.seen[w]
            if self.use_graphs and key in seen:   # recurring: capture it for the next time
                g = self._capture(launch, stream)
                with self.cv:
                    graphs[key] = g
                    while len(graphs) > MAX_GRAPHS:
                        graphs.popitem(last=False)
                    seen.pop(key, None)
                self.stats["graph_captures"] += 1
            elif self.use_graphs:
                seen[key] = True
                while len(seen) > 4 * MAX_GRAPHS:
                    seen.popitem(last=False)
        bufs["h_offs"][:nq + 1].copy_(d_offs, non_blocking=True)
        stream.synchronize()
        offs = bufs["h_offs"][:nq + 1].tolist()
        if offs[nq] > out.shape[0]:     # buffer too small: grow, drop this worker's graphs, rerun
            with self.cuda_lock:
                out = bufs["out"] = torch.empty((int(offs[nq] * 1.25) + 1, 3, 3), dtype=torch.float32,
                                                device=self.device)
            with self.cv:
                self.graphs[w].clear()
            amriso.iso_multi_async(ctxs, padded, d_isos, out, d_offs, ws, stream)
            bufs["h_offs"][:nq + 1].copy_(d_offs, non_blocking=True)
            stream.synchronize()
            offs = bufs["h_offs"][:nq + 1].tolist()
        first = {}
        q = 0
        for res, p in zip(residents, padded):
            first[res.name] = q
            q += p
        taken = collections.Counter()
        for r in batch:
            j = first[r.dataset] + taken[r.dataset]
            taken[r.dataset] += len(r.isos)
            r.counts = [offs[j + i + 1] - offs[j + i] for i in range(len(r.isos))]
            if self.keep_results:
                r.tris = [out[offs[j + i]:offs[j + i + 1]].cpu() for i in range(len(r.isos))]

    def _capture(self, launch, stream):
        """CUDA graph of the batched step (counts, prefix sums, emission),
        captured on the worker's own stream. (torch.cuda.graph's context
        manager would also synchronise the whole device, run the garbage
        collector and empty the allocator's cache on every capture, stalling
        the other workers' batches.)"""
        g = torch.cuda.CUDAGraph()
        with self.cuda_lock, torch.cuda.stream(stream):
            g.capture_begin(capture_error_mode="thread_local")
            try:
                launch()
            finally:
                g.capture_end()
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
