"""Serving: scheduling logic on the CPU (fake resident contexts), and on the
GPU every request's result in a mixed, concurrently batched stream (with LRU
eviction under a small budget and CUDA-graph replays) equals the same
request served alone by the plain context path."""
import threading
import time

import numpy as np
import pytest
import torch


class _FakeCtx:
    def __init__(self):
        self.closed = False

    def close(self):
        self.closed = True


def _server(budget):
    from paper_2004_08475_b300.serve import Server, _Resident
    srv = Server.__new__(Server)
    srv.budget = budget
    srv.datasets = {}
    srv.resident = __import__("collections").OrderedDict()
    srv.queue = []
    srv.cv = threading.Condition()
    srv.used = 0
    srv.stats = __import__("collections").Counter()
    srv._rid = 0
    srv.graphs = __import__("collections").defaultdict(__import__("collections").OrderedDict)
    return srv, _Resident


def _req(rid, ds, k):
    from paper_2004_08475_b300.serve import Request
    return Request(rid, ds, [0.5] * k, time.perf_counter())


def test_batch_coalesces_same_dataset_up_to_64_isos():
    srv, _ = _server(1 << 30)
    srv.queue = [_req(1, "a", 10), _req(2, "b", 3), _req(3, "a", 40), _req(4, "a", 20), _req(5, "a", 5)]
    with srv.cv:
        batch, entries = srv._take_batch()
    assert [r.rid for r in batch] == [1, 3, 5]          # 10 + 40 + 5 <= 64; 20 would exceed
    assert [r.rid for r in srv.queue] == [2, 4]
    (res, fresh), = entries                             # a needs its dual-mesh pass: a placeholder
    assert fresh and res.ctx is None and srv.resident["a"] is res and res.users == 1


def test_batch_skips_dataset_being_prepared():
    srv, Res = _server(1 << 30)
    busy = Res("a", None, 10)   # another worker runs its dual-mesh pass
    busy.users = 1
    srv.resident["a"] = busy
    srv.queue = [_req(1, "a", 1), _req(2, "b", 1)]
    with srv.cv:
        batch, entries = srv._take_batch()
    assert [r.rid for r in batch] == [2]


def test_batch_joins_ready_datasets():
    """Requests for other data sets join a batch whose head is ready when
    those are resident and ready (even while another batch reads them), not
    when they still need their dual-mesh pass; a batch whose head needs its
    dual-mesh pass takes nothing else. Every data set taken is pinned."""
    srv, Res = _server(1 << 30)
    for name in ("a", "c"):
        srv.resident[name] = Res(name, _FakeCtx(), 10)
    srv.resident["c"].users = 1
    srv.queue = [_req(1, "a", 3), _req(2, "b", 2), _req(3, "d", 1), _req(4, "c", 62), _req(5, "c", 4)]
    with srv.cv:
        batch, entries = srv._take_batch()
    assert [r.rid for r in batch] == [1, 5]             # b, d not resident; c's 62 would pass 64 values
    assert [(e.name, fresh) for e, fresh in entries] == [("a", False), ("c", False)]
    assert srv.resident["a"].users == 1 and srv.resident["c"].users == 2
    with srv.cv:
        batch, entries = srv._take_batch()
    assert [r.rid for r in batch] == [2] and entries[0][1]   # b alone, as a placeholder
    assert [r.rid for r in srv.queue] == [3, 4]


def test_lru_eviction_under_budget():
    from paper_2004_08475_b300 import serve
    srv, Res = _server(1000)

    class D:
        def __init__(self, n):
            self.xyz = torch.zeros((n, 3))
    srv.datasets = {"a": D(4), "b": D(4), "c": D(4)}
    old = serve.BYTES_PER_CELL_ESTIMATE
    serve.BYTES_PER_CELL_ESTIMATE = 100          # 400 bytes per data set
    try:
        for rid, name in enumerate(("a", "b")):
            srv.queue = [_req(rid, name, 1)]
            with srv.cv:
                _, entries = srv._take_batch()
                (res, fresh), = entries
                assert fresh and not srv._reserve(res)
            res.ctx = _FakeCtx()
            srv._release([res])
        srv.queue = [_req(3, "a", 1)]            # touch a: b becomes least recent
        with srv.cv:
            _, entries = srv._take_batch()
        assert not entries[0][1]
        srv._release([entries[0][0]])
        victim_ctx = srv.resident["b"].ctx
        srv.queue = [_req(4, "c", 1)]
        with srv.cv:
            _, entries = srv._take_batch()
            ev = srv._reserve(entries[0][0])      # 1200 > 1000: evict b
        assert "b" not in srv.resident and ev == [victim_ctx]
        assert srv.stats["evictions"] == 1 and srv.used == 800
    finally:
        serve.BYTES_PER_CELL_ESTIMATE = old


@pytest.mark.gpu
def test_mix_equals_alone():
    from paper_2004_08475_b300 import amriso, synth
    from paper_2004_08475_b300.serve import Server
    from tests.parity import canonical
    data = {
        "sphere": synth.sphere_tiny()[:4],
        "oct": synth.octree_gaussians(seed=31, roots=6, root_level=4)[:4],
        "rnd": synth.random_octree(5, levels=4, roots=5, p_hole=0.05)[:4],
        "blk": synth.block_vortex(seed=33, dims=(3, 2, 2), scale=0.1, tau=0.01, iso=0.05)[:4],
    }
    rng = np.random.default_rng(0)
    srv = Server(budget_bytes=60 << 20, slots=3, keep_results=True, out_capacity=1 << 16)
    for name, (x, l, s, iso) in data.items():
        srv.add_dataset(name, x, l, s)
    srv.start()
    reqs = []
    names = list(data)
    for i in range(40):
        name = names[rng.integers(len(names))]
        s = data[name][2]
        qs = rng.uniform(0.3, 0.8, size=int(rng.integers(1, 6)))
        isos = [float(np.quantile(s.numpy(), q)) for q in qs]
        reqs.append(srv.submit(name, isos))
        if i % 7 == 0:
            time.sleep(0.01)
    for r in reqs:
        assert r.done.wait(120)
    # the large octree alone exceeds the budget, so in the burst any data set
    # may be evicted before it is served again; ten identical requests one
    # after another keep the sphere resident, and with three worker slots one
    # of them serves it at least four times: a combination is captured the
    # second time a worker meets it and replayed from the third
    iso_sphere = float(np.quantile(data["sphere"][2].numpy(), 0.5))
    for _ in range(10):
        r = srv.submit("sphere", [iso_sphere])
        assert r.done.wait(120)
        reqs.append(r)
    srv.stop()
    errs = [r.error for r in reqs if r.error]
    assert not errs, errs[0]
    assert srv.stats["prefills"] > len(data)          # the budget forced evictions
    assert srv.stats["graph_replays"] > 0
    assert any(r.batched_with > 1 for r in reqs)
    ctxs = {}
    for name, (x, l, s, iso) in data.items():
        c = amriso.AmrContext()
        c.upload(x.cuda(), l.cuda(), s.cuda())
        c.build_locator()
        c.dual_cells()
        ctxs[name] = c
    for r in reqs:
        for v, got in zip(r.isos, r.tris):
            want = ctxs[r.dataset].iso(v).cpu().numpy()
            assert got.shape[0] == want.shape[0]
            assert (canonical(got.numpy()) == canonical(want)).all()


@pytest.mark.gpu
def test_preload_then_serve():
    """preload() runs the dual-mesh pass of data sets in the given order while
    they fit the budget; requests for them are then served without another."""
    from paper_2004_08475_b300 import synth
    from paper_2004_08475_b300.serve import Server
    data = {"sphere": synth.sphere_tiny()[:4],
            "rnd": synth.random_octree(6, levels=3, roots=4)[:4]}
    srv = Server(budget_bytes=1 << 30, slots=2, keep_results=True, out_capacity=1 << 14)
    for name, (x, l, s, iso) in data.items():
        srv.add_dataset(name, x, l, s)
    srv.preload(["rnd", "sphere"])
    assert srv.stats["prefills"] == 2 and list(srv.resident) == ["rnd", "sphere"]
    assert all(r.users == 0 and r.ctx is not None for r in srv.resident.values())
    srv.start()
    reqs = [srv.submit(name, [float(iso)]) for name, (x, l, s, iso) in data.items()]
    for r in reqs:
        assert r.done.wait(60)
    srv.stop()
    assert not any(r.error for r in reqs) and srv.stats["prefills"] == 2
    assert all(r.counts[0] > 0 for r in reqs)
