"""Pins of the slab-sharded oracle and the multiset fingerprint (CPU only).

* the fingerprint's mixing function reproduces the published splitmix64
  outputs from seed 0, is blind to row order and sees a changed, dropped or
  swapped row;
* the slab windows partition the owners and hold every cell a slab's owners
  can snap to;
* the sharded oracle equals the unsharded one (bit-exact duals, cases,
  triangle counts, triangles and edge keys) for 1 to 13 slabs, and a shard
  planted without its halo does not: the comparison has the power to see a
  missing halo;
* two gloo ranks, each with half of the slabs, exchange three integers per
  rank, and the sum of their fingerprints is the unsharded output's.
"""
import os
import socket

import numpy as np
import pytest
import torch

import oracle
from oracle import shard
from paper_2004_08475_b300 import synth
from tests.parity import canonical


def test_splitmix64_published_outputs():
    """splitmix64 from seed 0 (state advanced by the golden-ratio gamma
    before each output) starts e220a8397b1dcdaf, 6e789e6aa1b965f4,
    06c45d188009454f."""
    states = np.array([0, shard.GAMMA, (2 * shard.GAMMA) % (1 << 64)], dtype=np.uint64)
    got = [int(v) for v in shard._mix(states)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_fingerprint_order_blind_and_sensitive():
    rng = np.random.default_rng(3)
    rows = rng.integers(0, 1 << 31, size=(5000, 8), dtype=np.int64)
    fp = shard.fingerprint(rows)
    assert fp == shard.fingerprint(rows[rng.permutation(rows.shape[0])])
    changed = rows.copy()
    changed[1234, 5] += 1
    assert shard.fingerprint(changed) != fp
    assert shard.fingerprint(rows[1:])[0] == fp[0] - 1
    swapped = rows.copy()
    swapped[7, [2, 3]] = swapped[7, [3, 2]]        # same multiset of values in the row
    assert shard.fingerprint(swapped) != fp
    # additive: the fingerprint of a union is the sum of the parts'
    a, b = shard.fingerprint(rows[:2000]), shard.fingerprint(rows[2000:])
    m = (1 << 64) - 1
    assert (a[0] + b[0], (a[1] + b[1]) & m, (a[2] + b[2]) & m) == fp
    tris = rng.standard_normal((100, 3, 3)).astype(np.float32)
    t2 = tris.copy()
    t2[50, 1, 1] = np.nextafter(t2[50, 1, 1], np.float32(np.inf))
    assert shard.fingerprint(tris) != shard.fingerprint(t2)


def test_slab_windows_partition_and_cover():
    xyz, lv, s, iso, info = synth.random_octree(8, levels=5, roots=4, p_hole=0.08)
    x, l = xyz.numpy().astype(np.int64), lv.numpy().astype(np.int64)
    w = 1 << l
    wins = shard.slab_windows(x, l, 6) + shard.slab_windows(x, l, 5, balance="count")
    for part in (wins[:6], wins[6:]):
        owners = np.concatenate([o for o, _ in part])
        assert np.array_equal(np.sort(owners), np.arange(x.shape[0]))
    counts = [o.shape[0] for o, _ in wins[6:]]
    assert max(counts) < 2 * x.shape[0] / 5
    for own, win in wins:
        assert (np.diff(win) > 0).all()
        assert np.isin(own, win).all()
        if own.shape[0] == 0:
            continue
        # every cell containing a query point x - w .. x + w of an owner is
        # in the window (checked cell by cell along x)
        qlo = (x[own, 0] - w[own]).min()
        qhi = (x[own, 0] + w[own]).max()
        touching = np.nonzero((x[:, 0] <= qhi) & (x[:, 0] + w > qlo))[0]
        assert np.isin(touching, win).all()


def _unsharded(x, l, s, iso):
    m = oracle.OracleMesh(x, l)
    d = m.duals()
    r = m.iso(s, d, iso, want_keys=True)
    return {"duals": d, "cases": r["cases"], "ntri": r["ntri"], "tris": r["tris"], "keys": r["keys"]}


def _same(a, b):
    oa, ob = np.lexsort(a["duals"].T[::-1]), np.lexsort(b["duals"].T[::-1])
    if a["duals"].shape != b["duals"].shape or not np.array_equal(a["duals"][oa], b["duals"][ob]):
        return False
    if not (np.array_equal(a["cases"][oa], b["cases"][ob]) and np.array_equal(a["ntri"][oa], b["ntri"][ob])):
        return False
    if a["tris"].shape != b["tris"].shape:
        return False
    if not np.array_equal(canonical(a["tris"]).view(np.int32), canonical(b["tris"]).view(np.int32)):
        return False
    ka = np.sort(a["keys"].reshape(-1, 3, 2), axis=1).reshape(-1, 6)
    kb = np.sort(b["keys"].reshape(-1, 3, 2), axis=1).reshape(-1, 6)
    return shard.fingerprint(ka) == shard.fingerprint(kb)


CASES = [
    ("random_octree", lambda: synth.random_octree(8, levels=5, roots=4, p_hole=0.08, field="sphere")),
    ("random_octree_holes", lambda: synth.random_octree(21, levels=4, roots=7, p_hole=0.2)),
    ("block_vortex", lambda: synth.block_vortex(seed=33, dims=(3, 2, 2), scale=0.1, tau=0.01, iso=0.05)),
    ("sphere_tiny", lambda: synth.sphere_tiny()),
]


@pytest.mark.parametrize("name,gen", CASES, ids=[c[0] for c in CASES])
def test_sharded_equals_unsharded(name, gen):
    xyz, lv, s, iso, info = gen()
    x, l, v = xyz.numpy(), lv.numpy(), s.numpy()
    ref = _unsharded(x, l, v, iso)
    assert ref["duals"].shape[0] > 100 and ref["tris"].shape[0] > 10
    for n, balance in ((1, "width"), (2, "width"), (5, "width"), (13, "width"), (3, "count"), (7, "count")):
        got = shard.run_sharded(x, l, v, iso, n_slabs=n, processes=1, balance=balance)
        assert _same(got, ref), (name, n, balance)
        assert shard.fingerprint(got["duals"]) == shard.fingerprint(ref["duals"])


def test_sharded_process_pool():
    xyz, lv, s, iso, info = synth.random_octree(21, levels=4, roots=7, p_hole=0.2)
    x, l, v = xyz.numpy(), lv.numpy(), s.numpy()
    got = shard.run_sharded(x, l, v, iso, n_slabs=4, processes=2)
    assert _same(got, _unsharded(x, l, v, iso))


def test_planted_missing_halo_is_caught():
    """A shard that holds only its owners' cells (a planted mistake: no
    halo) loses or changes duals at the slab faces."""
    xyz, lv, s, iso, info = synth.random_octree(8, levels=5, roots=4, p_hole=0.08, field="sphere")
    x, l, v = xyz.numpy(), lv.numpy(), s.numpy()
    ref = _unsharded(x, l, v, iso)
    parts = []
    for own, _win in shard.slab_windows(x, l, 5):
        job = (x[own], l[own], v[own], np.arange(own.shape[0]), own, float(iso))
        parts.append(shard._one_slab(job))
    planted = {k: np.concatenate([p[k] for p in parts]) for k in ("duals", "cases", "ntri", "tris", "keys")}
    assert not _same(planted, ref)
    assert shard.fingerprint(planted["duals"]) != shard.fingerprint(ref["duals"])


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    xyz, lv, s, iso, info = synth.random_octree(21, levels=4, roots=7, p_hole=0.2)
    jobs = shard.shard_jobs(xyz.numpy(), lv.numpy(), s.numpy(), iso, 6)
    mine = [shard._one_slab(j) for j in jobs[rank::world]]
    d = np.concatenate([p["duals"] for p in mine]).reshape(-1, 8)
    t = np.concatenate([p["tris"] for p in mine]).reshape(-1, 3, 3)
    fps = list(shard.fingerprint(d)) + list(shard.fingerprint(canonical(t).reshape(-1, 9)))
    # the fingerprints travel as exact integers: 32-bit halves in int64
    parts = [[v & 0xFFFFFFFF, v >> 32] for v in fps]
    mine_t = torch.tensor(parts, dtype=torch.int64)
    gathered = [torch.zeros_like(mine_t) for _ in range(world)]
    dist.all_gather(gathered, mine_t)
    if rank == 0:
        tot = [sum(int(g[i, 0]) + (int(g[i, 1]) << 32) for g in gathered) for i in range(6)]
        q.put([v % (1 << 64) for v in tot])
    dist.destroy_process_group()


def test_two_gloo_ranks_sum_fingerprints():
    """The multi-rank form of the sharded check: each rank runs its slabs
    and sends only its fingerprints; their sum is the whole output's."""
    import torch.multiprocessing as mp
    xyz, lv, s, iso, info = synth.random_octree(21, levels=4, roots=7, p_hole=0.2)
    ref = _unsharded(xyz.numpy(), lv.numpy(), s.numpy(), iso)
    want = list(shard.fingerprint(ref["duals"])) + list(shard.fingerprint(canonical(ref["tris"]).reshape(-1, 9)))
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=300)
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    assert got == want


def test_bench_cpu_leg_on_several_processes():
    """bench.py's CPU-baseline leg: the oracle cut into x slabs on a pool of
    processes counts the same duals and triangles as one process."""
    import bench
    xyz, lv, s, iso, info = synth.random_octree(8, levels=5, roots=4, p_hole=0.08, field="sphere")
    x, l, v = xyz.numpy(), lv.numpy(), s.numpy()
    one = bench.time_oracle(x, l, v, iso, seconds=0.01)
    pool = bench.oracle_pool(2)
    assert pool is not None
    try:
        two = bench.time_oracle(x, l, v, iso, seconds=0.01, pool=pool, processes=2)
    finally:
        pool.shutdown()
    assert one["cores"] == 1 and two["cores"] == 2
    assert one["cells"] == two["cells"] == x.shape[0]
    assert (one["duals"], one["tris"]) == (two["duals"], two["tris"])
    assert "2 x slabs" in bench.oracle_sample_text(two, "random_octree")


def test_bench_cpu_leg_survives_a_broken_pool():
    """A pool that fails leaves the CPU leg timing the one-process oracle."""
    import bench

    class Broken:
        def map(self, *a, **k):
            raise RuntimeError("planted pool failure")

    xyz, lv, s, iso, info = synth.random_octree(8, levels=5, roots=4, p_hole=0.08, field="sphere")
    x, l, v = xyz.numpy(), lv.numpy(), s.numpy()
    r = bench.time_oracle(x, l, v, iso, seconds=0.01, pool=Broken(), processes=4)
    one = bench.time_oracle(x, l, v, iso, seconds=0.01)
    assert r["cores"] == 1 and (r["duals"], r["tris"]) == (one["duals"], one["tris"])


def test_bench_oracle_window_is_a_box():
    """bench.py's sample: exactly the cells within a box around a finest-level
    cell (brute force over all cells), about the requested size, in input
    order."""
    import bench
    xyz, lv, s, iso, info = synth.octree_gaussians(seed=12, roots=4, root_level=4)
    x, l, v = xyz.numpy(), lv.numpy(), s.numpy()
    for target, sub_max in ((500, 1 << 30), (5000, 1 << 30), (50000, 1 << 30), (5000, 40000), (50000, 40000)):
        wx, wl, ws = bench.oracle_window(x, l, v, target, seed=3, sub_max=sub_max)
        # (the box grows in whole cell layers, so small targets land within a factor 2)
        assert 0.4 * target <= wx.shape[0] <= 2.5 * target
        # the box: the tightest box around the window, centred on a finest cell
        lo, hi = wx.min(0).astype(np.int64), wx.max(0).astype(np.int64)
        inside = np.all((x >= lo) & (x <= hi), axis=1)
        assert inside.sum() == wx.shape[0]
        assert np.array_equal(x[inside], wx) and np.array_equal(l[inside], wl) and np.array_equal(v[inside], ws)
        assert (wl == l.min()).any()
    empty = bench.oracle_window(x[:0], l[:0], v[:0], 100)
    assert empty[0].shape == (0, 3)
