"""Slab sharding of one data set (paper_2004_08475_b300.shard, the owner
filter of amr_dual_cells_owned).

CPU: the product's slab edges and halo windows are the partition of the
sharded oracle (oracle/shard.py), and two gloo ranks split the slabs between
them and gather every slab's counts once. GPU: the slabs' dual cells and
triangles, extracted one shard after another, are exactly the whole data
set's (as multisets), and each slab's dual cells equal the sharded oracle's
for that slab."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2004_08475_b300 import synth


def _xw(xyz, lv):
    x = torch.as_tensor(xyz)[:, 0].long()
    return x, torch.ones_like(x) << torch.as_tensor(lv).long()


def test_slab_windows_match_oracle_partition():
    from oracle import shard as oshard
    from paper_2004_08475_b300 import shard
    xyz, lv, s, iso, info = synth.random_octree(17, levels=4, roots=5, p_split=0.45, p_hole=0.06)
    x, w = _xw(xyz, lv)
    for n_slabs in (1, 3, 7):
        want = oshard.slab_windows(xyz.numpy(), lv.numpy(), n_slabs, balance="count")
        bounds = shard.slab_bounds(x, w, n_slabs)
        assert len(bounds) == n_slabs
        for (x0, x1), (owners, window) in zip(bounds, want):
            got_win = shard.slab_window(x, w, x0, x1, int(w.max())).numpy()
            got_own = torch.nonzero((x >= x0) & (x < x1)).squeeze(1).numpy()
            assert np.array_equal(got_win, window) and np.array_equal(got_own, owners)


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _fake_extract(xyz, level, scalar, iso, x0, x1, wmax, want_duals=True):
    """Stands in for the GPU extraction: one 'dual' per owner, one
    'triangle' per window cell."""
    from paper_2004_08475_b300 import shard
    x = xyz[:, 0].long()
    w = torch.ones_like(x) << level.long()
    own = torch.nonzero((x >= x0) & (x < x1)).squeeze(1)
    win = shard.slab_window(x, w, x0, x1, wmax)
    return own.reshape(-1, 1).repeat(1, 8), torch.zeros((win.shape[0], 3, 3))


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2004_08475_b300 import shard
    xyz, lv, s, iso, info = synth.random_octree(23, levels=3, roots=4)
    mine, counts = shard.run_sharded(xyz, lv, s, iso, 5, rank=rank, world=world, extract=_fake_extract)
    q.put((rank, [k for k, _, _ in mine], counts.tolist(), int(xyz.shape[0])))
    dist.destroy_process_group()


def test_two_rank_sharded_counts():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    (_, slabs0, c0, n), (_, slabs1, c1, _) = out
    assert slabs0 == [0, 2, 4] and slabs1 == [1, 3]           # slab k on rank k % 2
    assert c0 == c1                                           # both ranks see every slab's counts
    assert sum(c[0] for c in c0) == n                         # every cell owns its 'dual' in one slab
    assert all(c[1] >= c[0] > 0 for c in c0)                  # windows hold their owners and a halo


@pytest.mark.gpu
def test_sharded_equals_whole_and_oracle():
    from oracle import shard as oshard
    from paper_2004_08475_b300 import amriso, shard
    from tests.parity import canonical
    xyz, lv, s, iso, info = synth.octree_gaussians(seed=12, roots=6, root_level=4)
    ctx = amriso.AmrContext()
    ctx.upload(xyz.cuda(), lv.cuda(), s.cuda())
    ctx.build_locator()
    ctx.dual_cells()
    whole_d = ctx.get_duals().cpu().numpy().astype(np.int64)
    whole_t = ctx.iso(iso).cpu().numpy()
    ctx.close()
    mine, counts = shard.run_sharded(xyz.cuda(), lv.cuda(), s.cuda(), iso, 4)
    dd = np.concatenate([d.cpu().numpy() for _, d, _ in mine])
    tt = np.concatenate([t.cpu().numpy() for _, _, t in mine])

    def rows(a):
        return a[np.lexsort(a.T[::-1])]
    assert dd.shape == whole_d.shape and np.array_equal(rows(dd), rows(whole_d))
    assert np.array_equal(canonical(tt).view(np.int32), canonical(whole_t).view(np.int32))
    # each slab against the sharded oracle's slab
    jobs = oshard.shard_jobs(xyz.numpy(), lv.numpy(), s.numpy(), iso, 4, balance="count", want_keys=False)
    for (k, d, t), job in zip(mine, jobs):
        o = oshard._one_slab(job)
        assert np.array_equal(rows(d.cpu().numpy()), rows(o["duals"]))
        assert np.array_equal(canonical(t.cpu().numpy()).view(np.int32), canonical(o["tris"]).view(np.int32))
