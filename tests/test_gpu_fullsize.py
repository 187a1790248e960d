"""Parity at the full sizes of the block-structured (~126M cells) and wing
(~592M cells) workloads, in the launch configuration bench.py times.

Sampled boxes: every dual cell owned by the cells of a box, its case index,
its triangle count and its triangles (the GPU's own, selected through the
per-triangle dual index of amr_iso_tagged) equal the oracle's. The oracle
runs on the box plus a halo of two coarsest-cell widths, which holds every
vertex of those duals. On the wing the triangle buffer is 4.7 GB, so the
boxes' triangles include rows written past byte 2^32 of it.

Whole block: the multiset fingerprints (oracle.shard.fingerprint) of all
dual cells and all triangles equal those of the slab-sharded oracle run over
the whole data set on the host's cores."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2004_08475_b300 import synth
from tests.parity import canonical, compare

pytestmark = pytest.mark.gpu


def _owners_gpu(duals, xyz, lv, chunk=1 << 24):
    """Owner of each dual (vertex with the smallest (level, z, y, x))."""
    out = torch.empty(duals.shape[0], dtype=torch.int64, device="cuda")
    for a in range(0, duals.shape[0], chunk):
        d = duals[a:a + chunk].long()
        x = xyz[d].long()
        key = (lv[d].long() << 60) + ((x[..., 2] + (1 << 21)) << 40) + ((x[..., 1] + (1 << 21)) << 20) + \
            (x[..., 0] + (1 << 21))
        out[a:a + chunk] = torch.gather(d, 1, key.argmin(1, keepdim=True)).squeeze(1)
    return out


def _sampled_parity(gen, n_boxes=3, half=12, seed=0, tail_box=False):
    """One box of half-width `half` around a random finest cell, n_boxes
    around the owners of random triangles (boxes on the surface), and with
    tail_box one more around the owner of a triangle written past byte 2^32
    of the triangle buffer (triangles come out roughly in dual-list order,
    which is spatial, so a random box rarely reaches the buffer's tail)."""
    from paper_2004_08475_b300 import amriso
    xyz, lv, s, iso, info = gen
    ctx = amriso.AmrContext()
    ctx.upload(xyz, lv, s)
    ctx.build_locator()
    nd = ctx.dual_cells()
    duals = ctx.get_duals()
    cases, ntri = ctx.iso_cases(iso)
    tris, tags = ctx.iso_tagged(iso)
    assert tris.shape[0] == int(ntri.sum())
    owner = _owners_gpu(duals, xyz, lv)
    wmax = 1 << int(lv.max())
    rng = np.random.default_rng(seed)
    fine = torch.nonzero(lv == 0).squeeze(1)
    checked = 0
    max_row = 0
    def around_triangle(r):
        o = int(owner[int(tags[r])])
        return xyz[o].long(), max(half, 4 << int(lv[o])), True

    centres = [(xyz[fine[int(rng.integers(0, fine.shape[0]))]].long(), half, False)]
    centres += [around_triangle(int(rng.integers(0, tris.shape[0]))) for _ in range(n_boxes)]
    first_tail = -(-(2 ** 32) // 36)
    if tail_box and tris.shape[0] > first_tail:
        centres.append(around_triangle(int(rng.integers(first_tail, tris.shape[0]))))
    for c, hb, surface in centres:
        inner = ((xyz.long() - c).abs() <= hb).all(1)
        outer = ((xyz.long() - c).abs() <= hb + 2 * wmax).all(1)
        win = torch.nonzero(outer).squeeze(1)
        own = torch.nonzero(inner).squeeze(1)
        sel = torch.isin(owner, own)
        # the GPU's triangles of the selected duals
        dmask = torch.zeros(nd, dtype=torch.bool, device="cuda")
        dmask[torch.nonzero(sel).squeeze(1)] = True
        rows = torch.nonzero(dmask[tags]).squeeze(1)
        max_row = max(max_row, int(rows.max()) if rows.numel() else 0)
        g = {"duals": duals[sel].cpu().numpy().astype(np.int64), "cases": cases[sel].cpu().numpy(),
             "ntri": ntri[sel].cpu().numpy(), "tris": tris[rows].cpu().numpy()}
        wx, wl, ws = xyz[win].cpu().numpy(), lv[win].cpu().numpy(), s[win].cpu().numpy()
        m = oracle.OracleMesh(wx, wl)
        local_owner = torch.nonzero(torch.isin(win, own)).squeeze(1).cpu().numpy()
        od = m.duals(owners=local_owner)
        r = m.iso(ws, od, iso, want_keys=False)
        ids = win.cpu().numpy()
        o = {"duals": ids[od], "cases": r["cases"], "ntri": r["ntri"], "tris": r["tris"]}
        assert g["duals"].shape[0] > 100
        res = compare(g, o, float(max(info["domain"])))
        assert res["bit_exact_frac"] == 1.0
        assert res["tris"] > 0 or not surface
        checked += g["duals"].shape[0]
    assert int(ntri.sum()) == ctx.iso_count(iso, torch.empty((1, 3, 3), device="cuda"))
    ctx.close()
    return checked, nd, max_row, int(tris.shape[0])


def test_block_full_size_sampled():
    gen = synth.block_vortex(device="cuda")
    assert gen[4]["n"] > 100_000_000
    checked, nd, _, _ = _sampled_parity(gen, seed=1)
    assert nd > 100_000_000


def test_wing_full_size_sampled():
    gen = synth.wing_bands(device="cuda")
    assert gen[4]["n"] > 550_000_000
    checked, nd, max_row, nt = _sampled_parity(gen, n_boxes=3, seed=2, tail_box=True)
    assert nd > 550_000_000
    assert nt * 36 > 2 ** 32
    # at least one checked triangle sits past byte 2^32 of the output buffer
    assert max_row * 36 >= 2 ** 32, (max_row, nt)


def test_block_full_size_fingerprint():
    """All dual cells (as cell IDs) and all triangles of the 126M-cell block
    workload against the slab-sharded oracle over the whole data set, as
    multiset fingerprints (count, sum and sum of squares of a 64-bit row
    hash)."""
    from oracle import shard
    from paper_2004_08475_b300 import amriso
    xyz, lv, s, iso, info = synth.block_vortex(device="cuda")
    ctx = amriso.AmrContext()
    ctx.upload(xyz, lv, s)
    ctx.build_locator()
    nd = ctx.dual_cells()
    g_duals = ctx.get_duals().cpu().numpy()
    g_tris = ctx.iso(iso).cpu().numpy()
    ctx.close()
    x, l, v = xyz.cpu().numpy(), lv.cpu().numpy(), s.cpu().numpy()
    del xyz, lv, s
    torch.cuda.empty_cache()
    o = shard.run_sharded(x, l, v, iso, n_slabs=max(8, min(32, os.cpu_count() or 1)), balance="count",
                          want_keys=False)
    assert o["duals"].shape[0] == nd > 100_000_000
    assert shard.fingerprint(g_duals.astype(np.int64)) == shard.fingerprint(o["duals"])
    assert g_tris.shape[0] == o["tris"].shape[0] > 1_000_000
    # each triangle rotated to start at its smallest vertex (orientation kept)
    assert shard.fingerprint(canonical(g_tris)) == shard.fingerprint(canonical(o["tris"]))
