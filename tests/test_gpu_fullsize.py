"""Parity at the full sizes of the block-structured (~126M cells) and wing
(~592M cells) workloads, in the launch configuration bench.py times: every
dual cell owned by the cells of sampled boxes equals the oracle's (bit-exact
tuples, case indices and triangle counts). The oracle runs on the box plus a
halo of two coarsest-cell widths, which holds every vertex of those duals."""
import numpy as np
import pytest
import torch

import oracle
from paper_2004_08475_b300 import synth
from tests.parity import compare

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


def _sampled_parity(gen, n_boxes=3, half=12, seed=0):
    from paper_2004_08475_b300 import amriso
    xyz, lv, s, iso, info = gen
    ctx = amriso.AmrContext()
    ctx.upload(xyz, lv, s)
    ctx.build_locator()
    nd = ctx.dual_cells()
    duals = ctx.get_duals()
    cases, ntri = ctx.iso_cases(iso)
    owner = _owners_gpu(duals, xyz, lv)
    wmax = 1 << int(lv.max())
    rng = np.random.default_rng(seed)
    fine = torch.nonzero(lv == 0).squeeze(1)
    checked = 0
    for b in range(n_boxes):
        c = xyz[fine[int(rng.integers(0, fine.shape[0]))]].long()
        inner = ((xyz.long() - c).abs() <= half).all(1)
        outer = ((xyz.long() - c).abs() <= half + 2 * wmax).all(1)
        win = torch.nonzero(outer).squeeze(1)
        own = torch.nonzero(inner).squeeze(1)
        sel = torch.isin(owner, own)
        g = {"duals": duals[sel].cpu().numpy().astype(np.int64), "cases": cases[sel].cpu().numpy(),
             "ntri": ntri[sel].cpu().numpy()}
        wx, wl, ws = xyz[win].cpu().numpy(), lv[win].cpu().numpy(), s[win].cpu().numpy()
        m = oracle.OracleMesh(wx, wl)
        local_owner = torch.nonzero(torch.isin(win, own)).squeeze(1).cpu().numpy()
        od = m.duals(owners=local_owner)
        r = m.iso(ws, od, iso, want_keys=False)
        ids = win.cpu().numpy()
        o = {"duals": ids[od], "cases": r["cases"], "ntri": r["ntri"], "tris": r["tris"]}
        g["tris"] = r["tris"]
        assert g["duals"].shape[0] > 100
        compare(g, o, float(max(info["domain"])))
        checked += g["duals"].shape[0]
    assert int(ntri.sum()) == ctx.iso_count(iso, torch.empty((1, 3, 3), device="cuda"))
    ctx.close()
    return checked, nd


def test_block_full_size_sampled():
    gen = synth.block_vortex(device="cuda")
    assert gen[4]["n"] > 100_000_000
    checked, nd = _sampled_parity(gen, seed=1)
    assert nd > 100_000_000


def test_wing_full_size_sampled():
    gen = synth.wing_bands(device="cuda")
    assert gen[4]["n"] > 550_000_000
    checked, nd = _sampled_parity(gen, seed=2)
    assert nd > 550_000_000
