"""The indexed face set (amr_iso_indexed) against the oracle's weld of its
own triangles: the same vertices (by edge key, bit-exact positions) and the
same triangles (as edge-key triples, orientation kept)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2004_08475_b300 import synth
from tests.parity import canonical

pytestmark = pytest.mark.gpu


def _key_triangles(tri, vkeys):
    """Triangles as rows of three edge keys, each row rotated (orientation
    kept) to start at its smallest key; rows sorted."""
    k = vkeys[tri]                                   # [T,3,2]
    code = k[:, :, 0].astype(np.int64) * (1 << 32) + k[:, :, 1]
    first = np.argmin(code, axis=1)
    idx = (first[:, None] + np.arange(3)[None]) % 3
    r = np.take_along_axis(code, idx, axis=1)
    return r[np.lexsort(r.T[::-1])]


def _check(xyz, lv, s, iso, host=False):
    from paper_2004_08475_b300 import amriso
    ctx = amriso.AmrContext()
    ctx.upload(xyz.cuda(), lv.cuda(), s.cuda())
    ctx.build_locator()
    ctx.dual_cells()
    vtx, tri, vkeys = ctx.iso_indexed(iso, host=host)
    fat = ctx.iso(iso).cpu().numpy()
    vtx, tri, vkeys = vtx.cpu().numpy(), tri.cpu().numpy().astype(np.int64), vkeys.cpu().numpy().astype(np.int64)
    m = oracle.OracleMesh(xyz.cpu().numpy(), lv.cpu().numpy())
    r = m.iso(s.cpu().numpy(), m.duals(), iso, want_keys=True)
    ovtx, otri, okeys = oracle.weld(r["tris"], r["keys"])
    # vertices: one per edge key, same keys, bit-exact positions
    assert vtx.shape[0] == ovtx.shape[0] and tri.shape[0] == otri.shape[0]
    order = np.lexsort(vkeys.T[::-1])
    assert np.array_equal(vkeys[order], okeys)
    assert np.array_equal(vtx[order].view(np.int32), ovtx.view(np.int32))
    assert tri.min(initial=0) >= 0 and tri.max(initial=-1) < vtx.shape[0]
    # triangles: the same edge-key triples with the same orientation
    assert np.array_equal(_key_triangles(tri, vkeys), _key_triangles(otri, okeys))
    # and the same surface as the fat triangles of amr_iso
    assert np.array_equal(canonical(vtx[tri]).view(np.int32), canonical(fat).view(np.int32))
    return vtx.shape[0], tri.shape[0]


def test_sphere_indexed():
    nv, nt = _check(*synth.sphere_tiny()[:4])
    assert nv - (3 * nt // 2) + nt == 2   # closed sphere: V - E + F = 2


@pytest.mark.parametrize("seed", range(6))
def test_random_octrees_indexed(seed):
    xyz, lv, s, iso, info = synth.random_octree(300 + seed, levels=2 + seed % 3, roots=4, p_split=0.45,
                                                p_hole=0.05, field="random" if seed % 2 else "sphere")
    _check(xyz, lv, s, iso, host=bool(seed % 2))


def test_octree_gaussians_indexed():
    xyz, lv, s, iso, info = synth.octree_gaussians(seed=21, roots=6, root_level=4)
    _check(xyz, lv, s, iso)


def test_indexed_capacity_reports_exact_counts():
    from paper_2004_08475_b300 import amriso
    xyz, lv, s, iso, info = synth.sphere_tiny()
    ctx = amriso.AmrContext()
    ctx.upload(xyz.cuda(), lv.cuda(), s.cuda())
    ctx.build_locator()
    ctx.dual_cells()
    v, t, k = ctx.iso_indexed(iso)
    import ctypes
    nv, nt = ctypes.c_int64(0), ctypes.c_int64(0)
    vb = torch.empty((4, 3), dtype=torch.float32, device="cuda")
    tb = torch.empty((4, 3), dtype=torch.int32, device="cuda")
    rc = amriso.lib().amr_iso_indexed(ctx._h, ctypes.c_float(iso), vb.data_ptr(), 4, tb.data_ptr(), 4, None,
                                      ctypes.byref(nv), ctypes.byref(nt), amriso.DEVICE_PTRS)
    assert rc == amriso.ERR_CAPACITY and nv.value == v.shape[0] and nt.value == t.shape[0]


@pytest.mark.parametrize("host", [False, True])
def test_interpolate_matches_oracle(host):
    """amr_interpolate: a second field at the indexed vertices, bit-exact
    against the oracle; with the centres' x it reproduces the vertices' x."""
    from paper_2004_08475_b300 import amriso
    xyz, lv, s, iso, info = synth.octree_gaussians(seed=23, roots=6, root_level=4)
    ctx = amriso.AmrContext()
    ctx.upload(xyz.cuda(), lv.cuda(), s.cuda())
    ctx.build_locator()
    ctx.dual_cells()
    vtx, tri, vkeys = ctx.iso_indexed(iso)
    attr = synth.uniform01(77, torch.arange(xyz.shape[0])).to(torch.float32) * 100.0 - 50.0
    dev = "cpu" if host else "cuda"
    got = ctx.interpolate(iso, attr.to(dev), vkeys.to(dev)).cpu().numpy()
    want = oracle.interpolate(xyz.numpy(), s.numpy(), attr.numpy(), vkeys.cpu().numpy(), iso)
    assert np.array_equal(got.view(np.int32), want.view(np.int32))
    cx = xyz[:, 0].to(torch.float32) + (2.0 ** lv.to(torch.float32)) * 0.5
    gx = ctx.interpolate(iso, cx.to(dev), vkeys.to(dev)).cpu().numpy()
    assert np.array_equal(gx.view(np.int32), vtx[:, 0].cpu().numpy().view(np.int32))


def test_interpolate_rejects_bad_cell_index():
    from paper_2004_08475_b300 import amriso
    xyz, lv, s, iso, info = synth.sphere_tiny()
    ctx = amriso.AmrContext()
    ctx.upload(xyz.cuda(), lv.cuda(), s.cuda())
    keys = torch.tensor([[0, 1], [0, xyz.shape[0]]], dtype=torch.int32, device="cuda")
    with pytest.raises(amriso.AmrError) as e:
        ctx.interpolate(iso, s.cuda(), keys)
    assert e.value.code == amriso.ERR_RANGE


@pytest.mark.parametrize("seed", range(4))
def test_dual_shapes_match_oracle(seed):
    """amr_dual_shapes: per-dual distinct-cell counts and their histogram,
    against the oracle on the same dual list (matched through get_duals)."""
    from paper_2004_08475_b300 import amriso
    xyz, lv, s, iso, info = synth.random_octree(500 + seed, levels=2 + seed % 3, roots=4, p_split=0.45,
                                                p_hole=0.05)
    ctx = amriso.AmrContext()
    ctx.upload(xyz.cuda(), lv.cuda(), s.cuda())
    ctx.build_locator()
    ctx.dual_cells()
    counts, hist = ctx.dual_shapes()
    d = ctx.get_duals().cpu().numpy()
    want = oracle.dual_shapes(d)
    assert np.array_equal(counts.cpu().numpy(), want)
    assert np.array_equal(hist, np.bincount(want, minlength=9))
    m = oracle.OracleMesh(xyz.numpy(), lv.numpy())
    assert np.array_equal(np.sort(oracle.dual_shapes(m.duals())), np.sort(want))


def test_next_rows_on_empty_outputs():
    """Degenerate cases: an iso-value above every scalar (no triangles), an
    empty data set and a single cell (no duals) give empty indexed face sets,
    empty attribute lists and an all-zero shape histogram, like the oracle."""
    from paper_2004_08475_b300 import amriso
    xyz, lv, s, iso, info = synth.sphere_tiny()
    ctx = amriso.AmrContext()
    ctx.upload(xyz.cuda(), lv.cuda(), s.cuda())
    ctx.build_locator()
    ctx.dual_cells()
    above = float(s.max()) + 1.0
    for host in (False, True):
        vtx, tri, vkeys = ctx.iso_indexed(above, host=host)
        assert vtx.shape == (0, 3) and tri.shape == (0, 3) and vkeys.shape == (0, 2)
    assert ctx.interpolate(above, s.cuda(), vkeys.cuda()).shape == (0,)
    assert ctx.interpolate(above, s.clone(), vkeys.cpu()).shape == (0,)
    m = oracle.OracleMesh(xyz.numpy(), lv.numpy())
    r = m.iso(s.numpy(), m.duals(), above, want_keys=True)
    assert r["tris"].shape[0] == 0 and oracle.weld(r["tris"], r["keys"])[0].shape == (0, 3)
    for cells in (0, 1):
        ctx.upload(torch.tensor([[4, 8, -12]][:cells], dtype=torch.int32, device="cuda").reshape(-1, 3),
                   torch.tensor([2][:cells], dtype=torch.uint8, device="cuda"),
                   torch.tensor([1.0][:cells], dtype=torch.float32, device="cuda"))
        ctx.build_locator()
        assert ctx.dual_cells() == 0
        counts, hist = ctx.dual_shapes()
        assert counts.shape == (0,) and not hist.any()
        assert oracle.dual_shapes(np.zeros((0, 8), np.int64)).shape == (0,)
        vtx, tri, vkeys = ctx.iso_indexed(0.5)
        assert vtx.shape[0] == 0 and tri.shape[0] == 0
    ctx.close()
