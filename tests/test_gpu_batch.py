"""Batched iso-values (amr_iso_batch, amr_iso_batch_async) against the oracle,
segment by segment: every iso-value's segment holds exactly the triangles the
oracle's Marching Cubes gives at that value (Sec. 5), bit for bit after
canonical ordering.

Cases: the 16 iso-values iso0 * 2^((k-8)/4), k = 0..15, of the large wing
workload on a reduced wing (all four levels, holes); a dense field (uniform
random scalars) where more than 80 triangles fall among 32 consecutive dual
cells; +inf padding (no triangles, as the server pads batches); and a
capacity shorter than the total on the device-side entry point, where only
rows below the capacity are written and each holds a triangle of its
iso-value."""
from collections import Counter

import numpy as np
import pytest
import torch

import oracle
from paper_2004_08475_b300 import synth
from tests.parity import canonical

pytestmark = pytest.mark.gpu


def _reduced_wing():
    # 146k cells, widths 1-8, holes inside the wing, log-normal scalar
    return synth.wing_bands(dims=(32, 32, 8), scale=1 / 14, bands=(25.0, 40.0, 62.0))


def _context(xyz, lv, s):
    from paper_2004_08475_b300 import amriso
    ctx = amriso.AmrContext()
    ctx.upload(xyz.cuda(), lv.cuda(), s.cuda())
    ctx.build_locator()
    ctx.dual_cells()
    return ctx


def _rows(t):
    """Multiset of canonical triangle rows (orientation kept) as bytes."""
    c = canonical(np.asarray(t, dtype=np.float32))
    return Counter(r.tobytes() for r in c.reshape(-1, 9))


def _check_segments(tris, offs, m, duals, s, isos):
    total = 0
    for k, v in enumerate(isos):
        r = m.iso(s, duals, np.float32(v), want_keys=False)
        seg = tris[int(offs[k]):int(offs[k + 1])].cpu().numpy()
        assert seg.shape[0] == r["tris"].shape[0], (k, v)
        assert (canonical(seg) == canonical(r["tris"])).all(), (k, v)
        total += seg.shape[0]
    return total


def test_batch_16_isos_reduced_wing_match_oracle():
    xyz, lv, s, iso0, info = _reduced_wing()
    assert int(lv.max()) == 3 and info["n"] > 100_000
    isos = [float(np.float32(iso0 * 2.0 ** ((k - 8) / 4))) for k in range(16)]
    ctx = _context(xyz, lv, s)
    tris, offs = ctx.iso_batch(isos)
    m = oracle.OracleMesh(xyz.numpy(), lv.numpy())
    d = m.duals()
    assert d.shape[0] == ctx.n_dual
    total = _check_segments(tris, offs, m, d, s.numpy(), isos)
    assert total == int(offs[-1]) > 10_000
    ctx.close()


def test_batch_dense_field_and_inf_padding_match_oracle():
    xyz, lv, s, iso, info = synth.uniform_grid(40, 0, field="random")
    isos = [0.5, 0.3, float("inf"), 0.7, 0.5, float("inf")]
    ctx = _context(xyz, lv, s)
    # the dense case: some 32 consecutive duals carry more than 80 triangles
    _, ntri = ctx.iso_cases(0.5)
    n = ntri.shape[0] // 32 * 32
    assert int(ntri[:n].view(-1, 32).int().sum(1).max()) > 80
    tris, offs = ctx.iso_batch(isos)
    m = oracle.OracleMesh(xyz.numpy(), lv.numpy())
    d = m.duals()
    _check_segments(tris, offs, m, d, s.numpy(), isos)
    assert int(offs[3]) == int(offs[2]) and int(offs[6]) == int(offs[5])   # +inf: empty segments
    ctx.close()


def test_batch_async_short_capacity():
    xyz, lv, s, iso0, info = _reduced_wing()
    isos = [iso0 * 0.8, iso0, iso0 * 1.3]
    ctx = _context(xyz, lv, s)
    _, offs_full = ctx.iso_batch(isos)
    total = int(offs_full[-1])
    cap = total * 2 // 3
    sentinel = 1234.5
    out = torch.full((total + 64, 3, 3), sentinel, dtype=torch.float32, device="cuda")
    d_iso = torch.tensor(isos, dtype=torch.float32, device="cuda")
    d_off = torch.zeros(len(isos) + 1, dtype=torch.int64, device="cuda")
    ctx.iso_batch_async(d_iso, out[:cap], d_off)
    torch.cuda.synchronize()
    offs = d_off.cpu().tolist()
    assert offs == offs_full.tolist() and offs[-1] > cap
    assert (out[cap:] == sentinel).all(), "rows past the capacity were written"
    m = oracle.OracleMesh(xyz.numpy(), lv.numpy())
    d = m.duals()
    for k, v in enumerate(isos):
        lo, hi = offs[k], min(offs[k + 1], cap)
        if hi <= lo:
            continue
        want = _rows(m.iso(s.numpy(), d, np.float32(v), want_keys=False)["tris"])
        got = _rows(out[lo:hi].cpu().numpy())
        assert sum(got.values()) == hi - lo
        assert all(want[r] >= c for r, c in got.items()), f"segment {k}: a row that is not the oracle's"
    ctx.close()


def test_multi_dataset_batch_matches_oracle():
    """One batch over three data sets of different sizes, depths and brick
    sizes (amr_iso_multi_async): every (data set, iso-value) segment holds
    exactly the oracle's triangles."""
    from paper_2004_08475_b300 import amriso
    sets = [(_reduced_wing(), 3, 5), (synth.random_octree(31, levels=4, roots=5, p_split=0.45, p_hole=0.06,
                                                          field="random"), 2, 3),
            (synth.sphere_tiny(), 3, 2)]
    ctxs, isos, n_isos, refs = [], [], [], []
    for (xyz, lv, s, iso0, info), logb, k in sets:
        ctx = amriso.AmrContext()
        ctx.upload(xyz.cuda(), lv.cuda(), s.cuda())
        ctx.build_locator(log2_brick=logb)
        ctx.dual_cells()
        vals = [float(np.float32(iso0 * (0.8 + 0.15 * q))) for q in range(k)]
        ctxs.append(ctx)
        isos += vals
        n_isos.append(k)
        m = oracle.OracleMesh(xyz.numpy(), lv.numpy())
        d = m.duals()
        refs += [m.iso(s.numpy(), d, np.float32(v), want_keys=False)["tris"] for v in vals]
    total = sum(r.shape[0] for r in refs)
    ws = torch.empty(amriso.iso_multi_workspace(ctxs, n_isos), dtype=torch.uint8, device="cuda")
    out = torch.empty((total + 16, 3, 3), dtype=torch.float32, device="cuda")
    d_iso = torch.tensor(isos, dtype=torch.float32, device="cuda")
    d_off = torch.zeros(len(isos) + 1, dtype=torch.int64, device="cuda")
    amriso.iso_multi_async(ctxs, n_isos, d_iso, out, d_off, ws)
    torch.cuda.synchronize()
    offs = d_off.cpu().tolist()
    assert offs[-1] == total > 0
    for q, ref in enumerate(refs):
        seg = out[offs[q]:offs[q + 1]].cpu().numpy()
        assert seg.shape[0] == ref.shape[0], q
        assert (canonical(seg) == canonical(ref)).all(), q
    for c in ctxs:
        c.close()
