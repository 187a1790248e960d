"""GPU-vs-oracle parity helpers (used by the gpu-marked tests, the smoke check
and nothing in the product)."""
from __future__ import annotations

import numpy as np
import torch

import oracle


def run_gpu(xyz, lv, s, iso, log2_brick=3, check_overlap=False, host_upload=False, partitioned=0):
    from paper_2004_08475_b300 import amriso
    ctx = amriso.AmrContext()
    if host_upload:
        ctx.upload(xyz.cpu(), lv.cpu(), s.cpu())
    else:
        ctx.upload(xyz.cuda(), lv.cuda(), s.cuda())
    ctx.build_locator(log2_brick=log2_brick, check_overlap=check_overlap, partitioned=partitioned)
    nd = ctx.dual_cells()
    duals = ctx.get_duals().cpu().numpy().astype(np.int64)
    cases, ntri = ctx.iso_cases(iso)
    tris = ctx.iso(iso).cpu().numpy()
    info = ctx.info()
    torch.cuda.synchronize()
    return {"ctx": ctx, "nd": nd, "duals": duals, "cases": cases.cpu().numpy(),
            "ntri": ntri.cpu().numpy(), "tris": tris, "info": info}


def run_oracle(xyz, lv, s, iso):
    x = xyz.cpu().numpy()
    l = lv.cpu().numpy()
    v = s.cpu().numpy()
    m = oracle.OracleMesh(x, l)
    d = m.duals()
    r = m.iso(v, d, iso, want_keys=False)
    return {"duals": d, "cases": r["cases"], "ntri": r["ntri"], "tris": r["tris"],
            "max_err": r["max_err"]}


def _by_tuple(d, *cols):
    order = np.lexsort(d.T[::-1])
    return (d[order],) + tuple(c[order] for c in cols)


def canonical(tris):
    """Each triangle rotated (orientation kept) to start at its smallest
    vertex by (z, y, x) bit patterns; then the rows sorted."""
    t = np.asarray(tris, dtype=np.float32).reshape(-1, 3, 3)
    bits = t.view(np.int32).astype(np.int64)
    k = np.stack([bits[:, :, 2], bits[:, :, 1], bits[:, :, 0]], -1)
    best = np.zeros(t.shape[0], dtype=np.int64)
    rows = np.arange(t.shape[0])
    for c in (1, 2):
        a = k[rows, c]
        b = k[rows, best]
        less = (a[:, 0] < b[:, 0]) | ((a[:, 0] == b[:, 0]) & ((a[:, 1] < b[:, 1]) |
                                                              ((a[:, 1] == b[:, 1]) & (a[:, 2] < b[:, 2]))))
        best = np.where(less, c, best)
    idx = (best[:, None] + np.arange(3)[None]) % 3
    r = np.take_along_axis(t, idx[:, :, None], axis=1).reshape(-1, 9)
    order = np.lexsort(r.view(np.int32).T[::-1])
    return r[order].reshape(-1, 3, 3)


def compare(g, o, extent, tol_rel=1e-5):
    """Bit-exact duals, cases and triangle counts; vertices within
    tol_rel * extent after canonical ordering. Returns a summary dict."""
    gd, gc, gn = _by_tuple(g["duals"], g["cases"], g["ntri"])
    od, oc, on = _by_tuple(o["duals"], o["cases"], o["ntri"])
    assert gd.shape == od.shape, (gd.shape, od.shape)
    assert (gd == od).all(), "dual cells differ"
    assert (gc == oc).all(), "case indices differ"
    assert (gn == on).all(), "per-dual triangle counts differ"
    assert g["tris"].shape[0] == o["tris"].shape[0] == int(on.sum())
    gt, ot = canonical(g["tris"]), canonical(o["tris"])
    diff = np.abs(gt.astype(np.float64) - ot.astype(np.float64)).max() if gt.size else 0.0
    assert diff <= tol_rel * extent, diff
    exact = float((gt == ot).all(axis=(1, 2)).mean()) if gt.size else 1.0
    return {"duals": int(gd.shape[0]), "tris": int(gt.shape[0]), "max_diff": float(diff),
            "bit_exact_frac": exact}


def owners_of(duals, xyz, lv):
    """Owner cell of each dual: the vertex with the smallest (level, z, y, x)
    (rules 2 and 3 make the owner the finest, then lowest, vertex)."""
    x = xyz[duals].astype(np.int64)   # [D, 8, 3]
    l = lv[duals].astype(np.int64)    # [D, 8]
    key = (l << 60) + ((x[..., 2] + (1 << 21)) << 40) + ((x[..., 1] + (1 << 21)) << 20) + \
        (x[..., 0] + (1 << 21))
    j = np.argmin(key, axis=1)
    return duals[np.arange(duals.shape[0]), j]
