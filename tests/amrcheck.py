"""Shared test helpers: brute-force dual enumeration, mesh topology checks and
canonicalisation. These restate definitions (not the oracle's code) so that
they can pin the oracle."""
from __future__ import annotations

import numpy as np

# corner e = ex + 2 ey + 4 ez of a hexahedron
CORNERS = np.array([[e & 1, (e >> 1) & 1, (e >> 2) & 1] for e in range(8)], dtype=np.int64)


def voxelize(xyz, level, pad=0):
    """Dense finest-level array of cell indices (-1: no cell); origin at the
    bounding-box minimum minus `pad`."""
    xyz = np.asarray(xyz, dtype=np.int64)
    level = np.asarray(level, dtype=np.int64)
    w = 1 << level
    lo = xyz.min(0) - pad
    hi = (xyz + w[:, None]).max(0) + pad
    dims = hi - lo
    vox = -np.ones(tuple(dims[::-1]), dtype=np.int64)   # [z, y, x]
    for c in range(xyz.shape[0]):
        x, y, z = xyz[c] - lo
        ww = w[c]
        blk = vox[z:z + ww, y:y + ww, x:x + ww]
        assert (blk == -1).all(), "overlapping cells"
        blk[...] = c
    return vox, lo


def brute_duals(xyz, level):
    """Every logical dual D^(l) on every level whose 8 vertices (logical
    level-l cells) all lie in actual cells, none finer than l, at least one of
    level l. Vertex cells are found through a dense voxel array (a different
    mechanism from the oracle's ordered map). Returns sorted [D, 8] tuples."""
    xyz = np.asarray(xyz, dtype=np.int64)
    level = np.asarray(level, dtype=np.int64)
    wmax = 1 << int(level.max())
    vox, lo = voxelize(xyz, level, pad=2 * wmax)
    nz, ny, nx = vox.shape
    out = []
    for l in range(int(level.max()) + 1):
        w = 1 << l
        # lattice of level-l logical cells (in voxel coordinates, aligned)
        start = [(-int(lo[a])) % w for a in range(3)]
        axes = [np.arange(start[a], dim - w, w) for a, dim in enumerate((nx, ny, nz))]
        X, Y, Z = np.meshgrid(*axes, indexing="ij")
        base = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
        verts = np.empty((base.shape[0], 8), dtype=np.int64)
        for e in range(8):
            q = base + CORNERS[e] * w
            ok = (q < np.array([nx, ny, nz])).all(1)
            v = -np.ones(base.shape[0], dtype=np.int64)
            v[ok] = vox[q[ok, 2], q[ok, 1], q[ok, 0]]
            verts[:, e] = v
        good = (verts >= 0).all(1)
        verts = verts[good]
        if verts.shape[0] == 0:
            continue
        lv = level[verts]
        keep = lv.min(1) == l
        out.append(verts[keep])
    if not out:
        return np.zeros((0, 8), dtype=np.int64)
    return sort_rows(np.concatenate(out))


def sort_rows(a):
    a = np.asarray(a)
    if a.shape[0] == 0:
        return a
    idx = np.lexsort(a.T[::-1])
    return a[idx]


def edge_mesh(keys):
    """Vertex ids and directed edges of a triangle mesh whose vertices are
    identified by edge keys [T,3,2] (pairs of cell ids)."""
    k = np.asarray(keys, dtype=np.int64).reshape(-1, 2)
    uniq, inv = np.unique(k, axis=0, return_inverse=True)
    tri = inv.reshape(-1, 3)
    return uniq, tri


def manifold_report(tri):
    """Counts of undirected edges by multiplicity and orientation consistency."""
    tri = np.asarray(tri, dtype=np.int64)
    a = np.concatenate([tri[:, 0], tri[:, 1], tri[:, 2]])
    b = np.concatenate([tri[:, 1], tri[:, 2], tri[:, 0]])
    und = np.stack([np.minimum(a, b), np.maximum(a, b)], 1)
    ue, cnt = np.unique(und, axis=0, return_counts=True)
    directed = np.stack([a, b], 1)
    de, dcnt = np.unique(directed, axis=0, return_counts=True)
    return {"edges": ue, "edge_count": cnt, "directed_max": int(dcnt.max()) if len(dcnt) else 0,
            "V": int(np.unique(tri).shape[0]), "E": int(ue.shape[0]), "F": int(tri.shape[0])}


def signed_volume(tris):
    """Volume enclosed by a closed oriented triangle mesh (divergence theorem)."""
    t = np.asarray(tris, dtype=np.float64)
    return float(np.einsum("ij,ij->i", t[:, 0], np.cross(t[:, 1], t[:, 2])).sum() / 6.0)


def canonical_triangles(tris, keys=None):
    """Rotate each triangle (keeping orientation) so that its smallest vertex
    comes first, then sort the list. With `keys`, order by edge keys."""
    t = np.asarray(tris, dtype=np.float32).reshape(-1, 3, 3)
    if keys is not None:
        k = np.asarray(keys, dtype=np.int64).reshape(-1, 3, 2)
        sk = k[:, :, 0] * (1 << 31) + k[:, :, 1]
        first = np.argmin(sk, axis=1)
    else:
        v = t.view(np.int32).astype(np.int64)
        sk = (v[:, :, 0] << 40) ^ (v[:, :, 1] << 20) ^ v[:, :, 2]
        first = np.argmin(sk, axis=1)
    idx = (first[:, None] + np.arange(3)[None]) % 3
    rt = np.take_along_axis(t, idx[:, :, None], axis=1)
    flat = rt.reshape(-1, 9)
    order = np.lexsort(flat.view(np.int32).T[::-1])
    if keys is not None:
        rk = np.take_along_axis(k, idx[:, :, None], axis=1).reshape(-1, 6)
        order = np.lexsort(rk.T[::-1])
        return rt[order], rk[order].reshape(-1, 3, 2)
    return rt[order], None
