"""Pins of the oracle's Marching Cubes on dual cells (Sec. 5) against
properties that do not depend on its triangulation code: the face rule checked
from its definition on all 256 cases, closed oriented 2-manifolds with the
right Euler characteristic and enclosed volume, the table-independent vertex
set, the convexity bound on the sphere, the fp64 cross-check, ties, and a
hand-derived golden example."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2004_08475_b300 import synth
from tests.amrcheck import CORNERS, edge_mesh, manifold_report, signed_volume, voxelize

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
EDGES = oracle.EDGES


def _np(*ts):
    return [t.numpy() if hasattr(t, "numpy") else t for t in ts]


def _faces_of_edge(e):
    a, b = EDGES[e]
    ca, cb = CORNERS[a], CORNERS[b]
    out = []
    for axis in range(3):
        if ca[axis] == cb[axis]:
            out.append((axis, int(ca[axis])))
    return out


def _face_corners(face):
    axis, side = face
    return [v for v in range(8) if CORNERS[v][axis] == side]


@pytest.mark.parametrize("case", range(256))
def test_case_face_rule(case):
    """Definition of the face rule: the loops' boundary on each face of the
    cube pairs the crossed edges of that face, and on a face with four crossed
    edges each pair shares an inside corner (inside corners are cut off)."""
    inside = [(case >> v) & 1 for v in range(8)]
    crossed = {e for e, (a, b) in enumerate(EDGES) if inside[a] != inside[b]}
    tri = oracle.case_triangles(case)
    assert tri.shape[0] <= 5
    used = set(tri.ravel().tolist())
    assert used == crossed
    # boundary of the triangle fan: undirected sides used once
    sides = {}
    for t in tri:
        for i in range(3):
            a, b = int(t[i]), int(t[(i + 1) % 3])
            k = (min(a, b), max(a, b))
            sides[k] = sides.get(k, 0) + 1
            assert a != b
    assert all(c <= 2 for c in sides.values())
    boundary = [k for k, c in sides.items() if c == 1]
    interior = [k for k, c in sides.items() if c == 2]
    # every boundary side lies on exactly one cube face
    per_face = {}
    for (a, b) in boundary:
        common = set(_faces_of_edge(a)) & set(_faces_of_edge(b))
        assert len(common) == 1, (case, a, b)
        per_face.setdefault(common.pop(), []).append((a, b))
    # interior sides (fan diagonals) are never both on one face
    for face in [(ax, sd) for ax in range(3) for sd in range(2)]:
        fc = _face_corners(face)
        fe = [e for e, (a, b) in enumerate(EDGES) if a in fc and b in fc]
        fx = [e for e in fe if e in crossed]
        segs = sorted(per_face.get(face, []))
        if len(fx) == 0:
            assert segs == []
        elif len(fx) == 2:
            assert segs == [tuple(sorted(fx))]
        else:
            assert len(fx) == 4
            want = []
            for v in fc:
                if inside[v]:
                    inc = sorted(e for e in fe if v in EDGES[e])
                    want.append(tuple(inc))
            assert segs == sorted(want)
    # orientation consistency inside the case: interior sides run both ways
    directed = set()
    for t in tri:
        for i in range(3):
            d = (int(t[i]), int(t[(i + 1) % 3]))
            assert d not in directed
            directed.add(d)


def test_no_triangle_lies_in_a_cube_face():
    """Face rule, last clause: no triangle of any case has its three vertices
    on one face of the cube (a neighbouring dual shares that face, and a flat
    triangle there would fold the surface into the face)."""
    for case in range(256):
        for t in oracle.case_triangles(case):
            common = set(_faces_of_edge(int(t[0]))) & set(_faces_of_edge(int(t[1]))) & \
                set(_faces_of_edge(int(t[2])))
            assert not common, (case, t.tolist())


def test_case_count_histogram():
    """Up to 5 triangles per case (Sec. 5.2); cases 0 and 255 are empty."""
    counts = [oracle.case_triangles(c).shape[0] for c in range(256)]
    assert max(counts) == 5 and counts[0] == 0 and counts[255] == 0
    assert all(counts[c] == 1 for c in (1, 2, 4, 8, 16, 32, 64, 128))


def test_single_corner_orientation():
    """A lone inside corner (s > iso) gets one triangle whose normal points
    away from it, toward decreasing s."""
    for v in range(8):
        tri = oracle.case_triangles(1 << v)[0]
        p = []
        for e in tri:
            a, b = EDGES[e]
            p.append(0.5 * (CORNERS[a] + CORNERS[b]))
        n = np.cross(p[1] - p[0], p[2] - p[0])
        assert np.dot(n, np.mean(p, 0) - CORNERS[v]) > 0


def _run(gen):
    xyz, lv, s, iso, info = gen
    xyz, lv, s = _np(xyz, lv, s)
    m = oracle.OracleMesh(xyz, lv)
    d = m.duals()
    r = m.iso(s, d, iso)
    return xyz, lv, s, iso, m, d, r


def _crossed_dual_edges(d, s, iso):
    inside = s[d] > iso
    keys = set()
    for a, b in EDGES:
        x = inside[:, a] != inside[:, b]
        ca, cb = d[x, a], d[x, b]
        for u, v in zip(np.minimum(ca, cb), np.maximum(ca, cb)):
            keys.add((int(u), int(v)))
    return keys


def test_sphere_closed_manifold():
    xyz, lv, s, iso, m, d, r = _run(synth.sphere_tiny())
    uniq, tri = edge_mesh(r["keys"])
    rep = manifold_report(tri)
    assert (rep["edge_count"] == 2).all(), "every edge shared by exactly two triangles"
    assert rep["directed_max"] == 1, "consistent orientation"
    assert rep["V"] - rep["E"] + rep["F"] == 2, "Euler characteristic of a sphere"
    # vertex set = the sign-changing dual edges (independent of any table)
    assert {tuple(k) for k in uniq.tolist()} == _crossed_dual_edges(d, s, iso)
    # convexity: interpolated vertices lie inside the radius-8 sphere
    dist = np.sqrt(((r["tris"].reshape(-1, 3).astype(np.float64) - 16.0) ** 2).sum(1))
    assert dist.max() <= 8.0 + 1e-4
    assert dist.min() > 6.0
    # normals point toward decreasing s, i.e. inward here: negative volume
    vol = signed_volume(r["tris"])
    assert abs(vol + 4.0 / 3.0 * math.pi * 512.0) < 0.05 * 4.0 / 3.0 * math.pi * 512.0
    # fp32 against fp64: within 4 ulp of the extent (32)
    assert r["max_err"] <= 4 * np.spacing(np.float32(32.0))


@pytest.mark.parametrize("seed", range(12))
def test_random_octree_sphere_field(seed):
    """Smooth field on random octrees without holes: the surface is a closed,
    consistently oriented 2-manifold with one component per sphere."""
    gen = synth.random_octree(seed, levels=3 + seed % 2, roots=4 if seed % 2 == 0 else 3,
                              p_split=0.5, p_hole=0.0, field="sphere")
    xyz, lv, s, iso, m, d, r = _run(gen)
    assert r["tris"].shape[0] > 0
    uniq, tri = edge_mesh(r["keys"])
    rep = manifold_report(tri)
    assert (rep["edge_count"] == 2).all()
    assert rep["directed_max"] == 1
    assert rep["V"] - rep["E"] + rep["F"] == 2
    assert {tuple(k) for k in uniq.tolist()} <= _crossed_dual_edges(d, s, iso)
    assert signed_volume(r["tris"]) < 0


def _interior_cells(xyz, lv):
    """Cells whose one-width neighbourhood is fully covered by cells."""
    vox, lo = voxelize(xyz, lv, pad=2 * (1 << int(lv.max())))
    covered = vox >= 0
    cs = np.pad(np.cumsum(np.cumsum(np.cumsum(covered, 0), 1), 2), ((1, 0), (1, 0), (1, 0)))
    out = np.zeros(xyz.shape[0], dtype=bool)
    for c in range(xyz.shape[0]):
        w = 1 << int(lv[c])
        a = xyz[c] - lo - w
        b = xyz[c] - lo + 2 * w
        x0, y0, z0 = a
        x1, y1, z1 = b
        tot = (cs[z1, y1, x1] - cs[z0, y1, x1] - cs[z1, y0, x1] - cs[z1, y1, x0]
               + cs[z0, y0, x1] + cs[z0, y1, x0] + cs[z1, y0, x0] - cs[z0, y0, x0])
        out[c] = tot == (3 * w) ** 3
    return out


def _oriented_boundary(tri):
    """Undirected edges whose forward and backward uses do not cancel."""
    a = np.concatenate([tri[:, 0], tri[:, 1], tri[:, 2]])
    b = np.concatenate([tri[:, 1], tri[:, 2], tri[:, 0]])
    lo_, hi_ = np.minimum(a, b), np.maximum(a, b)
    sign = np.where(a < b, 1, -1)
    key = lo_ * (int(tri.max()) + 1) + hi_
    uk, inv = np.unique(key, return_inverse=True)
    net = np.zeros(uk.shape[0], dtype=np.int64)
    np.add.at(net, inv, sign)
    bad = uk[net != 0]
    n = int(tri.max()) + 1
    return np.stack([bad // n, bad % n], 1)


@pytest.mark.parametrize("seed", range(16))
@pytest.mark.parametrize("p_hole", [0.0, 0.07])
def test_random_field_crack_free(seed, p_hole):
    """Random fields, level jumps, holes: crack-freeness (Sec. 5) in the
    oriented sense - the boundary of the oriented triangle chain vanishes
    except at cells next to holes or the domain boundary. (On degenerate
    duals two neighbours may both emit one flat triangle on their shared,
    collapsed face with opposite orientations; those cancel in the chain.)
    No triangle repeats a vertex key."""
    gen = synth.random_octree(seed, levels=2 + seed % 3, roots=4, p_split=0.4, p_hole=p_hole)
    xyz, lv, s, iso, m, d, r = _run(gen)
    keys = r["keys"]
    if keys.shape[0] == 0:
        return
    uniq, tri = edge_mesh(keys)
    assert (tri[:, 0] != tri[:, 1]).all() and (tri[:, 1] != tri[:, 2]).all() and \
        (tri[:, 0] != tri[:, 2]).all()
    inner = _interior_cells(xyz.astype(np.int64), lv.astype(np.int64))
    for u, v in _oriented_boundary(tri):
        cells = np.concatenate([uniq[u], uniq[v]])
        assert not inner[cells].all(), (seed, uniq[u], uniq[v])
    assert r["max_err"] <= 4 * np.spacing(np.float32(64.0))


def test_uniform_random_field_boundary():
    """On a uniform grid with a random field, edges used once lie on the
    boundary of the grid of cell centres."""
    n = 9
    xyz, lv, s, iso, m, d, r = _run(synth.uniform_grid(n, 0, (0, 0, 0), seed=3))
    uniq, tri = edge_mesh(r["keys"])
    rep = manifold_report(tri)
    assert rep["edge_count"].max() <= 2 and rep["directed_max"] == 1
    once = rep["edges"][rep["edge_count"] == 1]
    for u, v in once:
        cells = np.concatenate([uniq[u], uniq[v]])
        p = xyz[cells]
        on = [(p[:, a] == 0).all() or (p[:, a] == n - 1).all() for a in range(3)]
        assert any(on)
    # count check: every case's triangle count from the face walk
    cases = r["cases"]
    per_case = np.array([oracle.case_triangles(c).shape[0] for c in range(256)])
    assert int(per_case[cases].sum()) == r["tris"].shape[0]


def test_uniform_sphere_euler():
    xyz, lv, s, iso, m, d, r = _run(synth.uniform_grid(14, 1, (4, 4, 4), field="sphere"))
    uniq, tri = edge_mesh(r["keys"])
    rep = manifold_report(tri)
    assert (rep["edge_count"] == 2).all() and rep["directed_max"] == 1
    assert rep["V"] - rep["E"] + rep["F"] == 2
    # closed sphere: F = 2V - 4 with V = number of sign-changing lattice edges
    assert rep["F"] == 2 * len(_crossed_dual_edges(d, s, iso)) - 4


def test_ties_kept_as_zero_area():
    """s == iso exactly: the corner counts as outside (strict >), and vertices
    on its edges land exactly on its centre (t = 0 from the canonical first
    endpoint). A 2^3 grid with s = 1 except s = iso at the origin cell is case
    254: one triangle with three different edge keys and zero area, kept."""
    xyz, lv, s, iso, info = synth.uniform_grid(2, 0, (0, 0, 0))
    xyz, lv = _np(xyz, lv)
    s = np.ones(xyz.shape[0], dtype=np.float32)
    tie = int(np.where((xyz == 0).all(1))[0][0])
    s[tie] = 0.5
    m = oracle.OracleMesh(xyz, lv)
    d = m.duals()
    r = m.iso(s, d, 0.5)
    corner0 = [e for e in range(8) if d[0][e] == tie][0]
    assert corner0 == 0 and int(r["cases"][0]) == 254
    assert r["tris"].shape[0] == 1
    k = r["keys"][0]
    assert len({tuple(x) for x in k.tolist()}) == 3 and (k == tie).any(1).all()
    assert (r["tris"][0] == np.float32(0.5)).all()


def test_golden_pyramid_mc():
    with open(os.path.join(GOLDEN, "two_level_pyramid.json")) as f:
        g = json.load(f)
    xyz = np.array(g["xyz"], dtype=np.int32)
    lv = np.array(g["level"], dtype=np.uint8)
    s = np.array(g["scalar"], dtype=np.float32)
    m = oracle.OracleMesh(xyz, lv)
    d = m.duals()
    r = m.iso(s, d, g["iso"])
    for t, c in zip(d, r["cases"]):
        assert g["cases"][" ".join(str(x) for x in t)] == int(c)
    assert r["tris"].shape[0] == g["n_triangles"]
    got = {tuple(v) for v in r["tris"].reshape(-1, 3).tolist()}
    assert got == {tuple(v) for v in g["triangle_vertices"]}


def test_weld_sphere_indexed_face_set():
    """The oracle's indexed face set (Sec. 5.2, vertices identified by edge
    key): it reproduces every fat triangle bit for bit, has one vertex per
    sign-changing dual edge, and is a closed sphere (V - E + F = 2)."""
    xyz, lv, s, iso, m, d, r = _run(synth.sphere_tiny())
    vtx, tri, vkeys = oracle.weld(r["tris"], r["keys"])
    assert np.array_equal(vtx[tri].view(np.int32), r["tris"].view(np.int32))
    assert {tuple(k) for k in vkeys.tolist()} == _crossed_dual_edges(d, s, iso)
    assert vtx.shape[0] < 3 * tri.shape[0] // 2   # vertices are shared
    rep = manifold_report(tri)
    assert rep["V"] - rep["E"] + rep["F"] == 2


def test_weld_rejects_two_positions_for_one_key():
    tris = np.zeros((2, 3, 3), np.float32)
    keys = np.array([[[0, 1], [1, 2], [0, 2]], [[0, 1], [1, 3], [0, 3]]], np.int64)
    oracle.weld(tris, keys)   # same positions: fine
    tris[1, 0, 0] = 1.0       # key (0,1) now at two positions
    with pytest.raises(oracle.OracleError):
        oracle.weld(tris, keys)
    v, t, k = oracle.weld(np.zeros((0, 3, 3), np.float32), np.zeros((0, 3, 2), np.int64))
    assert v.shape == (0, 3) and t.shape == (0, 3) and k.shape == (0, 2)


def test_interpolate_closed_forms():
    """Interpolating the centres' x coordinate reproduces every vertex's x
    bit for bit (the same formula on another field); interpolating the
    scalar itself gives the iso-value within a few ulp."""
    xyz, lv, s, iso, m, d, r = _run(synth.sphere_tiny())
    vtx, tri, vkeys = oracle.weld(r["tris"], r["keys"])
    x = np.asarray(xyz)
    centre_x = (x[:, 0].astype(np.float32) + (np.float32(1) * (1 << np.asarray(lv).astype(np.int64))).astype(np.float32)
                * np.float32(0.5)).astype(np.float32)
    fx = oracle.interpolate(x, s, centre_x, vkeys, iso)
    assert np.array_equal(fx.view(np.int32), vtx[:, 0].view(np.int32))
    fs = oracle.interpolate(x, s, s, vkeys, iso)
    assert np.abs(fs - np.float32(iso)).max() <= 8 * np.spacing(np.float32(abs(iso) + np.abs(np.asarray(s)).max()))
