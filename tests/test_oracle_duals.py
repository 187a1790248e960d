"""Pins of the oracle's dual-cell construction (Sec. 3-4) against definitions
that do not go through its code: brute-force snapping of every logical dual,
closed forms on uniform grids, a hand-derived two-level example, and the
containment invariant of every emitted vertex."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2004_08475_b300 import synth
from tests.amrcheck import CORNERS, brute_duals, sort_rows

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _np(*ts):
    return [t.numpy() if hasattr(t, "numpy") else t for t in ts]


def test_sphere_tiny_shape():
    """Config: 16^3 level-1 cells, 280 refined into 2240 level-0 cells."""
    xyz, lv, s, iso, info = synth.sphere_tiny()
    assert info["n"] == 6056 and info["refined"] == 280
    assert int((lv == 0).sum()) == 2240 and int((lv == 1).sum()) == 3816


def test_sphere_brute_force():
    xyz, lv, s, iso, info = synth.sphere_tiny()
    xyz, lv = _np(xyz, lv)
    m = oracle.OracleMesh(xyz, lv)
    got = sort_rows(m.duals())
    ref = brute_duals(xyz, lv)
    assert got.shape == ref.shape
    assert (got == ref).all()


@pytest.mark.parametrize("seed", list(range(60)))
def test_random_octree_brute_force(seed):
    levels = 2 + seed % 3
    xyz, lv, s, iso, info = synth.random_octree(seed, levels=levels, roots=4 if levels < 4 else 3,
                                                p_split=0.3 + 0.05 * (seed % 5),
                                                p_hole=0.0 if seed % 4 == 0 else 0.08)
    xyz, lv = _np(xyz, lv)
    m = oracle.OracleMesh(xyz, lv)
    d = m.duals()
    got = sort_rows(d)
    ref = brute_duals(xyz, lv)
    assert got.shape == ref.shape, (got.shape, ref.shape)
    assert (got == ref).all()
    # exactly once: no tuple twice
    if got.shape[0] > 1:
        assert not (got[1:] == got[:-1]).all(1).any()


@pytest.mark.parametrize("n,l,origin", [(2, 0, (0, 0, 0)), (5, 0, (3, -7, 11)), (4, 2, (-8, 4, 0)),
                                         (7, 1, (0, 0, -6))])
def test_uniform_closed_form(n, l, origin):
    """A uniform n^3 grid of one level has exactly (n-1)^3 duals, each the
    lattice cube p + e w (Sec. 3.1, dual definition)."""
    xyz, lv, s, iso, info = synth.uniform_grid(n, l, origin)
    xyz, lv = _np(xyz, lv)
    m = oracle.OracleMesh(xyz, lv)
    d = m.duals()
    assert d.shape[0] == (n - 1) ** 3
    w = 1 << l
    index = {tuple(p): i for i, p in enumerate(xyz.tolist())}
    exp = []
    for k in range(n - 1):
        for j in range(n - 1):
            for i in range(n - 1):
                p = np.array(origin) + np.array([i, j, k]) * w
                exp.append([index[tuple((p + CORNERS[e] * w).tolist())] for e in range(8)])
    assert (sort_rows(d) == sort_rows(np.array(exp))).all()


def test_vertex_containment_invariant():
    """Every vertex e of a dual owned by S lies in an actual cell that contains
    the logical cell q_e = p_S + (e - e_S) w; all vertices are level >= l_S."""
    xyz, lv, s, iso, info = synth.random_octree(11, levels=4, roots=3, p_split=0.45, p_hole=0.05)
    xyz, lv = _np(xyz, lv)
    xyz = xyz.astype(np.int64)
    lv = lv.astype(np.int64)
    m = oracle.OracleMesh(xyz, lv)
    d, owner = m.duals(with_owner=True)
    assert d.shape[0] > 100
    for t, o in zip(d, owner):
        es = [e for e in range(8) if t[e] == o]
        assert len(es) == 1
        es = es[0]
        w = 1 << lv[o]
        for e in range(8):
            q = xyz[o] + (CORNERS[e] - CORNERS[es]) * w
            c = t[e]
            wc = 1 << lv[c]
            assert lv[c] >= lv[o]
            assert (xyz[c] <= q).all() and (q + w <= xyz[c] + wc).all()


def test_golden_two_level():
    """Hand-derived example (Sec. 4.3): eight level-0 cells filling [0,2)^3 and
    one level-1 cell at (2,0,0). Exactly one cube dual (owned by the cell at
    the origin) and one pyramid dual (owned by (1,0,0)); the coarse cell owns
    nothing because all its level-1 duals reach finer cells or the outside."""
    with open(os.path.join(GOLDEN, "two_level_pyramid.json")) as f:
        g = json.load(f)
    xyz = np.array(g["xyz"], dtype=np.int32)
    lv = np.array(g["level"], dtype=np.uint8)
    m = oracle.OracleMesh(xyz, lv)
    d = sort_rows(m.duals())
    assert (d == sort_rows(np.array(g["duals"]))).all()


def test_invalid_inputs_rejected():
    with pytest.raises(oracle.OracleError):
        oracle.OracleMesh(np.array([[1, 0, 0]]), np.array([1]))      # unaligned
    with pytest.raises(oracle.OracleError):
        oracle.OracleMesh(np.array([[0, 0, 0], [0, 0, 0]]), np.array([0, 0]))  # duplicate


def test_snap_levels():
    """snap() returns the unique cell containing the point, at any level, or
    none (Sec. 3.2)."""
    xyz, lv, s, iso, info = synth.random_octree(5, levels=3, roots=4, p_hole=0.1)
    xyz, lv = _np(xyz, lv)
    m = oracle.OracleMesh(xyz, lv)
    from tests.amrcheck import voxelize
    vox, lo = voxelize(xyz, lv, pad=3)
    rng = np.random.default_rng(0)
    pts = rng.integers(0, np.array(vox.shape[::-1]), size=(2000, 3))
    for p in pts:
        want = vox[p[2], p[1], p[0]]
        got = m.snap(*(p + lo))
        assert got == want


def test_dual_shapes_pins():
    """Shapes of the snapped duals (Sec. 4.1): a uniform grid gives only
    hexahedra; the hand-derived two-level example gives one hexahedron and
    one pyramid (5 distinct cells); on random octrees no emitted dual
    collapses below 2 distinct cells (a level-l-owned dual reaches at least
    one other cell), and shapes appear only at level changes."""
    xyz, lv, s, iso, info = synth.uniform_grid(5, 1, (0, 0, 0))
    xyz, lv = _np(xyz, lv)
    assert (oracle.dual_shapes(oracle.OracleMesh(xyz, lv).duals()) == 8).all()
    with open(os.path.join(GOLDEN, "two_level_pyramid.json")) as f:
        g = json.load(f)
    m = oracle.OracleMesh(np.array(g["xyz"], dtype=np.int32), np.array(g["level"], dtype=np.uint8))
    assert sorted(oracle.dual_shapes(m.duals()).tolist()) == [5, 8]
    for seed in range(4):
        xyz, lv, s, iso, info = synth.random_octree(40 + seed, levels=3, roots=3, p_split=0.45, p_hole=0.0)
        xyz, lv = _np(xyz, lv)
        m = oracle.OracleMesh(xyz, lv)
        d = m.duals()
        k = oracle.dual_shapes(d)
        assert k.min() >= 2 and (k == 8).any() and (k < 8).any()
        same_level = np.array([len(set(lv[row].tolist())) == 1 for row in d])
        assert (k[same_level] == 8).all()
