"""Oracle for the AMR dual-mesh / iso-surface method (Wald, Sec. 3-5).

TEST INFRASTRUCTURE ONLY: a plain single-threaded CPU implementation (C++ in
``oracle.cpp``, loaded through ctypes) that the tests, the smoke check and the
benchmark's CPU-baseline leg compare the CUDA library against. The product
path never imports this package, and this package imports nothing from the
product.

Functions follow the paper's steps:
  * ``OracleMesh``      - the set of actual cells and snap() (Sec. 3.1, 3.2)
  * ``.duals()``        - doCell / doDualCell with rules 1-3 (Sec. 4.2-4.4)
  * ``.iso()``          - Marching Cubes on the dual hexahedra (Sec. 5, 5.2)
  * ``case_triangles``  - the run-time face walk for one MC case (Sec. 5.1)
  * ``weld``            - the indexed face set of a triangle list (Sec. 5.2),
                          vertices identified by their edge key
  * ``interpolate``     - a second per-cell field at those vertices (the
                          attribute mapping of Sec. 1)
  * ``dual_shapes``     - distinct cells per dual (the shapes snapping
                          produces, Sec. 4.1)

Pins (tests/test_oracle_*.py): brute-force snapping of every logical dual on
tiny inputs, the (n-1)^3 closed form on uniform grids, the sphere's Euler
characteristic and enclosed volume, watertightness and orientation, the face
rule checked from its definition, and the fp64 cross-check of every vertex.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None
# A variant build of oracle.cpp to load instead (tests/test_oracle_mutants.py
# runs the pins against copies with planted mistakes this way).
_VARIANT = os.environ.get("AMR_ORACLE_VARIANT_LIB")

COMPILE = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC"]


def build(force: bool = False) -> str:
    """Compile oracle.cpp into liboracle.so (g++, no FMA contraction)."""
    if _VARIANT:
        return _VARIANT
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(COMPILE + ["-o", _LIB + ".tmp", _SRC])
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.c_void_p
    I64 = ctypes.c_int64
    lib.oracle_mesh_create.restype = P
    lib.oracle_mesh_create.argtypes = [P, P, I64, ctypes.POINTER(ctypes.c_int)]
    lib.oracle_mesh_destroy.restype = None
    lib.oracle_mesh_destroy.argtypes = [P]
    lib.oracle_num_levels.restype = ctypes.c_int
    lib.oracle_num_levels.argtypes = [P]
    lib.oracle_snap.restype = I64
    lib.oracle_snap.argtypes = [P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
    lib.oracle_duals.restype = I64
    lib.oracle_duals.argtypes = [P, P, I64, P, P, I64]
    lib.oracle_case_triangles.restype = ctypes.c_int
    lib.oracle_case_triangles.argtypes = [ctypes.c_int, P]
    lib.oracle_iso.restype = I64
    lib.oracle_iso.argtypes = [P, P, P, I64, ctypes.c_float, P, P, P, P, P, I64,
                               ctypes.POINTER(ctypes.c_double)]
    _lib = lib
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class OracleError(ValueError):
    pass


_ERR = {-2: "unaligned lower corner", -3: "level out of range", -5: "duplicate cell"}


class OracleMesh:
    """The set of actual cells of one data set and the snap() operator."""

    def __init__(self, xyz, level):
        self.xyz = np.ascontiguousarray(xyz, dtype=np.int32).reshape(-1, 3)
        self.level = np.ascontiguousarray(level, dtype=np.uint8).reshape(-1)
        assert self.xyz.shape[0] == self.level.shape[0]
        lib = _load()
        err = ctypes.c_int(0)
        self._h = lib.oracle_mesh_create(_ptr(self.xyz), _ptr(self.level),
                                         self.xyz.shape[0], ctypes.byref(err))
        if not self._h:
            raise OracleError(_ERR.get(err.value, f"error {err.value}"))
        self.n = self.xyz.shape[0]

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.oracle_mesh_destroy(h)
            self._h = None

    @property
    def num_levels(self) -> int:
        return _load().oracle_num_levels(self._h)

    def snap(self, i, j, k) -> int:
        return _load().oracle_snap(self._h, int(i), int(j), int(k))

    def duals(self, owners=None, with_owner=False):
        """Dual cells [D, 8] (local cell indices, vertex order ex+2ey+4ez)."""
        lib = _load()
        own = None if owners is None else np.ascontiguousarray(owners, dtype=np.int64)
        n_own = 0 if own is None else own.shape[0]
        nd = lib.oracle_duals(self._h, _ptr(own), n_own, None, None, 0)
        out = np.empty((nd, 8), dtype=np.int64)
        owner = np.empty(nd, dtype=np.int64)
        nd2 = lib.oracle_duals(self._h, _ptr(own), n_own, _ptr(out), _ptr(owner), nd)
        assert nd2 == nd
        return (out, owner) if with_owner else out

    def iso(self, scalar, duals, iso, want_keys=True):
        """Marching Cubes over `duals` at `iso`.

        Returns dict: cases [D] u8, ntri [D] u8, tris [T,3,3] f32,
        keys [T,3,2] i64 (edge keys, local indices), tri_dual [T] i64,
        max_err (max |fp32 - fp64| over vertex coordinates).
        """
        lib = _load()
        s = np.ascontiguousarray(scalar, dtype=np.float32).reshape(-1)
        d = np.ascontiguousarray(duals, dtype=np.int64).reshape(-1, 8)
        nd = d.shape[0]
        cases = np.empty(nd, dtype=np.uint8)
        ntri = np.empty(nd, dtype=np.uint8)
        err = ctypes.c_double(0.0)
        nt = lib.oracle_iso(self._h, _ptr(s), _ptr(d), nd, ctypes.c_float(iso), _ptr(cases),
                            _ptr(ntri), None, None, None, 0, ctypes.byref(err))
        tris = np.empty((nt, 3, 3), dtype=np.float32)
        keys = np.empty((nt, 3, 2), dtype=np.int64) if want_keys else None
        tdual = np.empty(nt, dtype=np.int64)
        nt2 = lib.oracle_iso(self._h, _ptr(s), _ptr(d), nd, ctypes.c_float(iso), None, None,
                             _ptr(tris), _ptr(keys), _ptr(tdual), nt, ctypes.byref(err))
        assert nt2 == nt
        return {"cases": cases, "ntri": ntri, "tris": tris, "keys": keys,
                "tri_dual": tdual, "max_err": err.value}


def weld(tris, keys):
    """Indexed face set of fat triangles (Sec. 5.2). The paper merges
    vertices at equal positions after sorting; here a vertex is identified by
    its edge key (the unordered pair of cells it interpolates between), so
    each distinct key becomes one vertex.

    tris [T,3,3] f32 and keys [T,3,2] (from ``OracleMesh.iso``) -> (vtx [V,3]
    f32, tri [T,3] i64, vkeys [V,2] i64), vertices in increasing key order.
    Raises if one key carries two different positions."""
    k = np.asarray(keys, dtype=np.int64).reshape(-1, 2)
    p = np.asarray(tris, dtype=np.float32).reshape(-1, 3)
    if k.shape[0] == 0:
        return (np.zeros((0, 3), np.float32), np.zeros((0, 3), np.int64), np.zeros((0, 2), np.int64))
    vkeys, first, inv = np.unique(k, axis=0, return_index=True, return_inverse=True)
    vtx = p[first]
    if not np.array_equal(vtx[inv.reshape(-1)].view(np.int32), p.view(np.int32)):
        raise OracleError("one edge key with two vertex positions")
    return vtx, inv.reshape(-1, 3).astype(np.int64), vkeys


def interpolate(xyz, scalar, attr, vkeys, iso):
    """A per-cell field at the vertices of an indexed face set: for a vertex
    on the edge of cells (a, b), taken from the one whose lower corner is
    lower in (z, y, x) order, t = (iso - s_a) / (s_b - s_a) and
    f = f_a + t (f_b - f_a), every step in fp32 (the vertex formula of
    Sec. 5 applied to another field)."""
    x = np.asarray(xyz, dtype=np.int64).reshape(-1, 3)
    s = np.asarray(scalar, dtype=np.float32).reshape(-1)
    f = np.asarray(attr, dtype=np.float32).reshape(-1)
    k = np.asarray(vkeys, dtype=np.int64).reshape(-1, 2)
    a, b = k[:, 0].copy(), k[:, 1].copy()
    za, zb = x[a][:, ::-1], x[b][:, ::-1]   # (z, y, x)
    swap = np.array([tuple(q) < tuple(p) for p, q in zip(za.tolist(), zb.tolist())], dtype=bool)
    a[swap], b[swap] = k[swap, 1], k[swap, 0]
    iso32 = np.float32(iso)
    t = (iso32 - s[a]) / (s[b] - s[a])
    return (f[a] + t * (f[b] - f[a])).astype(np.float32)


def dual_shapes(duals) -> np.ndarray:
    """Number of distinct cells among each dual's 8 vertices (Sec. 4.1:
    snapping makes hexahedra, wedges, pyramids, tetrahedra and flatter
    shapes): 8, 6, 5, 4, ..."""
    d = np.sort(np.asarray(duals, dtype=np.int64).reshape(-1, 8), axis=1)
    return (1 + (d[:, 1:] != d[:, :-1]).sum(axis=1)).astype(np.uint8)


def case_triangles(case: int) -> np.ndarray:
    """Triangles [k,3] (edge indices) of one MC case from the run-time face walk."""
    buf = np.zeros(48, dtype=np.int32)
    n = _load().oracle_case_triangles(int(case), _ptr(buf))
    return buf[:3 * n].reshape(n, 3).copy()


# The 12 hexahedron edges as corner pairs (a, b), a < b, corners e = x+2y+4z.
EDGES = [(a, b) for a in range(8) for b in range(a + 1, 8) if (a ^ b) in (1, 2, 4)]
