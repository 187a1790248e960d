"""Host-side checks of the C-ABI library: it builds, loads, exports every
symbol include/amriso.h declares, and its host-generated MC table agrees case
by case with the oracle's run-time face walk. No device calls."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_2004_08475_b300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "amriso.h")


@pytest.fixture(scope="module")
def amriso():
    build.build()
    from paper_2004_08475_b300 import amriso as m
    return m


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(amr_[a-z_]+)\s*\(", text)))


def test_exports_every_declared_symbol(amriso):
    lib = ctypes.CDLL(amriso.LIB_PATH)
    names = declared_symbols()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(amriso.EXPORTS)


def test_abi_version_matches_header(amriso):
    m = re.search(r"#define AMR_ABI_VERSION (\d+)", open(HEADER).read())
    assert m and int(m.group(1)) == amriso.ABI_VERSION == amriso.lib().amr_abi_version()


def test_strerror(amriso):
    for code in range(0, -12, -1):
        assert amriso.strerror(code)
    assert amriso.strerror(0) == "ok"


def test_mc_table_matches_oracle_face_walk(amriso):
    count, edges = amriso.mc_table()
    for case in range(256):
        want = oracle.case_triangles(case)
        assert count[case] == want.shape[0]
        got = edges[case][:3 * count[case]].reshape(-1, 3).astype(np.int32)
        assert (got == want).all(), case
        assert (edges[case][3 * count[case]:] == 255).all()


def test_mc_table_edge_numbering(amriso):
    """Edge k joins corners (a,b), a<b, in increasing (a,b) order: both sides
    use the numbering the oracle lists."""
    count, edges = amriso.mc_table()
    # case 1 (corner 0 inside) uses exactly the edges touching corner 0
    e0 = {k for k, (a, b) in enumerate(oracle.EDGES) if 0 in (a, b)}
    assert set(edges[1][:3].tolist()) == e0


def test_create_without_device_fails_cleanly(amriso):
    import torch
    if torch.cuda.is_available():
        pytest.skip("device present")
    h = ctypes.c_void_p()
    rc = amriso.lib().amr_create(ctypes.byref(h), 0, None)
    assert rc == amriso.ERR_INVALID_ARG and not h.value
