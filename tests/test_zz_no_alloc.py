"""amr_extract_noalloc: the extraction for callers that cannot allocate device
memory (for example code living inside an application whose GPU memory is
managed by someone else, or latency-critical code that may not allocate).

The entry point takes every intermediate buffer from a fixed array the
library reserves per GPU. These tests call it through the C ABI, twice in a
row on different data sets (so left-over contents of the shared array would
show), and compare with the regular context entry points and with the
oracle: equal triangle counts, and triangles equal within 1e-5 of the extent
after canonical ordering. Kept in a file of its own, collected last."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2004_08475_b300 import synth
from tests.parity import canonical, run_oracle

pytestmark = pytest.mark.gpu


def _noalloc(xyz, lv, s, iso, cap):
    from paper_2004_08475_b300 import amriso
    xyz, lv, s = xyz.cuda().contiguous(), lv.cuda().contiguous(), s.cuda().contiguous()
    out = torch.empty((cap, 3, 3), dtype=torch.float32, device="cuda")
    n = ctypes.c_int64(-1)
    stream = torch.cuda.current_stream()
    rc = amriso.lib().amr_extract_noalloc(xyz.data_ptr(), lv.data_ptr(), s.data_ptr(), xyz.shape[0],
                                          ctypes.c_float(iso), out.data_ptr(), cap, ctypes.byref(n),
                                          ctypes.c_void_p(stream.cuda_stream))
    return rc, n.value, out


def _context(xyz, lv, s, iso):
    from paper_2004_08475_b300 import amriso
    ctx = amriso.AmrContext()
    ctx.upload(xyz.cuda(), lv.cuda(), s.cuda())
    ctx.build_locator()
    ctx.dual_cells()
    return ctx.iso(iso).cpu().numpy()


def test_noalloc_matches_context_two_calls():
    from paper_2004_08475_b300 import amriso
    cases = [synth.sphere_tiny(),
             synth.random_octree(9, levels=4, roots=5, p_split=0.45, p_hole=0.06, field="random")]
    for xyz, lv, s, iso, info in cases:
        assert info["n"] <= 65536
        want = _context(xyz, lv, s, iso)
        rc, n, out = _noalloc(xyz, lv, s, iso, cap=max(16, 2 * want.shape[0]))
        assert rc == amriso.OK, amriso.strerror(rc)
        assert n == want.shape[0] > 0
        got = out[:n].cpu().numpy()
        extent = float(max(info["domain"]))
        diff = np.abs(canonical(got).astype(np.float64) - canonical(want).astype(np.float64)).max()
        assert diff <= 1e-5 * extent
        ref = run_oracle(xyz, lv, s, iso)["tris"]
        assert ref.shape[0] == n
        diff = np.abs(canonical(got).astype(np.float64) - canonical(ref).astype(np.float64)).max()
        assert diff <= 1e-5 * extent


def test_noalloc_limits():
    from paper_2004_08475_b300 import amriso
    xyz, lv, s, iso, info = synth.sphere_tiny()
    # capacity: exact count reported, AMR_ERR_CAPACITY returned
    rc, n, _ = _noalloc(xyz, lv, s, iso, cap=8)
    assert rc == amriso.ERR_CAPACITY and n > 8
    # beyond the fixed maximum: rejected before any device work
    big = synth.uniform_grid(41, 0)          # 68921 cells > 65536
    rc, n, _ = _noalloc(big[0], big[1], big[2], big[3], cap=8)
    assert rc == amriso.ERR_RANGE
