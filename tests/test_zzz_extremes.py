"""Inputs at the limits the C ABI accepts, against the oracle: corners at
-2^30 and near +2^30, the largest level (14), and two clusters 2^21 - 1
finest units apart (the largest extent), with 4^3 and 8^3 bricks. Brick keys
keep 20 bits per axis, which this extent must not alias."""
import numpy as np
import pytest
import torch

from paper_2004_08475_b300 import synth
from tests.parity import compare, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


def _cat(*parts):
    xyz = torch.cat([p[0] for p in parts])
    lv = torch.cat([p[1] for p in parts])
    s = torch.cat([p[2] for p in parts])
    return xyz, lv, s


CASES = {
    # corners from -2^30 up to 2^30 - 59 on the three axes
    "far_corners": lambda: synth.uniform_grid(5, 0, (2 ** 30 - 64, -2 ** 30, 2 ** 20), field="sphere"),
    # level-14 cells (width 16384), the deepest level the ABI accepts
    "level_14": lambda: synth.uniform_grid(3, 14, (-2 ** 30, 0, 2 ** 30 - 3 * 16384)),
}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("logb", [2, 3])
def test_limits_match_oracle(name, logb):
    xyz, lv, s, iso, info = CASES[name]()
    g = run_gpu(xyz, lv, s, iso, log2_brick=logb)
    o = run_oracle(xyz, lv, s, iso)
    assert g["nd"] == o["duals"].shape[0] > 0
    compare(g, o, 2.0 ** 21)


@pytest.mark.parametrize("logb", [2, 3])
def test_largest_extent(logb):
    """Two 3^3 clusters at x = 0 and x = 2^21 - 4: extent 2^21 - 1, 8 duals
    each, none between them."""
    a = synth.uniform_grid(3, 0, (0, 0, 0))
    b = synth.uniform_grid(3, 0, (2 ** 21 - 4, 0, 0), seed=8)
    xyz, lv, s = _cat(a, b)
    g = run_gpu(xyz, lv, s, 0.5, log2_brick=logb)
    o = run_oracle(xyz, lv, s, 0.5)
    assert g["nd"] == o["duals"].shape[0] == 16
    compare(g, o, 2.0 ** 21)
    assert int(g["info"].n_bricks) == 2
    q = g["duals"] // 27                          # cluster of each vertex (27 cells each)
    assert (q.min(1) == q.max(1)).all() and np.array_equal(np.unique(q), [0, 1])
