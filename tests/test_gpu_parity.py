"""CUDA path vs oracle, element by element: bit-exact dual cells (sorted
8-tuples of cell IDs), case indices and per-dual triangle counts; triangle
vertices within 1e-5 of the domain extent after canonical ordering (the
kernels use the oracle's fp32 operation order, so they are expected to be
bit-exact)."""
import numpy as np
import pytest
import torch

from paper_2004_08475_b300 import synth
from tests.parity import canonical, compare, owners_of, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


def _extent(info):
    return float(max(info["domain"]))


@pytest.mark.parametrize("logb", [2, 3])
def test_sphere_tiny(logb):
    xyz, lv, s, iso, info = synth.sphere_tiny()
    g = run_gpu(xyz, lv, s, iso, log2_brick=logb)
    o = run_oracle(xyz, lv, s, iso)
    r = compare(g, o, _extent(info))
    assert r["duals"] == 5827
    assert r["bit_exact_frac"] == 1.0


@pytest.mark.parametrize("part", [-1, 1])
def test_partitioned_placement(part):
    """Both cell-placement paths of the locator build (direct scatter and
    binned by slot range) give the oracle's result."""
    for seed in range(6):
        gen = synth.random_octree(200 + seed, levels=2 + seed % 4, roots=5 if seed % 4 < 3 else 3,
                                  p_split=0.45, p_hole=0.06, field="random" if seed % 2 else "sphere")
        xyz, lv, s, iso, info = gen
        g = run_gpu(xyz, lv, s, iso, log2_brick=2 + seed % 2, partitioned=part)
        o = run_oracle(xyz, lv, s, iso)
        compare(g, o, _extent(info))
    xyz, lv, s, iso, info = synth.octree_gaussians(seed=12, roots=6, root_level=4)
    compare(run_gpu(xyz, lv, s, iso, partitioned=part), run_oracle(xyz, lv, s, iso), _extent(info))


@pytest.mark.parametrize("case", range(8))
def test_fused_dual_iso_equals_separate(case):
    """amr_dual_cells_iso gives the same resident dual list and the same
    triangles (bit for bit after canonical ordering) as amr_dual_cells
    followed by amr_iso, and both match the oracle."""
    from paper_2004_08475_b300 import amriso
    if case < 5:
        gen = synth.random_octree(300 + case, levels=2 + case % 4, roots=5, p_split=0.45, p_hole=0.06,
                                  field="random" if case % 2 else "sphere")
    elif case == 5:
        gen = synth.sphere_tiny()
    elif case == 6:
        gen = synth.octree_gaussians(seed=12, roots=6, root_level=4)
    else:
        gen = synth.wing_bands(seed=14, dims=(24, 24, 8), bands=(3.0, 7.0, 14.0), iso=8.0)
    xyz, lv, s, iso, info = gen
    for logb in (2, 3):
        ctx = amriso.AmrContext()
        ctx.upload(xyz.cuda(), lv.cuda(), s.cuda())
        ctx.build_locator(log2_brick=logb)
        out = torch.empty((200000, 3, 3), dtype=torch.float32, device="cuda")
        nd, nt = ctx.dual_cells_iso(iso, out)
        fused_tris = out[:nt].cpu().numpy()
        fused_duals = ctx.get_duals().cpu().numpy().astype(np.int64)
        cases, ntri = ctx.iso_cases(iso)
        assert int(ntri.sum()) == nt
        sep = ctx.iso(iso).cpu().numpy()
        assert sep.shape[0] == nt
        assert (canonical(fused_tris) == canonical(sep)).all()
        g = {"duals": fused_duals, "cases": cases.cpu().numpy(), "ntri": ntri.cpu().numpy(), "tris": fused_tris}
        compare(g, run_oracle(xyz, lv, s, iso), _extent(info))


def test_partitioned_duplicate_detected():
    from paper_2004_08475_b300 import amriso
    xyz = torch.tensor([[0, 0, 0], [2, 0, 0], [2, 0, 0]], dtype=torch.int32)
    lv = torch.tensor([1, 1, 1], dtype=torch.uint8)
    s = torch.tensor([0.0, 1.0, 2.0])
    ctx = amriso.AmrContext()
    ctx.upload(xyz.cuda(), lv.cuda(), s.cuda())
    with pytest.raises(amriso.AmrError) as e:
        ctx.build_locator(partitioned=1)
    assert e.value.code == amriso.ERR_DUPLICATE


def test_placement_paths_agree_and_are_reported():
    """From 2^20 cells on the default placement is binned, below it a direct
    scatter; both give the same dual list and triangles."""
    from paper_2004_08475_b300 import amriso
    xyz, lv, s, iso, info = synth.uniform_grid(104, field="sphere")   # 1,124,864 cells
    assert xyz.shape[0] >= 1 << 20
    out = {}
    for part in (0, -1):
        ctx = amriso.AmrContext()
        ctx.upload(xyz.cuda(), lv.cuda(), s.cuda())
        ctx.build_locator(partitioned=part)
        out[part] = (ctx.info().placement, ctx.dual_cells(), ctx.get_duals().cpu().numpy(),
                     canonical(ctx.iso(iso).cpu().numpy()))
        ctx.close()
    assert out[0][0] == 1 and out[-1][0] == 0

    def rows_sorted(d):   # brick numbering (hence dual order) differs between builds
        return d[np.lexsort(d.T[::-1])]
    assert out[0][1] == out[-1][1] and np.array_equal(rows_sorted(out[0][2]), rows_sorted(out[-1][2]))
    assert np.array_equal(out[0][3].view(np.int32), out[-1][3].view(np.int32))
    small = synth.sphere_tiny()
    ctx = amriso.AmrContext()
    ctx.upload(small[0].cuda(), small[1].cuda(), small[2].cuda())
    ctx.build_locator()
    assert ctx.info().placement == 0


def test_trim_keeps_results():
    """amr_trim frees the placement workspace; the resident locator and dual
    cells still give the same triangles."""
    from paper_2004_08475_b300 import amriso
    xyz, lv, s, iso, info = synth.octree_gaussians(seed=5, roots=8, root_level=5)
    ctx = amriso.AmrContext()
    ctx.upload(xyz.cuda(), lv.cuda(), s.cuda())
    ctx.build_locator(partitioned=1)
    ctx.dual_cells()
    before = ctx.info().device_bytes
    a = canonical(ctx.iso(iso).cpu().numpy())
    ctx.trim()
    after = ctx.info().device_bytes
    assert after < before
    b = canonical(ctx.iso(iso, host=True).numpy())   # host delivery re-creates its staging
    assert a.shape[0] > 0 and np.array_equal(a.view(np.int32), b.view(np.int32))


@pytest.mark.parametrize("copies", [3, 9000])
def test_binned_window_overflow_is_duplicate(copies):
    """More copies of one cell than a window of the binned placement holds
    are caught by the capacity check, not written past the window."""
    from paper_2004_08475_b300 import amriso
    xyz = torch.zeros((copies + 1, 3), dtype=torch.int32)
    xyz[0, 0] = 8
    lv = torch.zeros(copies + 1, dtype=torch.uint8)
    s = torch.arange(copies + 1, dtype=torch.float32)
    ctx = amriso.AmrContext()
    ctx.upload(xyz.cuda(), lv.cuda(), s.cuda())
    with pytest.raises(amriso.AmrError) as e:
        ctx.build_locator(partitioned=1)
    assert e.value.code == amriso.ERR_DUPLICATE


@pytest.mark.parametrize("seed", range(24))
def test_random_octrees(seed):
    levels = 2 + seed % 4
    gen = synth.random_octree(seed, levels=levels, roots=5 if levels < 5 else 3, p_split=0.45,
                              p_hole=0.0 if seed % 3 == 0 else 0.08,
                              field="random" if seed % 2 else "sphere")
    xyz, lv, s, iso, info = gen
    g = run_gpu(xyz, lv, s, iso, log2_brick=2 + seed % 2)
    o = run_oracle(xyz, lv, s, iso)
    compare(g, o, _extent(info))


@pytest.mark.parametrize("n,l,origin", [(2, 0, (0, 0, 0)), (9, 0, (-5, 3, 17)), (12, 3, (-64, 0, 8)),
                                         (17, 1, (1000, -2000, 30))])
def test_uniform_grid(n, l, origin):
    xyz, lv, s, iso, info = synth.uniform_grid(n, l, origin)
    g = run_gpu(xyz, lv, s, iso)
    assert g["nd"] == (n - 1) ** 3
    o = run_oracle(xyz, lv, s, iso)
    compare(g, o, float(n << l))


def test_octree_gaussians_small():
    gen = synth.octree_gaussians(seed=12, roots=6, root_level=4)
    xyz, lv, s, iso, info = gen
    assert info["n"] > 10000
    for logb in (2, 3):
        g = run_gpu(xyz, lv, s, iso, log2_brick=logb)
        o = run_oracle(xyz, lv, s, iso)
        compare(g, o, _extent(info))


def test_block_vortex_small():
    gen = synth.block_vortex(seed=13, dims=(4, 2, 2), scale=0.12, tau=0.004, iso=0.05)
    xyz, lv, s, iso, info = gen
    assert info["n"] > 10000
    g = run_gpu(xyz, lv, s, iso)
    o = run_oracle(xyz, lv, s, iso)
    compare(g, o, _extent(info))


def test_wing_small():
    gen = synth.wing_bands(seed=14, dims=(24, 24, 8), bands=(3.0, 7.0, 14.0), iso=8.0)
    xyz, lv, s, iso, info = gen
    assert info["n"] > 10000
    g = run_gpu(xyz, lv, s, iso)
    o = run_oracle(xyz, lv, s, iso)
    compare(g, o, _extent(info))


def test_host_pointer_upload():
    xyz, lv, s, iso, info = synth.random_octree(77, levels=4, roots=4, p_hole=0.05)
    g = run_gpu(xyz, lv, s, iso, host_upload=True)
    o = run_oracle(xyz, lv, s, iso)
    compare(g, o, _extent(info))


@pytest.mark.parametrize("part", [-1, 1])
def test_misaligned_device_arrays(part):
    """Cell arrays that start one cell into their allocations (corners 12
    bytes, levels 1 byte past an aligned address, so the insert pass reads
    them cell by cell instead of in 16-byte groups), with a cell count that
    leaves a ragged last group: the oracle's result on both placement paths."""
    from paper_2004_08475_b300 import amriso
    xyz, lv, s, iso, info = synth.random_octree(78, levels=4, roots=5, p_split=0.45, p_hole=0.05)
    n = xyz.shape[0] - 3 if (xyz.shape[0] - 3) % 4 else xyz.shape[0] - 2   # not a multiple of 4
    xb = torch.zeros((n + 1, 3), dtype=torch.int32, device="cuda")
    lb = torch.zeros(n + 1, dtype=torch.uint8, device="cuda")
    sb = torch.zeros(n + 1, dtype=torch.float32, device="cuda")
    xb[1:] = xyz[:n].cuda()
    lb[1:] = lv[:n].cuda()
    sb[1:] = s[:n].cuda()
    x1, l1, s1 = xb[1:], lb[1:], sb[1:]
    assert x1.data_ptr() % 16 and l1.data_ptr() % 4
    ctx = amriso.AmrContext()
    ctx.upload(x1, l1, s1)
    ctx.build_locator(partitioned=part)
    ctx.dual_cells()
    cases, ntri = ctx.iso_cases(iso)
    g = {"duals": ctx.get_duals().cpu().numpy().astype(np.int64), "cases": cases.cpu().numpy(),
         "ntri": ntri.cpu().numpy(), "tris": ctx.iso(iso).cpu().numpy()}
    ctx.close()
    r = compare(g, run_oracle(xyz[:n], lv[:n], s[:n], iso), _extent(info))
    assert r["bit_exact_frac"] == 1.0


def test_empty_and_single():
    from paper_2004_08475_b300 import amriso
    ctx = amriso.AmrContext()
    ctx.upload(torch.zeros((0, 3), dtype=torch.int32, device="cuda"),
               torch.zeros(0, dtype=torch.uint8, device="cuda"),
               torch.zeros(0, dtype=torch.float32, device="cuda"))
    ctx.build_locator()
    assert ctx.dual_cells() == 0
    assert ctx.iso(0.5).shape[0] == 0
    ctx.upload(torch.tensor([[4, 8, -12]], dtype=torch.int32, device="cuda"),
               torch.tensor([2], dtype=torch.uint8, device="cuda"),
               torch.tensor([1.0], device="cuda"))
    ctx.build_locator()
    assert ctx.dual_cells() == 0


def test_deep_jumps_collapsed_duals():
    """Five levels on a 2^3 root grid with heavy splitting: transition duals
    with many repeated vertices and level jumps up to 4."""
    for seed in range(4):
        gen = synth.random_octree(100 + seed, levels=5, roots=2, p_split=0.7, p_hole=0.0,
                                  field="random")
        xyz, lv, s, iso, info = gen
        g = run_gpu(xyz, lv, s, iso, log2_brick=2)
        o = run_oracle(xyz, lv, s, iso)
        compare(g, o, _extent(info))


@pytest.mark.parametrize("what", ["duplicate", "unaligned", "nonfinite", "level", "overlap", "extent"])
def test_invalid_input_codes(what):
    from paper_2004_08475_b300 import amriso
    xyz = torch.tensor([[0, 0, 0], [2, 0, 0], [4, 0, 0]], dtype=torch.int32)
    lv = torch.tensor([1, 1, 1], dtype=torch.uint8)
    s = torch.tensor([0.0, 1.0, 2.0])
    overlap = False
    want = {"duplicate": amriso.ERR_DUPLICATE, "unaligned": amriso.ERR_UNALIGNED,
            "nonfinite": amriso.ERR_NONFINITE, "level": amriso.ERR_RANGE,
            "overlap": amriso.ERR_OVERLAP, "extent": amriso.ERR_RANGE}[what]
    if what == "duplicate":
        xyz[2] = xyz[1]
    elif what == "unaligned":
        xyz[1, 0] = 3
    elif what == "nonfinite":
        s[2] = float("nan")
    elif what == "level":
        lv[0] = 15
    elif what == "overlap":
        xyz[2] = torch.tensor([2, 0, 0])
        lv[2] = 0
        overlap = True
    elif what == "extent":
        xyz[2, 1] = 1 << 22
    ctx = amriso.AmrContext()
    ctx.upload(xyz.cuda(), lv.cuda(), s.cuda())
    with pytest.raises(amriso.AmrError) as e:
        ctx.build_locator(check_overlap=overlap)
    assert e.value.code == want
    with pytest.raises(amriso.AmrError) as e:
        ctx.dual_cells()
    assert e.value.code == amriso.ERR_STATE


def test_capacity_and_exact_count():
    from paper_2004_08475_b300 import amriso
    xyz, lv, s, iso, info = synth.sphere_tiny()
    ctx = amriso.AmrContext()
    ctx.upload(xyz.cuda(), lv.cuda(), s.cuda())
    ctx.build_locator()
    ctx.dual_cells()
    full = ctx.iso(iso)
    small = torch.empty((10, 3, 3), dtype=torch.float32, device="cuda")
    n = ctx.iso_count(iso, small)
    assert n == full.shape[0] > 10
    host = torch.empty((n, 3, 3), dtype=torch.float32).pin_memory()
    assert ctx.iso_count(iso, host) == n
    assert (canonical(host.numpy()) == canonical(full.cpu().numpy())).all()


def test_iso_batch_equals_single():
    from paper_2004_08475_b300 import amriso
    gen = synth.octree_gaussians(seed=21, roots=5, root_level=4)
    xyz, lv, s, iso, info = gen
    ctx = amriso.AmrContext()
    ctx.upload(xyz.cuda(), lv.cuda(), s.cuda())
    ctx.build_locator()
    ctx.dual_cells()
    isos = [iso * (0.5 + 0.1 * k) for k in range(12)]
    tris, offs = ctx.iso_batch(isos)
    for k, v in enumerate(isos):
        one = ctx.iso(v).cpu().numpy()
        seg = tris[offs[k]:offs[k + 1]].cpu().numpy()
        assert seg.shape == one.shape
        assert (canonical(seg) == canonical(one)).all()


def test_octree_full_size_complete():
    """The 10M-cell octree at full size, complete: every dual cell, case
    index and per-dual triangle count equals the oracle's bit for bit, and
    every triangle matches within 1e-5 of the extent (bit-exact in fact).
    The oracle runs slab by slab on the host cores (``oracle.shard``: each
    slab with a halo of the widest cell, exact)."""
    import os
    from oracle import shard
    xyz, lv, s, iso, info = synth.octree_gaussians()
    assert 9_000_000 < info["n"] < 11_000_000
    x, l, v = xyz.numpy(), lv.numpy(), s.numpy()
    o = shard.run_sharded(x, l, v, iso, n_slabs=max(4, min(16, os.cpu_count() or 1)), balance="count")
    g = run_gpu(xyz, lv, s, iso)
    assert g["nd"] == o["duals"].shape[0]
    r = compare(g, o, _extent(info))
    assert r["duals"] > 10_000_000 and r["tris"] > 500_000
    assert r["bit_exact_frac"] == 1.0
    assert o["max_err"] <= 4 * np.spacing(np.float32(_extent(info)))
