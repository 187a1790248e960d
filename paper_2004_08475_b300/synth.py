"""Seeded synthetic AMR inputs.

This module only draws inputs: integer lower corners (finest-level units),
levels and fp32 scalars, in shuffled order. It holds none of the dual-mesh or
Marching Cubes arithmetic; both the CUDA library's tests and the oracle's
tests consume what it returns.

Every generator returns ``(xyz int32 [N,3], level uint8 [N], scalar fp32 [N],
iso float, info dict)`` as torch tensors on ``device`` (CPU by default).
Randomness comes from numpy ``PCG64`` generators for the few global
parameters and from a counter-based 32-bit hash of (seed, key) for per-cell
decisions, so results do not depend on thread counts.

Workloads (stand-ins for the paper's data sets of its results figure, which
are not available here):
  * ``sphere_tiny``       2 levels, 32^3 domain, ~6k cells, iso 8
  * ``random_octree``     tiny random AMR with holes and arbitrary level jumps
  * ``uniform_grid``      one level, n^3 cells
  * ``octree_gaussians``  octree AMR, 512^3, 5 levels, ~10M cells
  * ``block_vortex``      block-structured AMR, 8^3 blocks, 4 levels, holes,
                          ~100M cells, |curl| of vortex rings
  * ``wing_bands``        ~600M cells in distance bands around a swept wing,
                          holes in the solid, log-normal scalar
  * ``serving_set``       24 data sets of 50k-50M cells for the server
"""
from __future__ import annotations

import math

import numpy as np
import torch

_M32 = 0xFFFFFFFF


def hash32(seed: int, key: torch.Tensor) -> torch.Tensor:
    """Counter-based 32-bit hash of (seed, key) in int64 containers.

    A xorshift-multiply integer mixer (the 'lowbias32' construction); only the
    low 32 bits of each product are kept, so int64 wrap-around is harmless.
    """
    h = (key.to(torch.int64) ^ (seed * 0x9E3779B9)) & _M32
    h = (h ^ (h >> 16)) & _M32
    h = (h * 0x7FEB352D) & _M32
    h = (h ^ (h >> 15)) & _M32
    h = (h * 0x846CA68B) & _M32
    h = (h ^ (h >> 16)) & _M32
    return h


def uniform01(seed: int, key: torch.Tensor) -> torch.Tensor:
    """Uniform [0,1) doubles from hash32."""
    return hash32(seed, key).to(torch.float64) / 4294967296.0


def _shuffle(seed, *arrays):
    n = arrays[0].shape[0]
    g = torch.Generator(device="cpu").manual_seed(int(seed))
    perm = torch.randperm(n, generator=g).to(arrays[0].device)
    return tuple(a[perm] for a in arrays)


def _pack(xyz, level, s, iso, seed, info, shuffle=True):
    xyz = xyz.to(torch.int32).contiguous()
    level = level.to(torch.uint8).contiguous()
    s = s.to(torch.float32).contiguous()
    if shuffle:
        xyz, level, s = _shuffle(seed, xyz, level, s)
    info = dict(info)
    info["n"] = int(xyz.shape[0])
    return xyz.contiguous(), level.contiguous(), s.contiguous(), float(iso), info


def _children(lower: torch.Tensor, child_w: int) -> torch.Tensor:
    """Lower corners of the 8 children (width child_w) of each cell."""
    o = torch.tensor([[x, y, z] for z in (0, 1) for y in (0, 1) for x in (0, 1)],
                     dtype=lower.dtype, device=lower.device) * child_w
    return (lower[:, None, :] + o[None]).reshape(-1, 3)


def _grid(nx, ny, nz, w, device, origin=(0, 0, 0)):
    ax = [torch.arange(n, device=device, dtype=torch.int64) * w + o
          for n, o in zip((nx, ny, nz), origin)]
    Z, Y, X = torch.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return torch.stack([X.reshape(-1), Y.reshape(-1), Z.reshape(-1)], 1)


def centres(xyz: torch.Tensor, level: torch.Tensor) -> torch.Tensor:
    """Cell centres in float64 (lower corner + width / 2)."""
    w = (torch.ones_like(level, dtype=torch.int64) << level.to(torch.int64)).to(torch.float64)
    return xyz.to(torch.float64) + 0.5 * w[:, None]


# ---------------------------------------------------------------------------
# Tiny cases
# ---------------------------------------------------------------------------

def sphere_tiny(seed: int = 1, device="cpu"):
    """32^3 domain; level-1 cells except level-0 cells inside radius 8.

    All 16^3 level-1 cells; a level-1 cell whose centre is closer than 8 to
    (16,16,16) is replaced by its 8 level-0 children. s = |centre - (16,16,16)|
    in fp32, iso = 8.
    """
    lower = _grid(16, 16, 16, 2, device)
    c = lower.to(torch.float64) + 1.0
    refine = ((c - 16.0) ** 2).sum(1) < 64.0
    fine = _children(lower[refine], 1)
    coarse = lower[~refine]
    xyz = torch.cat([fine, coarse])
    level = torch.cat([torch.zeros(fine.shape[0], dtype=torch.int64, device=device),
                       torch.ones(coarse.shape[0], dtype=torch.int64, device=device)])
    s = torch.sqrt(((centres(xyz, level) - 16.0) ** 2).sum(1))
    return _pack(xyz, level, s, 8.0, seed,
                 {"workload": "sphere_tiny", "domain": [32, 32, 32], "levels": 2,
                  "refined": int(refine.sum())})


def uniform_grid(n: int, level: int = 0, origin=(0, 0, 0), seed: int = 7, field: str = "random",
                 device="cpu"):
    """n^3 cells of one level; field 'random' (hash uniform) or 'sphere'."""
    w = 1 << level
    xyz = _grid(n, n, n, w, device, origin)
    lv = torch.full((xyz.shape[0],), level, dtype=torch.int64, device=device)
    if field == "random":
        key = (xyz[:, 0] * 73856093) ^ (xyz[:, 1] * 19349663) ^ (xyz[:, 2] * 83492791)
        s = uniform01(seed, key)
        iso = 0.5
    else:
        mid = torch.tensor(origin, dtype=torch.float64, device=device) + 0.5 * n * w
        s = torch.sqrt(((centres(xyz, lv) - mid) ** 2).sum(1))
        iso = 0.3 * n * w + 0.1234 * w
    return _pack(xyz, lv, s, iso, seed, {"workload": "uniform_grid", "n": n, "level": level})


def random_octree(seed: int, levels: int = 3, roots: int = 4, p_split: float = 0.45,
                  p_hole: float = 0.06, field: str = "random", device="cpu"):
    """Tiny random octree AMR with holes and unrestricted level jumps.

    roots^3 cells of level levels-1 are split recursively with probability
    p_split (per cell, seeded hash); each final cell is removed with
    probability p_hole. Finest domain: roots * 2^(levels-1) per axis.
    """
    top = levels - 1
    cells = _grid(roots, roots, roots, 1 << top, device)
    lv = torch.full((cells.shape[0],), top, dtype=torch.int64, device=device)
    out_x, out_l = [], []
    l = top
    while True:
        key = cells[:, 0] * 1000003 + cells[:, 1] * 1009 + cells[:, 2] * 7 + l * 131071
        split = (uniform01(seed * 31 + l, key) < p_split) if l > 0 else \
            torch.zeros(cells.shape[0], dtype=torch.bool, device=device)
        out_x.append(cells[~split])
        out_l.append(lv[~split])
        if l == 0 or not bool(split.any()):
            break
        cells = _children(cells[split], 1 << (l - 1))
        l -= 1
        lv = torch.full((cells.shape[0],), l, dtype=torch.int64, device=device)
    xyz = torch.cat(out_x)
    level = torch.cat(out_l)
    key = xyz[:, 0] * 7919 + xyz[:, 1] * 104729 + xyz[:, 2] * 1299709 + level
    keep = uniform01(seed * 17 + 5, key) >= p_hole
    xyz, level = xyz[keep], level[keep]
    dom = roots * (1 << top)
    if field == "random":
        s = uniform01(seed * 13 + 1, key[keep])
        iso = 0.5
    else:
        c = centres(xyz, level) - 0.5 * dom
        s = torch.sqrt((c ** 2).sum(1))
        iso = 0.31 * dom
    return _pack(xyz, level, s, iso, seed,
                 {"workload": "random_octree", "domain": [dom] * 3, "levels": levels})


# ---------------------------------------------------------------------------
# Octree AMR: 512^3, widths 1..16, refined by |grad f| * w > tau
# ---------------------------------------------------------------------------

def _gauss_params(seed, n_gauss, dom):
    rng = np.random.Generator(np.random.PCG64(seed))
    mu = rng.uniform(0, dom, size=(n_gauss, 3))
    sigma = np.exp(rng.uniform(math.log(4.0), math.log(64.0), size=n_gauss))
    amp = rng.uniform(0.5, 1.5, size=n_gauss)
    return mu, sigma, amp


def _gauss_eval(x, mu, sigma, amp, grad: bool):
    """f = sum_g a_g exp(-|x-mu_g|^2 / (2 sigma_g^2)) and optionally |grad f|."""
    f = torch.zeros(x.shape[0], dtype=torch.float64, device=x.device)
    g = torch.zeros_like(x) if grad else None
    for m, sg, a in zip(mu, sigma, amp):
        d = x - torch.tensor(m, dtype=torch.float64, device=x.device)
        e = a * torch.exp(-(d * d).sum(1) / (2.0 * sg * sg))
        f += e
        if grad:
            g -= e[:, None] * d / (sg * sg)
    return f, (torch.sqrt((g * g).sum(1)) if grad else None)


# refinement threshold giving ~10M cells at the default size (found by
# bisection on the cell count and frozen here)
OCTREE_TAU = 0.02788


def octree_gaussians(seed: int = 2, roots: int = 32, root_level: int = 4, tau: float = OCTREE_TAU,
                     n_gauss: int = 32, device="cpu", chunk: int = 1 << 22):
    """Octree AMR: roots^3 cells of width 2^root_level; a cell of width w > 1
    is split while |grad f(centre)| * w > tau (no 2:1 balancing, so level
    jumps up to root_level occur). s = f(centre); iso = the 60th percentile
    (element floor(0.6 N) of sorted s)."""
    dom = roots << root_level
    mu, sigma, amp = _gauss_params(seed, n_gauss, dom)
    cells = _grid(roots, roots, roots, 1 << root_level, device)
    l = root_level
    out_x, out_l = [], []
    while cells.shape[0]:
        w = 1 << l
        if l == 0:
            out_x.append(cells)
            out_l.append(torch.zeros(cells.shape[0], dtype=torch.int64, device=device))
            break
        split = torch.empty(cells.shape[0], dtype=torch.bool, device=device)
        for a in range(0, cells.shape[0], chunk):
            c = cells[a:a + chunk].to(torch.float64) + 0.5 * w
            _, gn = _gauss_eval(c, mu, sigma, amp, True)
            split[a:a + chunk] = gn * w > tau
        out_x.append(cells[~split])
        out_l.append(torch.full((int((~split).sum()),), l, dtype=torch.int64, device=device))
        cells = _children(cells[split], w // 2)
        l -= 1
    xyz = torch.cat(out_x)
    level = torch.cat(out_l)
    s = torch.empty(xyz.shape[0], dtype=torch.float64, device=device)
    for a in range(0, xyz.shape[0], chunk):
        f, _ = _gauss_eval(centres(xyz[a:a + chunk], level[a:a + chunk]), mu, sigma, amp, False)
        s[a:a + chunk] = f
    s32 = s.to(torch.float32)
    srt = torch.sort(s32).values
    iso = float(srt[int(0.6 * (s32.shape[0] - 1))]) if s32.shape[0] else 0.0
    return _pack(xyz, level, s32, iso, seed,
                 {"workload": "octree_gaussians", "domain": [dom] * 3, "levels": root_level + 1,
                  "tau": tau})


# ---------------------------------------------------------------------------
# Block-structured AMR: 8^3-cell blocks, widths 1..8, holes, vortex rings
# ---------------------------------------------------------------------------

def _ring_params(seed, n_rings, dom):
    rng = np.random.Generator(np.random.PCG64(seed))
    cen = rng.uniform(0.15, 0.85, size=(n_rings, 3)) * np.asarray(dom, dtype=np.float64)
    axis = rng.normal(size=(n_rings, 3))
    axis /= np.linalg.norm(axis, axis=1, keepdims=True)
    radius = rng.uniform(100.0, 600.0, size=n_rings)
    core = rng.uniform(8.0, 40.0, size=n_rings)
    gamma = math.pi * core ** 2 * rng.uniform(0.5, 1.5, size=n_rings)
    return cen, axis, radius, core, gamma


def vortex_vorticity(x: torch.Tensor, params) -> torch.Tensor:
    """|sum_r omega_r(x)|, omega_r = Gamma_r/(pi a_r^2) exp(-d_r^2/a_r^2) phi_r:
    a Gaussian vortex tube around each ring core circle, directed along the
    core tangent (d_r: distance to the core circle)."""
    cen, axis, radius, core, gamma = params
    acc = torch.zeros_like(x)
    for c, n, R, a, G in zip(cen, axis, radius, core, gamma):
        nt = torch.tensor(n, dtype=torch.float64, device=x.device)
        v = x - torch.tensor(c, dtype=torch.float64, device=x.device)
        h = (v * nt).sum(1)
        rho = v - h[:, None] * nt
        rn = torch.sqrt((rho * rho).sum(1)).clamp_min(1e-9)
        d2 = (rn - R) ** 2 + h * h
        tang = torch.cross(nt.expand_as(rho), rho / rn[:, None], dim=1)
        acc += (G / (math.pi * a * a) * torch.exp(-d2 / (a * a)))[:, None] * tang
    return torch.sqrt((acc * acc).sum(1))


BLOCK_TAU = 0.12        # split threshold on the variation of s (frozen: ~126M cells)
BLOCK_ISO = 0.2         # iso-value near the triangle-count maximum (~9M triangles)


def block_vortex(seed: int = 3, dims=(64, 32, 32), tau: float = BLOCK_TAU, iso: float = BLOCK_ISO,
                 p_hole: float = 0.05, n_rings: int = 8, device="cpu", chunk: int = 1 << 22,
                 scale: float = 1.0):
    """Block-structured AMR without hierarchy. Level-3 blocks (8^3 cells of
    width 8, edge 64) tile a dims*64 domain; a level-l block splits into 8
    level-(l-1) blocks iff s varies by more than tau over its 8 octant centres
    (refinement on variation, as block-AMR codes refine where the solution
    changes); 5% of the final blocks are removed as holes; every block
    expands to its 512 cells. `scale` shrinks ring geometry for small test
    domains."""
    dom = [d * 64 for d in dims]
    prm = list(_ring_params(seed, n_rings, dom))
    prm[2] = prm[2] * scale          # ring radius
    prm[3] = prm[3] * scale          # core radius
    prm[4] = prm[4] * scale ** 2     # circulation, keeps the peak vorticity
    blocks = _grid(*dims, 64, device)
    l = 3
    out_b, out_l = [], []
    while blocks.shape[0]:
        edge = 8 << l
        if l == 0:
            out_b.append(blocks)
            out_l.append(torch.zeros(blocks.shape[0], dtype=torch.int64, device=device))
            break
        octs = _children(blocks, edge // 2).to(torch.float64) + edge / 4.0
        vals = torch.empty(octs.shape[0], dtype=torch.float64, device=device)
        for a in range(0, octs.shape[0], chunk):
            vals[a:a + chunk] = vortex_vorticity(octs[a:a + chunk], prm)
        v8 = vals.reshape(-1, 8)
        split = (v8.amax(1) - v8.amin(1)) > tau
        out_b.append(blocks[~split])
        out_l.append(torch.full((int((~split).sum()),), l, dtype=torch.int64, device=device))
        blocks = _children(blocks[split], edge // 2)
        l -= 1
    blocks = torch.cat(out_b)
    blev = torch.cat(out_l)
    key = blocks[:, 0] * 3 + blocks[:, 1] * 7919 + blocks[:, 2] * 6291469 + blev
    keep = uniform01(seed * 101 + 9, key) >= p_hole
    blocks, blev = blocks[keep], blev[keep]
    cell_off = _grid(8, 8, 8, 1, device)                          # [512,3]
    w = (torch.ones_like(blev) << blev)
    xyz = (blocks[:, None, :] + cell_off[None] * w[:, None, None]).reshape(-1, 3)
    level = blev[:, None].expand(-1, 512).reshape(-1)
    s = torch.empty(xyz.shape[0], dtype=torch.float32, device=device)
    for a in range(0, xyz.shape[0], chunk):
        s[a:a + chunk] = vortex_vorticity(centres(xyz[a:a + chunk], level[a:a + chunk]), prm).float()
    return _pack(xyz, level, s, iso, seed,
                 {"workload": "block_vortex", "domain": dom, "levels": 4, "tau": tau,
                  "blocks": int(blocks.shape[0])})


# ---------------------------------------------------------------------------
# ~600M cells in distance bands around a swept, tapered wing
# ---------------------------------------------------------------------------

def wing_sdf(x: torch.Tensor, wing) -> torch.Tensor:
    """Approximate signed distance to a swept, tapered wing with a symmetric
    4-digit-style thickness profile (negative inside the solid)."""
    x0, y0, z0, span, c_root, c_tip, sweep, thick = wing
    px, py, pz = x[:, 0], x[:, 1], x[:, 2]
    eta = ((py - y0) / span).clamp(0.0, 1.0)
    chord = c_root + (c_tip - c_root) * eta
    xle = x0 + eta * span * math.tan(sweep)
    u = ((px - xle) / chord).clamp(0.0, 1.0)
    yt = 5.0 * thick * (0.2969 * torch.sqrt(u) - 0.1260 * u - 0.3516 * u ** 2
                        + 0.2843 * u ** 3 - 0.1015 * u ** 4) * chord
    dz = (pz - z0).abs() - yt                                  # thickness direction
    dx = torch.maximum(xle - px, px - (xle + chord)).clamp_min(0.0)   # off the chord
    dy = torch.maximum(y0 - py, py - (y0 + span)).clamp_min(0.0)      # off the span
    outside = torch.sqrt(dx * dx + dy * dy + dz.clamp_min(0.0) ** 2)
    inside = torch.minimum(dz, torch.zeros_like(dz))
    return torch.where((dx > 0) | (dy > 0) | (dz > 0), outside, inside)


def lognormal_field(x: torch.Tensor, seed: int, n_waves: int = 64, waves=(32.0, 512.0)) -> torch.Tensor:
    """s = exp(2 g), g = sqrt(2/n) sum_m cos(k_m . x + phi_m): a unit-variance
    random-phase field, so s is log-normal with sigma = 2 (wavelengths
    log-uniform in `waves`)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lam = np.exp(rng.uniform(math.log(waves[0]), math.log(waves[1]), size=n_waves))
    dirs = rng.normal(size=(n_waves, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    k = dirs * (2 * math.pi / lam)[:, None]
    phi = rng.uniform(0, 2 * math.pi, size=n_waves)
    kt = torch.tensor(k, dtype=torch.float64, device=x.device)
    pt = torch.tensor(phi, dtype=torch.float64, device=x.device)
    g = torch.cos(x @ kt.T + pt).sum(1) * math.sqrt(2.0 / n_waves)
    return torch.exp(2.0 * g)


# Frozen by probing cell and triangle counts: ~590M cells, ~130M triangles.
WING_DIMS = (448, 448, 96)        # level-3 (width 8) root grid
WING_BANDS = (75.0, 125.0, 195.0)  # |sdf| thresholds for widths 1, 2, 4
WING_ISO = 2.7


WING_WAVES = (12.0, 192.0)


def wing_bands(seed: int = 4, dims=WING_DIMS, bands=WING_BANDS, iso: float = WING_ISO,
               device="cpu", chunk: int = 1 << 24, scale: float = 1.0, waves=None):
    """Exajet-sized AMR: widths 1,2,4,8. The domain is tiled with width-8
    cells; a cell of width w splits while |sdf(centre)| < band(w/2); cells
    whose centre lies inside the wing (sdf < 0) are dropped as holes. The
    scalar is log-normal (sigma = 2)."""
    dom = [d * 8 for d in dims]
    wing = (0.22 * dom[0], 0.12 * dom[1], 0.5 * dom[2], 0.7 * dom[1] * scale,
            0.45 * dom[0] * scale, 0.18 * dom[0] * scale, math.radians(28.0), 0.14)
    cells = _grid(*dims, 8, device)
    out_x, out_l = [], []
    l = 3
    while cells.shape[0]:
        w = 1 << l
        sd = torch.empty(cells.shape[0], dtype=torch.float64, device=device)
        for a in range(0, cells.shape[0], chunk):
            sd[a:a + chunk] = wing_sdf(cells[a:a + chunk].to(torch.float64) + 0.5 * w, wing)
        if l == 0:
            keep = sd >= 0
            out_x.append(cells[keep])
            out_l.append(torch.zeros(int(keep.sum()), dtype=torch.int64, device=device))
            break
        split = sd.abs() < bands[l - 1]
        final = (~split) & (sd >= 0)
        out_x.append(cells[final])
        out_l.append(torch.full((int(final.sum()),), l, dtype=torch.int64, device=device))
        cells = _children(cells[split], w // 2)
        del sd, split, final
        l -= 1
    xyz = torch.cat(out_x)
    level = torch.cat(out_l)
    del out_x, out_l
    s = torch.empty(xyz.shape[0], dtype=torch.float32, device=device)
    for a in range(0, xyz.shape[0], chunk):
        s[a:a + chunk] = lognormal_field(centres(xyz[a:a + chunk], level[a:a + chunk]), seed,
                                         waves=waves or WING_WAVES).float()
    return _pack(xyz, level, s, iso, seed,
                 {"workload": "wing_bands", "domain": dom, "levels": 4, "bands": list(bands)})


# ---------------------------------------------------------------------------
# Serving: 24 data sets of 50k..50M cells
# ---------------------------------------------------------------------------

def serving_sizes(count: int = 24, lo: float = 5e4, hi: float = 5e7):
    return [int(lo * (hi / lo) ** (i / (count - 1))) for i in range(count)]


def crop(xyz, level, s, target: int, seed: int):
    """The cells inside a box around a finest-level cell, the box grown or
    shrunk until it holds about `target` cells (a crop of an AMR data set is
    an AMR data set whose border acts as a hole)."""
    g = torch.Generator(device="cpu").manual_seed(int(seed))
    fine = torch.nonzero(level == level.min()).reshape(-1)
    c = xyz[fine[torch.randint(0, fine.shape[0], (1,), generator=g)]].to(torch.float64).reshape(1, 3)
    x = xyz.to(torch.float64)
    lo, hi = x.min(0).values, x.max(0).values
    half = (hi - lo) * min(1.0, target / xyz.shape[0]) ** (1 / 3) / 2 + 1
    m = None
    for _ in range(60):
        m = ((x - c).abs() <= half).all(1)
        k = int(m.sum())
        if 0.9 * target <= k <= 1.1 * target or k == xyz.shape[0]:
            break
        half = half * (target / max(k, 1)) ** (1 / 3)
    return xyz[m].contiguous(), level[m].contiguous(), s[m].contiguous()


def serving_set(count: int = 24, lo: float = 5e4, hi: float = 5e7, device="cpu"):
    """Serving mix: `count` data sets of lo..hi cells (geometric sizes), cut
    alternately from the octree workload (5 levels) and the block-structured
    workload (4 levels, holes); sizes above the octree's ~10M cells come from
    the block workload. Returns [(name, xyz, level, scalar, (iso_lo, iso_hi))]
    with iso_lo/hi the 40th/95th percentiles of the data set's scalar."""
    oct_ = octree_gaussians(device=device)
    blk = block_vortex(device=device)
    out = []
    for i, n in enumerate(serving_sizes(count, lo, hi)):
        src = oct_ if (i % 2 == 0 and n <= 0.8 * oct_[4]["n"]) else blk
        x, l, v = crop(src[0], src[1], src[2], n, seed=500 + i)
        srt = torch.sort(v).values
        lo_q = float(srt[int(0.40 * (v.shape[0] - 1))])
        hi_q = float(srt[int(0.95 * (v.shape[0] - 1))])
        out.append((f"ds{i:02d}_{src[4]['workload']}", x, l, v, (lo_q, hi_q)))
    return out
