"""The pins have the power to see plausible mistakes in the oracle.

Each mutant is a copy of oracle/oracle.cpp with one planted mistake (a
dropped rejection rule or a non-strict rule-3 order, the other dual offsets,
an unmasked snap query, a wrong sign or a transposed operand in the vertex
formula, a dropped half in the cell centre, the ambiguous-face pairing
around outside corners, loops fanned from their first edge, the
degenerate-triangle drop removed, ties counted as inside). The oracle pin
suites (test_oracle_duals.py, test_oracle_mc.py) run against each mutant in a
child process and must fail with an assertion (or crash partway); against
an unmodified copy they must pass. The oracle's Python functions (weld,
interpolate, dual_shapes, the sharded oracle) get the same treatment
in-process: a mutated copy is patched in and one of their pins must fail.
CPU only.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.cpp")
PINS = [os.path.join(ROOT, "tests", "test_oracle_duals.py"), os.path.join(ROOT, "tests", "test_oracle_mc.py")]

# name -> [(text in oracle.cpp, replacement)], each text found exactly once
MUTANTS = {
    "rule1_dropped": [("if (v < 0) return false;                       // rule #1: outside / hole",
                       "if (v < 0) v = self;")],
    "rule2_dropped": [("if (m.level[v] < l) return false;              // rule #2: finer level",
                       "")],
    # (rule 3 with the order reversed, or cell IDs as the order, is not a
    # mistake: any strict total order emits the same set of duals)
    "rule3_non_strict": [("return std::tie(pa[2], pa[1], pa[0]) < std::tie(pb[2], pb[1], pb[0]);",
                          "return std::tie(pa[2], pa[1], pa[0]) <= std::tie(pb[2], pb[1], pb[0]);")],
    "rule3_dropped": [("if (m.level[v] == l && lower_than(m, v, self))", "if (false)")],
    "dual_offsets_0_1": [("for (int dk = -1; dk <= 0; ++dk)", "for (int dk = 0; dk <= 1; ++dk)"),
                         ("for (int dj = -1; dj <= 0; ++dj)", "for (int dj = 0; dj <= 1; ++dj)"),
                         ("for (int di = -1; di <= 0; ++di)", "for (int di = 0; di <= 1; ++di)")],
    "snap_unmasked": [("Label{l, project(k, l), project(j, l), project(i, l)}", "Label{l, k, j, i}")],
    "t_wrong_sign": [("const float t = (iso - sa) / d;", "const float t = (sa - iso) / d;"),
                     ("const double t64 = (double(iso) - double(sa)) / d64;",
                      "const double t64 = (double(sa) - double(iso)) / d64;")],
    "lerp_transposed": [("out.p32[x] = ca + tdc;", "out.p32[x] = cb - tdc;"),
                        ("out.p64[x] = double(ca) + t64 * (double(cb) - double(ca));",
                         "out.p64[x] = double(cb) - t64 * (double(cb) - double(ca));")],
    "centre_half_dropped": [("const float ha = float(int32_t(1) << m.level[va]) * 0.5f;",
                             "const float ha = float(int32_t(1) << m.level[va]);"),
                            ("const float hb = float(int32_t(1) << m.level[vb]) * 0.5f;",
                             "const float hb = float(int32_t(1) << m.level[vb]);")],
    "ambiguous_face_outside": [("""        for (int r = 0; r < 4; ++r)
          if (inside[ring[r]]) {
            pr[np][0] = (r + 3) % 4;""", """        for (int r = 0; r < 4; ++r)
          if (!inside[ring[r]]) {
            pr[np][0] = (r + 3) % 4;""")],
    "fan_apex_first": [("    int apex = -1;\n    for (int cand", "    int apex = 0;\n    for (int cand")],
    "degenerate_kept": [("if (same(vt[0], vt[1]) || same(vt[1], vt[2]) || same(vt[0], vt[2]))\n        continue;",
                         "if (false)\n        continue;")],
    "ties_inside": [("if (s[v[e]] > iso) cas |= 1 << e;", "if (s[v[e]] >= iso) cas |= 1 << e;")],
}


def _compile(name, edits, tmp):
    text = open(SRC).read()
    for old, new in edits:
        assert text.count(old) == 1, (name, old)
        text = text.replace(old, new)
    src = os.path.join(tmp, f"{name}.cpp")
    lib = os.path.join(tmp, f"lib{name}.so")
    with open(src, "w") as f:
        f.write(text)
    subprocess.check_call(oracle.COMPILE + ["-o", lib, src])
    return lib


def _run_pins(lib, first_failure=True):
    env = dict(os.environ, AMR_ORACLE_VARIANT_LIB=lib, PYTHONDONTWRITEBYTECODE="1")
    cmd = [sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider", "-m", "not gpu"] + \
        (["-x"] if first_failure else []) + PINS
    p = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return p.returncode, p.stdout + p.stderr


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    tmp = str(tmp_path_factory.mktemp("mutants"))
    libs = {"unmodified": _compile("unmodified", [], tmp)}
    for name, edits in MUTANTS.items():
        libs[name] = _compile(name, edits, tmp)
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        futs = {name: ex.submit(_run_pins, lib) for name, lib in libs.items()}
        return {name: f.result() for name, f in futs.items()}


def test_unmodified_copy_passes_the_pins(results):
    rc, out = results["unmodified"]
    assert rc == 0, out[-3000:]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_fails_a_pin(results, name):
    rc, out = results[name]
    if rc < 0:   # the mutant crashed the child while the pins ran (after some passed)
        assert "." in out.split("Fatal Python error")[0], out[-3000:]
        return
    assert rc == 1, out[-3000:]                    # 1: tests failed (not a usage or collection error)
    assert "failed" in out and ("AssertionError" in out or "assert" in out), out[-3000:]


# ---- the oracle's Python functions: mutants planted in-process -------------

def _mutated(fn, edits):
    """`fn` recompiled from its source with the textual edits applied, in the
    namespace of its module."""
    import inspect
    import textwrap
    src = textwrap.dedent(inspect.getsource(fn))
    for old, new in edits:
        assert src.count(old) == 1, (fn.__name__, old)
        src = src.replace(old, new)
    ns = dict(fn.__globals__)
    exec(compile(src, f"<mutant of {fn.__name__}>", "exec"), ns)
    return ns[fn.__name__]


def _pins():
    from tests import test_oracle_duals as duals_pins
    from tests import test_oracle_mc as mc_pins
    from tests import test_oracle_shard as shard_pins
    return {
        "interpolate": [mc_pins.test_interpolate_closed_forms],
        "weld": [mc_pins.test_weld_sphere_indexed_face_set, mc_pins.test_weld_rejects_two_positions_for_one_key],
        "dual_shapes": [duals_pins.test_dual_shapes_pins],
        "shard": [lambda: shard_pins.test_sharded_equals_unsharded(*shard_pins.CASES[0])],
    }


PY_MUTANTS = {
    "interpolate_higher_first": ("interpolate", [("tuple(q) < tuple(p)", "tuple(q) > tuple(p)")]),
    "interpolate_t_sign": ("interpolate", [("t = (iso32 - s[a]) / (s[b] - s[a])", "t = (s[a] - iso32) / (s[b] - s[a])")]),
    "interpolate_from_b": ("interpolate", [("f[a] + t * (f[b] - f[a])", "f[b] + t * (f[a] - f[b])")]),
    "weld_unchecked": ("weld", [("if not np.array_equal(vtx[inv.reshape(-1)].view(np.int32), p.view(np.int32)):",
                                 "if False:")]),
    "weld_wrong_index": ("weld", [("return vtx, inv.reshape(-1, 3).astype(np.int64), vkeys",
                                   "return vtx, np.sort(inv.reshape(-1, 3), axis=1).astype(np.int64), vkeys")]),
    "dual_shapes_off_by_one": ("dual_shapes", [("return (1 + (d[:, 1:] != d[:, :-1]).sum(axis=1))",
                                                "return ((d[:, 1:] != d[:, :-1]).sum(axis=1))")]),
}


@pytest.mark.parametrize("name", sorted(PY_MUTANTS))
def test_python_mutant_fails_a_pin(monkeypatch, name):
    fn_name, edits = PY_MUTANTS[name]
    mutant = _mutated(getattr(oracle, fn_name), edits)
    monkeypatch.setattr(oracle, fn_name, mutant)
    caught = False
    for pin in _pins()[fn_name]:
        try:
            pin()
        except (AssertionError, oracle.OracleError, pytest.fail.Exception):   # a failed pin
            caught = True
    assert caught, name


def test_python_pins_pass_unmodified():
    for pins in _pins().values():
        for pin in pins:
            pin()


def test_shard_without_owner_filter_fails_a_pin(monkeypatch):
    """The sharded oracle keeping every dual its window emits (halo owners
    included) instead of the slab's own: duplicates and wrong duals."""
    from oracle import shard
    mutant = _mutated(shard._one_slab, [("d = m.duals(owners=owners_local)", "d = m.duals()")])
    monkeypatch.setattr(shard, "_one_slab", mutant)
    with pytest.raises(AssertionError):
        _pins()["shard"][0]()
