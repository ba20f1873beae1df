"""The C-ABI library builds, loads without a GPU and exports every entry point
declared in include/trk.h; the ctypes structures match the C layouts."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1710_07350_gb300 import build, trk

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in os.listdir(os.path.join(ROOT, "include")) if h.endswith(".h")]


def declared_functions():
    names = set()
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(trk_[A-Za-z0-9_]+)\s*\(", src, re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_core_calls():
    names = declared_functions()
    for must in ("trk_create_lattice", "trk_track", "trk_moments", "trk_wake", "trk_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(build.build())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_struct_layouts_match_header(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text("""
#include <stddef.h>
#include <stdio.h>
#include "trk.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(trk_element_desc), offsetof(trk_element_desc, C),
         offsetof(trk_element_desc, charge), sizeof(trk_lattice_opts), offsetof(trk_lattice_opts, p0c_ev),
         sizeof(trk_schedule));
  printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(trk_triage_opts), offsetof(trk_triage_opts, lr),
         offsetof(trk_triage_opts, expand_radius), sizeof(trk_triage_stats),
         offsetof(trk_triage_stats, ms_retrack), offsetof(trk_triage_stats, n_passes), sizeof(trk_stats));
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    want = [ctypes.sizeof(trk.trk_element_desc), trk.trk_element_desc.C.offset, trk.trk_element_desc.charge.offset,
            ctypes.sizeof(trk.trk_lattice_opts), trk.trk_lattice_opts.p0c_ev.offset, ctypes.sizeof(trk.trk_schedule),
            ctypes.sizeof(trk.trk_triage_opts), trk.trk_triage_opts.lr.offset, trk.trk_triage_opts.expand_radius.offset,
            ctypes.sizeof(trk.trk_triage_stats), trk.trk_triage_stats.ms_retrack.offset,
            trk.trk_triage_stats.n_passes.offset, ctypes.sizeof(trk.trk_stats)]
    assert got == want


def test_invalid_descriptors_rejected_without_gpu():
    """Argument validation happens on the host before any device call."""
    lib = trk.lib()
    h = ctypes.c_void_p()
    o = trk.trk_lattice_opts()
    o.p0c_ev = 1e9
    d = (trk.trk_element_desc * 1)()
    d[0].type = 99
    assert lib.trk_create_lattice(d, 1, ctypes.byref(o), ctypes.byref(h)) == 1
    assert b"unknown type" in lib.trk_last_error()
    d[0].type = trk.TYPES["MAP"]
    d[0].order = 2
    assert lib.trk_create_lattice(d, 1, ctypes.byref(o), ctypes.byref(h)) == 1
    assert b"needs R" in lib.trk_last_error()
    d[0].type = trk.TYPES["KQUAD"]
    d[0].n_kicks = 0
    assert lib.trk_create_lattice(d, 1, ctypes.byref(o), ctypes.byref(h)) == 1
    o.p0c_ev = -1.0
    assert lib.trk_create_lattice(d, 1, ctypes.byref(o), ctypes.byref(h)) == 1
    o.p0c_ev = 1e9
    o.aperture = 1
    o.a = 0.0
    assert lib.trk_create_lattice(d, 1, ctypes.byref(o), ctypes.byref(h)) == 1
    assert lib.trk_bunch_wrap(None, 0, None, -1, None, ctypes.byref(h)) == 1
    assert lib.trk_bunch_wrap(None, 5, None, 10, None, ctypes.byref(h)) == 1
    assert lib.trk_track(None, None, 1) == 1


def test_space_charge_and_bend_descriptors_rejected_without_gpu():
    """The impedance space charge and the sector bend validate on the host."""
    lib = trk.lib()
    h = ctypes.c_void_p()
    o = trk.trk_lattice_opts()
    o.p0c_ev = 1e9
    d = (trk.trk_element_desc * 1)()
    d[0].type = trk.TYPES["LSC"]
    d[0].length, d[0].charge, d[0].lsc_rb, d[0].lsc_mc2 = 1.0, 1e-9, 1e-3, 0.511e6
    for nbins in (1000, 8192):                       # a power of two up to 4096
        d[0].nbins = nbins
        assert lib.trk_create_lattice(d, 1, ctypes.byref(o), ctypes.byref(h)) == 1
        assert b"impedance" in lib.trk_last_error()
    d[0].nbins = 256
    for field, value in (("lsc_mc2", 0.0), ("lsc_rb", -1e-3), ("lsc_rb", float("nan")), ("lsc_f1", 1.5)):
        old = getattr(d[0], field)
        setattr(d[0], field, value)
        assert lib.trk_create_lattice(d, 1, ctypes.byref(o), ctypes.byref(h)) == 1
        setattr(d[0], field, old)
    d[0].lsc_f0, d[0].lsc_f1 = 0.6, 0.5                # f0 < f1 when filtering
    assert lib.trk_create_lattice(d, 1, ctypes.byref(o), ctypes.byref(h)) == 1
    d = (trk.trk_element_desc * 1)()
    d[0].type = trk.TYPES["SBEND"]
    for length, angle in ((1.0, 3.2), (0.0, 0.1), (-1.0, 0.1), (1.0, float("nan"))):
        d[0].length, d[0].angle = length, angle
        assert lib.trk_create_lattice(d, 1, ctypes.byref(o), ctypes.byref(h)) == 1
        assert b"sector bend" in lib.trk_last_error()


def test_collective_and_bend_flop_accounting():
    from paper_1710_07350_gb300 import flops
    assert flops.element_flops({"type": "LSC", "nbins": 64}) == 0
    assert flops.element_flops({"type": "SBEND", "L": 1.0, "angle": 0.1}) == 64
    assert flops.element_flops({"type": "SBEND", "L": 1.0, "angle": 0.0}) == 12
    # two complex transforms of N = 8192 points (5 N log2 N each) and N impedance values
    assert flops.lsc_imp_flops(4096) == 2 * 5 * 8192 * 13 + 8192 * (flops.LSC_BRACKET_FLOPS + 6)


def test_reference_arm_prints_one_line_on_the_host(tmp_path):
    """`bench.py --impl reference` times the oracle on the host cores and prints
    the contract's line without touching a GPU."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=root,
                         env={**os.environ, "CUDA_VISIBLE_DEVICES": ""})
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "config",
              "cpu_baseline", "e2e", "impl"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1


def test_step_work_accounting():
    """Passes and flops of a step from loss records (used by the bench)."""
    import numpy as np
    import synthetic as syn
    from paper_1710_07350_gb300 import flops
    lat = syn.lattice_c2(cells=1)
    ne = len(lat["elements"])
    p, f = flops.step_work(lat, 10, 3)
    assert p == 10 * 3 * ne
    per = flops.lattice_pass_flops(lat)
    assert f == 10 * 3 * (per.sum() + flops.MOMENTS_FLOPS)
    p2, f2 = flops.step_work(lat, 10, 3, [1], [2])
    assert p2 == 9 * 3 * ne + (1 * ne + 3)
    assert f2 == 9 * 3 * (per.sum() + 54) + (per.sum() + 54) + per[:3].sum()
    # kick-drift quad with 4 steps: strengths 2 + 13 drifts x 14 + 12 kicks x 4 (+ run entry 9)
    assert flops.element_flops({"type": "KQUAD", "L": 0.2, "K1": 1.2, "n_kicks": 4}, canonical=True) == 232
    assert flops.element_flops({"type": "KQUAD", "L": 0.2, "K1": 1.2, "n_kicks": 4}) == 241
    assert flops.element_flops({"type": "KSEXT", "L": 0.1, "K2": 20.0, "n_kicks": 4}, canonical=True) == 282
    # one c2 cell: the run [QF, SF, D, QD, SF, D] converts at entry (QF) and before the RF cavity
    ell = flops.APERTURE_FLOPS["ellipse"]
    assert list(per) == [241 + ell, 282 + ell, 14 + ell, 232 + ell, 282 + ell, 14 + ell, 12 + 10 + ell]


def test_flop_runs_at_the_turn_end():
    """A run that reaches the end of the turn converts back there; an exact
    drift before the first kick-drift element works on slopes."""
    from paper_1710_07350_gb300 import flops
    q = {"type": "KQUAD", "L": 0.2, "K1": 1.2, "n_kicks": 1}
    d = {"type": "EDRIFT", "L": 1.0}
    lat = {"elements": [d, q, d], "aperture": None}
    body = 2 + 4 * 14 + 3 * 4
    assert list(flops.lattice_pass_flops(lat)) == [12, body + 9, 14 + 10]
    sb = {"type": "SBEND", "L": 1.0, "angle": 0.1}
    lat = {"elements": [q, sb, q], "aperture": ("rect", 0.02, 0.02)}
    assert list(flops.lattice_pass_flops(lat)) == [body + 9 + 4, 10 + 64 + 4, body + 9 + 10 + 4]


def test_da_boundary_metric():
    import numpy as np
    from paper_1710_07350_gb300 import da_metrics as dm
    exh = np.zeros((9, 9), bool)
    exh[2:7, 2:7] = True
    b = dm.boundary(exh)
    assert b[2, 2] and b[1, 1] and b[4, 1] and not b[4, 4] and not b[0, 4]
    ok, nd, r = dm.boundary_difference(exh, exh)
    assert ok and nd == 0
    tri = exh.copy()
    tri[2, 4] = False            # on the boundary: distance 0
    tri[1, 4] = True             # just outside: distance 0 (neighbour of the edge)
    assert dm.boundary_difference(tri, exh)[0]
    tri2 = exh.copy()
    tri2[4, 4] = False           # deep inside: 2 cells from the boundary
    ok, nd, r = dm.boundary_difference(tri2, exh)
    assert not ok and nd == 1 and r == 2
