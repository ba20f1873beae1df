"""GPU parity of the fused tracking path (through the C ABI) against the oracle."""
import math

import numpy as np
import pytest

import synthetic as syn
from oracle import oracle as orc
from paper_1710_07350_gb300 import trk

from gpu_util import (MARGIN, TOL_100, TOL_PASS, by_id, compare_moments, compare_tracking, gpu_track, tol_turns,
                      reduction_check)

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def rand_particles(n, seed, scale=(1e-3, 1e-4, 1e-3, 1e-4, 1e-3, 1e-3), big=0.1):
    """Mostly beam-like particles plus a fraction with large angles that take
    the exact (non-series) branches."""
    rng = np.random.default_rng(seed)
    z = rng.normal(size=(n, 6)) * np.array(scale)
    k = int(big * n)
    z[:k, 1] = rng.uniform(-2e-2, 2e-2, k)
    z[:k, 3] = rng.uniform(-2e-2, 2e-2, k)
    return z


ONE_ELEMENT = [
    ("MAP.o2", lambda: {"type": "MAP", "map": syn.stored_map("QF.o2")}),
    ("MAP.o3", lambda: {"type": "MAP", "map": syn.stored_map("QD.o3")}),
    ("MAP.drift", lambda: {"type": "MAP", "map": syn.stored_map("D1.0.o2")}),
    ("EDRIFT", lambda: {"type": "EDRIFT", "L": 0.9}),
    ("KQUAD", lambda: {"type": "KQUAD", "L": 0.2, "K1": 1.2, "n_kicks": 4}),
    ("KQUAD-", lambda: {"type": "KQUAD", "L": 0.2, "K1": -1.2, "n_kicks": 1}),
    ("KSEXT", lambda: {"type": "KSEXT", "L": 0.1, "K2": 20.0, "n_kicks": 4}),
    ("KSEXT+K1", lambda: {"type": "KSEXT", "L": 0.3, "K1": 0.5, "K2": -20.0, "n_kicks": 3}),
    ("THINSEXT", lambda: {"type": "THINSEXT", "K2L": 20.0}),
    ("RFCA", lambda: {"type": "RFCA", "volt": 20e6, "phase_deg": -10.0, "freq_hz": 2.856e9}),
]


@pytest.mark.parametrize("name,mk", ONE_ELEMENT, ids=[n for n, _ in ONE_ELEMENT])
def test_single_element_one_pass(name, mk):
    lat = {"elements": [mk()], "aperture": None, "p0c": syn.P0C_1GEV}
    z = rand_particles(1000, 7)
    g = gpu_track(lat, z, 1)
    o = orc.track(lat, z, 1)
    compare_tracking(g, o, TOL_PASS)
    compare_moments(g["moments"], o["moments"])
    assert g["p0c"] == o["p0c"]


@pytest.mark.parametrize("block,per_thread", [(128, 1), (64, 2), (256, 1), (96, 2)])
def test_c1_100_turns(block, per_thread):
    """Config 1 at full size (10k particles, 100 turns) in several schedules."""
    lat = syn.lattice_c1()
    z = syn.bunch("c1")
    g = gpu_track(lat, z, 100, schedule={"block": block, "per_thread": per_thread, "chunk_turns": 37})
    o = orc.track(lat, z, 100)
    assert g["n_alive"] == o["n_alive"] == 10000
    err = compare_tracking(g, o, TOL_100)
    compare_moments(g["moments"][:1], o["moments"][:1])
    compare_moments(g["moments"], o["moments"], coord_err=err)
    reduction_check(g)


def test_c1_losses_ragged_tiles():
    """Small aperture: many losses at many elements and turns; n not a multiple
    of the tile; lost ids, turns and elements exact outside the margin."""
    lat = syn.lattice_c1()
    lat["aperture"] = ("rect", 7e-4, 4e-4)
    z = syn.bunch("c1", n=3001, seed=21)
    g = gpu_track(lat, z, 30, schedule={"block": 64, "per_thread": 1, "chunk_turns": 7})
    o = orc.track(lat, z, 30)
    assert 0 < o["n_alive"] < 3001
    err = compare_tracking(g, o, TOL_100)
    compare_moments(g["moments"], o["moments"], coord_err=err)
    reduction_check(g)
    # compaction: alive slots hold exactly the survivors, in id order (stable)
    alive_ids = g["ids"][:g["n_alive"]]
    assert np.all(np.diff(alive_ids) > 0)


def test_c2_one_pass_and_100_turns():
    lat = syn.lattice_c2()
    z = syn.bunch("c2", n=600)
    g1 = gpu_track(lat, z, 1)
    o1 = orc.track(lat, z, 1)
    compare_tracking(g1, o1, TOL_PASS)
    compare_moments(g1["moments"], o1["moments"])
    g = gpu_track(lat, z, 100, schedule={"chunk_turns": 30})
    o = orc.track(lat, z, 100)
    err = compare_tracking(g, o, TOL_100)
    compare_moments(g["moments"], o["moments"], coord_err=err)
    reduction_check(g)
    assert g["p0c"] == o["p0c"]


def test_c2_ellipse_losses():
    lat = syn.lattice_c2(cells=5)
    lat["aperture"] = ("ellipse", 1.2e-3, 6e-4)
    z = syn.bunch("c2", n=2000, seed=9)
    g = gpu_track(lat, z, 12, schedule={"block": 128, "per_thread": 2, "chunk_turns": 5})
    o = orc.track(lat, z, 12)
    assert 0 < o["n_alive"] < 2000
    err = compare_tracking(g, o, TOL_100)
    compare_moments(g["moments"], o["moments"], coord_err=err)
    reduction_check(g)


def test_resume_bit_identical():
    lat = syn.lattice_c2(cells=3)
    lat["aperture"] = ("ellipse", 1.5e-3, 8e-4)
    z = syn.bunch("c2", n=1500, seed=4)
    a = gpu_track(lat, z, 9)
    b = gpu_track(lat, z, 9, calls=[2, 3, 4])
    za, al_a, lt_a, le_a = by_id(a, 1500)
    zb, al_b, lt_b, le_b = by_id(b, 1500)
    assert np.array_equal(za, zb) and np.array_equal(al_a, al_b)
    assert np.array_equal(lt_a, lt_b) and np.array_equal(le_a, le_b)
    assert 0 < a["n_alive"] < 1500
    # survivors keep their relative order whatever the chunking
    assert np.array_equal(a["ids"][:a["n_alive"]], b["ids"][:b["n_alive"]])
    assert np.array_equal(a["moments"][:, 0], b["moments"][:, 0])
    assert np.allclose(a["moments"], b["moments"], rtol=1e-13, atol=0)


def test_schedule_invariance_of_coordinates():
    """The per-particle arithmetic does not depend on the launch shape."""
    lat = syn.lattice_c2(cells=2)
    z = syn.bunch("c2", n=999, seed=5)
    a = gpu_track(lat, z, 5, schedule={"block": 64, "per_thread": 1, "chunk_turns": 1})
    b = gpu_track(lat, z, 5, schedule={"block": 256, "per_thread": 2, "chunk_turns": 5})
    za, _, _, _ = by_id(a, 999)
    zb, _, _, _ = by_id(b, 999)
    assert np.array_equal(za, zb)


def test_edge_cases_empty_single_nan():
    lat = syn.lattice_c1()
    g = gpu_track(lat, np.zeros((0, 6)), 5)
    assert g["n_alive"] == 0 and g["moments"].shape == (0, 28)
    z = np.zeros((3, 6))
    z[0, 0] = np.nan
    z[1, 0] = 0.02
    z[2, 2] = 1e-4
    g = gpu_track(lat, z, 2)
    o = orc.track(lat, z, 2)
    compare_tracking(g, o, tol_turns(2))
    k = list(g["lost"][0]).index(0)      # the NaN particle is lost at element 0 of turn 0
    assert g["lost"][1][k] == 0 and g["lost"][2][k] == 0
    one = syn.bunch("c1", n=1)
    g = gpu_track(lat, one, 3)
    o = orc.track(lat, one, 3)
    compare_tracking(g, o, tol_turns(3))
    compare_moments(g["moments"], o["moments"])


def test_all_lost():
    lat = syn.lattice_c1()
    lat["aperture"] = ("rect", 1e-7, 1e-7)
    z = syn.bunch("c1", n=500)
    g = gpu_track(lat, z, 3)
    o = orc.track(lat, z, 3)
    assert g["n_alive"] == 0 == o["n_alive"]
    compare_tracking(g, o, TOL_PASS)
    assert np.all(g["moments"] == 0.0)


def test_order3_maps_ring():
    lat = syn.lattice_c1(order=3)
    z = syn.bunch("c1", n=2000, seed=3)
    g = gpu_track(lat, z, 20)
    o = orc.track(lat, z, 20)
    err = compare_tracking(g, o, TOL_100)
    compare_moments(g["moments"], o["moments"], coord_err=err)
    reduction_check(g)


def test_fp64_probe_rates_are_plausible():
    """The measured DFMA rate backs the derived FP64 peak of the roofline:
    152 SMs x 2 lanes x 2.07 GHz = 6.3e11 FMA/s at most, and a working
    device reaches a large part of it."""
    fma_rate, mul_rate, add_rate = trk.trk_probe_fp64()
    assert 2e11 < fma_rate < 7e11
    assert 0.3 * fma_rate < mul_rate <= 1.05 * fma_rate
    assert 0.3 * fma_rate < add_rate <= 1.05 * fma_rate


def test_checkpoint_restart_bit_identical():
    """Checkpoint after 4 turns (alive slots, ids, p0c, turn counter copied to the
    host), restart in a new bunch for 5 more: the coordinates and loss records
    equal one straight 9-turn run; the moments agree to reduction order."""
    lat = syn.lattice_c2(cells=3)
    lat["aperture"] = ("ellipse", 1.5e-3, 8e-4)
    z = syn.bunch("c2", n=1500, seed=4)
    a = gpu_track(lat, z, 9)
    za, al_a, lt_a, le_a = by_id(a, 1500)
    L = trk.trk_create_lattice(lat)
    coords, ids = trk.upload(z)
    b = trk.trk_bunch_wrap(coords, ids)
    trk.trk_track(b, L, 4)
    m1 = trk.trk_moments(b)
    na = trk.trk_n_alive(b)
    zz, ii = trk.download(b)
    p0, turn, lost1 = trk.trk_bunch_p0c(b), trk.trk_bunch_turn(b), trk.trk_lost(b)
    assert turn == 4 and 0 < na < 1500
    c2, _ = trk.upload(zz[:na])
    ids2 = torch.from_numpy(np.ascontiguousarray(ii[:na]).astype(np.int32)).cuda()
    b2 = trk.trk_bunch_wrap(c2, ids2)
    trk.trk_bunch_set_p0c(b2, p0)
    trk.trk_bunch_set_turn(b2, turn)
    trk.trk_track(b2, L, 5)
    m2 = trk.trk_moments(b2)
    assert trk.trk_bunch_turn(b2) == 9 and trk.trk_bunch_p0c(b2) == a["p0c"]
    zb = np.full((1500, 6), np.nan)
    z2, i2 = trk.download(b2)
    zb[i2] = z2
    zb[ii[na:]] = zz[na:]          # lost before the checkpoint: slots [n_alive, n) of the first bunch
    lt_b = np.full(1500, -1)
    le_b = np.full(1500, -1)
    for lid, lt, le in (lost1, trk.trk_lost(b2)):
        lt_b[lid] = lt
        le_b[lid] = le
    al_b = np.zeros(1500, bool)
    al_b[i2[:trk.trk_n_alive(b2)]] = True
    assert np.array_equal(al_a, al_b)
    assert np.array_equal(lt_a, lt_b) and np.array_equal(le_a, le_b)
    assert np.array_equal(za, zb)
    assert np.allclose(a["moments"], np.concatenate([m1, m2]), rtol=1e-13, atol=0)
    assert np.array_equal(a["moments"][:, 0], np.concatenate([m1, m2])[:, 0])


def test_repeated_runs_bit_identical():
    """Run-to-run reproducibility of the reductions (moments) and of the
    coordinates: no order depends on scheduling or atomics."""
    lat = syn.lattice_c2(cells=4)
    lat["aperture"] = ("ellipse", 1.5e-3, 8e-4)
    z = syn.bunch("c2", n=30_000, seed=8)
    r1 = gpu_track(lat, z, 6)
    r2 = gpu_track(lat, z, 6)
    assert np.array_equal(r1["moments"], r2["moments"])
    assert np.array_equal(r1["z"], r2["z"]) and np.array_equal(r1["ids"], r2["ids"])


def test_bend_ring_one_pass_and_50_turns():
    """Sector dipoles (exact orbit in a uniform field) between kick-drift
    quadrupoles, with the ellipse aperture: one pass and 50 turns."""
    lat = syn.lattice_bend_ring()
    z = syn.bend_ring_bunch(3000)
    g1 = gpu_track(lat, z, 1)
    o1 = orc.track(lat, z, 1)
    compare_tracking(g1, o1, TOL_PASS)
    compare_moments(g1["moments"], o1["moments"])
    g = gpu_track(lat, z, 50, schedule={"block": 128, "per_thread": 2, "chunk_turns": 20})
    o = orc.track(lat, z, 50)
    err = compare_tracking(g, o, TOL_100)
    compare_moments(g["moments"], o["moments"], coord_err=err)


def test_sbend_zero_angle_is_the_exact_drift():
    lat = {"elements": [{"type": "SBEND", "L": 1.5, "angle": 0.0}, {"type": "SBEND", "L": 0.7, "angle": -0.05}],
           "aperture": ("rect", 0.02, 0.02), "p0c": syn.P0C_1GEV}
    z = syn.bend_ring_bunch(1000, seed=5)
    g = gpu_track(lat, z, 3)
    o = orc.track(lat, z, 3)
    compare_tracking(g, o, tol_turns(3))


def test_sbend_particles_that_cannot_reach_the_exit_face_are_lost_alike():
    """Far off-axis and steep particles (asin argument outside [-1, 1], |y'| beyond
    the momentum, momentum down to 0.1 of the reference): their coordinates turn
    NaN and both sides lose them at the bend; the steep survivors agree to
    rounding amplified by the near-tangent exits (relative 1e-11)."""
    lat = {"elements": [{"type": "SBEND", "L": 1.0, "angle": 0.5}, {"type": "EDRIFT", "L": 0.1}],
           "aperture": ("rect", 5.0, 5.0), "p0c": syn.P0C_1GEV}
    g = np.random.Generator(np.random.Philox(key=23))
    n = 4000
    z = np.zeros((n, 6))
    z[:, 0] = g.uniform(-3.0, 3.0, n)
    z[:, 1] = g.uniform(-2.0, 2.0, n)
    z[:, 2] = g.uniform(-0.01, 0.01, n)
    z[:, 3] = g.uniform(-1.5, 1.5, n)
    z[:, 5] = g.uniform(-0.9, 0.5, n)
    gp = gpu_track(lat, z, 1)
    o = orc.track(lat, z, 1)
    gz, alive, lt, le = by_id(gp, n)
    oa = o["alive"].astype(bool)
    assert np.array_equal(alive, oa) and 1000 < np.sum(~oa) < n - 1000
    assert np.all(le[~oa] == 0) and np.all(o["loss_elem"][~oa] == 0)
    rel = np.abs(gz[oa] - o["z"][oa]) / np.maximum(1.0, np.abs(o["z"][oa]))
    assert np.max(rel) <= 1e-11


@pytest.mark.parametrize("ap", [("rect", 0.01, 0.01), ("ellipse", 0.01, 0.01)])
def test_nan_of_either_sign_is_lost(ap):
    """NaN coordinates with the sign bit set or clear are outside every aperture."""
    n = 512
    z = np.zeros((n, 6))
    z[:, 0] = 1e-3
    neg = np.copysign(np.nan, -1.0)
    z[0::4, 0] = neg
    z[1::4, 2] = neg
    z[2::4, 0] = np.nan
    lat = {"elements": [{"type": "EDRIFT", "L": 0.1}], "aperture": ap, "p0c": syn.P0C_1GEV}
    g = gpu_track(lat, z, 1)
    o = orc.track(lat, z, 1)
    _, alive, lt, le = by_id(g, n)
    assert np.array_equal(alive, o["alive"].astype(bool)) and np.sum(~alive) == 3 * n // 4
    assert np.all(le[~alive] == 0)
