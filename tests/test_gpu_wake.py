"""GPU parity of the longitudinal wake path (histogram, convolution, kick)."""
import numpy as np
import pytest

import synthetic as syn
from oracle import oracle as orc
from paper_1710_07350_gb300 import trk

from gpu_util import TOL_PASS, compare_moments, compare_tracking, gpu_track, tol_turns

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def gpu_wake(z, nbins, w0, sc, charge, p0c, schedule=None):
    coords, ids = trk.upload(z)
    b = trk.trk_bunch_wrap(coords, ids)
    if schedule:
        trk.trk_bunch_set_schedule(b, **schedule)
    hist = torch.zeros(nbins, dtype=torch.int32, device="cuda")
    volt = torch.zeros(nbins, dtype=torch.float64, device="cuda")
    trk.trk_wake(b, nbins, w0, sc, charge, p0c, hist=hist, volt=volt)
    zz, ii = trk.download(b)
    out = np.empty_like(zz)
    out[ii] = zz
    return out, hist.cpu().numpy().astype(np.int64), volt.cpu().numpy()


@pytest.mark.parametrize("n,nbins", [(20_000, 4096), (12_345, 1000), (5000, 16384), (3000, 1)])
def test_wake_standalone(n, nbins):
    z = syn.bunch("c3", n=n)
    W0, sc, Q, p0 = syn.C3_W0, syn.C3_SC, syn.C3_CHARGE, 2.0e9
    g, gh, gV = gpu_wake(z, nbins, W0, sc, Q, p0)
    o, oh, oV = orc.wake(z, nbins, W0, sc, Q, p0)
    assert np.array_equal(gh, oh), "histogram must be bit-exact on identical l"
    assert np.allclose(gV, oV, rtol=1e-13, atol=0)
    assert np.array_equal(g[:, :5], z[:, :5])
    assert np.max(np.abs(g[:, 5] - o[:, 5])) <= 1e-15


def test_wake_degenerate():
    p0 = 1e9
    z = np.zeros((7, 6))
    z[:, 4] = 3e-5                       # all equal: dl = 0, everything in bin 0
    g, gh, gV = gpu_wake(z, 64, 4e11, 1e-5, 1e-12, p0)
    o, oh, oV = orc.wake(z, 64, 4e11, 1e-5, 1e-12, p0)
    assert np.array_equal(gh, oh) and gh[0] == 7
    assert np.allclose(gV, oV, rtol=1e-14, atol=0)
    assert np.allclose(g, o, rtol=0, atol=1e-18)
    g, gh, gV = gpu_wake(z[:1], 8, 4e11, 1e-5, 1e-12, p0)
    o, oh, oV = orc.wake(z[:1], 8, 4e11, 1e-5, 1e-12, p0)
    assert np.array_equal(gh, oh) and np.allclose(g, o, rtol=0, atol=1e-18)


def test_wake_zero_strength_identity():
    z = syn.bunch("c3", n=4000)
    g, gh, gV = gpu_wake(z, 512, 0.0, 1e-5, 250e-12, 1e9)
    assert np.array_equal(g, z) and np.all(gV == 0.0) and gh.sum() == 4000


def test_c3_linac_reduced():
    """Config-3 structure (RF, WAKE, drift, quad per period) at reduced size."""
    lat = syn.lattice_c3(periods=6, nbins=512)
    z = syn.bunch("c3", n=20_000)
    g = gpu_track(lat, z, 1, schedule={"block": 128, "per_thread": 2})
    o = orc.track(lat, z, 1)
    err = compare_tracking(g, o, TOL_PASS)
    compare_moments(g["moments"], o["moments"], coord_err=err)
    assert g["p0c"] == o["p0c"]


def test_wake_last_and_first_element():
    """A lattice that starts and ends with a wake (segments of zero length)."""
    wk = {"type": "WAKE", "nbins": 128, "W0": syn.C3_W0, "sc": syn.C3_SC, "charge": syn.C3_CHARGE}
    rf = {"type": "RFCA", "volt": 20e6, "phase_deg": -10.0, "freq_hz": 2.856e9}
    lat = {"elements": [wk, rf, wk, wk, {"type": "EDRIFT", "L": 1.0}, wk], "aperture": None, "p0c": syn.P0C_1GEV}
    z = syn.bunch("c3", n=3000)
    g = gpu_track(lat, z, 2)
    o = orc.track(lat, z, 2)
    err = compare_tracking(g, o, tol_turns(2))
    compare_moments(g["moments"], o["moments"], coord_err=err)


def offset_bunch(n, seed=3):
    z = syn.bunch("c3", n=n, seed=seed)
    z[:, 0] += 1.0e-4
    z[:, 2] -= 5.0e-5
    return z


def test_transverse_wake_linac_reduced():
    """Linac periods with longitudinal and transverse wakes on an offset bunch:
    coordinates after one pass and the per-pass moments against the oracle."""
    lat = syn.lattice_c3(periods=6, nbins=512, transverse=True)
    z = offset_bunch(20_000)
    g = gpu_track(lat, z, 1, schedule={"block": 128, "per_thread": 2})
    o = orc.track(lat, z, 1)
    err = compare_tracking(g, o, TOL_PASS)
    compare_moments(g["moments"], o["moments"], coord_err=err)
    # the transverse wake acts: the mean slope differs from the run without it
    o0 = orc.track(syn.lattice_c3(periods=6, nbins=512), z, 1)
    assert abs(o["moments"][-1, 2] - o0["moments"][-1, 2]) > 1e-9


@pytest.mark.parametrize("nbins", [4096, 6000])
def test_transverse_wake_single_element(nbins):
    """One wake element with a transverse part, shared-memory dipole sums
    (4096 bins) and global ones (6000 bins), against the oracle."""
    wk = {"type": "WAKE", "nbins": nbins, "W0": syn.C3_W0, "sc": syn.C3_SC, "charge": syn.C3_CHARGE,
          "W0T": syn.C3_W0T}
    lat = {"elements": [wk, {"type": "EDRIFT", "L": 0.5}], "aperture": None, "p0c": 2.0e9}
    z = offset_bunch(50_000, seed=7)
    g = gpu_track(lat, z, 2)
    o = orc.track(lat, z, 2)
    compare_tracking(g, o, TOL_PASS)
    oz, _, _, Vx, Vy = orc.wake2(z, nbins, syn.C3_W0, syn.C3_W0T, syn.C3_SC, syn.C3_CHARGE, 2.0e9)
    assert np.max(np.abs(Vx)) > 0 and np.max(np.abs(Vy)) > 0


@pytest.mark.parametrize("nbins,passes", [(256, 4), (4096, 0), (1, 3)])
def test_space_charge_against_oracle(nbins, passes):
    """Long-wavelength space charge between drifts, twice per turn, two turns;
    the field is computed from bit-exact counts with the oracle's rounding."""
    sc = {"type": "LSC", "nbins": nbins, "L": 2.0, "K": 4.0e4, "charge": syn.C3_CHARGE, "passes": passes}
    lat = {"elements": [sc, {"type": "EDRIFT", "L": 1.0}, sc, {"type": "EDRIFT", "L": 0.5}], "aperture": None,
           "p0c": 1.0e8}
    z = syn.bunch("c3", n=30_000, seed=11)
    g = gpu_track(lat, z, 2)
    o = orc.track(lat, z, 2)
    err = compare_tracking(g, o, TOL_PASS)
    compare_moments(g["moments"], o["moments"], coord_err=err)
    if nbins > 1:
        o0 = orc.track({**lat, "elements": [e for e in lat["elements"] if e["type"] != "LSC"]}, z, 2)
        assert np.max(np.abs(o["z"][:, 5] - o0["z"][:, 5])) > 1e-9


MC2_E = 0.51099895e6   # electron rest energy [eV]


@pytest.mark.parametrize("nbins,f0,f1,p0c", [(256, 0.0, 0.0, 1.0e8), (4096, 0.2, 0.6, 1.0e8), (1024, 0.0, 0.5, 5e6),
                                             (1, 0.0, 0.0, 1.0e8)])
def test_space_charge_impedance_against_oracle(nbins, f0, f1, p0c):
    """Round-beam impedance space charge (radix-2 transforms on the GPU, direct
    transforms in the oracle) between drifts, twice per turn, two turns; the
    counts are bit-exact, the fields agree to the transforms' rounding."""
    sc = {"type": "LSC", "nbins": nbins, "L": 2.0, "charge": syn.C3_CHARGE, "rb": 1e-3, "mc2": MC2_E,
          "f0": f0, "f1": f1}
    lat = {"elements": [sc, {"type": "EDRIFT", "L": 1.0}, sc, {"type": "EDRIFT", "L": 0.5}], "aperture": None,
           "p0c": p0c}
    z = syn.bunch("c3", n=30_000, seed=13)
    g = gpu_track(lat, z, 2)
    o = orc.track(lat, z, 2)
    err = compare_tracking(g, o, TOL_PASS)
    compare_moments(g["moments"], o["moments"], coord_err=err)
    if nbins > 1:
        o0 = orc.track({**lat, "elements": [e for e in lat["elements"] if e["type"] != "LSC"]}, z, 2)
        assert np.max(np.abs(o["z"][:, 5] - o0["z"][:, 5])) > 1e-9


def test_space_charge_impedance_in_accelerating_lattice():
    """gamma follows the reference momentum through an RF cavity between two
    impedance kicks."""
    sc = {"type": "LSC", "nbins": 512, "L": 1.0, "charge": syn.C3_CHARGE, "rb": 5e-4, "mc2": MC2_E}
    rf = {"type": "RFCA", "volt": 2.0e7, "phase_deg": 80.0, "freq_hz": 2.856e9}
    lat = {"elements": [sc, rf, {"type": "EDRIFT", "L": 1.0}, sc], "aperture": None, "p0c": 2.0e7}
    z = syn.bunch("c3", n=20_000, seed=17)
    g = gpu_track(lat, z, 3)
    o = orc.track(lat, z, 3)
    err = compare_tracking(g, o, TOL_PASS)
    compare_moments(g["moments"], o["moments"], coord_err=err)


@pytest.mark.parametrize("bad", [{"nbins": 1000}, {"nbins": 8192}, {"rb": -1e-3}, {"mc2": 0.0},
                                 {"f0": 0.6, "f1": 0.5}, {"f1": 1.5}, {"rb": float("nan")}])
def test_space_charge_impedance_rejects_bad_parameters(bad):
    sc = {"type": "LSC", "nbins": 256, "L": 1.0, "charge": 1e-9, "rb": 1e-3, "mc2": MC2_E, **bad}
    with pytest.raises(trk.TrkError):
        trk.trk_create_lattice({"elements": [sc], "aperture": None, "p0c": 1e8})


@pytest.mark.parametrize("lmin,lmax,nb", [
    (-1.234e-4, 3.21e-4, 1000),      # a window about zero
    (0.75, 0.75 + 2.5e-5, 4096),     # a narrow window far from zero (fixed point set by |l| ~ 1)
    (-3.0e2, -2.9999e2, 777),        # negative, far from zero, odd bin count
    (1e-300, 7e-300, 64),            # tiny magnitudes
    (-5e-3, 5e-3, 65536),            # the largest bin count of the integer path
    (1e6, 1e6 + 1e-3, 4096),         # bins about 2000 units of rounding of l wide
    (2.0, 2.0 + 2.0 ** -40, 16),     # bins a few units of rounding wide
])
def test_wake_histogram_on_and_next_to_bin_edges(lmin, lmax, nb):
    """Particles placed on the bin edges and one ulp either side (where both
    division-free bin indices defer to the division), plus uniform particles:
    counts bit-exact for windows near and far from zero, tiny and wide."""
    dl = (lmax - lmin) / nb
    k = np.arange(nb + 1) if nb <= 5000 else np.random.default_rng(3).integers(0, nb + 1, 5000)
    edges = lmin + k * dl
    rng = np.random.default_rng(nb)
    l = np.concatenate([edges, np.nextafter(edges, np.inf), np.nextafter(edges, -np.inf),
                        rng.uniform(lmin, lmax, 20000), [lmin, lmax]])
    z = np.zeros((l.size, 6))
    z[:, 4] = np.clip(l, lmin, lmax)
    g, gh, gV = gpu_wake(z, nb, syn.C3_W0, syn.C3_SC, syn.C3_CHARGE, 2.0e9)
    o, oh, oV = orc.wake(z, nb, syn.C3_W0, syn.C3_SC, syn.C3_CHARGE, 2.0e9)
    assert np.array_equal(gh, oh)
    assert np.allclose(gV, oV, rtol=1e-13, atol=0)


@pytest.mark.parametrize("order", ["wake-lsc", "lsc-wake", "three", "at-ends"])
def test_adjacent_collective_elements_against_oracle(order):
    """Adjacent collective elements (the parts of an RFCW cavity) share one l
    window on the GPU and kick together, in lattice order, in the next segment's
    prologue; the oracle applies them one after the other.  Different bin
    counts, a transverse wake, impedance and long-wavelength space charge, a run
    of three (a pair and a single), and groups at both ends of the lattice."""
    wk = {"type": "WAKE", "nbins": 512, "W0": syn.C3_W0, "sc": syn.C3_SC, "charge": syn.C3_CHARGE,
          "W0T": syn.C3_W0T}
    sc = {"type": "LSC", "nbins": 1024, "L": 2.0, "charge": syn.C3_CHARGE, "rb": 1e-3, "mc2": MC2_E,
          "f0": 0.2, "f1": 0.6}
    lw = {"type": "LSC", "nbins": 256, "L": 1.0, "K": 4.0e4, "charge": syn.C3_CHARGE, "passes": 2}
    rf = {"type": "RFCA", "volt": syn.C3_VOLT, "phase_deg": syn.C3_PHASE, "freq_hz": syn.C3_FREQ}
    dr = {"type": "EDRIFT", "L": 1.0}
    els = {"wake-lsc": [rf, wk, sc, dr], "lsc-wake": [rf, sc, wk, dr], "three": [rf, wk, sc, lw, dr, rf],
           "at-ends": [wk, sc, rf, dr, lw, wk]}[order]
    lat = {"elements": els, "aperture": None, "p0c": 1.0e8}
    z = offset_bunch(20_000, seed=21)
    g = gpu_track(lat, z, 2)
    o = orc.track(lat, z, 2)
    err = compare_tracking(g, o, TOL_PASS)
    compare_moments(g["moments"], o["moments"], coord_err=err)


def test_space_charge_and_wake_with_losses_and_bends():
    """A sector-bend ring with a wake + impedance space-charge group and an
    aperture that removes part of a wide bunch: the collective elements see only
    the particles still alive, on both sides."""
    ring = syn.lattice_bend_ring(cells=2, aperture=("rect", 2.0e-3, 1.5e-3))
    wk = {"type": "WAKE", "nbins": 512, "W0": syn.C3_W0, "sc": syn.C3_SC, "charge": syn.C3_CHARGE}
    sc = {"type": "LSC", "nbins": 512, "L": 2.0, "charge": syn.C3_CHARGE, "rb": 1e-3, "mc2": MC2_E,
          "f0": 0.25, "f1": 0.5}
    els = ring["elements"]
    lat = {**ring, "elements": els[:4] + [wk, sc] + els[4:]}
    z = syn.bend_ring_bunch(20_000, seed=31)
    z[:, 0] *= 1.5
    z[:, 2] *= 1.5
    z[:, 4] = np.random.Generator(np.random.Philox(key=32)).normal(0.0, 1e-4, z.shape[0])
    g = gpu_track(lat, z, 3)
    o = orc.track(lat, z, 3)
    assert 0.05 < 1.0 - o["n_alive"] / z.shape[0] < 0.6
    err = compare_tracking(g, o, tol_turns(3))
    compare_moments(g["moments"], o["moments"], coord_err=err)


def _parts_run(lat, z, sizes, n_turns, schedule=None):
    """Track z split into parts of the given sizes (ids stay global); returns
    the coordinates by id, the loss records and the reference momentum."""
    L = trk.trk_create_lattice(lat)
    bunches, keep = [], []
    start = 0
    for m in sizes:
        coords, _ = trk.upload(z[start:start + m])
        ids = torch.arange(start, start + m, dtype=torch.int32, device="cuda")
        b = trk.trk_bunch_wrap(coords, ids, n=m)
        if schedule:
            trk.trk_bunch_set_schedule(b, **schedule)
        bunches.append(b)
        keep.append((coords, ids))
        start += m
    trk.trk_track_parts(bunches, L, n_turns)
    out = np.full(z.shape, np.nan)
    lost = {}
    for b in bunches:
        zz, ii = trk.download(b)
        out[ii] = zz
        lid, lt, le = trk.trk_lost(b)
        for a, t, e in zip(lid, lt, le):
            lost[int(a)] = (int(t), int(e))
    return out, lost, trk.trk_bunch_p0c(bunches[0])


def _one_run(lat, z, n_turns, schedule=None):
    g = gpu_track(lat, z, n_turns, schedule=schedule)
    out = np.full(z.shape, np.nan)
    out[g["ids"]] = g["z"]
    lost = {int(a): (int(t), int(e)) for a, t, e in zip(*g["lost"])}
    return out, lost, g["p0c"]


@pytest.mark.parametrize("sizes", [(7000, 1, 12999), (0, 10000, 10000), (5000, 5000, 5000, 5000)])
def test_bunch_in_parts_equals_one_bunch_and_the_oracle(sizes):
    """A bunch held in parts (uneven, one empty or a single particle) through
    linac periods with wakes, transverse wakes and impedance space charge: the
    coordinates equal those of the same particles as one bunch bit for bit,
    and the oracle's (on the whole bunch) to the one-pass tolerance."""
    lat = syn.lattice_c3(periods=3, nbins=512, transverse=True, lsc=True)
    z = offset_bunch(sum(sizes), seed=41)
    got, _, p0 = _parts_run(lat, z, sizes, 1, schedule={"block": 128, "per_thread": 2})
    one, _, p1 = _one_run(lat, z, 1, schedule={"block": 128, "per_thread": 2})
    assert p0 == p1
    assert np.array_equal(got, one)
    o = orc.track(lat, z, 1)
    assert np.max(np.abs(got - o["z"])) <= TOL_PASS


def test_bunch_in_parts_with_losses():
    """Parts lose particles at the aperture between collective elements: the
    window, histogram and charge per particle still cover every part; loss
    records and coordinates equal the one-bunch run's."""
    ring = syn.lattice_bend_ring(cells=2, aperture=("rect", 2.0e-3, 1.5e-3))
    wk = {"type": "WAKE", "nbins": 512, "W0": syn.C3_W0, "sc": syn.C3_SC, "charge": syn.C3_CHARGE}
    sc = {"type": "LSC", "nbins": 512, "L": 2.0, "charge": syn.C3_CHARGE, "rb": 1e-3, "mc2": MC2_E,
          "f0": 0.25, "f1": 0.5}
    els = ring["elements"]
    lat = {**ring, "elements": els[:4] + [wk, sc] + els[4:]}
    z = syn.bend_ring_bunch(12_000, seed=31)
    z[:, 0] *= 1.5
    z[:, 2] *= 1.5
    z[:, 4] = np.random.Generator(np.random.Philox(key=32)).normal(0.0, 1e-4, z.shape[0])
    got, lost_p, _ = _parts_run(lat, z, (3000, 4000, 5000), 3)
    one, lost_1, _ = _one_run(lat, z, 3)
    assert len(lost_1) > 0.05 * z.shape[0]
    assert lost_p == lost_1
    assert np.array_equal(got, one, equal_nan=True)
