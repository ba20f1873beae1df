"""Pins of the CPU oracle to closed forms, invariants, published constants and
brute force (no GPU).  Each test is chosen so that a plausible slip in the
oracle (a dropped term, a wrong sign or index, a transposed operand) fails it.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate

import synthetic as syn
from oracle import flows, maps
from oracle import oracle as orc
from oracle.tpsa import TPS, identity

HERE = os.path.dirname(os.path.abspath(__file__))
T_IDX = {}
_q = 0
for _j in range(6):
    for _k in range(_j, 6):
        T_IDX[(_j, _k)] = _q
        _q += 1

J2 = np.array([[0.0, 1.0], [-1.0, 0.0]])
# (x, px), (y, py) and (l, delta): H = -pz + delta gives dz/ds = dH/d delta with
# z = -l, so the (l, delta) pair enters with the opposite sign.
J6 = np.zeros((6, 6))
J6[0:2, 0:2] = J2
J6[2:4, 2:4] = J2
J6[4:6, 4:6] = -J2


def linear_map_by_tracking(lat, eps=1e-7):
    """Cell matrix from the oracle tracker by central differences (exact for a
    linear lattice up to rounding)."""
    R = np.zeros((6, 6))
    for j in range(6):
        z = np.zeros((2, 6))
        z[0, j], z[1, j] = eps, -eps
        s = orc.track(lat, z, 1, moments=False)
        R[:, j] = (s["z"][0] - s["z"][1]) / (2 * eps)
    return R


def map_elem(m):
    return {"type": "MAP", "map": m}


# ------------------------------------------------------------ linear optics --

def test_thin_lens_fodo_cos_mu_and_beta():
    """Thin-lens FODO (QF f, drift L, QD -f, drift L): cos mu = 1 - L^2/(2 f^2)
    and beta at QF = 2L(1 + sin(mu/2))/sin(mu) (textbook closed forms)."""
    Lq, K1, L = 0.2, 1.2, 1.2
    f = 1.0 / (K1 * Lq)
    lat = {"elements": [map_elem(maps.thin_quad_map(K1 * Lq)), map_elem(maps.drift_map(L, 1)),
                        map_elem(maps.thin_quad_map(-K1 * Lq)), map_elem(maps.drift_map(L, 1))],
           "aperture": None, "p0c": syn.P0C_1GEV}
    M = linear_map_by_tracking(lat)
    cmu = 1.0 - L * L / (2.0 * f * f)
    assert abs(0.5 * (M[0, 0] + M[1, 1]) - cmu) < 1e-12
    assert abs(0.5 * (M[2, 2] + M[3, 3]) - cmu) < 1e-12
    mu = math.acos(cmu)
    beta_max = 2 * L * (1 + math.sin(mu / 2)) / math.sin(mu)
    assert abs(M[0, 1] / math.sin(mu) - beta_max) < 1e-9
    beta_min = 2 * L * (1 - math.sin(mu / 2)) / math.sin(mu)
    assert abs(M[2, 3] / math.sin(mu) - beta_min) < 1e-9


def _quad_R_closed(K, L):
    if K > 0:
        k = math.sqrt(K)
        return np.array([[math.cos(k * L), math.sin(k * L) / k], [-k * math.sin(k * L), math.cos(k * L)]])
    k = math.sqrt(-K)
    return np.array([[math.cosh(k * L), math.sinh(k * L) / k], [k * math.sinh(k * L), math.cosh(k * L)]])


@pytest.mark.parametrize("key,K", [("QF.o2", 1.2), ("QD.o2", -1.2), ("QF.o3", 1.2)])
def test_thick_quad_R_closed_form(key, K):
    m = syn.stored_map(key)
    R = m["R"]
    assert np.allclose(R[0:2, 0:2], _quad_R_closed(K, 0.2), rtol=0, atol=1e-14)
    assert np.allclose(R[2:4, 2:4], _quad_R_closed(-K, 0.2), rtol=0, atol=1e-14)
    assert np.allclose(R[4:6, 4:6], np.eye(2), atol=1e-15)
    off = R.copy()
    for p in range(3):
        off[2 * p:2 * p + 2, 2 * p:2 * p + 2] = 0
    assert np.max(np.abs(off)) < 1e-15
    assert np.max(np.abs(m["C"])) < 1e-16


def test_thick_quad_order2_chromatic_T():
    """In slope coordinates K -> K/(1+delta), so T_{i,j6} = -K dR_ij/dK."""
    K, L = 1.2, 0.2
    m = syn.stored_map("QF.o2")
    for plane, Kp in ((0, K), (2, -K)):
        h = 1e-6 * abs(Kp)
        dR = (_quad_R_closed(Kp + h, L) - _quad_R_closed(Kp - h, L)) / (2 * h)
        for a in range(2):
            for b in range(2):
                t = m["T"][plane + a, T_IDX[(plane + b, 5)]]
                assert abs(t - (-Kp) * dR[a, b]) < 1e-9, (plane, a, b)
    # no other T terms in the transverse rows besides x_j * delta
    for i in range(4):
        for (j, k), q in T_IDX.items():
            if k != 5 or j > 3 or (j // 2) != (i // 2):
                assert abs(m["T"][i, q]) < 1e-15, (i, j, k)


def test_path_length_row_closed_form():
    """l-row: l1 = l0 + 1/2 int (x'^2 + y'^2) ds to second order, i.e.
    T_5,(jk) = (2 - [j==k]) * 1/2 int R2j(s) R2k(s) ds (+ y plane)."""
    K, L = 1.2, 0.2
    m = syn.stored_map("QF.o2")
    for plane, Kp in ((0, K), (2, -K)):
        def Rp(s, a):
            return _quad_R_closed(Kp, s)[1, a]
        for a in range(2):
            for b in range(a, 2):
                val, _ = integrate.quad(lambda s: Rp(s, a) * Rp(s, b), 0.0, L, epsabs=1e-16, epsrel=1e-14)
                expect = 0.5 * val * (1 if a == b else 2)
                assert abs(m["T"][4, T_IDX[(plane + a, plane + b)]] - expect) < 1e-13
    d = syn.stored_map("D1.0.o2")
    assert abs(d["T"][4, T_IDX[(1, 1)]] - 0.5) < 1e-15
    assert abs(d["T"][4, T_IDX[(3, 3)]] - 0.5) < 1e-15
    assert abs(d["R"][0, 1] - 1.0) < 1e-15 and abs(d["R"][2, 3] - 1.0) < 1e-15


def _flow_reference(z):
    return flows.thick_multipole(list(z), 0.2, 1.2, 0.0, 256, flows.YOSHIDA6)


def test_map_truncation_error_scaling_brute_force():
    """|M(eps v) - flow(eps v)| scales as eps^3 for order 2 and eps^4 for order 3."""
    v = np.array([1.0, 0.7, -0.8, 0.5, 0.0, 0.9]) * 1e-2
    for order, slope in ((2, 3), (3, 4)):
        key = "QF.o%d" % order
        lat = {"elements": [map_elem(syn.stored_map(key))], "aperture": None, "p0c": syn.P0C_1GEV}
        errs = []
        for eps in (1.0, 0.5, 0.25):
            z = eps * v
            got = orc.track(lat, z[None, :], 1, moments=False)["z"][0]
            errs.append(np.max(np.abs(got - np.array(_flow_reference(z)))))
        rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
        assert all(abs(r - slope) < 0.25 for r in rates), (order, rates)


def test_T_coefficients_by_central_differences():
    """T_ijk from second central differences of the high-accuracy flow."""
    m = syn.stored_map("QF.o2")
    h = 1e-4
    for (j, k), q in T_IDX.items():
        if j == 4 or k == 4:
            continue
        def f(a, b):
            z = np.zeros(6)
            z[j] += a
            z[k] += b
            return np.array(_flow_reference(z))
        if j == k:
            d2 = (f(h, 0) - 2 * f(0, 0) + f(-h, 0)) / (h * h)
            est = 0.5 * d2
        else:
            est = (f(h, h) - f(h, -h) - f(-h, h) + f(-h, -h)) / (4 * h * h)
        for i in range(6):
            t = m["T"][i, q]
            assert abs(t - est[i]) <= 1e-6 * max(abs(t), 1e-2), (i, j, k, t, est[i])


# ------------------------------------------------------------ symplecticity --

@pytest.mark.parametrize("key", ["QF.o2", "QD.o2", "D1.0.o2", "QF.o3", "QD.o3", "D1.0.o3", "c5.0.QF", "c5.17.QD"])
def test_stored_maps_symplectic(key):
    R = syn.stored_map(key)["R"]
    assert np.max(np.abs(R.T @ J6 @ R - J6)) < 1e-13
    assert abs(np.linalg.det(R) - 1.0) < 1e-13


@pytest.mark.parametrize("k1,k2", [(1.2, 0.0), (-1.2, 0.0), (0.0, 20.0), (0.0, -20.0)])
def test_kickdrift_core_symplectic_off_axis(k1, k2):
    """The Yoshida-4 kick-drift core has an exactly symplectic Jacobian at any
    point (dual-number differentiation through the same integrator)."""
    z0 = [3e-3, 2e-3, -2e-3, 1e-3, 1e-4, 5e-3]
    M = maps.element_map(lambda z: flows.integrate_canonical(z, 0.2, k1, k2, 4), 1, z0)["R"]
    assert np.max(np.abs(M.T @ J6 @ M - J6)) < 1e-13
    assert abs(np.linalg.det(M) - 1.0) < 1e-13


def test_kickdrift_element_on_axis_symplectic():
    M = maps.jacobian(lambda z: flows.thick_multipole(z, 0.2, 1.2, 0.0, 4))
    assert np.max(np.abs(M.T @ J6 @ M - J6)) < 1e-13


def test_rf_jacobian_determinant():
    """Accelerating cavity: each plane's 2x2 block has det p0/p0' (adiabatic
    damping), so R^T J R = J does not hold by construction."""
    p0 = syn.P0C_1GEV
    V, ph, f = 20e6, -10.0, 2.856e9
    p1 = p0 + V * math.cos(math.radians(ph))
    M = maps.element_map(lambda z: flows.rfca(z, V, ph, f, p0)[0], 1)["R"]
    for p in range(3):
        assert abs(np.linalg.det(M[2 * p:2 * p + 2, 2 * p:2 * p + 2]) - p0 / p1) < 1e-14


# ------------------------------------------------------------ the integrator --

def test_yoshida4_coefficients_published():
    vals = {}
    with open(os.path.join(HERE, "golden", "yoshida4.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    ops = flows.YOSHIDA4
    assert [o for o, _ in ops] == ["D", "K", "D", "K", "D", "K", "D"]
    assert abs(ops[1][1] - vals["w1"]) < 1e-15 and abs(ops[3][1] - vals["w0"]) < 1e-15
    assert abs(ops[0][1] - vals["w1"] / 2) < 1e-15 and abs(ops[2][1] - (vals["w0"] + vals["w1"]) / 2) < 1e-15
    assert abs(sum(f for o, f in ops if o == "D") - 1) < 1e-15
    assert abs(sum(f for o, f in ops if o == "K") - 1) < 1e-15


def test_yoshida4_global_error_is_fourth_order():
    """Oracle C kick-drift element vs a 256-step 6th-order reference."""
    z = np.array([5e-3, 1e-3, -4e-3, 2e-3, 0.0, 1e-2])
    ref = np.array(flows.thick_multipole(list(z), 0.2, 1.2, 20.0, 256, flows.YOSHIDA6))
    errs = []
    for n in (2, 4, 8, 16):
        lat = {"elements": [{"type": "KQUAD", "L": 0.2, "K1": 1.2, "K2": 20.0, "n_kicks": n}],
               "aperture": None, "p0c": syn.P0C_1GEV}
        got = orc.track(lat, z[None, :], 1, moments=False)["z"][0]
        errs.append(np.max(np.abs(got - ref)))
    slopes = [math.log2(errs[i] / errs[i + 1]) for i in range(3)]
    assert all(abs(s - 4.0) < 0.2 for s in slopes), slopes


def test_c_and_python_kickdrift_agree():
    rng = np.random.default_rng(0)
    z = rng.normal(size=(20, 6)) * [1e-3, 1e-4, 1e-3, 1e-4, 1e-3, 1e-3]
    for el in ({"type": "KQUAD", "L": 0.2, "K1": -1.2, "n_kicks": 4},
               {"type": "KSEXT", "L": 0.1, "K2": 20.0, "n_kicks": 4}):
        lat = {"elements": [el], "aperture": None, "p0c": syn.P0C_1GEV}
        got = orc.track(lat, z, 1, moments=False)["z"]
        for i in range(len(z)):
            ref = flows.thick_multipole(list(z[i]), el["L"], el.get("K1", 0.0), el.get("K2", 0.0), 4)
            assert np.max(np.abs(got[i] - ref)) < 1e-17


def test_kickdrift_reduces_to_exact_drift_and_quad():
    rng = np.random.default_rng(1)
    z = rng.normal(size=(50, 6)) * [1e-3, 1e-3, 1e-3, 1e-3, 1e-3, 1e-2]
    def run(el):
        return orc.track({"elements": [el], "aperture": None, "p0c": 1e9}, z, 1, moments=False)["z"]
    dr = run({"type": "EDRIFT", "L": 0.2})
    q0 = run({"type": "KQUAD", "L": 0.2, "K1": 0.0, "n_kicks": 4})
    assert np.max(np.abs(dr - q0)) < 1e-15
    q = run({"type": "KQUAD", "L": 0.2, "K1": 1.2, "n_kicks": 4})
    s = run({"type": "KSEXT", "L": 0.2, "K1": 1.2, "K2": 0.0, "n_kicks": 4})
    assert np.array_equal(q, s)
    # the exact drift keeps x' and y' and moves x by L x'
    assert np.array_equal(dr[:, 1], z[:, 1]) and np.allclose(dr[:, 0], z[:, 0] + 0.2 * z[:, 1], atol=1e-18)


def test_kickdrift_quad_linear_part_matches_thick_lens():
    """Small amplitudes, delta = 0: 4 Yoshida-4 steps reproduce the textbook
    thick-quadrupole matrix to the integrator's truncation error."""
    eps = 1e-9
    lat = {"elements": [{"type": "KQUAD", "L": 0.2, "K1": 1.2, "n_kicks": 4}], "aperture": None, "p0c": 1e9}
    R = linear_map_by_tracking(lat, eps)
    assert np.allclose(R[0:2, 0:2], _quad_R_closed(1.2, 0.2), atol=1e-8)
    assert np.allclose(R[2:4, 2:4], _quad_R_closed(-1.2, 0.2), atol=1e-8)


# ------------------------------------------------------------------- RF -----

def test_rf_invariants():
    p0 = syn.P0C_1GEV
    V, ph, f = 20e6, -10.0, 2.856e9
    rng = np.random.default_rng(2)
    z = rng.normal(size=(200, 6)) * [1e-3, 1e-4, 1e-3, 1e-4, 1e-4, 1e-3]
    lat = {"elements": [{"type": "RFCA", "volt": V, "phase_deg": ph, "freq_hz": f}], "aperture": None, "p0c": p0}
    s = orc.track(lat, z, 1, moments=False)
    out, p1 = s["z"], s["p0c"]
    assert abs(p1 - (p0 + V * math.cos(math.radians(ph)))) < 1e-6
    P, P1 = (1 + z[:, 5]) * p0, (1 + out[:, 5]) * p1
    # transverse momentum P x' is unchanged by a longitudinal kick
    assert np.allclose(P1 * out[:, 1], P * z[:, 1], rtol=1e-14, atol=0)
    assert np.allclose(P1 * out[:, 3], P * z[:, 3], rtol=1e-14, atol=0)
    # energy gain follows the cavity voltage at each particle's phase
    k = 2 * math.pi * f / flows.C_LIGHT
    gain = P1 - P
    assert np.allclose(gain, V * np.cos(math.radians(ph) + k * z[:, 4]), rtol=1e-9, atol=1e-3)
    # positions and l untouched; one RF wavelength later the kick repeats
    assert np.array_equal(out[:, [0, 2, 4]], z[:, [0, 2, 4]])
    z2 = z.copy()
    z2[:, 4] += flows.C_LIGHT / f
    s2 = orc.track(lat, z2, 1, moments=False)
    assert np.allclose(s2["z"][:, 5], out[:, 5], rtol=0, atol=1e-12)


def test_rf_zero_voltage_identity():
    z = np.random.default_rng(3).normal(size=(10, 6)) * 1e-3
    lat = {"elements": [{"type": "RFCA", "volt": 0.0, "phase_deg": 30.0, "freq_hz": 1e9}],
           "aperture": None, "p0c": 1e9}
    s = orc.track(lat, z, 1, moments=False)
    # delta goes through (1 + delta) p0 / p0 - 1: equal up to rounding of 1 + delta
    assert np.allclose(s["z"], z, rtol=0, atol=5e-16)
    assert np.array_equal(s["z"][:, :5], z[:, :5]) or np.allclose(s["z"][:, :5], z[:, :5], rtol=1e-15, atol=0)


def test_thin_sextupole_kick():
    z = np.array([[2e-3, 0.0, 1e-3, 0.0, 0.0, 0.0]])
    s = orc.track({"elements": [{"type": "THINSEXT", "K2L": 2.0}], "aperture": None, "p0c": 1e9}, z, 1, moments=False)
    # gradient kick of V = (K2L/6)(x^3 - 3 x y^2)
    assert abs(s["z"][0, 1] - (-(4e-6 - 1e-6))) < 1e-20
    assert abs(s["z"][0, 3] - 2.0 * 2e-3 * 1e-3) < 1e-20


# -------------------------------------------------------------- moments -----

def test_moments_vs_numpy_cov():
    rng = np.random.default_rng(4)
    z = rng.normal(size=(5000, 6)) * [1e-3, 1e-4, 2e-3, 1e-4, 1e-3, 1e-3] + [0.5, 1e-3, -0.2, 0, 3.0, 1e-2]
    alive = (rng.uniform(size=5000) > 0.1).astype(np.uint8)
    m = orc.moments(z, alive)
    za = z[alive == 1]
    assert m[0] == za.shape[0]
    assert np.allclose(m[1:7], za.mean(axis=0), rtol=1e-14, atol=0)
    C = np.cov(za.T, bias=True)
    q = 7
    for j in range(6):
        for k in range(j, 6):
            assert abs(m[q] - C[j, k]) <= 1e-11 * math.sqrt(C[j, j] * C[k, k]), (j, k)
            q += 1


def test_moments_degenerate():
    z = np.ones((3, 6))
    assert np.array_equal(orc.moments(z, np.zeros(3, np.uint8)), np.zeros(28))
    m = orc.moments(z[:1])
    assert m[0] == 1 and np.array_equal(m[1:7], np.ones(6)) and np.array_equal(m[7:], np.zeros(21))


def test_linear_ring_conserves_emittance():
    """Order-1 maps (no chromatic terms): sqrt(det Sigma) per plane is invariant."""
    lat = syn.lattice_c1(order=2)
    for el in lat["elements"]:
        m = dict(el["map"])
        m["order"] = 1
        el["map"] = m
    lat["aperture"] = None
    z = syn.bunch("c1", n=2000)
    s = orc.track(lat, z, 100)
    M = s["moments"]
    def emit(row, p):
        sxx, sxp, spp = row[7 + T_IDX[(p, p)]], row[7 + T_IDX[(p, p + 1)]], row[7 + T_IDX[(p + 1, p + 1)]]
        return math.sqrt(sxx * spp - sxp * sxp)
    # each map's 2x2 determinants are 1 to ~3e-16 (rounding of the series
    # integration), so the invariant holds to ~1e-14 per 40-element turn
    for p in (0, 2):
        e = np.array([emit(r, p) for r in M])
        assert np.max(np.abs(e[1:] / e[:-1] - 1)) < 1e-13
        assert np.max(np.abs(e / e[0] - 1)) < 1e-11


def test_generated_bunch_matches_twiss():
    (bx, ax), (by, ay) = syn.twiss("c1")
    z = syn.bunch("c1", n=200_000, seed=11)
    m = orc.moments(z)
    n = m[0]
    for p, beta, alpha in ((0, bx, ax), (2, by, ay)):
        sxx = m[7 + T_IDX[(p, p)]]
        sxp = m[7 + T_IDX[(p, p + 1)]]
        assert abs(sxx / (syn.EMIT * beta) - 1) < 5 * math.sqrt(2 / n)
        assert abs(sxp / (-syn.EMIT * alpha) - 1) < 5 * math.sqrt(2 / n) * (1 + 1 / abs(alpha))


# ----------------------------------------------------------------- losses ---

def test_loss_records_match_independent_predicate():
    """Lost set and (turn, element) records equal an independent element-by-
    element recomputation with the aperture predicate evaluated in numpy."""
    lat = syn.lattice_c1()
    lat["aperture"] = ("rect", 6e-4, 5e-4)
    z = syn.bunch("c1", n=400)
    s = orc.track(lat, z, 3, moments=False)
    zz = z.copy()
    alive = np.ones(len(z), bool)
    lt = np.full(len(z), -1)
    le = np.full(len(z), -1)
    for t in range(3):
        for e, el in enumerate(lat["elements"]):
            one = {"elements": [el], "aperture": None, "p0c": lat["p0c"]}
            idx = np.nonzero(alive)[0]
            zz[idx] = orc.track(one, zz[idx], 1, moments=False)["z"]
            bad = alive & ~((np.abs(zz[:, 0]) <= 6e-4) & (np.abs(zz[:, 2]) <= 5e-4))
            lt[bad], le[bad] = t, e
            alive &= ~bad
    assert 0 < (~alive).sum() < len(z)
    assert np.array_equal(s["alive"].astype(bool), alive)
    assert np.array_equal(s["loss_turn"], lt) and np.array_equal(s["loss_elem"], le)
    assert np.array_equal(s["z"], zz)


def test_nan_is_lost_and_edge_is_kept():
    lat = {"elements": [{"type": "THINSEXT", "K2L": 0.0}], "aperture": ("rect", 1e-3, 1e-3), "p0c": 1e9}
    z = np.zeros((3, 6))
    z[0, 0] = np.nan
    z[1, 0] = 1e-3          # exactly on the edge: alive
    z[2, 2] = -1.0000000000000002e-3
    s = orc.track(lat, z, 1, moments=False)
    assert list(s["alive"]) == [0, 1, 0]
    ell = {"elements": [{"type": "THINSEXT", "K2L": 0.0}], "aperture": ("ellipse", 2e-3, 1e-3), "p0c": 1e9}
    z = np.zeros((3, 6))
    z[0, 0], z[1, 2], z[2, 0], z[2, 2] = 2e-3, 1e-3, 1.5e-3, 0.7e-3
    s = orc.track(ell, z, 1, moments=False)
    assert list(s["alive"]) == [1, 1, 0]   # (0.75)^2 + (0.7)^2 > 1


def test_resume_equals_single_run():
    lat = syn.lattice_c1()
    z = syn.bunch("c1", n=300)
    a = orc.track(lat, z, 7)
    b = orc.track(lat, z, 3)
    b = orc.track(lat, None, 4, turn0=3, state=b)
    assert np.array_equal(a["z"], b["z"]) and np.array_equal(a["loss_turn"], b["loss_turn"])
    assert np.array_equal(a["moments"][3:], b["moments"])


# ------------------------------------------------------------------- wake ---

def test_histogram_vs_numpy_and_degenerate():
    rng = np.random.default_rng(5)
    l = np.concatenate([rng.normal(0, 1e-4, 9500), rng.uniform(-6e-4, 6e-4, 500)])
    h, lmin, dl, na = orc.wake_hist(l, 4096)
    assert lmin == l.min() and dl == (l.max() - l.min()) / 4096 and na == len(l)
    b = np.clip(np.floor((l - lmin) / dl).astype(np.int64), 0, 4095)
    assert np.array_equal(h, np.bincount(b, minlength=4096))
    assert h.sum() == len(l) and h[-1] >= 1 and h[0] >= 1
    h1, lmin1, dl1, _ = orc.wake_hist(np.array([3e-5]), 16)
    assert dl1 == 0.0 and h1[0] == 1 and h1.sum() == 1
    h2, _, dl2, _ = orc.wake_hist(np.full(7, -2e-5), 16)
    assert dl2 == 0.0 and h2[0] == 7
    alive = np.zeros(7, np.uint8)
    h3, _, _, na3 = orc.wake_hist(np.arange(7.0), 4, alive)
    assert na3 == 0 and h3.sum() == 0


def test_convolution_vs_numpy_and_closed_forms():
    nb, dl, w0, sc, qm = 512, 2e-7, 4e11, 1e-5, 2.5e-17
    w = w0 / np.sqrt(np.maximum(np.arange(nb) * dl, sc))
    rng = np.random.default_rng(6)
    h = rng.integers(0, 5000, nb)
    V = orc.wake_conv(h, dl, w0, sc, qm)
    ref = -qm * np.convolve(h.astype(np.float64), w)[:nb]
    assert np.allclose(V, ref, rtol=1e-13, atol=0)
    # uniform histogram: V_k = -q h sum_{m<=k} W(m dl)
    Vu = orc.wake_conv(np.full(nb, 3), dl, w0, sc, qm)
    assert np.allclose(Vu, -qm * 3 * np.cumsum(w), rtol=1e-13, atol=0)
    # single source bin reproduces the wake function, causal (zero ahead)
    hd = np.zeros(nb, np.int64)
    hd[10] = 1
    Vd = orc.wake_conv(hd, dl, w0, sc, qm)
    assert np.all(Vd[:10] == 0.0)
    assert np.allclose(Vd[10:], -qm * w[: nb - 10], rtol=1e-15, atol=0)


def test_wake_kick_identity_and_interpolation():
    z = syn.bunch("c3", n=5000)
    out, h, V = orc.wake(z, 64, 0.0, 1e-5, 250e-12, 1e9)
    assert np.array_equal(out, z) and np.all(V == 0)
    out, h, V = orc.wake(z, 64, 4e11, 1e-5, 250e-12, 1e9)
    assert h.sum() == len(z)
    lmin, dl = z[:, 4].min(), (z[:, 4].max() - z[:, 4].min()) / 64
    for k in (0, 5, 63):
        assert orc.wake_interp(V, lmin, dl, lmin + (k + 0.5) * dl) == pytest.approx(V[k], rel=1e-14)
    assert orc.wake_interp(V, lmin, dl, lmin) == V[0]
    assert orc.wake_interp(V, lmin, dl, lmin + 64 * dl) == V[63]
    mid = orc.wake_interp(V, lmin, dl, lmin + 6.0 * dl)
    assert mid == pytest.approx(0.5 * (V[5] + V[6]), rel=1e-14)
    dE = (out[:, 5] - z[:, 5]) * 1e9
    assert np.all(V < 0) and np.all(dE < 0)   # every particle loses energy to the wake
    assert np.array_equal(out[:, :5], z[:, :5])
