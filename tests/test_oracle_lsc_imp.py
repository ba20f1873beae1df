"""Pins of the oracle's impedance space-charge kick (CPU): the impedance bracket
1 - x K1(x) against scipy's K1 and its small-argument expansion, the transform
against the closed-form response to one Fourier mode (scale, sign, index and
filter), symmetry, linearity, degenerate cases and the element in tracking."""
import math

import numpy as np
import pytest

import synthetic as syn
from oracle import oracle as orc

sp = pytest.importorskip("scipy.special")

Z0 = 376.730313412
C = 299792458.0
EULER = 0.57721566490153286061


@pytest.mark.parametrize("x", np.logspace(-1, math.log10(600.0), 40))
def test_bracket_matches_scipy_k1(x):
    ref = 1.0 - x * sp.k1(x)
    assert orc.lsc_bracket(x) == pytest.approx(ref, rel=1e-13, abs=1e-16)


@pytest.mark.parametrize("x", [1e-7, 1e-5, 1e-4, 1e-3, 3e-3])
def test_bracket_small_argument_expansion(x):
    """1 - x K1(x) = (x^2/2)(ln(2/x) + 1/2 - gamma_E) + (x^4/16)(ln(2/x) + 5/4 - gamma_E) + O(x^6 ln x),
    from the ascending series of K1 and I1; here 1 - x k1(x) in double loses every
    digit to cancellation, so the expansion is the reference."""
    lg = math.log(2.0 / x)
    ref = 0.5 * x * x * (lg + 0.5 - EULER) + x ** 4 / 16.0 * (lg + 1.25 - EULER)
    assert orc.lsc_bracket(x) == pytest.approx(ref, rel=max(1e-14, x ** 4))


def test_bracket_continuous_between_series_and_integral_and_degenerate():
    # the series ends at 2, the integral starts above it; d/dx (1 - x K1(x)) = x K0(x)
    below, at, above = orc.lsc_bracket(2.0 - 1e-12), orc.lsc_bracket(2.0), orc.lsc_bracket(2.0 + 1e-12)
    step = 1e-12 * 2.0 * sp.k0(2.0)
    assert abs(at - below - step) < 2e-15 and abs(above - at - step) < 2e-15
    assert orc.lsc_bracket(0.0) == 0.0 and orc.lsc_bracket(1e6) == 1.0
    xs = np.linspace(0.01, 20, 500)
    assert np.all(np.diff([orc.lsc_bracket(x) for x in xs]) > 0)   # increasing towards 1


def mode_response(N, m0, dl, L, rb, gamma, f0=0.0, f1=0.0):
    """|Z| of mode m0 from scipy's K1 and the cosine taper, written out."""
    kap = 2 * math.pi * m0 / (N * dl)
    xi = kap * rb / gamma
    z = Z0 / (math.pi * kap * rb * rb) * (1.0 - xi * sp.k1(xi))
    f = m0 / (N / 2)
    if f1 > 0:
        z *= 1.0 if f <= f0 else (0.0 if f >= f1 else 0.5 * (1 + math.cos(math.pi * (f - f0) / (f1 - f0))))
    return z


@pytest.mark.parametrize("N,m0,phi,rb,gamma", [(64, 5, 0.3, 1e-3, 2000.0), (96, 1, -1.1, 5e-4, 50.0),
                                               (128, 40, 2.0, 2e-3, 10.0)])
def test_single_mode_closed_form(N, m0, phi, rb, gamma):
    """lambda_k = A cos(theta_k + phi), theta_k = 2 pi m0 k / N, gives
    V_k = -L c A |Z(kappa_m0)| sin(theta_k + phi): the field leads the density by a
    quarter wave, so the head (smaller l) of a density peak gains energy."""
    A, dl, L = 2e-9, 1e-5, 3.0
    k = np.arange(N)
    th = 2 * math.pi * m0 * k / N + phi
    V = orc.lsc_imp_apply(A * np.cos(th), dl, L, rb, gamma)
    ref = -L * C * A * mode_response(N, m0, dl, L, rb, gamma) * np.sin(th)
    assert np.max(np.abs(V - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_single_mode_long_wavelength_limit():
    """For xi << 1 the impedance tends to i kappa Z0 g / (4 pi gamma^2),
    g = 2 (ln(2 gamma / (kappa r_b)) + 1/2 - gamma_E): the field is the derivative
    of the density times c Z0 g L / (4 pi gamma^2)."""
    N, m0, dl, L, rb, gamma = 256, 3, 1e-4, 1.0, 1e-4, 1e4
    k = np.arange(N)
    kap = 2 * math.pi * m0 / (N * dl)
    lam = 1e-8 * np.cos(kap * k * dl)
    V = orc.lsc_imp_apply(lam, dl, L, rb, gamma)
    g = 2 * (math.log(2 * gamma / (kap * rb)) + 0.5 - EULER)
    ref = C * Z0 * g * L / (4 * math.pi * gamma ** 2) * (-1e-8 * kap * np.sin(kap * k * dl))
    assert np.max(np.abs(V - ref)) <= 1e-9 * np.max(np.abs(ref))


def test_filter_taper_and_cutoff():
    N, dl, L, rb, gamma, f0, f1 = 128, 1e-5, 1.0, 1e-3, 100.0, 0.25, 0.5
    k = np.arange(N)
    for m0, expect_zero in [(10, False), (24, False), (40, True), (63, True)]:
        lam = 1e-9 * np.cos(2 * math.pi * m0 * k / N)
        V = orc.lsc_imp_apply(lam, dl, L, rb, gamma, f0, f1)
        if expect_zero:   # rounding leaks into the other modes only
            full = L * C * 1e-9 * mode_response(N, m0, dl, L, rb, gamma)
            assert np.max(np.abs(V)) <= 1e-11 * full
        else:
            ref = -L * C * 1e-9 * mode_response(N, m0, dl, L, rb, gamma, f0, f1) * np.sin(2 * math.pi * m0 * k / N)
            assert np.max(np.abs(V - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_mean_and_nyquist_carry_no_field():
    N = 64
    V = orc.lsc_imp_apply(np.full(N, 3e-9) + 1e-9 * (-1.0) ** np.arange(N), 1e-5, 1.0, 1e-3, 100.0)
    scale = C * 3e-9 * mode_response(N, 1, 1e-5, 1.0, 1e-3, 100.0)   # the strongest mode's response
    assert np.max(np.abs(V)) <= 1e-11 * scale                        # rounding leakage only


def test_symmetric_histogram_gives_antisymmetric_field_and_linearity():
    nb = 256
    i = np.arange(nb)
    h = np.round(1000 * np.exp(-0.5 * ((i - (nb - 1) / 2) / 30.0) ** 2)).astype(np.int64)
    assert np.array_equal(h, h[::-1])
    V = orc.lsc_imp_field(h, 2e-6, 1e-15, 1.0, 1e-3, 200.0)
    assert np.max(np.abs(V + V[::-1])) <= 1e-12 * np.max(np.abs(V))
    assert V[nb // 2 - 20] > 0 > V[nb // 2 + 20]    # head gains, tail loses
    V2 = orc.lsc_imp_field(2 * h, 2e-6, 1e-15, 1.0, 1e-3, 200.0)
    assert np.max(np.abs(V2 - 2 * V)) <= 1e-13 * np.max(np.abs(V2))


def test_degenerate_cases():
    assert np.all(orc.lsc_imp_field(np.array([5], np.int64), 1e-6, 1e-15, 1.0, 1e-3, 100.0) == 0)
    assert np.all(orc.lsc_imp_field(np.array([5, 3, 0, 1], np.int64), 0.0, 1e-15, 1.0, 1e-3, 100.0) == 0)
    z = np.zeros((10, 6))
    z[:, 4] = 1e-4                                    # all at the same l: dl == 0
    out, _, V = orc.lsc_imp(z, 64, 1.0, 1e-3, 0.511e6, 1e-9, 1e8)
    assert np.all(V == 0) and np.array_equal(out, z)


def test_element_in_tracking_equals_single_kick():
    """An impedance LSC element in a lattice applies exactly the single kick of
    lsc_imp with gamma from p0c and the rest energy."""
    z = syn.bunch("c3", n=4000, seed=5)
    el = {"type": "LSC", "nbins": 128, "L": 2.0, "charge": syn.C3_CHARGE, "rb": 1e-3, "mc2": 0.51099895e6,
          "f0": 0.3, "f1": 0.6}
    lat = {"elements": [el], "aperture": None, "p0c": 1.0e8}
    o = orc.track(lat, z, 1)
    ref, _, V = orc.lsc_imp(z, 128, 2.0, 1e-3, 0.51099895e6, syn.C3_CHARGE, 1.0e8, 0.3, 0.6)
    assert np.array_equal(o["z"], ref)
    assert np.max(np.abs(V)) > 0
