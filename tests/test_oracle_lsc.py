"""Pins of the oracle's long-wavelength space-charge kick (CPU): the smoothing
and the difference against their definitions written independently, exact
results on polynomial densities, symmetry, and the Gaussian limit."""
import math

import numpy as np
import pytest

import synthetic as syn
from oracle import oracle as orc


def smooth_then_diff(h, dl, qm, KL, passes):
    """Independent restatement: 1-2-1 filter as a convolution with edge padding,
    then numpy.gradient (central inside, one-sided first order at the ends)."""
    a = qm * np.asarray(h, float) / dl
    for _ in range(passes):
        p = np.concatenate([[a[0]], a, [a[-1]]])
        a = (p[:-2] + 2.0 * p[1:-1] + p[2:]) / 4.0
    return KL * np.gradient(a, dl, edge_order=1)


@pytest.mark.parametrize("passes", [0, 1, 5])
def test_field_matches_independent_restatement(passes):
    g = np.random.Generator(np.random.Philox(key=51))
    h = g.integers(0, 1000, size=300)
    V = orc.lsc_field(h, 2e-6, 1e-15, 3e4, passes)
    assert np.allclose(V, smooth_then_diff(h, 2e-6, 1e-15, 3e4, passes), rtol=1e-12, atol=0)


def test_linear_density_has_constant_field_inside():
    """h_k = a + b k: the filter keeps a linear ramp away from the ends, so the
    field is KL q_m b / dl^2 on every bin more than `passes` from an end."""
    nb, dl, qm, KL, passes = 200, 1e-6, 2e-15, 5e3, 4
    h = 1000 + 7 * np.arange(nb)
    V = orc.lsc_field(h, dl, qm, KL, passes)
    want = KL * qm * 7 / dl ** 2
    assert np.allclose(V[passes + 1:nb - passes - 1], want, rtol=1e-12)


def test_flat_density_has_no_field_and_degenerate_cases():
    assert np.all(orc.lsc_field(np.full(64, 123), 1e-6, 1e-15, 1e4, 3) == 0.0)
    assert np.all(orc.lsc_field(np.array([50]), 1e-6, 1e-15, 1e4, 3) == 0.0)
    assert np.all(orc.lsc_field(np.array([5, 9, 1]), 0.0, 1e-15, 1e4, 3) == 0.0)


def test_symmetric_density_gives_antisymmetric_field():
    h = np.array([1, 4, 9, 20, 40, 60, 40, 20, 9, 4, 1] * 1)
    V = orc.lsc_field(h, 1e-6, 1e-15, 1e4, 2)
    assert np.allclose(V, -V[::-1], rtol=1e-13, atol=1e-30)


def test_gaussian_bunch_field_approaches_the_analytic_derivative():
    """A Gaussian bunch: V(l) -> KL d lambda/dl = -KL Q (l - mu) / sigma^2 g(l)
    near the core; 4e6 particles in 100 bins, 4 smoothing passes (whose
    broadening, about 0.15 sigma, accounts for most of the 3 % left)."""
    n, nb, sig, Q, KL, p0 = 4_000_000, 100, 1e-4, 1e-10, 1e3, 1e9
    g = np.random.Generator(np.random.Philox(key=52))
    z = np.zeros((n, 6))
    z[:, 4] = g.standard_normal(n) * sig
    out, h, V = orc.lsc(z, nb, KL, 4, Q, p0)
    lmin, lmax = z[:, 4].min(), z[:, 4].max()
    dl = (lmax - lmin) / nb
    c = lmin + (np.arange(nb) + 0.5) * dl
    lam = Q / (sig * math.sqrt(2 * math.pi)) * np.exp(-0.5 * (c / sig) ** 2)
    want = -KL * c / sig ** 2 * lam
    core = np.abs(c) < 1.5 * sig
    assert np.max(np.abs(V[core] - want[core])) < 0.05 * np.max(np.abs(want))
    # the kick: delta changes by V(l)/p0c, interpolated; the head (small l) gains
    head, tail = (z[:, 4] < -sig) & (z[:, 4] > -2 * sig), (z[:, 4] > sig) & (z[:, 4] < 2 * sig)
    assert np.all(out[head, 5] > 0.0) and np.all(out[tail, 5] < 0.0)
