"""Pins of the oracle's transverse dipole wake (CPU): per-bin dipole sums
against a numpy brute force, the closed forms of a rigidly offset bunch and of
a single particle, linearity, causality and the x/y independence."""
import math

import numpy as np
import pytest

import synthetic as syn
from oracle import oracle as orc

W0, W0T, SC, Q, P0 = 4e11, 3e13, 1e-5, 250e-12, 2e9


def bunch(n=4000, seed=41):
    z = syn.bunch("c3", n=n, seed=seed)
    return z


def numpy_bins(z, nb):
    l = z[:, 4]
    lmin, lmax = l.min(), l.max()
    dl = (lmax - lmin) / nb
    b = np.clip(np.floor((l - lmin) / dl), 0, nb - 1).astype(int)
    return b, lmin, dl


def test_dipole_sums_match_brute_force():
    z = bunch()
    for nb in (1, 64, 1000):
        b, _, _ = numpy_bins(z, nb) if nb > 1 else (np.zeros(len(z), int), 0, 0)
        for c in (0, 2):
            D = orc.wake_dipole(z, nb, c)
            want = np.bincount(b, weights=z[:, c], minlength=nb)
            assert np.allclose(D, want, rtol=1e-13, atol=1e-18)


def test_rigid_offset_relates_transverse_to_longitudinal_voltage():
    """All x = X0: D = X0 h, so Vx = -(W0T / W0) X0 V (same s_c), and Vy = 0."""
    z = bunch()
    z[:, 0] = 1.5e-4
    z[:, 2] = 0.0
    _, h, V, Vx, Vy = orc.wake2(z, 500, W0, W0T, SC, Q, P0)
    assert np.allclose(Vx, -(W0T / W0) * 1.5e-4 * V, rtol=1e-12, atol=0)
    assert np.all(Vy == 0.0)


def test_single_particle_self_kick_closed_form():
    z = np.array([[2e-4, 1e-5, -1e-4, 0.0, 3e-5, 2e-3]])
    out, h, V, Vx, Vy = orc.wake2(z, 16, W0, W0T, SC, Q, P0)
    w = W0T / math.sqrt(SC)
    assert Vx[0] == pytest.approx(Q * 2e-4 * w, rel=1e-15)
    assert Vy[0] == pytest.approx(Q * -1e-4 * w, rel=1e-15)
    P = P0 * (1.0 + 2e-3)
    assert out[0, 1] == pytest.approx(1e-5 + Vx[0] / P, rel=1e-15)
    assert out[0, 3] == pytest.approx(0.0 + Vy[0] / P, abs=1e-25)
    # the energy kick uses the same single-particle voltage, after the transverse kick
    assert out[0, 5] == pytest.approx(2e-3 + V[0] / P0, rel=1e-14)


def test_linearity_sign_and_xy_independence():
    z = bunch()
    _, _, _, Vx1, Vy1 = orc.wake2(z, 300, W0, W0T, SC, Q, P0)
    z2 = z.copy()
    z2[:, 0] *= 2.0
    z2[:, 2] *= -1.0
    _, _, _, Vx2, Vy2 = orc.wake2(z2, 300, W0, W0T, SC, Q, P0)
    assert np.allclose(Vx2, 2.0 * Vx1, rtol=1e-14, atol=1e-30)
    assert np.allclose(Vy2, -Vy1, rtol=1e-14, atol=1e-30)
    z3 = z.copy()
    z3[:, 0] = 0.0
    out, _, _, Vx3, _ = orc.wake2(z3, 300, W0, W0T, SC, Q, P0)
    assert np.all(Vx3 == 0.0) and np.array_equal(out[:, 1], z3[:, 1])


def test_causality_tail_offsets_act_on_no_bin_ahead():
    """Offsets only in the last bin: every earlier bin sees no transverse voltage."""
    z = bunch()
    b, _, _ = numpy_bins(z, 200)
    z[:, 0] = 0.0
    z[b == 199, 0] = 3e-4
    _, _, _, Vx, _ = orc.wake2(z, 200, W0, W0T, SC, Q, P0)
    assert np.all(Vx[:199] == 0.0) and Vx[199] != 0.0


def test_transverse_strength_zero_is_the_longitudinal_wake():
    z = bunch()
    a = orc.wake(z, 256, W0, SC, Q, P0)
    b = orc.wake2(z, 256, W0, 0.0, SC, Q, P0)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
