"""Pins of the oracle's exact sector dipole (CPU): a brute-force RK4
integration of the orbit in the laboratory plane, the textbook linear
sector-bend matrix, symplecticity, and the drift limit."""
import math

import numpy as np
import pytest

from oracle import oracle as orc

L, THETA = 1.5, 0.2


def rk4_bend(z, L, theta, steps=4000):
    """Brute force: the horizontal orbit dX/ds = cos psi, dY/ds = sin psi,
    dpsi/ds = 1/R (uniform field, R = rho p_h, s the horizontal arc length),
    integrated by RK4 from radius rho + x until it crosses the ray at angle
    theta (refined by bisection on the last step); the vertical motion is
    linear in s."""
    x, xp, y, yp, l, d = z
    rho = L / theta
    d1 = 1.0 + d
    r = math.sqrt(1 + xp * xp + yp * yp)
    px, py, pz = xp * d1 / r, yp * d1 / r, d1 / r
    ph = math.sqrt(d1 * d1 - py * py)
    R = rho * ph

    def f(u):
        return np.array([math.cos(u[2]), math.sin(u[2]), 1.0 / R])

    def step(u, h):
        k1 = f(u)
        k2 = f(u + 0.5 * h * k1)
        k3 = f(u + 0.5 * h * k2)
        k4 = f(u + h * k3)
        return u + h / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)

    def g(u):
        return u[1] * math.cos(theta) - u[0] * math.sin(theta)

    u = np.array([rho + x, 0.0, math.atan2(pz, px)])
    h = 1.2 * L / steps
    s = 0.0
    while True:
        v = step(u, h)
        if g(v) >= 0.0:
            lo, hi = 0.0, h
            for _ in range(80):
                mid = 0.5 * (lo + hi)
                if g(step(u, mid)) >= 0.0:
                    hi = mid
                else:
                    lo = mid
            u = step(u, hi)
            s += hi
            break
        u, s = v, s + h
    xf = math.hypot(u[0], u[1]) - rho
    pxf = ph * math.cos(u[2] - theta)
    pzf = math.sqrt(d1 * d1 - pxf * pxf - py * py)
    return np.array([xf, pxf / pzf, y + py / ph * s, py / pzf, l + s * d1 / ph - L, d])


POINTS = [[0, 0, 0, 0, 0, 0], [1e-3, 2e-4, -5e-4, 3e-4, 1e-5, 2e-3], [-4e-3, -1e-3, 2e-3, -2e-3, 0, -5e-3],
          [2e-2, 5e-3, 1e-2, 4e-3, 0, 3e-2]]


@pytest.mark.parametrize("z", POINTS)
def test_exact_bend_matches_brute_force_orbit(z):
    got = orc.sbend(z, L, THETA)
    want = rk4_bend(z, L, THETA)
    assert np.allclose(got, want, rtol=0, atol=5e-11), got - want


def jacobian(f, z0, eps=1e-7):
    z0 = np.asarray(z0, float)
    M = np.zeros((6, 6))
    for j in range(6):
        dp, dm = z0.copy(), z0.copy()
        dp[j] += eps
        dm[j] -= eps
        M[:, j] = (f(dp) - f(dm)) / (2 * eps)
    return M


def test_linear_map_is_the_textbook_sector_bend():
    rho = L / THETA
    c, s = math.cos(THETA), math.sin(THETA)
    M = jacobian(lambda z: orc.sbend(z, L, THETA), np.zeros(6))
    want_x = np.array([[c, rho * s, rho * (1 - c)], [-s / rho, c, s]])
    assert np.allclose(M[0:2][:, [0, 1, 5]], want_x, atol=1e-8)
    assert np.allclose(M[2:4, 2:4], [[1, L], [0, 1]], atol=1e-8)
    # path length: a larger radius and an outward slope lengthen the path
    assert M[4, 0] == pytest.approx(s, abs=1e-8) and M[4, 1] == pytest.approx(rho * (1 - c), abs=1e-8)


def to_canonical(z):
    x, xp, y, yp, l, d = z
    r = math.sqrt(1 + xp * xp + yp * yp)
    return np.array([x, xp * (1 + d) / r, y, yp * (1 + d) / r, -l, d])


def from_canonical(w):
    x, px, y, py, ml, d = w
    pz = math.sqrt((1 + d) ** 2 - px * px - py * py)
    return np.array([x, px / pz, y, py / pz, -ml, d])


@pytest.mark.parametrize("z", POINTS[:3])
def test_symplectic_in_canonical_coordinates(z):
    """In (x, px, y, py, -l, delta) the map's Jacobian satisfies M^T J M = J."""
    J = np.zeros((6, 6))
    for k in range(3):
        J[2 * k, 2 * k + 1], J[2 * k + 1, 2 * k] = 1.0, -1.0
    w0 = to_canonical(np.asarray(z, float))
    M = jacobian(lambda w: to_canonical(orc.sbend(from_canonical(w), L, THETA)), w0, eps=1e-6)
    assert np.max(np.abs(M.T @ J @ M - J)) < 1e-7


def test_small_angle_limit_is_the_drift_and_zero_angle_is_exact_drift():
    z = [1e-3, 2e-4, -5e-4, 3e-4, 1e-5, 2e-3]
    lat = {"elements": [{"type": "EDRIFT", "L": L}], "aperture": None, "p0c": 1e9}
    drift = orc.track(lat, np.array([z]), 1, moments=False)["z"][0]
    assert np.array_equal(orc.sbend(z, L, 0.0), drift)
    assert np.allclose(orc.sbend(z, L, 1e-7), drift, atol=1e-9)
