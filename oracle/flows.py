"""Element flows written once for floats and TPSA series alike.

Oracle / test infrastructure only.

Coordinates are (x, x', y, y', l, delta): slopes, as in the paper's CPU
exactDrift listing (Sec. 2.1), with l the path-length DEVIATION from the
reference particle (the paper adds the full path length; storing the deviation
keeps FP64 resolution over many turns).  Particles are ultra-relativistic
(beta = 1): no velocity slip, E = pc.

Kick-drift elements (KQUAD/KSEXT, "canonical kick ... 2nd or 4th order
symplectic integration", Sec. 3 / Table 1 multipole_tracking2) convert slopes to
canonical momenta normalised to the reference momentum,
    px = (1+delta) x' / sqrt(1 + x'^2 + y'^2),
integrate with the exact-Hamiltonian drift
    pz = sqrt((1+delta)^2 - px^2 - py^2),  x += h px/pz,  y += h py/pz,
    l += h ((1+delta)/pz - 1),
and the multipole kicks
    quadrupole: px -= K1 h x,  py += K1 h y,
    sextupole:  px -= (K2/2) h (x^2 - y^2),  py += K2 h x y,
then convert back.  Symplectic integrators of any even order are built by the
triple-jump composition of Yoshida (Phys. Lett. A 150 (1990) 262) starting from
the second-order leapfrog S2(t) = D(t/2) K(t) D(t/2).
"""
import math

from .tpsa import cos, sqrt

C_LIGHT = 299792458.0


def leapfrog():
    return [("D", 0.5), ("K", 1.0), ("D", 0.5)]


def triple_jump(scheme, order):
    """S_{order+2}(t) = S(z1 t) S(z0 t) S(z1 t), z1 = 1/(2 - 2^(1/(order+1)))."""
    z1 = 1.0 / (2.0 - 2.0 ** (1.0 / (order + 1)))
    z0 = 1.0 - 2.0 * z1
    out = []
    for z in (z1, z0, z1):
        out += [(op, f * z) for op, f in scheme]
    return out


def merged(scheme):
    out = []
    for op, f in scheme:
        if out and out[-1][0] == op == "D":
            out[-1] = ("D", out[-1][1] + f)
        else:
            out.append((op, f))
    return out


def yoshida(order):
    s = leapfrog()
    o = 2
    while o < order:
        s = triple_jump(s, o)
        o += 2
    return merged(s)


YOSHIDA4 = yoshida(4)   # D(w1/2) K(w1) D((w0+w1)/2) K(w0) D((w0+w1)/2) K(w1) D(w1/2)
YOSHIDA6 = yoshida(6)


def slopes_to_canonical(z):
    x, xp, y, yp, l, d = z
    P = 1.0 + d
    r = sqrt(1.0 + xp * xp + yp * yp)
    return [x, P * xp / r, y, P * yp / r, l, d]


def canonical_to_slopes(z):
    x, px, y, py, l, d = z
    P = 1.0 + d
    pz = sqrt(P * P - px * px - py * py)
    return [x, px / pz, y, py / pz, l, d]


def drift_canonical(z, h):
    """l += h (P/pz - 1), evaluated as h (px^2 + py^2) / (pz (P + pz))."""
    x, px, y, py, l, d = z
    P = 1.0 + d
    p2 = px * px + py * py
    pz = sqrt(P * P - p2)
    return [x + h * px / pz, px, y + h * py / pz, py, l + h * (p2 / (pz * (P + pz))), d]


def kick_canonical(z, h, k1, k2):
    x, px, y, py, l, d = z
    if k1 != 0.0:
        px = px - k1 * h * x
        py = py + k1 * h * y
    if k2 != 0.0:
        px = px - 0.5 * k2 * h * (x * x - y * y)
        py = py + k2 * h * x * y
    return [x, px, y, py, l, d]


def integrate_canonical(z, length, k1, k2, n_steps, scheme=YOSHIDA4):
    """n_steps steps of `scheme` in canonical coordinates (x, px, y, py, l, delta)."""
    h = length / n_steps
    for _ in range(n_steps):
        for op, f in scheme:
            z = drift_canonical(z, f * h) if op == "D" else kick_canonical(z, f * h, k1, k2)
    return z


def thick_multipole(z, length, k1, k2, n_steps, scheme=YOSHIDA4):
    """Kick-drift thick quadrupole/sextupole: n_steps steps of `scheme`."""
    z = slopes_to_canonical(z)
    z = integrate_canonical(z, length, k1, k2, n_steps, scheme)
    return canonical_to_slopes(z)


def exact_drift(z, length):
    """EDRIFT (Sec. 2.1 listings), storing the path-length deviation
    L (sqrt(1 + v) - 1), evaluated as L v / (sqrt(1 + v) + 1)."""
    x, xp, y, yp, l, d = z
    v = xp * xp + yp * yp
    return [x + length * xp, xp, y + length * yp, yp, l + length * (v / (sqrt(1.0 + v) + 1.0)), d]


def thin_quad(z, k1l):
    """Linear thin lens, R21 = -1/f with f = 1/(K1 L) (FODO pin only)."""
    x, xp, y, yp, l, d = z
    return [x, xp - k1l * x, y, yp + k1l * y, l, d]


def thin_sext(z, k2l):
    """Thin sextupole: exact quadratic kick on the slopes."""
    x, xp, y, yp, l, d = z
    return [x, xp - 0.5 * k2l * (x * x - y * y), y, yp + k2l * x * y, l, d]


def rfca(z, volt, phase_deg, freq_hz, p0c):
    """Thin RF cavity (RFCA row of Table 1), beta = 1:
    dE = V cos(phi_s + k_rf l), P' = P + dE, p0' = p0 + V cos(phi_s),
    delta' = P'/p0' - 1, slopes scaled by P/P'.  Returns (z, p0').
    Energies and momenta in eV (charge e)."""
    x, xp, y, yp, l, d = z
    phi = phase_deg * math.pi / 180.0
    k = 2.0 * math.pi * freq_hz / C_LIGHT
    P = (1.0 + d) * p0c
    P1 = P + volt * cos(phi + k * l)
    p0c1 = p0c + volt * math.cos(phi)
    s = P / P1
    return [x, xp * s, y, yp * s, l, P1 / p0c1 - 1.0], p0c1
