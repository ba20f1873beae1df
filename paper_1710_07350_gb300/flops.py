"""Algorithmic work of the tracking path, for the roofline.

Convention: one flop per +, -, *, /, sqrt or cos of the element model as the
paper and the oracle state it (an FMA is two flops); per-element constants
(K1 h, 0.5 K2 h, ...) are not counted.  This is the work the method needs,
whatever instructions the kernel spends on it.

Per particle and pass (alive particle entering the element):
  EDRIFT        x += L x', y += L y' (4); l += L (sqrt(1 + x'^2 + y'^2) - 1) (8)  -> 12
  kick-drift    entry P = 1 + delta, r = sqrt(1 + x'^2 + y'^2), px, py          -> 10
                per merged drift (n_steps * 3 + 1 of them): pz = sqrt(P^2 - px^2 - py^2) (6),
                x += h px/pz (3), y (3), l += h (P/pz - 1) (4)                     -> 16
                per quad kick (3 per step): px -= a x, py += a y                   -> 4
                per sextupole kick (3 per step): (x^2 - y^2) (3), *c, -= (2); x y * c += (3) -> 8
                exit: pz (6), x' = px/pz, y' = py/pz (2)                           -> 8
  THINSEXT      x' -= (K2L/2)(x^2 - y^2) (5), y' += K2L x y (3)                      -> 8
  SBEND         slopes -> px, py, pz (9), p_h (4), S (6), beta: atan2, asin, divide,
                add (4), alpha (1), sin and cos of alpha and beta (4), exit point
                (14), px_f (3), 1/pz_f (6), x_f (5), slopes, y, l (9)               -> 64
  RFCA          P (2), phi + k l (2), cos (1), V * (1), + (1), P/P' (1), 2 *, delta (2) -> 12
  MAP           per nonzero term of degree d (the R_rr = 1 diagonal is free): d * (products) + 1 add
                i.e. deg 0: 1, deg 1: 2, deg 2: 3, deg 3: 4
  aperture      RECT |x| <= a, |y| <= b: 4;  ELLIPSE (x/a)^2 + (y/b)^2 <= 1: 6
  moments       per alive particle and turn: 6 means + 21 centred products: 54
"""
import numpy as np

MOMENTS_FLOPS = 54
# Wake element per alive particle: min/max (2 compares), bin index (sub, div,
# floor: 3), kick (sub, div, sub, floor, sub, 2 for the interpolation, div by p0
# and add: 9) -> 14; the convolution adds nbins^2/2 multiply-adds per wake.
WAKE_FLOPS_PER_PARTICLE = 14


# Transverse part of a wake element per alive particle: the x and y dipole sums
# (2 adds), 1 / (p0c (1 + delta)) (add, multiply, divide: 3), two interpolated
# voltages (sub, 2 for the interpolation each, shared bin index: 5) and two
# slope kicks (FMA each: 4) -> 14; plus two nbins^2/2 convolutions per wake.
TRWAKE_FLOPS_PER_PARTICLE = 14


def wake_conv_flops(nbins):
    return float(nbins) * (nbins + 1)


# Space-charge element per alive particle: the same window, bin index and
# interpolated energy kick as the wake -> 14.
LSC_FLOPS_PER_PARTICLE = 14
# One value of the impedance bracket 1 - xi K1(xi): 39 series terms of about
# 8 flops (or as many quadrature points above xi = 2), plus kappa, Z and the taper.
LSC_BRACKET_FLOPS = 320


def lsc_imp_flops(nbins):
    """Impedance field of one element pass: two complex transforms of
    N = 2 nbins points (5 N log2 N each), N impedance values and the complex
    products (6 each)."""
    n = 2 * int(nbins)
    return 2 * 5.0 * n * np.log2(n) + n * (LSC_BRACKET_FLOPS + 6)


APERTURE_FLOPS = {None: 0, "rect": 4, "ellipse": 6}


def map_flops(m):
    order = int(m["order"])
    f = 0
    R = np.asarray(m["R"]).reshape(6, 6)
    C = np.asarray(m["C"]).ravel()
    for r in range(6):
        f += int(C[r] != 0.0)
        for j in range(6):
            if R[r, j] != 0.0 and not (j == r and R[r, j] == 1.0):
                f += 2
        if order >= 2:
            f += 3 * int(np.count_nonzero(np.asarray(m["T"]).reshape(6, 21)[r]))
        if order >= 3:
            f += 4 * int(np.count_nonzero(np.asarray(m["U"]).reshape(6, 56)[r]))
    return f


def element_flops(el):
    t = el["type"]
    if t == "EDRIFT":
        return 12
    if t in ("KQUAD", "KSEXT"):
        n = el["n_kicks"]
        kick = (4 if el.get("K1", 0.0) != 0.0 else 0) + (8 if el.get("K2", 0.0) != 0.0 and t == "KSEXT" else 0)
        return 10 + (3 * n + 1) * 16 + 3 * n * kick + 8
    if t == "THINSEXT":
        return 8
    if t == "SBEND":
        return 64 if el["angle"] != 0.0 else 12
    if t == "RFCA":
        return 12
    if t == "MAP":
        return map_flops(el["map"])
    if t in ("WAKE", "LSC"):
        return 0  # counted separately (histogram, field, kick)
    raise ValueError(t)


def lattice_pass_flops(lat):
    """Per element: flops of one particle pass including the aperture test."""
    ap = lat.get("aperture")
    fa = APERTURE_FLOPS[ap[0] if ap else None]
    return np.array([element_flops(el) + fa for el in lat["elements"]], dtype=np.float64)


def step_work(lat, n_start, n_turns, lost_turn_local=(), lost_elem=(), moments=True):
    """(passes, flops) of n_turns turns for n_start alive particles of which the
    listed ones are lost at (local turn, element)."""
    f = lattice_pass_flops(lat)
    ne = len(f)
    cum = np.cumsum(f)
    turn_f = cum[-1] + (MOMENTS_FLOPS if moments else 0)
    lt = np.asarray(lost_turn_local, dtype=np.int64)
    le = np.asarray(lost_elem, dtype=np.int64)
    n_surv = n_start - lt.size
    passes = n_surv * n_turns * ne + float(np.sum(lt * ne + le + 1))
    flops = n_surv * n_turns * turn_f + float(np.sum(lt * turn_f + cum[le])) if lt.size else n_surv * n_turns * turn_f
    return float(passes), float(flops)
