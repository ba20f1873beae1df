"""Algorithmic work of the tracking path, for the roofline.

Convention: one flop per +, -, *, /, sqrt, rsqrt or cos of the element model
(an FMA is two flops); per-element constants (K1 h, K2 h / 2, ...) are not
counted.  The model is counted in the form the method evaluates it: inside a
run of consecutive kick-drift elements and exact drifts the momenta are the
scaled canonical momenta q = p / (1 + delta) (Sec. 3 "canonical kick"; the
exit conversion of one element and the entry conversion of the next are
inverse maps, so a run converts once at each end), and the drifts of the
Yoshida scheme are the exact-Hamiltonian drift in those variables.  Every
operation counted is one the element model needs; no count exceeds the
instructions the fused kernel issues for it.

Per particle and pass (alive particle entering the element):
  EDRIFT, slopes     x += L x', y += L y' (4); v = x'^2 + y'^2 (3);
                     l += L (sqrt(1 + v) - 1) (5)                                 -> 12
  drift on q         u = qx^2 + qy^2 (3); g = (1 - u)^(-1/2) - 1 (3);
                     t = h (1 + g) (2); x += t qx, y += t qy (4); l += h g (2)    -> 14
                     (an EDRIFT inside a run, and every merged Yoshida drift)
  kick-drift body    strengths / (1 + delta): 2 (quad) or 4 (sextupole);
                     (3 n + 1) merged drifts (14 each); 3 n kicks:
                     quad qx -= a x, qy += a y (4);
                     sextupole w = x^2 - y^2 (3), qx -= hb w (2), qy += (b y) x (3) (8)
  run entry          1/(1 + delta) (2); v (3), (1 + v)^(-1/2) (2), q = c x' (2)     -> 9
  run exit           u (3), g (3), x' = q (1 + g) (4)                                 -> 10
                     charged to the element after the run (or the run's last
                     element at the end of the turn, where the moments need slopes)
  THINSEXT           x' -= (K2L/2)(x^2 - y^2) (5), y' += K2L x y (3)                  -> 8
  SBEND              slopes -> px, py, pz (9), p_h (4), S (6), beta: atan2, asin, divide,
                     add (4), alpha (1), sin and cos of alpha and beta (4), exit point
                     (14), px_f (3), 1/pz_f (6), x_f (5), slopes, y, l (9)               -> 64
  RFCA               P (2), phi + k l (2), cos (1), V * (1), + (1), P/P' (1), 2 *, delta (2) -> 12
  MAP                per nonzero term of degree d (the R_rr = 1 diagonal is free): d * (products) + 1 add
                     i.e. deg 0: 1, deg 1: 2, deg 2: 3, deg 3: 4
  aperture           RECT |x| <= a, |y| <= b: 4;  ELLIPSE (x/a)^2 + (y/b)^2 <= 1: 6
  moments            per alive particle and turn: 6 means + 21 centred products: 54
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


DRIFT_Q_FLOPS = 14          # exact-Hamiltonian drift on the scaled canonical momenta
EDRIFT_SLOPE_FLOPS = 12
RUN_ENTRY_FLOPS = 9
RUN_EXIT_FLOPS = 10
_RUN_TYPES = ("KQUAD", "KSEXT", "EDRIFT")


def kick_drift_body_flops(el):
    """One kick-drift element inside a run (no conversions)."""
    n = el["n_kicks"]
    quad = el.get("K1", 0.0) != 0.0
    sext = el["type"] == "KSEXT" and el.get("K2", 0.0) != 0.0
    setup = (2 if quad else 0) + (4 if sext else 0)
    kick = (4 if quad else 0) + (8 if sext else 0)
    return setup + (3 * n + 1) * DRIFT_Q_FLOPS + 3 * n * kick


def element_flops(el, canonical=False):
    """Flops of one pass through `el`; `canonical`: the particle arrives with
    scaled canonical momenta (inside a run of kick-drift elements)."""
    t = el["type"]
    if t == "EDRIFT":
        return DRIFT_Q_FLOPS if canonical else EDRIFT_SLOPE_FLOPS
    if t in ("KQUAD", "KSEXT"):
        return kick_drift_body_flops(el) + (0 if canonical else RUN_ENTRY_FLOPS)
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
    """Per element: flops of one particle pass including the aperture test and
    the representation changes at the ends of kick-drift runs (a run starts at a
    kick-drift element; an exact drift before any kick-drift element of the
    turn works on slopes; slopes are restored before any other element and at
    the end of the turn)."""
    ap = lat.get("aperture")
    fa = APERTURE_FLOPS[ap[0] if ap else None]
    els = lat["elements"]
    out = np.zeros(len(els), dtype=np.float64)
    canon = False
    for i, el in enumerate(els):
        t = el["type"]
        f = 0
        if canon and t not in _RUN_TYPES:
            f += RUN_EXIT_FLOPS
            canon = False
        f += element_flops(el, canonical=canon)
        if t in ("KQUAD", "KSEXT"):
            canon = True
        out[i] = f + fa
    if canon and len(els):
        out[-1] += RUN_EXIT_FLOPS
    return out


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
