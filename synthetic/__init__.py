"""Seeded synthetic inputs: lattice descriptions, bunches, DA grids, variants.

This module is shared by the product's tests and bench and by the oracle's
tests.  It holds none of the tracking arithmetic: it only lays out element
lists with their parameters, draws seeded random numbers, and loads data files.
Transport-map coefficients and matched Twiss parameters are data written by
``oracle/gen_inputs.py`` into ``synthetic/data/inputs.npz``.

Workloads (stand-ins for the paper's LCLS and Table-1 runs, which use 100k to
3.2M particles per kernel and 8M per GPU; the LCLS lattice is not available):
  c1  10-cell FODO ring of order-2 maps, 10k particles, 100 turns, rect +-20 mm
  c2  40-cell kick-drift ring (Yoshida-4, 4 steps) + 1 RF cavity, 1M particles,
      1000 turns, elliptical aperture 15 x 8 mm
  c3  linac: 200 x [RF -10 deg, WAKE 4096 bins, drift, quad], 10M particles
  c4  256 variants of c1 + thin sextupoles, log-uniform 1000..65536 particles,
      1000 turns
  c5  64 variants (6 lattice parameters) x 512^2 DA grid to +-25 mm, 1000 turns
"""
import math
import os

import numpy as np

DATA = os.path.join(os.path.dirname(__file__), "data", "inputs.npz")

ELECTRON_MASS_EV = 0.51099895e6
C_LIGHT = 299792458.0


def p0c_from_energy(e_total_ev):
    return math.sqrt(e_total_ev * e_total_ev - ELECTRON_MASS_EV * ELECTRON_MASS_EV)


P0C_1GEV = p0c_from_energy(1.0e9)

# Ring and linac constants (readings of the points the paper leaves open).
L_QUAD, K1_QUAD, L_DRIFT = 0.2, 1.2, 1.0
L_SEXT, K2_SEXT, L_DRIFT_C2, N_KICKS = 0.1, 20.0, 0.9, 4
C2_CELLS, C2_HARMONIC, C2_VOLT, C2_PHASE = 40, 400, 1.0e6, -90.0
C3_PERIODS, C3_VOLT, C3_PHASE, C3_FREQ = 200, 20.0e6, -10.0, 2.856e9
C3_NBINS, C3_W0, C3_CHARGE = 4096, 4.0e11, 250e-12
C3_SIGMA_L = 100e-6
C3_SC = 0.1 * C3_SIGMA_L
# transverse dipole wake of the linac variant with transverse wakes: about
# 1e-6 rad per cavity behind a bunch offset by 100 um (a readable kick, not a
# physical structure)
C3_W0T = 1.0e15
# impedance space charge of the linac variant with space charge: a 3 m
# structure, 1 mm round beam, low-pass taper from 1/4 to 1/2 of Nyquist
C3_LSC_L, C3_LSC_RB, C3_LSC_F0, C3_LSC_F1 = 3.0, 1.0e-3, 0.25, 0.5
K2L_THIN = K2_SEXT * L_SEXT
# c5 names no sextupole strength; 10x the c4 value makes the DA sextupole-limited
# inside the +-20 mm aperture (with K2L_THIN it is the aperture rectangle).
K2L_C5 = 10.0 * K2L_THIN
EMIT, SIGMA_D, SIGMA_L = 1e-8, 1e-3, 1e-3
DA_HALF_WIDTH, DA_N = 0.025, 512

_cache = {}


def data():
    """Maps and Twiss written by oracle/gen_inputs.py."""
    if "npz" not in _cache:
        if not os.path.exists(DATA):
            raise FileNotFoundError(
                "synthetic/data/inputs.npz is missing; it is written by oracle/gen_inputs.py")
        with np.load(DATA) as z:
            _cache["npz"] = {k: z[k] for k in z.files}
    return _cache["npz"]


def stored_map(key):
    d = data()
    order = int(d[key + ".order"])
    return {"order": order, "C": d[key + ".C"], "R": d[key + ".R"],
            "T": d[key + ".T"], "U": d[key + ".U"]}


def twiss(name):
    """((beta_x, alpha_x), (beta_y, alpha_y)) at the lattice entrance."""
    t = data()["twiss." + name]
    return (float(t[0]), float(t[1])), (float(t[2]), float(t[3]))


def _map_elem(key):
    return {"type": "MAP", "key": key, "map": stored_map(key)}


def lattice_c1(order=2):
    qf, dr, qd = _map_elem("QF.o%d" % order), _map_elem("D1.0.o%d" % order), _map_elem("QD.o%d" % order)
    return {"name": "c1", "elements": [qf, dr, qd, dr] * 10,
            "aperture": ("rect", 0.02, 0.02), "p0c": P0C_1GEV}


def lattice_c2(cells=C2_CELLS, rf=True):
    cell = [
        {"type": "KQUAD", "L": L_QUAD, "K1": K1_QUAD, "n_kicks": N_KICKS},
        {"type": "KSEXT", "L": L_SEXT, "K2": K2_SEXT, "n_kicks": N_KICKS},
        {"type": "EDRIFT", "L": L_DRIFT_C2},
        {"type": "KQUAD", "L": L_QUAD, "K1": -K1_QUAD, "n_kicks": N_KICKS},
        {"type": "KSEXT", "L": L_SEXT, "K2": -K2_SEXT, "n_kicks": N_KICKS},
        {"type": "EDRIFT", "L": L_DRIFT_C2},
    ]
    circ = C2_CELLS * (2 * L_QUAD + 2 * L_SEXT + 2 * L_DRIFT_C2)
    els = cell * cells
    if rf:
        els = els + [{"type": "RFCA", "volt": C2_VOLT, "phase_deg": C2_PHASE,
                      "freq_hz": C2_HARMONIC * C_LIGHT / circ}]
    return {"name": "c2", "elements": els, "aperture": ("ellipse", 0.015, 0.008), "p0c": P0C_1GEV}


def lattice_c3(periods=C3_PERIODS, nbins=C3_NBINS, transverse=False, lsc=False):
    """Per period [RFCA, WAKE, (LSC,) drift, quad]; with `transverse` the wake has
    its dipole part and with `lsc` an impedance space-charge kick follows it, so
    that a period holds the parts of an RFCW cavity (Table 1)."""
    rf = {"type": "RFCA", "volt": C3_VOLT, "phase_deg": C3_PHASE, "freq_hz": C3_FREQ}
    wk = {"type": "WAKE", "nbins": nbins, "W0": C3_W0, "sc": C3_SC, "charge": C3_CHARGE,
          "W0T": C3_W0T if transverse else 0.0}
    sc = {"type": "LSC", "nbins": nbins, "L": C3_LSC_L, "charge": C3_CHARGE, "rb": C3_LSC_RB,
          "mc2": ELECTRON_MASS_EV, "f0": C3_LSC_F0, "f1": C3_LSC_F1}
    dr = _map_elem("D1.0.o2")
    qf, qd = _map_elem("QF.o2"), _map_elem("QD.o2")
    els = []
    for p in range(periods):
        els += [rf, wk] + ([sc] if lsc else []) + [dr, qf if p % 2 == 0 else qd]
    return {"name": "c3", "elements": els, "aperture": None, "p0c": P0C_1GEV}


def _ring_with_thin_sext(qf, qd, k2l_f, k2l_d):
    els = []
    for c in range(10):
        f = k2l_f[c % len(k2l_f)]
        d = k2l_d[c % len(k2l_d)]
        els += [qf, {"type": "THINSEXT", "K2L": f}, _map_elem("D1.0.o2"),
                qd, {"type": "THINSEXT", "K2L": d}, _map_elem("D1.0.o2")]
    return els


def c4_variants(n_var=256, seed=4):
    """Per variant: (K2L_SF, K2L_SD, n_particles), drawn from Philox(seed)."""
    g = np.random.Generator(np.random.Philox(key=seed))
    u = g.uniform(-0.1, 0.1, size=(n_var, 2))
    n = np.rint(np.exp(g.uniform(math.log(1000.0), math.log(65536.0), size=n_var))).astype(np.int64)
    return [(K2L_THIN * (1 + u[v, 0]), -K2L_THIN * (1 + u[v, 1]), int(n[v])) for v in range(n_var)]


def lattice_bend_ring(cells=8, aperture=("ellipse", 0.02, 0.012)):
    """A ring with sector dipoles: per cell [B, D0.4, QF, D0.4, B, D0.4, QD, D0.4],
    B a 1.5 m sector bend of 2 pi / (2 cells), QF / QD kick-drift quadrupoles
    (0.2 m, K1 = +-1.2, 4 steps); no cavity (the momentum deviation slips)."""
    ang = 2.0 * math.pi / (2 * cells)
    b = {"type": "SBEND", "L": 1.5, "angle": ang}
    d = {"type": "EDRIFT", "L": 0.4}
    qf = {"type": "KQUAD", "L": L_QUAD, "K1": K1_QUAD, "n_kicks": N_KICKS}
    qd = {"type": "KQUAD", "L": L_QUAD, "K1": -K1_QUAD, "n_kicks": N_KICKS}
    return {"name": "bend ring", "elements": [b, d, qf, d, b, d, qd, d] * cells, "aperture": aperture,
            "p0c": P0C_1GEV}


def bend_ring_bunch(n, seed=77):
    """Gaussian bunch for the bend ring: 0.3 mm, 0.1 mrad, sigma_delta 1e-3."""
    g = np.random.Generator(np.random.Philox(key=seed))
    z = np.zeros((n, 6))
    z[:, 0], z[:, 1] = g.normal(0, 3e-4, n), g.normal(0, 1e-4, n)
    z[:, 2], z[:, 3] = g.normal(0, 3e-4, n), g.normal(0, 1e-4, n)
    z[:, 5] = g.normal(0, 1e-3, n)
    return z


def lattice_c4(variant):
    k2f, k2d, _ = variant
    qf, qd = _map_elem("QF.o2"), _map_elem("QD.o2")
    return {"name": "c4", "elements": _ring_with_thin_sext(qf, qd, [k2f], [k2d]),
            "aperture": ("rect", 0.02, 0.02), "p0c": P0C_1GEV}


def c5_params(n_var=64, seed=5):
    """Normalised lattice parameters in [-1, 1]: (K1_QF, K1_QD, K2L_SF1, K2L_SF2,
    K2L_SD1, K2L_SD2); K1 varies +-2 %, K2L +-10 %."""
    g = np.random.Generator(np.random.Philox(key=seed))
    return g.uniform(-1.0, 1.0, size=(n_var, 6))


def c5_strengths(p):
    return (K1_QUAD * (1 + 0.02 * p[0]), -K1_QUAD * (1 + 0.02 * p[1]),
            K2L_C5 * (1 + 0.1 * p[2]), K2L_C5 * (1 + 0.1 * p[3]),
            -K2L_C5 * (1 + 0.1 * p[4]), -K2L_C5 * (1 + 0.1 * p[5]))


def lattice_c5(v):
    p = c5_params()[v]
    _, _, f1, f2, d1, d2 = c5_strengths(p)
    qf, qd = _map_elem("c5.%d.QF" % v), _map_elem("c5.%d.QD" % v)
    return {"name": "c5", "elements": _ring_with_thin_sext(qf, qd, [f1, f2], [d1, d2]),
            "aperture": ("rect", 0.02, 0.02), "p0c": P0C_1GEV}


def da_grid(n=DA_N, half_width=DA_HALF_WIDTH):
    """Cell-centre amplitudes: -w + (i + 1/2) * 2w/n."""
    return -half_width + (np.arange(n) + 0.5) * (2.0 * half_width / n)


def da_particles(n=DA_N, half_width=DA_HALF_WIDTH, stride=1, offset=0):
    """(ny*nx, 6) initial coordinates of the DA grid, row-major [iy][ix], every
    `stride`-th cell starting at `offset`; x' = y' = l = delta = 0."""
    g = da_grid(n, half_width)[offset::stride]
    X, Y = np.meshgrid(g, g)
    z = np.zeros((X.size, 6))
    z[:, 0] = X.ravel()
    z[:, 2] = Y.ravel()
    return z


def gaussian_bunch(n, seed, tw, emit=EMIT, sigma_l=SIGMA_L, sigma_d=SIGMA_D,
                   tail_frac=0.0, tail_half_width=0.0):
    """6D Gaussian bunch matched to Twiss `tw`; a fraction `tail_frac` of the
    particles gets l uniform on [-tail_half_width, +tail_half_width]."""
    g = np.random.Generator(np.random.Philox(key=seed))
    u = g.standard_normal((n, 6))
    z = np.empty((n, 6))
    for p, (beta, alpha) in enumerate(tw):
        z[:, 2 * p] = math.sqrt(emit * beta) * u[:, 2 * p]
        z[:, 2 * p + 1] = math.sqrt(emit / beta) * (u[:, 2 * p + 1] - alpha * u[:, 2 * p])
    z[:, 4] = sigma_l * u[:, 4]
    z[:, 5] = sigma_d * u[:, 5]
    if tail_frac > 0.0:
        nt = int(round(tail_frac * n))
        z[n - nt:, 4] = g.uniform(-tail_half_width, tail_half_width, size=nt)
    return z


def gaussian_bunch_device(n, seed, tw, emit=EMIT, sigma_l=SIGMA_L, sigma_d=SIGMA_D, tail_frac=0.0,
                          tail_half_width=0.0, device="cuda"):
    """The distribution of gaussian_bunch drawn on the device (torch's own
    generator, so not the same particles as the host draw): a (6, n) float64
    CUDA tensor, for throughput runs whose bunch would be slow to make and
    copy from the host."""
    import torch
    g = torch.Generator(device=device).manual_seed(seed)
    u = torch.randn((6, n), dtype=torch.float64, device=device, generator=g)
    z = torch.empty((6, n), dtype=torch.float64, device=device)
    for p, (beta, alpha) in enumerate(tw):
        z[2 * p] = math.sqrt(emit * beta) * u[2 * p]
        z[2 * p + 1] = math.sqrt(emit / beta) * (u[2 * p + 1] - alpha * u[2 * p])
    z[4] = sigma_l * u[4]
    z[5] = sigma_d * u[5]
    if tail_frac > 0.0:
        nt = int(round(tail_frac * n))
        z[4, n - nt:] = (torch.rand(nt, dtype=torch.float64, device=device, generator=g) * 2.0 - 1.0) * tail_half_width
    return z


def c3_bunch_device(n, seed=3):
    """The config-3 bunch distribution (95 % Gaussian, 5 % uniform tail) drawn on the device."""
    return gaussian_bunch_device(n, seed, twiss("c3"), sigma_l=C3_SIGMA_L, tail_frac=0.05,
                                 tail_half_width=6 * C3_SIGMA_L)


def bunch(name, n=None, seed=None):
    """Standard bunch of a workload (n and seed may be overridden)."""
    if name == "c1":
        return gaussian_bunch(n or 10_000, 1 if seed is None else seed, twiss("c1"))
    if name == "c2":
        return gaussian_bunch(n or 1_000_000, 2 if seed is None else seed, twiss("c2"))
    if name == "c3":
        return gaussian_bunch(n or 10_000_000, 3 if seed is None else seed, twiss("c3"),
                              sigma_l=C3_SIGMA_L, tail_frac=0.05, tail_half_width=6 * C3_SIGMA_L)
    raise KeyError(name)


def c4_bunch(v, n):
    """Bunch of c4 variant v (its own Philox key, disjoint from the variant draw)."""
    return gaussian_bunch(n, (4 << 16) + v, twiss("c1"))


def mlp_init(seed=7):
    """Initial surrogate weights, [(W (out, in) float32, b (out,) float32)] for
    8 -> 256 -> 256 -> 256 -> 256 -> 1: W uniform on +-sqrt(6/fan_in) (He), b = 0."""
    g = np.random.Generator(np.random.Philox(key=seed))
    dims = [8, 256, 256, 256, 256, 1]
    out = []
    for i in range(5):
        lim = math.sqrt(6.0 / dims[i])
        W = g.uniform(-lim, lim, size=(dims[i + 1], dims[i])).astype(np.float32)
        out.append((W, np.zeros(dims[i + 1], np.float32)))
    return out
