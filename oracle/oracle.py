"""ctypes wrapper of the C oracle (trk_oracle.c) plus lattice marshalling.

Oracle / test infrastructure only (see oracle/__init__.py).
"""
import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "trk_oracle.c")
LIB = os.path.join(HERE, "_build", "liboracle.so")

TYPES = {"MAP": 1, "EDRIFT": 2, "KQUAD": 3, "KSEXT": 4, "THINSEXT": 5, "RFCA": 6, "WAKE": 7, "LSC": 8,
         "SBEND": 9}
APERTURES = {None: 0, "rect": 1, "ellipse": 2}
ED_N, EM_N = 20, 504


def build(force=False):
    """Compile the oracle (-O2 -ffp-contract=off: every operation rounds as written)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    tmp = LIB + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared",
                           "-o", tmp, SRC, "-lm"])
    os.replace(tmp, LIB)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        P = ctypes.c_void_p
        L.o_track.restype = ctypes.c_int64
        L.o_track.argtypes = [ctypes.c_int, P, P, P, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                              P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                              P, P, P, P, P, P]
        L.o_moments.restype = None
        L.o_moments.argtypes = [P, P, ctypes.c_int64, P]
        L.o_wake_hist.restype = ctypes.c_int64
        L.o_wake_hist.argtypes = [P, P, ctypes.c_int64, ctypes.c_int, P, P, P]
        L.o_wake_conv.restype = None
        L.o_wake_conv.argtypes = [P, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_double, P]
        L.o_wake_interp.restype = ctypes.c_double
        L.o_wake_interp.argtypes = [P, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.o_wake.restype = None
        L.o_wake.argtypes = [P, P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_double,
                             ctypes.c_double, ctypes.c_double, ctypes.c_double, P, P]
        L.o_wake2.restype = None
        L.o_wake2.argtypes = [P, P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_double,
                              ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, P, P, P, P]
        L.o_lsc.restype = None
        L.o_lsc.argtypes = [P, P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                            ctypes.c_double, ctypes.c_double, P, P]
        L.o_lsc_field.restype = None
        L.o_lsc_field.argtypes = [P, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int, P]
        L.o_lsc_bracket.restype = ctypes.c_double
        L.o_lsc_bracket.argtypes = [ctypes.c_double]
        L.o_lsc_imp_apply.restype = None
        L.o_lsc_imp_apply.argtypes = [P, ctypes.c_int] + [ctypes.c_double] * 6 + [P]
        L.o_lsc_imp_field.restype = None
        L.o_lsc_imp_field.argtypes = [P, ctypes.c_int] + [ctypes.c_double] * 7 + [P]
        L.o_lsc_imp.restype = None
        L.o_lsc_imp.argtypes = [P, P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int] + [ctypes.c_double] * 7 + [P, P]
        L.o_sbend.restype = None
        L.o_sbend.argtypes = [P, ctypes.c_double, ctypes.c_double]
        L.o_wake_dipole.restype = None
        L.o_wake_dipole.argtypes = [P, P, ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_int, P]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def lattice_arrays(lat):
    els = lat["elements"]
    ne = len(els)
    ei = np.zeros((ne, 4), np.int32)
    ed = np.zeros((ne, ED_N), np.float64)
    em = np.zeros((ne, EM_N), np.float64)
    for e, el in enumerate(els):
        t = el["type"]
        ei[e, 0] = TYPES[t]
        if t == "MAP":
            m = el["map"]
            ei[e, 1] = m["order"]
            em[e, 0:6] = m["C"]
            em[e, 6:42] = np.asarray(m["R"]).ravel()
            em[e, 42:168] = np.asarray(m["T"]).ravel()
            em[e, 168:504] = np.asarray(m["U"]).ravel()
        elif t == "EDRIFT":
            ed[e, 0] = el["L"]
        elif t in ("KQUAD", "KSEXT"):
            ed[e, 0] = el["L"]
            ed[e, 1] = el.get("K1", 0.0)
            ed[e, 2] = el.get("K2", 0.0)
            ei[e, 2] = el["n_kicks"]
        elif t == "THINSEXT":
            ed[e, 9] = el["K2L"]
        elif t == "RFCA":
            ed[e, 3], ed[e, 4], ed[e, 5] = el["volt"], el["phase_deg"], el["freq_hz"]
        elif t == "WAKE":
            ei[e, 3] = el["nbins"]
            ed[e, 6], ed[e, 7], ed[e, 8] = el["W0"], el["sc"], el["charge"]
            ed[e, 10] = el.get("W0T", 0.0)
        elif t == "SBEND":
            ed[e, 0], ed[e, 12] = el["L"], el["angle"]
        elif t == "LSC":
            ei[e, 3], ei[e, 1] = el["nbins"], el.get("passes", 0)
            ed[e, 0], ed[e, 11], ed[e, 8] = el["L"], el.get("K", 0.0), el["charge"]
            ed[e, 13], ed[e, 14] = el.get("rb", 0.0), el.get("mc2", 0.0)
            ed[e, 15], ed[e, 16] = el.get("f0", 0.0), el.get("f1", 0.0)
        else:
            raise ValueError(t)
    return ei, ed, em


def track(lat, z, n_turns, turn0=0, state=None, moments=True, p0c=None, n_total=None):
    """Track a copy of z (n x 6).  `state` (from a previous call) continues a run.
    Returns dict z, alive, loss_turn, loss_elem, margin, moments, p0c, n_alive."""
    ei, ed, em = lattice_arrays(lat)
    if state is None:
        z = np.array(z, dtype=np.float64, order="C", copy=True)
        n = z.shape[0]
        state = {"z": z, "alive": np.ones(n, np.uint8), "loss_turn": np.full(n, -1, np.int32),
                 "loss_elem": np.full(n, -1, np.int32), "margin": np.full(n, np.inf),
                 "p0c": lat["p0c"] if p0c is None else p0c, "n_total": n if n_total is None else n_total}
    else:
        state = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in state.items()}
    n = state["z"].shape[0]
    mom = np.zeros((max(n_turns, 1), 28)) if moments else None
    p0 = ctypes.c_double(state["p0c"])
    ap = lat.get("aperture")
    ap_t, ap_a, ap_b = (APERTURES[ap[0]], ap[1], ap[2]) if ap else (0, 0.0, 0.0)
    na = lib().o_track(len(lat["elements"]), _p(ei), _p(ed), _p(em), ap_t, ap_a, ap_b,
                       _p(state["z"]), n, state["n_total"], n_turns, turn0,
                       _p(state["alive"]), _p(state["loss_turn"]), _p(state["loss_elem"]),
                       _p(state["margin"]), _p(mom) if moments else None, ctypes.byref(p0))
    state["p0c"] = p0.value
    state["n_alive"] = int(na)
    state["moments"] = mom[:n_turns] if moments else None
    return state


def moments(z, alive=None):
    z = np.ascontiguousarray(z, dtype=np.float64)
    alive = np.ones(z.shape[0], np.uint8) if alive is None else np.ascontiguousarray(alive, np.uint8)
    out = np.zeros(28)
    lib().o_moments(_p(z), _p(alive), z.shape[0], _p(out))
    return out


def wake_hist(l, nbins, alive=None):
    n = len(l)
    z = np.zeros((n, 6))
    z[:, 4] = l
    alive = np.ones(n, np.uint8) if alive is None else np.ascontiguousarray(alive, np.uint8)
    h = np.zeros(nbins, np.int64)
    lmin, dl = ctypes.c_double(), ctypes.c_double()
    na = lib().o_wake_hist(_p(z), _p(alive), n, nbins, ctypes.byref(lmin), ctypes.byref(dl), _p(h))
    return h, lmin.value, dl.value, int(na)


def wake_conv(hist, dl, w0, sc, qm):
    hist = np.ascontiguousarray(hist, np.int64)
    V = np.zeros(len(hist))
    lib().o_wake_conv(_p(hist), len(hist), dl, w0, sc, qm, _p(V))
    return V


def wake_interp(V, lmin, dl, l):
    V = np.ascontiguousarray(V, np.float64)
    return lib().o_wake_interp(_p(V), len(V), lmin, dl, l)


def wake(z, nbins, w0, sc, charge, p0c, alive=None, n_total=None):
    """One wake element on a copy of z; returns (z, hist, V)."""
    z = np.array(z, dtype=np.float64, order="C", copy=True)
    n = z.shape[0]
    alive = np.ones(n, np.uint8) if alive is None else np.ascontiguousarray(alive, np.uint8)
    h = np.zeros(nbins, np.int64)
    V = np.zeros(nbins)
    lib().o_wake(_p(z), _p(alive), n, n if n_total is None else n_total, nbins, w0, sc, charge, p0c,
                 _p(h), _p(V))
    return z, h, V


def wake2(z, nbins, w0, w0t, sc, charge, p0c, alive=None, n_total=None):
    """Longitudinal and transverse wake on a copy of z; returns (z, hist, V, Vx, Vy)."""
    z = np.array(z, dtype=np.float64, order="C", copy=True)
    n = z.shape[0]
    alive = np.ones(n, np.uint8) if alive is None else np.ascontiguousarray(alive, np.uint8)
    h = np.zeros(nbins, np.int64)
    V, Vx, Vy = np.zeros(nbins), np.zeros(nbins), np.zeros(nbins)
    lib().o_wake2(_p(z), _p(alive), n, n if n_total is None else n_total, nbins, w0, w0t, sc, charge, p0c,
                  _p(h), _p(V), _p(Vx), _p(Vy))
    return z, h, V, Vx, Vy


def lsc(z, nbins, KL, passes, charge, p0c, alive=None, n_total=None):
    """One space-charge kick on a copy of z; returns (z, hist, V)."""
    z = np.array(z, dtype=np.float64, order="C", copy=True)
    n = z.shape[0]
    alive = np.ones(n, np.uint8) if alive is None else np.ascontiguousarray(alive, np.uint8)
    h = np.zeros(nbins, np.int64)
    V = np.zeros(nbins)
    lib().o_lsc(_p(z), _p(alive), n, n if n_total is None else n_total, nbins, KL, passes, charge, p0c, _p(h),
                _p(V))
    return z, h, V


def lsc_field(hist, dl, qm, KL, passes):
    h = np.ascontiguousarray(hist, np.int64)
    V = np.zeros(len(h))
    lib().o_lsc_field(_p(h), len(h), dl, qm, KL, passes, _p(V))
    return V


def lsc_bracket(x):
    """1 - x K1(x), the bracket of the round-beam space-charge impedance."""
    return lib().o_lsc_bracket(float(x))


def lsc_imp_apply(lam, dl, L, rb, gamma, f0=0.0, f1=0.0):
    """Impedance kick voltage on a periodic line density lam (C/m), all bins."""
    lam = np.ascontiguousarray(lam, np.float64)
    V = np.zeros(len(lam))
    lib().o_lsc_imp_apply(_p(lam), len(lam), dl, L, rb, gamma, f0, f1, _p(V))
    return V


def lsc_imp_field(hist, dl, qm, L, rb, gamma, f0=0.0, f1=0.0):
    """Impedance kick voltage on the bins of a histogram (zero-padded to 2 nb)."""
    h = np.ascontiguousarray(hist, np.int64)
    V = np.zeros(len(h))
    lib().o_lsc_imp_field(_p(h), len(h), dl, qm, L, rb, gamma, f0, f1, _p(V))
    return V


def lsc_imp(z, nbins, L, rb, mc2, charge, p0c, f0=0.0, f1=0.0, alive=None, n_total=None):
    """One impedance space-charge kick on a copy of z; returns (z, hist, V)."""
    z = np.array(z, dtype=np.float64, order="C", copy=True)
    n = z.shape[0]
    alive = np.ones(n, np.uint8) if alive is None else np.ascontiguousarray(alive, np.uint8)
    h = np.zeros(nbins, np.int64)
    V = np.zeros(nbins)
    lib().o_lsc_imp(_p(z), _p(alive), n, n if n_total is None else n_total, nbins, L, rb, mc2, f0, f1, charge,
                    p0c, _p(h), _p(V))
    return z, h, V


def sbend(z, L, angle):
    """The exact sector bend on a copy of one particle's 6 coordinates."""
    zz = np.array(z, dtype=np.float64, copy=True)
    lib().o_sbend(_p(zz), L, angle)
    return zz


def wake_dipole(z, nbins, coord, alive=None):
    """Per-bin sums of coordinate `coord` (0 = x, 2 = y) on the bins of wake_hist."""
    z = np.ascontiguousarray(z, dtype=np.float64)
    n = z.shape[0]
    alive = np.ones(n, np.uint8) if alive is None else np.ascontiguousarray(alive, np.uint8)
    h = np.zeros(nbins, np.int64)
    lmin, dl = ctypes.c_double(), ctypes.c_double()
    lib().o_wake_hist(_p(z), _p(alive), n, nbins, ctypes.byref(lmin), ctypes.byref(dl), _p(h))
    D = np.zeros(nbins)
    lib().o_wake_dipole(_p(z), _p(alive), n, nbins, lmin.value, dl.value, coord, _p(D))
    return D


def survival_turns(lat, z0, n_turns):
    """DA survival turn per particle: the 1-based turn of the loss, n_turns + 1
    if it survives."""
    s = track(lat, z0, n_turns, moments=False)
    return np.where(s["alive"] == 1, n_turns + 1, s["loss_turn"] + 1).astype(np.int32)
