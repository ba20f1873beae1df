"""Thin Python binding of the C ABI declared in include/trk.h.

Argument marshalling only: every step of the tracking path runs in the CUDA
kernels of libtrk.so.  Device arrays are PyTorch CUDA tensors (PyTorch supplies
device memory and streams); the library borrows them.  There is no CPU
fallback: if libtrk.so cannot be built or loaded, every call raises.
"""
import ctypes
import os

import numpy as np

from . import build as _build

c_int32, c_int64, c_double, c_void_p = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
PD = ctypes.POINTER(c_double)

TRK_OK = 0
TYPES = {"MAP": 1, "EDRIFT": 2, "KQUAD": 3, "KSEXT": 4, "THINSEXT": 5, "RFCA": 6, "WAKE": 7}
APERTURES = {None: 0, "rect": 1, "ellipse": 2}
STATUS = {0: "TRK_OK", 1: "TRK_EINVAL", 2: "TRK_ENOMEM", 3: "TRK_ECUDA", 4: "TRK_EKERNEL",
          5: "TRK_ETIMEOUT", 6: "TRK_EUNSUPPORTED"}


class TrkError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class trk_element_desc(ctypes.Structure):
    _fields_ = [("type", c_int32), ("order", c_int32), ("n_kicks", c_int32), ("nbins", c_int32),
                ("length", c_double), ("k1", c_double), ("k2", c_double), ("k2l", c_double),
                ("volt", c_double), ("phase_deg", c_double), ("freq_hz", c_double),
                ("wake_w0", c_double), ("wake_sc", c_double), ("charge", c_double),
                ("C", PD), ("R", PD), ("T", PD), ("U", PD)]


class trk_lattice_opts(ctypes.Structure):
    _fields_ = [("aperture", c_int32), ("moments", c_int32), ("a", c_double), ("b", c_double),
                ("p0c_ev", c_double)]


class trk_stats(ctypes.Structure):
    _fields_ = [("track_kernel_ms", c_double), ("track_launches", c_int64), ("launches", c_int64)]


class trk_schedule(ctypes.Structure):
    _fields_ = [("block", c_int32), ("per_thread", c_int32), ("chunk_turns", c_int32), ("pad", c_int32)]


_lib = None


def lib_path():
    return _build.LIB


def lib():
    """Load (building first if needed) libtrk.so; raises if that is impossible."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = c_void_p
        sig = {
            "trk_create_lattice": [P, c_int32, P, P],
            "trk_destroy_lattice": [P],
            "trk_bunch_wrap": [P, c_int64, P, c_int64, P, P],
            "trk_bunch_free": [P],
            "trk_bunch_set_p0c": [P, c_double],
            "trk_bunch_p0c": [P, P],
            "trk_bunch_set_schedule": [P, P],
            "trk_track": [P, P, c_int32],
            "trk_moments": [P, P, c_int32, P],
            "trk_lost": [P, P, P, P, c_int64, P],
            "trk_n_alive": [P, P],
            "trk_wake": [P, c_int32, c_double, c_double, c_double, c_double, P, P],
            "trk_bunch_enable_timing": [P, c_int32],
            "trk_bunch_stats": [P, P, c_int32],
            "trk_wake_static": [P, c_int64, c_int64, c_int32, c_double, c_double, c_double, c_double, P, P, P],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = c_int32
        L.trk_last_error.argtypes = []
        L.trk_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _check(status):
    if status != TRK_OK:
        raise TrkError(status, lib().trk_last_error().decode())


def _dptr(t):
    """Device pointer of a CUDA tensor (no copy)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    return c_void_p(t.data_ptr())


class Lattice:
    """Owns a trk_lattice handle."""

    def __init__(self, handle, n_elem, desc):
        self.handle = handle
        self.n_elem = n_elem
        self.desc = desc

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.trk_destroy_lattice(self.handle)
            self.handle = None


def trk_create_lattice(lattice, moments=True):
    """lattice: {"elements": [...], "aperture": (kind, a, b) | None, "p0c": eV}."""
    els = lattice["elements"]
    descs = (trk_element_desc * max(len(els), 1))()
    keep = []
    for i, el in enumerate(els):
        d = descs[i]
        t = el["type"]
        d.type = TYPES[t]
        if t == "MAP":
            m = el["map"]
            d.order = int(m["order"])
            for f in ("C", "R", "T", "U"):
                a = np.ascontiguousarray(np.asarray(m[f], dtype=np.float64).ravel())
                keep.append(a)
                setattr(d, f, a.ctypes.data_as(PD))
        elif t == "EDRIFT":
            d.length = el["L"]
        elif t in ("KQUAD", "KSEXT"):
            d.length, d.k1, d.k2, d.n_kicks = el["L"], el.get("K1", 0.0), el.get("K2", 0.0), el["n_kicks"]
        elif t == "THINSEXT":
            d.k2l = el["K2L"]
        elif t == "RFCA":
            d.volt, d.phase_deg, d.freq_hz = el["volt"], el["phase_deg"], el["freq_hz"]
        elif t == "WAKE":
            d.nbins, d.wake_w0, d.wake_sc, d.charge = el["nbins"], el["W0"], el["sc"], el["charge"]
        else:
            raise ValueError(t)
    o = trk_lattice_opts()
    ap = lattice.get("aperture")
    o.aperture = APERTURES[ap[0] if ap else None]
    if ap:
        o.a, o.b = ap[1], ap[2]
    o.moments = 1 if moments else 0
    o.p0c_ev = lattice["p0c"]
    h = c_void_p()
    _check(lib().trk_create_lattice(descs, len(els), ctypes.byref(o), ctypes.byref(h)))
    return Lattice(h, len(els), lattice)


class Bunch:
    """Owns a trk_bunch handle; keeps the borrowed tensors alive."""

    def __init__(self, handle, coords, ids, n, stream):
        self.handle = handle
        self.coords = coords
        self.ids = ids
        self.n = n
        self.stream = stream

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.trk_bunch_free(self.handle)
            self.handle = None


def upload(z, device="cuda", pitch=None):
    """(n, 6) host array -> (coords (6, pitch) float64, ids (n,) int32) CUDA tensors."""
    import torch
    z = np.asarray(z, dtype=np.float64)
    n = z.shape[0]
    pitch = n if pitch is None else pitch
    coords = torch.zeros((6, max(pitch, 1)), dtype=torch.float64, device=device)
    if n:
        coords[:, :n] = torch.from_numpy(np.ascontiguousarray(z.T)).to(device)
    ids = torch.arange(n, dtype=torch.int32, device=device)
    return coords, ids


def trk_bunch_wrap(coords, ids, n=None, stream=None):
    """coords: (6, pitch) float64 CUDA tensor; ids: (>= n,) int32 CUDA tensor."""
    import torch
    if coords.dtype != torch.float64 or coords.dim() != 2 or coords.shape[0] != 6 or not coords.is_contiguous():
        raise ValueError("coords must be a contiguous (6, pitch) float64 tensor")
    if ids.dtype != torch.int32:
        raise ValueError("ids must be int32")
    n = ids.shape[0] if n is None else n
    if stream is None:
        stream = torch.cuda.current_stream(coords.device)
    h = c_void_p()
    _check(lib().trk_bunch_wrap(_dptr(coords), coords.shape[1], _dptr(ids), n,
                                c_void_p(stream.cuda_stream), ctypes.byref(h)))
    return Bunch(h, coords, ids, n, stream)


def trk_bunch_set_schedule(b, block=0, per_thread=0, chunk_turns=0):
    s = trk_schedule(block, per_thread, chunk_turns, 0)
    _check(lib().trk_bunch_set_schedule(b.handle, ctypes.byref(s)))


def trk_bunch_set_p0c(b, p0c):
    _check(lib().trk_bunch_set_p0c(b.handle, p0c))


def trk_bunch_p0c(b):
    v = c_double()
    _check(lib().trk_bunch_p0c(b.handle, ctypes.byref(v)))
    return v.value


def trk_track(b, lat, n_turns):
    _check(lib().trk_track(b.handle, lat.handle, n_turns))


def trk_moments(b, cap_turns=1 << 30):
    nt = c_int32()
    _check(lib().trk_moments(b.handle, None, 0, ctypes.byref(nt)))
    out = np.zeros((max(nt.value, 0), 28))
    if nt.value:
        _check(lib().trk_moments(b.handle, out.ctypes.data_as(c_void_p), min(cap_turns, nt.value), ctypes.byref(nt)))
    return out


def trk_n_alive(b):
    v = c_int64()
    _check(lib().trk_n_alive(b.handle, ctypes.byref(v)))
    return v.value


def trk_lost(b):
    """(ids, turn, elem) int32 arrays of the lost particles, in slot order."""
    m = c_int64()
    _check(lib().trk_lost(b.handle, None, None, None, 0, ctypes.byref(m)))
    k = m.value
    ids = np.zeros(k, np.int32)
    turn = np.zeros(k, np.int32)
    elem = np.zeros(k, np.int32)
    if k:
        _check(lib().trk_lost(b.handle, ids.ctypes.data_as(c_void_p), turn.ctypes.data_as(c_void_p),
                              elem.ctypes.data_as(c_void_p), k, ctypes.byref(m)))
    return ids, turn, elem


def trk_wake(b, nbins, w0, sc, charge, p0c, hist=None, volt=None):
    _check(lib().trk_wake(b.handle, nbins, w0, sc, charge, p0c, _dptr(hist), _dptr(volt)))


def trk_bunch_enable_timing(b, on=True):
    _check(lib().trk_bunch_enable_timing(b.handle, 1 if on else 0))


def trk_bunch_stats(b, reset=False):
    s = trk_stats()
    _check(lib().trk_bunch_stats(b.handle, ctypes.byref(s), 1 if reset else 0))
    return {"track_kernel_ms": s.track_kernel_ms, "track_launches": s.track_launches, "launches": s.launches}


def trk_wake_static(coords, n, nbins, w0, sc, charge, p0c, hist=None, volt=None, stream=None):
    """Allocation-free standalone wake on a (6, pitch) float64 CUDA tensor."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream(coords.device)
    _check(lib().trk_wake_static(_dptr(coords), coords.shape[1], n, nbins, w0, sc, charge, p0c,
                                 _dptr(hist), _dptr(volt), c_void_p(stream.cuda_stream)))


def download(b):
    """Host copy (n, 6) of the bunch coordinates and (n,) ids, in slot order."""
    import torch
    torch.cuda.current_stream(b.coords.device).synchronize()
    b.stream.synchronize()
    z = b.coords[:, :b.n].T.contiguous().cpu().numpy()
    return z, b.ids[:b.n].cpu().numpy()
