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
TYPES = {"MAP": 1, "EDRIFT": 2, "KQUAD": 3, "KSEXT": 4, "THINSEXT": 5, "RFCA": 6, "WAKE": 7, "LSC": 8,
         "SBEND": 9}
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
                ("wake_w0", c_double), ("wake_sc", c_double), ("charge", c_double), ("wake_w0t", c_double),
                ("lsc_k", c_double), ("angle", c_double), ("lsc_rb", c_double), ("lsc_mc2", c_double),
                ("lsc_f0", c_double), ("lsc_f1", c_double),
                ("C", PD), ("R", PD), ("T", PD), ("U", PD)]


class trk_lattice_opts(ctypes.Structure):
    _fields_ = [("aperture", c_int32), ("moments", c_int32), ("a", c_double), ("b", c_double),
                ("p0c_ev", c_double)]


class trk_stats(ctypes.Structure):
    _fields_ = [("track_kernel_ms", c_double), ("track_launches", c_int64), ("launches", c_int64)]


class trk_triage_opts(ctypes.Structure):
    _fields_ = [("nx", c_int32), ("ny", c_int32), ("half_width", c_double), ("n_turns", c_int32),
                ("coarse_stride", c_int32), ("band_radius", c_int32), ("use_mlp", c_int32),
                ("epochs", c_int32), ("batch", c_int32), ("lr", ctypes.c_float), ("max_passes", c_int32),
                ("sentinel_stride", c_int32), ("expand_radius", c_int32)]


class trk_triage_stats(ctypes.Structure):
    _fields_ = [("n_cells", c_int64), ("n_coarse", c_int64), ("n_band", c_int64), ("n_audit", c_int64),
                ("n_tracked", c_int64), ("n_audit_wrong", c_int64), ("ms_coarse", c_double),
                ("ms_train", c_double), ("ms_infer", c_double), ("ms_band", c_double), ("ms_retrack", c_double),
                ("n_passes", c_int64), ("pass_cells", c_int64 * 16), ("pass_ms", c_double * 16),
                ("n_sentinel", c_int64), ("n_region", c_int64)]


class trk_schedule(ctypes.Structure):
    _fields_ = [("block", c_int32), ("per_thread", c_int32), ("chunk_turns", c_int32), ("growth", c_int32)]


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
            "trk_track_parts": [P, c_int32, P, c_int32],
            "trk_moments": [P, P, c_int32, P],
            "trk_lost": [P, P, P, P, c_int64, P],
            "trk_n_alive": [P, P],
            "trk_wake": [P, c_int32, c_double, c_double, c_double, c_double, P, P],
            "trk_bunch_enable_timing": [P, c_int32],
            "trk_batch_create": [P, P, c_int32, P],
            "trk_batch_set_schedule": [P, P],
            "trk_batch_get_schedule": [P, P],
            "trk_batch_track": [P, c_int32],
            "trk_batch_destroy": [P],
            "trk_track_batch": [P, P, c_int32, c_int32, P],
            "trk_autotune": [P, P, c_int32, c_int32, P, P],
            "trk_da_survival": [P, c_int32, P, P, P, c_int32, P, P, P],
            "trk_mlp_create": [P, P, P],
            "trk_mlp_destroy": [P],
            "trk_mlp_forward": [P, P, c_int64, P, P],
            "trk_mlp_forward_hidden": [P, P, c_int64, P, P, P],
            "trk_mlp_grad": [P, P, P, c_int32, P, P],
            "trk_mlp_adam": [P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, P],
            "trk_mlp_train": [P, P, P, c_int64, c_int32, c_int32, P, ctypes.c_float, P, P],
            "trk_mlp_get": [P, P, P, P, P],
            "trk_da_triage": [P, c_int32, P, P, P, P, P, P, P, P, P],
            "trk_bunch_stats": [P, P, c_int32],
            "trk_wake_static": [P, c_int64, c_int64, c_int32, c_double, c_double, c_double, c_double, P, P, P],
            "trk_bunch_set_turn": [P, c_int64],
            "trk_bunch_turn": [P, P],
            "trk_probe_fp64": [P, P],
            "trk_da_survival_lanes": [P, c_int32, P, P, P, c_int32, P, P],
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
    """lattice: {"elements": [...], "aperture": (kind, a, b) | None, "p0c": eV}.

    Element dicts by "type" (units as in include/trk.h):
      MAP      {"map": {"order", "C", "R", "T", "U"}}
      EDRIFT   {"L"}
      KQUAD / KSEXT {"L", "K1", "K2", "n_kicks"}
      THINSEXT {"K2L"}
      RFCA     {"volt", "phase_deg", "freq_hz"}
      WAKE     {"nbins", "W0", "sc", "charge", "W0T" (transverse, optional)}
      LSC      {"nbins", "L", "charge"} and either {"K", "passes"} (long-wavelength
               limit) or {"rb", "mc2", "f0", "f1"} (round-beam impedance)
      SBEND    {"L", "angle"}
    """
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
            d.wake_w0t = el.get("W0T", 0.0)
        elif t == "SBEND":
            d.length, d.angle = el["L"], el["angle"]
        elif t == "LSC":
            d.nbins, d.length, d.lsc_k, d.charge = el["nbins"], el["L"], el.get("K", 0.0), el["charge"]
            d.n_kicks = el.get("passes", 0)
            d.lsc_rb, d.lsc_mc2 = el.get("rb", 0.0), el.get("mc2", 0.0)
            d.lsc_f0, d.lsc_f1 = el.get("f0", 0.0), el.get("f1", 0.0)
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


def trk_track_parts(parts, lat, n_turns):
    """Track one bunch held in several Bunch parts (see include/trk.h)."""
    _check(lib().trk_track_parts(_handles(parts), len(parts), lat.handle, n_turns))


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


class Batch:
    """Owns a trk_batch handle; keeps the bunches and lattices alive."""

    def __init__(self, handle, bunches, lattices):
        self.handle = handle
        self.bunches = list(bunches)
        self.lattices = list(lattices)

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.trk_batch_destroy(self.handle)
            self.handle = None


def _handles(objs):
    arr = (c_void_p * len(objs))()
    for i, o in enumerate(objs):
        arr[i] = o.handle
    return arr


def trk_batch_create(bunches, lattices):
    if len(bunches) != len(lattices):
        raise ValueError("one lattice per bunch")
    h = c_void_p()
    _check(lib().trk_batch_create(_handles(bunches), _handles(lattices), len(bunches), ctypes.byref(h)))
    return Batch(h, bunches, lattices)


def trk_batch_set_schedule(B, block=0, per_thread=0, chunk_turns=0, growth=0):
    s = trk_schedule(block, per_thread, chunk_turns, growth)
    _check(lib().trk_batch_set_schedule(B.handle, ctypes.byref(s)))


def trk_batch_get_schedule(B):
    s = trk_schedule()
    _check(lib().trk_batch_get_schedule(B.handle, ctypes.byref(s)))
    return {"block": s.block, "per_thread": s.per_thread, "chunk_turns": s.chunk_turns, "growth": s.growth}


def trk_batch_track(B, n_turns):
    _check(lib().trk_batch_track(B.handle, n_turns))


def trk_autotune(bunches, lattices, probe_turns):
    """Fastest batched schedule for these pairs: (schedule dict, probe ms)."""
    s = trk_schedule()
    ms = c_double()
    _check(lib().trk_autotune(_handles(bunches), _handles(lattices), len(bunches), probe_turns, ctypes.byref(s),
                              ctypes.byref(ms)))
    return {"block": s.block, "per_thread": s.per_thread, "chunk_turns": s.chunk_turns, "growth": s.growth}, ms.value


def trk_track_batch(bunches, lattices, n_turns, schedule=None):
    s = None
    if schedule is not None:
        s = ctypes.byref(trk_schedule(schedule.get("block", 0), schedule.get("per_thread", 0),
                                      schedule.get("chunk_turns", 0), schedule.get("growth", 0)))
    _check(lib().trk_track_batch(_handles(bunches), _handles(lattices), len(bunches), n_turns, s))


def trk_da_survival(lattices, x0, y0, offsets, n_turns, schedule=None, stream=None):
    """x0, y0: float64 CUDA tensors of all points; offsets: n_var + 1 host ints.
    Returns an int32 CUDA tensor of survival turns (1-based loss turn, or
    n_turns + 1)."""
    import torch
    offs = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    surv = torch.empty(int(offs[-1]), dtype=torch.int32, device=x0.device)
    if stream is None:
        stream = torch.cuda.current_stream(x0.device)
    s = None
    if schedule is not None:
        s = ctypes.byref(trk_schedule(schedule.get("block", 0), schedule.get("per_thread", 0),
                                      schedule.get("chunk_turns", 0), schedule.get("growth", 0)))
    _check(lib().trk_da_survival(_handles(lattices), len(lattices), offs.ctypes.data_as(c_void_p), _dptr(x0),
                                 _dptr(y0), n_turns, s, _dptr(surv), c_void_p(stream.cuda_stream)))
    return surv


def trk_da_survival_lanes(lattices, x0, y0, offsets, n_turns, stream=None):
    """As trk_da_survival, 4 or 8 lanes per particle (few points; MAP, EDRIFT and
    THINSEXT lattices)."""
    import torch
    offs = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    surv = torch.empty(int(offs[-1]), dtype=torch.int32, device=x0.device)
    if stream is None:
        stream = torch.cuda.current_stream(x0.device)
    _check(lib().trk_da_survival_lanes(_handles(lattices), len(lattices), offs.ctypes.data_as(c_void_p), _dptr(x0),
                                       _dptr(y0), n_turns, _dptr(surv), c_void_p(stream.cuda_stream)))
    return surv


MLP_SHAPES = [(256, 8), (256, 256), (256, 256), (256, 256), (1, 256)]


class MLP:
    """Owns a trk_mlp handle."""

    def __init__(self, handle):
        self.handle = handle

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.trk_mlp_destroy(self.handle)
            self.handle = None


def _fptrs(arrays):
    arr = (c_void_p * len(arrays))()
    for i, a in enumerate(arrays):
        arr[i] = None if a is None else a.ctypes.data
    return arr


def trk_mlp_create(params):
    """params: [(W (out, in), b (out,))] x 5 host arrays (converted to FP32)."""
    Ws = [np.ascontiguousarray(W, dtype=np.float32) for W, _ in params]
    bs = [np.ascontiguousarray(b, dtype=np.float32) for _, b in params]
    for (o, i), W, b in zip(MLP_SHAPES, Ws, bs):
        if W.shape != (o, i) or b.shape != (o,):
            raise ValueError("MLP parameter shapes must be %s" % MLP_SHAPES)
    h = c_void_p()
    _check(lib().trk_mlp_create(_fptrs(Ws), _fptrs(bs), ctypes.byref(h)))
    return MLP(h)


def _stream(t, stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream(t.device)
    return c_void_p(s.cuda_stream)


def trk_mlp_forward(net, X, stream=None):
    """X: float32 CUDA tensor (M, 8) -> logits float32 CUDA tensor (M,)."""
    import torch
    out = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
    _check(lib().trk_mlp_forward(net.handle, _dptr(X), X.shape[0], _dptr(out), _stream(X, stream)))
    return out


def trk_mlp_forward_hidden(net, X, stream=None):
    """X: float32 CUDA tensor (M, 8) -> (logits (M,) float32, hidden (4, M, 256)
    int16 CUDA tensor holding each hidden layer's BF16 outputs bit for bit)."""
    import torch
    M = X.shape[0]
    out = torch.empty(M, dtype=torch.float32, device=X.device)
    hid = torch.empty((4, M, 256), dtype=torch.int16, device=X.device)
    _check(lib().trk_mlp_forward_hidden(net.handle, _dptr(X), M, _dptr(out), _dptr(hid), _stream(X, stream)))
    return out, hid


def trk_mlp_grad(net, X, y, stream=None):
    import torch
    loss = torch.zeros(1, dtype=torch.float32, device=X.device)
    _check(lib().trk_mlp_grad(net.handle, _dptr(X), _dptr(y), X.shape[0], _dptr(loss), _stream(X, stream)))
    return loss


def trk_mlp_adam(net, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    _check(lib().trk_mlp_adam(net.handle, lr, beta1, beta2, eps, c_void_p(s.cuda_stream)))


def trk_mlp_train(net, X, y, batch, epochs, perm=None, lr=1e-3, stream=None):
    """Returns the per-step loss history (float32 CUDA tensor)."""
    import torch
    n = X.shape[0]
    steps = epochs * ((n + batch - 1) // batch)
    hist = torch.zeros(steps, dtype=torch.float32, device=X.device)
    _check(lib().trk_mlp_train(net.handle, _dptr(X), _dptr(y), n, batch, epochs, _dptr(perm), lr, _dptr(hist),
                               _stream(X, stream)))
    return hist


def trk_mlp_get(net):
    """Host copies: (params [(W, b)], grads [(gW, gb)]) as float32 arrays."""
    Ws = [np.zeros(s, np.float32) for s in MLP_SHAPES]
    bs = [np.zeros(s[0], np.float32) for s in MLP_SHAPES]
    gWs = [np.zeros(s, np.float32) for s in MLP_SHAPES]
    gbs = [np.zeros(s[0], np.float32) for s in MLP_SHAPES]
    _check(lib().trk_mlp_get(net.handle, _fptrs(Ws), _fptrs(bs), _fptrs(gWs), _fptrs(gbs)))
    return list(zip(Ws, bs)), list(zip(gWs, gbs))


def trk_da_triage(lattices, params, opts, net=None, audit=None, perm=None, stream=None):
    """params: float32 CUDA tensor (n_var, 6); audit: uint8 CUDA tensor
    (n_var, ny, nx) or None; opts: dict of trk_triage_opts fields.
    Returns (mask uint8, survival int32 CUDA tensors (n_var, ny, nx), stats dict)."""
    import torch
    o = trk_triage_opts()
    for k, v in opts.items():
        setattr(o, k, v)
    nv = len(lattices)
    mask = torch.zeros((nv, o.ny, o.nx), dtype=torch.uint8, device=params.device)
    surv = torch.zeros((nv, o.ny, o.nx), dtype=torch.int32, device=params.device)
    st = trk_triage_stats()
    _check(lib().trk_da_triage(_handles(lattices), nv, _dptr(params), _dptr(audit),
                               net.handle if net is not None else None, _dptr(perm), ctypes.byref(o),
                               _dptr(mask), _dptr(surv), ctypes.byref(st), _stream(params, stream)))
    stats = {f: getattr(st, f) for f, _ in trk_triage_stats._fields_}
    for f in ("pass_cells", "pass_ms"):
        stats[f] = list(stats[f])[:max(1, min(st.n_passes, 16))]
    return mask, surv, stats


def trk_bunch_enable_timing(b, on=True):
    _check(lib().trk_bunch_enable_timing(b.handle, 1 if on else 0))


def trk_bunch_stats(b, reset=False):
    s = trk_stats()
    _check(lib().trk_bunch_stats(b.handle, ctypes.byref(s), 1 if reset else 0))
    return {"track_kernel_ms": s.track_kernel_ms, "track_launches": s.track_launches, "launches": s.launches}


def trk_wake_static(coords, n, nbins, w0, sc, charge, p0c, hist=None, volt=None, stream=None):
    """Allocation-free standalone wake on the first n columns of a contiguous
    (6, pitch) float64 CUDA tensor (every one of the n particles counts as
    alive).  hist (int32) and volt (float64), if given, are CUDA tensors of at
    least nbins elements on the same device; the library itself checks nbins
    against its fixed maximum.  The shapes, types and devices are checked here
    because the C call receives bare device pointers and cannot."""
    import torch
    if not (isinstance(coords, torch.Tensor) and coords.is_cuda and coords.dtype == torch.float64
            and coords.dim() == 2 and coords.shape[0] == 6 and coords.is_contiguous()):
        raise ValueError("trk_wake_static: coords must be a contiguous (6, pitch) float64 CUDA tensor")
    n = int(n)
    if n < 0 or n > coords.shape[1]:
        raise ValueError("trk_wake_static: n must be in 0..pitch")
    for name, t, dt in (("hist", hist, torch.int32), ("volt", volt, torch.float64)):
        if t is None:
            continue
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dt and t.is_contiguous()):
            raise ValueError("trk_wake_static: %s must be a contiguous %s CUDA tensor" % (name, dt))
        if t.device != coords.device:
            raise ValueError("trk_wake_static: %s is on %s, coords on %s" % (name, t.device, coords.device))
        if t.numel() < int(nbins):
            raise ValueError("trk_wake_static: %s holds %d elements, nbins is %d" % (name, t.numel(), nbins))
    with torch.cuda.device(coords.device):
        if stream is None:
            stream = torch.cuda.current_stream(coords.device)
        _check(lib().trk_wake_static(_dptr(coords), coords.shape[1], n, nbins, w0, sc, charge, p0c,
                                     _dptr(hist), _dptr(volt), c_void_p(stream.cuda_stream)))


def trk_probe_fp64(stream=None):
    """Measured FP64 rates of the current device: (DFMA, DMUL, DADD) thread
    operations per second."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    out = (c_double * 3)()
    _check(lib().trk_probe_fp64(out, c_void_p(stream.cuda_stream)))
    return tuple(out)


def trk_bunch_set_turn(b, turn):
    _check(lib().trk_bunch_set_turn(b.handle, int(turn)))


def trk_bunch_turn(b):
    t = c_int64()
    _check(lib().trk_bunch_turn(b.handle, ctypes.byref(t)))
    return t.value


def download(b):
    """Host copy (n, 6) of the bunch coordinates and (n,) ids, in slot order."""
    import torch
    torch.cuda.current_stream(b.coords.device).synchronize()
    b.stream.synchronize()
    z = b.coords[:, :b.n].T.contiguous().cpu().numpy()
    return z, b.ids[:b.n].cpu().numpy()
