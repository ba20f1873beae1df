"""Truncated power series algebra (TPSA) in 6 variables to order 3.

Oracle / test infrastructure only.

Used to generate element transport maps (the R, T, U coefficients of the
"transport matrices up to third order" of the paper's introduction and the
track_particles M1/M2/M3 rows of Table 1) by pushing a series "particle"
through a numerical flow, and to take exact Jacobians of the oracle's
kick-drift integrator (symplecticity pins).

Monomial order (shared layout of the map arrays): index 0 is the constant,
1..6 the variables x_j, 7..27 the products x_j x_k (j <= k, lexicographic),
28..83 the products x_j x_k x_l (j <= k <= l, lexicographic).  A map stores,
per output i, C_i, R_ij, T_i,(jk) and U_i,(jkl) with the coefficient
multiplying the monomial directly (no 1/2 factors).
"""
import itertools
import math

import numpy as np

NV = 6
MAXO = 3

MONOS = [()]
for _deg in range(1, MAXO + 1):
    MONOS += list(itertools.combinations_with_replacement(range(NV), _deg))
NMONO = len(MONOS)  # 84
INDEX = {m: i for i, m in enumerate(MONOS)}
DEG = np.array([len(m) for m in MONOS])
T_MONOS = [m for m in MONOS if len(m) == 2]   # 21
U_MONOS = [m for m in MONOS if len(m) == 3]   # 56


def _product_table(order):
    ia, ib, ic = [], [], []
    for a, ma in enumerate(MONOS):
        for b, mb in enumerate(MONOS):
            if len(ma) + len(mb) <= order:
                ia.append(a)
                ib.append(b)
                ic.append(INDEX[tuple(sorted(ma + mb))])
    return np.array(ia), np.array(ib), np.array(ic)


_TABLES = {o: _product_table(o) for o in range(0, MAXO + 1)}


class TPS:
    """A truncated power series; ``order`` is the truncation order (<= 3)."""

    __slots__ = ("c", "order")

    def __init__(self, c=None, order=MAXO):
        self.order = order
        self.c = np.zeros(NMONO) if c is None else np.asarray(c, dtype=np.float64)

    @staticmethod
    def const(v, order=MAXO):
        t = TPS(order=order)
        t.c[0] = v
        return t

    @staticmethod
    def var(j, v0=0.0, order=MAXO):
        t = TPS(order=order)
        t.c[0] = v0
        t.c[1 + j] = 1.0
        return t

    def _lift(self, o):
        return o if isinstance(o, TPS) else TPS.const(float(o), self.order)

    def __add__(self, o):
        o = self._lift(o)
        return TPS(self.c + o.c, self.order)

    __radd__ = __add__

    def __sub__(self, o):
        o = self._lift(o)
        return TPS(self.c - o.c, self.order)

    def __rsub__(self, o):
        return self._lift(o) - self

    def __neg__(self):
        return TPS(-self.c, self.order)

    def __mul__(self, o):
        if not isinstance(o, TPS):
            return TPS(self.c * float(o), self.order)
        ia, ib, ic = _TABLES[self.order]
        return TPS(np.bincount(ic, weights=self.c[ia] * o.c[ib], minlength=NMONO), self.order)

    __rmul__ = __mul__

    def __truediv__(self, o):
        if not isinstance(o, TPS):
            return TPS(self.c / float(o), self.order)
        return self * o.inv()

    def __rtruediv__(self, o):
        return self._lift(o) * self.inv()

    def _compose(self, derivs):
        """f(a0 + t) = sum_n f^(n)(a0)/n! t^n, t = self - a0 (no constant term)."""
        t = TPS(self.c.copy(), self.order)
        t.c[0] = 0.0
        out = TPS.const(derivs[0], self.order)
        p = TPS.const(1.0, self.order)
        for n in range(1, self.order + 1):
            p = p * t
            out = out + p * (derivs[n] / math.factorial(n))
        return out

    def inv(self):
        a = self.c[0]
        return self._compose([1 / a, -1 / a**2, 2 / a**3, -6 / a**4])

    def sqrt(self):
        a = self.c[0]
        r = math.sqrt(a)
        return self._compose([r, 0.5 / r, -0.25 / (a * r), 0.375 / (a * a * r)])

    def cos(self):
        a = self.c[0]
        ca, sa = math.cos(a), math.sin(a)
        return self._compose([ca, -sa, -ca, sa])

    @property
    def value(self):
        return self.c[0]


def sqrt(v):
    """sqrt for floats and TPS alike (lets one integrator serve both)."""
    return v.sqrt() if isinstance(v, TPS) else math.sqrt(v)


def cos(v):
    return v.cos() if isinstance(v, TPS) else math.cos(v)


def identity(order=MAXO, z0=None):
    z0 = [0.0] * NV if z0 is None else z0
    return [TPS.var(j, z0[j], order) for j in range(NV)]


def extract_map(z):
    """Series particle -> (C[6], R[6,6], T[6,21], U[6,56]) arrays."""
    C = np.array([t.c[0] for t in z])
    R = np.array([t.c[1:7] for t in z])
    T = np.array([t.c[7:28] for t in z])
    U = np.array([t.c[28:84] for t in z])
    return C, R, T, U
