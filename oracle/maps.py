"""Transport-map generation by TPSA through numerical flows.

Oracle / test infrastructure only.

The paper's QUAD and DRIFT elements are "implemented as a transport matrix, up
to 3rd and 2nd order" (Sec. 3, Table 1 track_particles M1/M2/M3).  Here a map is
the order-n Taylor expansion, about the reference orbit, of the element's flow
in slope coordinates.  For a thick quadrupole the flow is integrated with a
6th-order Yoshida scheme and many steps (truncation far below FP64 rounding);
for a drift the exact closed form is expanded.
"""
import numpy as np

from . import flows
from .tpsa import identity, extract_map


def element_map(flow, order, z0=None):
    """Map of `flow` (a function of a 6-list) expanded to `order` about z0."""
    z = flow(identity(order, z0))
    C, R, T, U = extract_map(z)
    return {"order": order, "C": C, "R": R, "T": T, "U": U}


def quad_map(length, k1, order, n_steps=64):
    return element_map(
        lambda z: flows.thick_multipole(z, length, k1, 0.0, n_steps, flows.YOSHIDA6), order)


def drift_map(length, order):
    return element_map(lambda z: flows.exact_drift(z, length), order)


def thin_quad_map(k1l):
    return element_map(lambda z: flows.thin_quad(z, k1l), 1)


def jacobian(flow, z0=None):
    """Exact Jacobian (order-1 series) of `flow` at z0."""
    return element_map(flow, 1, z0)["R"]


def compose_linear(Rs):
    """Product R_n ... R_2 R_1 of element matrices given in beam order."""
    M = np.eye(6)
    for R in Rs:
        M = R @ M
    return M


def twiss_from_cell(M):
    """Periodic (beta, alpha) per transverse plane from the one-cell matrix."""
    out = []
    for p in (0, 2):
        m = M[p:p + 2, p:p + 2]
        cmu = 0.5 * (m[0, 0] + m[1, 1])
        if abs(cmu) >= 1.0:
            raise ValueError("cell is not stable in plane %d" % (p // 2))
        smu = np.sign(m[0, 1]) * np.sqrt(1.0 - cmu * cmu)
        out.append((m[0, 1] / smu, (m[0, 0] - m[1, 1]) / (2.0 * smu)))
    return out
