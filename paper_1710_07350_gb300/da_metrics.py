"""Host-side evaluation of dynamic-aperture masks (numpy).

A boundary cell of a survival mask is a cell whose 8-neighbourhood (within the
grid) holds both classes.  A triaged mask agrees with the exhaustive one "to one
grid cell" when every cell where they differ lies within Chebyshev distance 1
of a boundary cell of the exhaustive mask.
"""
import numpy as np


def _neighbour_counts(mask):
    m = np.asarray(mask, dtype=np.int32)
    ny, nx = m.shape
    pad = np.pad(m, 1)
    ones = np.zeros((ny, nx), np.int32)
    cnt = np.zeros((ny, nx), np.int32)
    valid = np.pad(np.ones_like(m), 1)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            ones += pad[1 + dy:1 + dy + ny, 1 + dx:1 + dx + nx]
            cnt += valid[1 + dy:1 + dy + ny, 1 + dx:1 + dx + nx]
    return ones, cnt


def boundary(mask):
    ones, cnt = _neighbour_counts(mask)
    return (ones > 0) & (ones < cnt)


def dilate(b, r):
    b = np.asarray(b, bool)
    ny, nx = b.shape
    pad = np.pad(b, r)
    out = np.zeros_like(b)
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            out |= pad[r + dy:r + dy + ny, r + dx:r + dx + nx]
    return out


def boundary_difference(tri, exh, r_max=8):
    """(ok, n_diff, max Chebyshev distance in cells from a differing cell to the
    nearest exhaustive boundary cell, capped at r_max + 1) for one variant's masks."""
    tri = np.asarray(tri, bool)
    exh = np.asarray(exh, bool)
    diff = tri != exh
    if not diff.any():
        return True, 0, 0
    b = boundary(exh)
    r = 0
    d = b.copy()
    while np.any(diff & ~d) and r <= r_max:
        r += 1
        d = dilate(b, r)
    return r <= 1, int(diff.sum()), r
