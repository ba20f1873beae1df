"""Triage oracle: the band-refinement steps of the surrogate-triaged
dynamic-aperture scan, written out plainly in numpy, cell by cell where it
matters.  Test infrastructure only.

The paper has no learned or triaged part; this is the scan of the hot-path
scope (dynamic aperture over a grid of initial amplitudes, a cheap prediction,
exact FP64 re-tracking of a band around the predicted boundary).  The exact
labels are an input (survival turns of every cell, from the oracle tracker);
the oracle returns which cells the procedure tracks and the merged result, so
the GPU pipeline can be compared with it exactly when the prediction is the
deterministic nearest-coarse-cell rule.

Steps, per variant (grid ny x nx, cells indexed [iy, ix]):
  1. coarse cells: ix, iy in {off, off + s, ...} with off = s // 2 (s = coarse
     stride), and sentinel cells (positions of sentinel_axis on both axes);
     their exact labels are known;
  2. prediction of every cell (use_mlp = 0): the label of the nearest known
     cell -- the nearest coarse cell, index j = (i - off + s // 2) // s (0
     below off) clamped to the last coarse index, or, when sentinels are on
     and strictly closer (squared index distance), the nearest sentinel cell
     (per axis the sentinel position closest to i, the lower one on a tie);
  3. the merged mask starts as the prediction with the known labels applied;
  4. pass 0: track every unknown cell that is within Chebyshev distance r of a
     boundary cell of the merged mask, or an audit cell; pass p > 0: every
     unknown cell within r of a boundary cell or within R of a cell whose label
     the previous merge flipped; merging sets the exact label; passes stop when
     one finds nothing to track (or after max_passes);
  5. survival: exact where known, n_turns + 1 / 0 from the merged mask
     elsewhere.
A boundary cell is a cell whose 8-neighbourhood within the grid holds both
classes.
"""
import numpy as np


def boundary(mask):
    """Cells whose 8-neighbourhood (within the grid) holds both classes."""
    ny, nx = mask.shape
    out = np.zeros_like(mask, dtype=bool)
    for iy in range(ny):
        for ix in range(nx):
            blk = mask[max(iy - 1, 0):iy + 2, max(ix - 1, 0):ix + 2]
            out[iy, ix] = blk.any() and not blk.all()
    return out


def dilate(b, r):
    """Cells within Chebyshev distance r (inside the grid) of a set cell."""
    ny, nx = b.shape
    out = np.zeros_like(b, dtype=bool)
    if r < 0:
        return out
    for iy, ix in zip(*np.nonzero(b)):
        out[max(iy - r, 0):iy + r + 1, max(ix - r, 0):ix + r + 1] = True
    return out


def coarse_index(n, stride):
    off = stride // 2
    return np.arange(off, n, stride)


def sentinel_axis(n, stride):
    """Positions off, off + stride, ... up to n - 1 - off, plus n - 1 - off."""
    off = stride // 2
    last = n - 1 - off
    pos = set(range(off, last + 1, stride))
    pos.add(last)
    return np.array(sorted(p for p in pos if 0 <= p < n), dtype=np.int64)


def nearest_coarse_index(n, stride):
    """Per axis: index of the nearest coarse position of every cell."""
    off = stride // 2
    c = len(coarse_index(n, stride))
    return np.array([0 if i < off else min((i - off + stride // 2) // stride, c - 1) for i in range(n)])


def nearest_sentinel_position(n, stride):
    """Per axis: the sentinel position closest to every cell (lower on a tie)."""
    pos = sentinel_axis(n, stride)
    out = np.zeros(n, dtype=np.int64)
    for i in range(n):
        d = np.abs(pos - i)
        out[i] = pos[np.argmin(d)]   # argmin takes the first (lower) on a tie
    return out


def nearest_coarse_prediction(coarse_labels, n, stride):
    """(ny, nx) prediction from the (cy, cx) coarse labels (square grid n)."""
    j = nearest_coarse_index(n, stride)
    return coarse_labels[np.ix_(j, j)]


def nearest_known_prediction(exact, n, stride, sentinel):
    """Label of the nearest known cell: the nearest coarse cell, or the nearest
    sentinel cell where it is strictly closer (squared index distance)."""
    ci = coarse_index(n, stride)
    jc = nearest_coarse_index(n, stride)
    pc = ci[jc]                                   # nearest coarse position per axis
    ps = nearest_sentinel_position(n, sentinel)   # nearest sentinel position per axis
    pred = np.zeros((n, n), bool)
    for iy in range(n):
        for ix in range(n):
            dc = (pc[iy] - iy) ** 2 + (pc[ix] - ix) ** 2
            ds = (ps[iy] - iy) ** 2 + (ps[ix] - ix) ** 2
            pred[iy, ix] = exact[ps[iy], ps[ix]] if ds < dc else exact[pc[iy], pc[ix]]
    return pred


def triage_variant(exact_surv, n_turns, stride, r, prediction=None, audit=None, sentinel=0, expand=0,
                   max_passes=64):
    """One variant.  exact_surv: (n, n) int survival turns (n_turns + 1 =
    survives).  Returns (mask bool, survival int, tracked bool (cells tracked
    in the band passes; coarse and sentinel cells are tracked before them),
    passes)."""
    n = exact_surv.shape[0]
    exact = exact_surv == n_turns + 1
    ci = coarse_index(n, stride)
    known = np.zeros((n, n), bool)
    known[np.ix_(ci, ci)] = True
    if sentinel > 0:
        sa = sentinel_axis(n, sentinel)
        known[np.ix_(sa, sa)] = True
    if prediction is None:
        if sentinel > 0:
            prediction = nearest_known_prediction(exact, n, stride, sentinel)
        else:
            prediction = nearest_coarse_prediction(exact[np.ix_(ci, ci)], n, stride)
    mask = np.array(prediction, dtype=bool)
    mask[known] = exact[known]
    flip = np.zeros((n, n), bool)
    tracked = np.zeros((n, n), bool)
    passes = 0
    for p in range(max_passes):
        near = dilate(boundary(mask), r)
        if p == 0:
            want = near
            if audit is not None:
                want = want | np.asarray(audit, bool)
        else:
            want = near | (dilate(flip, expand) if expand > 0 else False)
        todo = want & ~known
        if not todo.any():
            break
        passes = p + 1
        flip = todo & (exact != mask)
        mask[todo] = exact[todo]
        known |= todo
        tracked |= todo
    surv = np.where(known, exact_surv, np.where(mask, n_turns + 1, 0))
    return mask, surv, tracked, passes
