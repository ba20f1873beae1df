"""Pins of the triage oracle (CPU): its helpers against brute-force
definitions, and the band procedure against the one-cell boundary criterion it
is built to meet, on label fields with islands the coarse grid cannot see."""
import numpy as np
import pytest

from oracle import triage as tri
from paper_1710_07350_gb300 import da_metrics as dm


def brute_boundary(mask):
    ny, nx = mask.shape
    out = np.zeros_like(mask, dtype=bool)
    for iy in range(ny):
        for ix in range(nx):
            vals = {bool(mask[jy, jx]) for jy in range(ny) for jx in range(nx)
                    if abs(jy - iy) <= 1 and abs(jx - ix) <= 1}
            out[iy, ix] = len(vals) == 2
    return out


def test_boundary_and_dilation_match_brute_force():
    g = np.random.Generator(np.random.Philox(key=21))
    m = g.uniform(size=(13, 11)) < 0.3
    assert np.array_equal(tri.boundary(m), brute_boundary(m))
    assert np.array_equal(tri.boundary(m), dm.boundary(m))
    b = g.uniform(size=(13, 11)) < 0.05
    for r in (0, 1, 3):
        want = np.zeros_like(b)
        pts = np.argwhere(b)
        for iy in range(13):
            for ix in range(11):
                want[iy, ix] = any(max(abs(iy - py), abs(ix - px)) <= r for py, px in pts)
        assert np.array_equal(tri.dilate(b, r), want)


@pytest.mark.parametrize("n,stride", [(64, 5), (61, 5), (512, 5), (40, 3), (7, 5)])
def test_sentinel_axis_covers_every_window(n, stride):
    pos = tri.sentinel_axis(n, stride)
    off = stride // 2
    assert pos[0] == off and pos[-1] == n - 1 - off
    assert np.all(np.diff(pos) >= 1) and np.all(np.diff(pos) <= stride)
    # every window of `stride` consecutive cells, and every edge-clipped window
    # of off + 1 cells, holds a sentinel
    s = set(pos.tolist())
    for a in range(0, n - stride + 1):
        assert any(i in s for i in range(a, a + stride))
    assert any(i in s for i in range(0, off + 1)) and any(i in s for i in range(n - 1 - off, n))


def label_field(g, n, n_turns):
    """Survival turns: a stable ellipse, islands of every size from 1 to 9 cells
    on both sides of its edge, and a ragged fringe."""
    yy, xx = np.mgrid[0:n, 0:n]
    c = (n - 1) / 2.0
    r2 = ((xx - c) / (0.33 * n)) ** 2 + ((yy - c) / (0.27 * n)) ** 2
    surv = r2 < 1.0
    fringe = (r2 > 0.85) & (r2 < 1.15)
    surv ^= fringe & (g.uniform(size=(n, n)) < 0.3)
    for _ in range(16):
        s = int(g.integers(1, 10))
        iy, ix = (int(v) for v in g.integers(0, n - s, size=2))
        surv[iy:iy + s, ix:ix + s] = not surv[iy + s // 2, ix + s // 2]
    return np.where(surv, n_turns + 1, 1 + g.integers(0, n_turns, size=(n, n)))


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("predict", ["nearest", "all_survive", "noise"])
def test_sentinels_make_the_one_cell_criterion_hold(seed, predict):
    g = np.random.Generator(np.random.Philox(key=100 + seed))
    n, turns = 80, 50
    surv = label_field(g, n, turns)
    exact = surv == turns + 1
    pred = None
    if predict == "all_survive":
        pred = np.ones((n, n), bool)
    elif predict == "noise":
        pred = exact ^ (g.uniform(size=(n, n)) < 0.01)
    mask, out, tracked, passes = tri.triage_variant(surv, turns, stride=8, r=2, prediction=pred,
                                                    sentinel=5, expand=4)
    ok, nd, dist = dm.boundary_difference(mask, exact)
    assert ok, (nd, dist)
    assert passes >= 1
    # every tracked or coarse cell carries its exact survival turn; the rest the merged label
    ci = tri.coarse_index(n, 8)
    sa = tri.sentinel_axis(n, 5)
    pre = np.zeros((n, n), bool)
    pre[np.ix_(ci, ci)] = True
    pre[np.ix_(sa, sa)] = True
    known = tracked | pre
    assert np.array_equal(out[known], surv[known])
    assert np.array_equal(out[~known], np.where(mask[~known], turns + 1, 0))
    assert np.array_equal(mask[known], exact[known])


def test_label_fields_defeat_the_band_without_sentinels():
    """The fields above are hard enough: without sentinels the band misses
    islands in some of them."""
    fails = 0
    for seed in range(6):
        g = np.random.Generator(np.random.Philox(key=100 + seed))
        surv = label_field(g, 80, 50)
        mask, _, _, _ = tri.triage_variant(surv, 50, stride=8, r=2, expand=4)
        fails += not dm.boundary_difference(mask, surv == 51)[0]
    assert fails >= 2


def test_island_between_coarse_cells_is_missed_without_sentinels():
    """A 7 x 7 lost island inside the stable region, between stride-8 coarse
    cells: the band alone never reaches it, and its centre is three cells from
    the exhaustive boundary; one sentinel inside it is enough."""
    n, turns = 64, 50
    surv = np.full((n, n), turns + 1)
    surv[:, :4] = 3                      # a lost strip on the left edge keeps a boundary elsewhere
    surv[21:28, 37:44] = 7               # island: coarse cells sit at 4, 12, 20, 28, 36, 44
    exact = surv == turns + 1
    mask, _, tracked, _ = tri.triage_variant(surv, turns, stride=8, r=2)
    ok, nd, dist = dm.boundary_difference(mask, exact)
    assert not ok and dist == 3 and not tracked[21:28, 37:44].any()
    mask, _, tracked, _ = tri.triage_variant(surv, turns, stride=8, r=2, sentinel=5)
    assert dm.boundary_difference(mask, exact)[0]
    assert np.array_equal(mask, exact)


def test_nearest_known_prediction_brute_force():
    """Nearest known cell by brute force over coarse and sentinel cells:
    squared index distance, coarse cells win ties, and among sentinels the
    lower position per axis."""
    g = np.random.Generator(np.random.Philox(key=22))
    n, s, t = 37, 8, 5
    exact = g.uniform(size=(n, n)) < 0.5
    pred = tri.nearest_known_prediction(exact, n, s, t)
    ci, sa = tri.coarse_index(n, s), tri.sentinel_axis(n, t)
    for iy in range(n):
        for ix in range(n):
            dc = min((cy - iy) ** 2 + (cx - ix) ** 2 for cy in ci for cx in ci)
            ds = min((sy - iy) ** 2 + (sx - ix) ** 2 for sy in sa for sx in sa)
            if ds < dc:
                best = min(((sy - iy) ** 2 + (sx - ix) ** 2, sy, sx) for sy in sa for sx in sa)
                want = exact[best[1], best[2]]
            else:
                # the coarse rule: per-axis nearest, the upper one on a tie
                jy = tri.nearest_coarse_index(n, s)[iy]
                jx = tri.nearest_coarse_index(n, s)[ix]
                assert (ci[jy] - iy) ** 2 + (ci[jx] - ix) ** 2 == dc
                want = exact[ci[jy], ci[jx]]
            assert pred[iy, ix] == want, (iy, ix)


def test_nearest_coarse_prediction_indices():
    labels = np.arange(16).reshape(4, 4)
    pred = tri.nearest_coarse_prediction(labels, 30, 8)
    # coarse cells at 4, 12, 20, 28; cell 8 is equidistant from 4 and 12 and takes 12
    cols = [pred[0, i] for i in (0, 3, 4, 7, 8, 15, 16, 29)]
    assert cols == [0, 0, 0, 0, 1, 1, 2, 3]
