"""GPU dynamic-aperture scans: survival turns against the oracle, batched scans
against per-lattice scans, and the surrogate-triaged scan against the
exhaustive one (boundary within one grid cell)."""
import numpy as np
import pytest

import synthetic as syn
from oracle import oracle as orc
from oracle import triage as otri
from paper_1710_07350_gb300 import da_metrics as dm
from paper_1710_07350_gb300 import trk

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def grid_points(n, w=syn.DA_HALF_WIDTH):
    z = syn.da_particles(n=n, half_width=w)
    return torch.from_numpy(z[:, 0].copy()).cuda(), torch.from_numpy(z[:, 2].copy()).cuda(), z


def test_da_survival_vs_oracle():
    n, turns = 24, 150
    x0, y0, z = grid_points(n)
    lats = [syn.lattice_c5(v) for v in (0, 3)]
    L = [trk.trk_create_lattice(l, moments=False) for l in lats]
    surv = trk.trk_da_survival(L, torch.cat([x0, x0]), torch.cat([y0, y0]), [0, n * n, 2 * n * n], turns)
    surv = surv.cpu().numpy()
    for k, lat in enumerate(lats):
        o = orc.track(lat, z, turns, moments=False)
        want = np.where(o["alive"] == 1, turns + 1, o["loss_turn"] + 1)
        exempt = ~(o["margin"] >= 1e-9)
        got = surv[k * n * n:(k + 1) * n * n]
        assert np.array_equal(got[~exempt], want[~exempt])
        assert 0 < np.sum(want == turns + 1) < n * n


def test_batched_scan_equals_per_lattice_scan():
    n, turns = 32, 200
    x0, y0, _ = grid_points(n)
    L = [trk.trk_create_lattice(syn.lattice_c5(v), moments=False) for v in range(5)]
    all_x = torch.cat([x0] * 5)
    all_y = torch.cat([y0] * 5)
    batched = trk.trk_da_survival(L, all_x, all_y, [k * n * n for k in range(6)], turns).cpu().numpy()
    for v in range(5):
        one = trk.trk_da_survival([L[v]], x0, y0, [0, n * n], turns).cpu().numpy()
        assert np.array_equal(one, batched[v * n * n:(v + 1) * n * n])


@pytest.mark.parametrize("use_mlp", [1, 0])
def test_triage_matches_exhaustive_boundary(use_mlp):
    nv, n, turns = 4, 96, 300
    L = [trk.trk_create_lattice(syn.lattice_c5(v), moments=False) for v in range(nv)]
    params = torch.from_numpy(syn.c5_params()[:nv].astype(np.float32)).cuda()
    x0, y0, _ = grid_points(n)
    exh = trk.trk_da_survival(L, torch.cat([x0] * nv), torch.cat([y0] * nv),
                              [k * n * n for k in range(nv + 1)], turns).cpu().numpy().reshape(nv, n, n)
    g = np.random.Generator(np.random.Philox(key=11))
    audit = torch.from_numpy((g.uniform(size=(nv, n, n)) < 0.005).astype(np.uint8)).cuda()
    opts = {"nx": n, "ny": n, "half_width": syn.DA_HALF_WIDTH, "n_turns": turns, "coarse_stride": 4,
            "band_radius": 2, "use_mlp": use_mlp, "epochs": 60, "batch": 256, "lr": 2e-3,
            "sentinel_stride": 5, "expand_radius": 4}
    net = trk.trk_mlp_create(syn.mlp_init(7)) if use_mlp else None
    ncoarse = nv * ((n - 2 + 3) // 4) ** 2
    perm = None
    if use_mlp:
        perm = torch.from_numpy(np.stack([g.permutation(ncoarse) for _ in range(60)]).astype(np.int32)).cuda()
    mask, surv, st = trk.trk_da_triage(L, params, opts, net=net, audit=audit, perm=perm)
    mask, surv = mask.cpu().numpy(), surv.cpu().numpy()
    for v in range(nv):
        ok, nd, r = dm.boundary_difference(mask[v], exh[v] == turns + 1)
        assert ok, (v, nd, r)
    # every exactly tracked cell carries the exhaustive survival turn
    exact = (surv > 0) & (surv <= turns)
    assert np.array_equal(surv[exact], exh[exact])
    assert st["n_tracked"] < nv * n * n and st["n_coarse"] == ncoarse
    assert 1 <= st["n_passes"] < 64


def test_nonlearned_triage_matches_triage_oracle():
    """With the nearest-coarse prediction the whole pipeline is deterministic:
    the merged mask, the survival turns and the number of band-tracked cells
    equal the triage oracle's, run on the oracle tracker's exact labels."""
    nv, n, turns, stride = 2, 48, 200, 8
    lats = [syn.lattice_c5(v) for v in range(nv)]
    L = [trk.trk_create_lattice(l, moments=False) for l in lats]
    params = torch.from_numpy(syn.c5_params()[:nv].astype(np.float32)).cuda()
    z = syn.da_particles(n=n)
    g = np.random.Generator(np.random.Philox(key=13))
    audit = (g.uniform(size=(nv, n, n)) < 0.01).astype(np.uint8)
    opts = {"nx": n, "ny": n, "half_width": syn.DA_HALF_WIDTH, "n_turns": turns, "coarse_stride": stride,
            "band_radius": 2, "use_mlp": 0, "sentinel_stride": 5, "expand_radius": 4}
    mask, surv, st = trk.trk_da_triage(L, params, opts, audit=torch.from_numpy(audit).cuda())
    mask, surv = mask.cpu().numpy().astype(bool), surv.cpu().numpy()
    n_tracked, passes, strict = 0, 0, True
    for v, lat in enumerate(lats):
        o = orc.track(lat, z, turns, moments=False)
        exact = np.where(o["alive"] == 1, turns + 1, o["loss_turn"] + 1).reshape(n, n)
        m, sv, tracked, p = otri.triage_variant(exact, turns, stride, 2, audit=audit[v], sentinel=5, expand=4)
        assert dm.boundary_difference(m, exact == turns + 1)[0]
        if np.any(~(o["margin"] >= 1e-9)):
            strict = False    # a label within rounding of the aperture may differ; compared above only
            continue
        assert np.array_equal(mask[v], m)
        assert np.array_equal(surv[v], sv)
        n_tracked += int(tracked.sum())
        passes = max(passes, p)
    if strict:
        assert st["n_tracked"] == n_tracked
        assert st["n_passes"] == passes


def test_lane_scan_bit_identical_to_batched_scan():
    """8 lanes per particle give the batched tracker's survival turns exactly,
    on maps, thin sextupoles and exact drifts, rectangle and ellipse apertures."""
    n, turns = 40, 300
    x0, y0, _ = grid_points(n)
    lats = [syn.lattice_c5(v) for v in (0, 1, 2)]
    lats[1]["elements"] = lats[1]["elements"][:5] + [{"type": "EDRIFT", "L": 0.05}] + lats[1]["elements"][5:]
    lats[2]["aperture"] = ("ellipse", 0.02, 0.015)
    L = [trk.trk_create_lattice(l, moments=False) for l in lats]
    offs = [k * n * n for k in range(4)]
    ax, ay = torch.cat([x0] * 3), torch.cat([y0] * 3)
    batched = trk.trk_da_survival(L, ax, ay, offs, turns, schedule={"block": 128, "per_thread": 1,
                                                                     "chunk_turns": 7}).cpu().numpy()
    lanes = trk.trk_da_survival_lanes(L, ax, ay, offs, turns).cpu().numpy()
    assert np.array_equal(batched, lanes)
    assert 0 < np.sum(lanes == turns + 1) < lanes.size
    # ragged variant sizes, an empty variant, a single point
    offs2 = [0, 7, 7, 8]
    sub_x = torch.cat([x0[:7], x0[100:101]])
    sub_y = torch.cat([y0[:7], y0[100:101]])
    a = trk.trk_da_survival(L, sub_x, sub_y, offs2, turns, schedule={"block": 64, "per_thread": 1}).cpu().numpy()
    b = trk.trk_da_survival_lanes(L, sub_x, sub_y, offs2, turns).cpu().numpy()
    assert np.array_equal(a, b)


def test_lane_scan_rejects_kick_drift_lattice():
    L = [trk.trk_create_lattice(syn.lattice_c2(cells=1), moments=False)]
    x0, y0, _ = grid_points(4)
    with pytest.raises(RuntimeError, match="MAP, EDRIFT and THINSEXT"):
        trk.trk_da_survival_lanes(L, x0, y0, [0, 16], 5)
    # the general entry point falls back to the batched tracker
    s = trk.trk_da_survival(L, x0, y0, [0, 16], 5).cpu().numpy()
    assert np.all((s >= 1) & (s <= 6))
