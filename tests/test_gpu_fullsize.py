"""Parity at the full workload sizes, in the launch configurations bench.py
times: the whole bunch (or every variant, or the whole DA grid) runs on the
GPU, and a seeded sample of particles is tracked one by one by the oracle.
Each particle's arithmetic is independent of the others, so the sample is
compared element by element; the moments of the full bunch are checked by a
property that holds at any size (they are the moments of the coordinates the
GPU returns)."""
import numpy as np
import pytest

import synthetic as syn
from oracle import oracle as orc
from paper_1710_07350_gb300 import trk

from gpu_util import MARGIN, TOL_100, TOL_PASS, compare_moments, compare_tracking, gpu_track, reduction_check

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def sample(n, k, key):
    g = np.random.Generator(np.random.Philox(key=key))
    return np.sort(g.choice(n, size=k, replace=False))


def compare_sample(z_gpu, alive_gpu, lost_turn, lost_elem, o, tol):
    """GPU results of the sampled particles (by id) against oracle run `o` on
    the same particles; particles within MARGIN of an aperture are exempt."""
    exempt = ~(o["margin"] >= MARGIN)
    keep = ~exempt
    assert np.array_equal(alive_gpu[keep], o["alive"][keep] == 1)
    lost = keep & (o["alive"] == 0)
    assert np.array_equal(lost_turn[lost], o["loss_turn"][lost])
    assert np.array_equal(lost_elem[lost], o["loss_elem"][lost])
    # survivors, and lost particles at the point of loss: max coordinate error
    err = float(np.max(np.abs(z_gpu[keep] - o["z"][keep]))) if keep.any() else 0.0
    assert err <= tol, "max coordinate error %.3e > %.1e" % (err, tol)
    return err


def gather(coords_host, ids_host, n_alive, lost, n, idx):
    z = np.full((n, 6), np.nan)
    z[ids_host] = coords_host
    alive = np.zeros(n, bool)
    alive[ids_host[:n_alive]] = True
    lt = np.full(n, -1)
    le = np.full(n, -1)
    lid, lturn, lel = lost
    lt[lid] = lturn
    le[lid] = lel
    return z[idx], alive[idx], lt[idx], le[idx]


def test_c2_full_bunch_bench_launch():
    """1e6 particles, block 128 x 2 particles per thread, one 100-turn launch."""
    lat = syn.lattice_c2()
    z = syn.bunch("c2")
    n = z.shape[0]
    L = trk.trk_create_lattice(lat)
    coords, ids = trk.upload(z)
    b = trk.trk_bunch_wrap(coords, ids)
    trk.trk_bunch_set_schedule(b, block=128, per_thread=2, chunk_turns=100)
    trk.trk_track(b, L, 100)
    mom = trk.trk_moments(b)
    zz, ii = trk.download(b)
    res = {"z": zz, "ids": ii, "n_alive": trk.trk_n_alive(b), "lost": trk.trk_lost(b), "moments": mom}
    idx = sample(n, 96, key=31)
    o = orc.track(lat, z[idx], 100)
    zs, al, lt, le = gather(zz, ii, res["n_alive"], res["lost"], n, idx)
    compare_sample(zs, al, lt, le, o, TOL_100)
    reduction_check(res)


def test_c4_all_variants_bench_batch():
    """256 variants, log-uniform 1000..65536 particles, one batched call with
    the autotuned schedule; 100 turns; 4 sampled particles in each of 16
    sampled variants."""
    vs = syn.c4_variants()
    lats = [syn.lattice_c4(v) for v in vs]
    Ls = [trk.trk_create_lattice(l) for l in lats]
    zs = [syn.c4_bunch(k, v[2]) for k, v in enumerate(vs)]
    inputs = [trk.upload(z) for z in zs]
    tuned, _ = trk.trk_autotune([trk.trk_bunch_wrap(c.clone(), i.clone()) for c, i in inputs], Ls, 20)
    bs = [trk.trk_bunch_wrap(c, i) for c, i in inputs]
    B = trk.trk_batch_create(bs, Ls)
    trk.trk_batch_set_schedule(B, **tuned)
    trk.trk_batch_track(B, 100)
    for v in sample(len(vs), 16, key=32):
        n = zs[v].shape[0]
        zz, ii = trk.download(bs[v])
        idx = sample(n, 4, key=1000 + int(v))
        o = orc.track(lats[v], zs[v][idx], 100, moments=False)
        zg, al, lt, le = gather(zz, ii, trk.trk_n_alive(bs[v]), trk.trk_lost(bs[v]), n, idx)
        compare_sample(zg, al, lt, le, o, TOL_100)


def oracle_survival(lat, z, turns):
    o = orc.track(lat, z, turns, moments=False)
    return np.where(o["alive"] == 1, turns + 1, o["loss_turn"] + 1), o["margin"]


def test_c5_full_da_grid_bench_scan():
    """64 variants x 512^2 cells x 1000 turns in one batched scan (the bench's
    exhaustive scan); about 48 sampled cells of each of 4 variants against the
    oracle's survival turns.  Over 1000 turns the chaotic orbits near the DA
    boundary amplify rounding differences exponentially, so a survival turn is
    compared only where it is well-conditioned: where the oracle gives the
    same turn with the start moved by 1e-12 relative (about the rounding that
    1000 turns accumulate) both ways, and the orbit stays MARGIN clear of the
    aperture.  Cells lost within the first turns and survivors deep inside the
    DA always qualify."""
    n, turns, nv = syn.DA_N, 1000, 64
    L = [trk.trk_create_lattice(syn.lattice_c5(v), moments=False) for v in range(nv)]
    z = syn.da_particles(n=n)
    x0 = torch.from_numpy(z[:, 0].copy()).cuda()
    y0 = torch.from_numpy(z[:, 2].copy()).cuda()
    surv = trk.trk_da_survival(L, torch.cat([x0] * nv), torch.cat([y0] * nv),
                               [k * n * n for k in range(nv + 1)], turns).cpu().numpy().reshape(nv, n * n)
    assert np.all((surv >= 1) & (surv <= turns + 1))
    for v in (0, 21, 42, 63):
        # half the sample near the DA boundary (where long survival is decided)
        idx = sample(n * n, 24, key=40 + v)
        s = surv[v]
        edge = np.nonzero((s > 50) & (s <= turns))[0]
        if edge.size:
            idx = np.unique(np.concatenate([idx, edge[sample(edge.size, min(24, edge.size), key=80 + v)]]))
        lat = syn.lattice_c5(v)
        want, margin = oracle_survival(lat, z[idx], turns)
        keep = margin >= MARGIN
        for sgn in (1.0, -1.0):
            zp = z[idx].copy()
            zp[:, 0] *= 1.0 + sgn * 1e-12
            zp[:, 2] *= 1.0 - sgn * 1e-12
            keep &= oracle_survival(lat, zp, turns)[0] == want
        assert keep.sum() >= len(idx) // 3
        assert np.array_equal(s[idx][keep], want[keep])


def test_c3_full_bunch_bench_launch():
    """The wake linac at its full size in the bench's launch configuration: the
    whole 1e7-particle bunch (95 % Gaussian, 5 % uniform tail), 4096-bin wakes,
    block 128 x 2 particles per thread, through the first three periods (RF
    cavity, wake, drift, quadrupole).  The wakes couple every particle, so the
    oracle tracks the whole bunch and every particle is compared; after one pass
    the tolerance is the one-pass 1e-12, and the per-element moments follow."""
    lat = syn.lattice_c3(periods=3)
    z = syn.bunch("c3")
    assert z.shape[0] == 10_000_000
    g = gpu_track(lat, z, 1, schedule={"block": 128, "per_thread": 2})
    o = orc.track(lat, z, 1)
    assert g["p0c"] == o["p0c"]
    assert g["n_alive"] == z.shape[0]                # no aperture in the linac
    err = compare_tracking(g, o, TOL_PASS)
    compare_moments(g["moments"], o["moments"], coord_err=err)
