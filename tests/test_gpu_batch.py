"""GPU batched tracking: many lattice variants with uneven particle counts in one
launch per chunk (CUDA graph), against the plain per-lattice path and the oracle."""
import numpy as np
import pytest

import synthetic as syn
from oracle import oracle as orc
from paper_1710_07350_gb300 import trk

from gpu_util import TOL_100, by_id, compare_moments, compare_tracking, reduction_check

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def variants(k, scale_n=0.05):
    vs = syn.c4_variants()[:k]
    return [(f, d, max(1, int(n * scale_n))) for f, d, n in vs]


def make(vs, aperture=None):
    lats, bunches, inputs = [], [], []
    for v, var in enumerate(vs):
        lat = syn.lattice_c4(var)
        if aperture is not None:
            lat["aperture"] = aperture
        z = syn.c4_bunch(v, var[2])
        coords, ids = trk.upload(z)
        bunches.append(trk.trk_bunch_wrap(coords, ids))
        lats.append(trk.trk_create_lattice(lat))
        inputs.append((lat, z))
    return lats, bunches, inputs


def result(b):
    zz, ii = trk.download(b)
    return {"z": zz, "ids": ii, "n_alive": trk.trk_n_alive(b), "lost": trk.trk_lost(b),
            "moments": trk.trk_moments(b), "p0c": trk.trk_bunch_p0c(b)}


@pytest.mark.parametrize("per_thread,growth", [(1, 0), (2, 2), (4, 0)])
def test_batch_equals_plain_bit_exact(per_thread, growth):
    vs = variants(9)
    ap = ("rect", 1.2e-3, 1.0e-3)     # small aperture: losses in every variant
    lats, bunches, _ = make(vs, ap)
    sched = {"block": 64, "per_thread": per_thread, "chunk_turns": 3, "growth": growth}
    B = trk.trk_batch_create(bunches, lats)
    trk.trk_batch_set_schedule(B, **sched)
    trk.trk_batch_track(B, 20)
    batched = [result(b) for b in bunches]
    # the same chunk sequence through trk_track, one lattice at a time
    chunks, t, first = [], 0, 3
    while t < 20:
        k = min(first, 20 - t)
        chunks.append(k)
        t += k
        if growth:
            first = min(first * growth, 128)
    lats2, bunches2, _ = make(vs, ap)
    for b, L in zip(bunches2, lats2):
        trk.trk_bunch_set_schedule(b, block=64, per_thread=per_thread, chunk_turns=128)
        moms = []
        for k in chunks:
            trk.trk_track(b, L, k)
            moms.append(trk.trk_moments(b))
        b.moms = np.concatenate(moms)
    n_lost = 0
    for r, b in zip(batched, bunches2):
        p = result(b)
        assert np.array_equal(r["z"], p["z"]) and np.array_equal(r["ids"], p["ids"])
        assert r["n_alive"] == p["n_alive"]
        for x, y in zip(r["lost"], p["lost"]):
            assert np.array_equal(x, y)
        assert np.array_equal(r["moments"], b.moms)
        n_lost += len(r["lost"][0])
    assert n_lost > 0


def test_batch_vs_oracle():
    vs = variants(6, scale_n=0.02)
    lats, bunches, inputs = make(vs)
    B = trk.trk_batch_create(bunches, lats)
    trk.trk_batch_set_schedule(B, block=128, per_thread=2, chunk_turns=25)
    trk.trk_batch_track(B, 50)
    for b, (lat, z) in zip(bunches, inputs):
        g = result(b)
        o = orc.track(lat, z, 50)
        err = compare_tracking(g, o, TOL_100)
        compare_moments(g["moments"][:1], o["moments"][:1])
        compare_moments(g["moments"], o["moments"], coord_err=err)
        reduction_check(g)


def test_batch_graph_replay_and_one_shot():
    vs = variants(5)
    lats, bunches, _ = make(vs)
    B = trk.trk_batch_create(bunches, lats)
    trk.trk_batch_set_schedule(B, block=128, per_thread=2, chunk_turns=4)
    trk.trk_batch_track(B, 8)
    trk.trk_batch_track(B, 8)          # replays the captured graph
    lats2, bunches2, _ = make(vs)
    trk.trk_track_batch(bunches2, lats2, 16, {"block": 128, "per_thread": 2, "chunk_turns": 4})
    for b1, b2 in zip(bunches, bunches2):
        z1, _, _, _ = by_id(result(b1), b1.n)
        z2, _, _, _ = by_id(result(b2), b2.n)
        assert np.array_equal(z1, z2)
    assert trk.trk_batch_get_schedule(B)["chunk_turns"] == 4


def test_batch_rejects_wake_lattice():
    lat = syn.lattice_c3(periods=1, nbins=16)
    L = trk.trk_create_lattice(lat)
    coords, ids = trk.upload(syn.bunch("c3", n=100))
    b = trk.trk_bunch_wrap(coords, ids)
    with pytest.raises(trk.TrkError):
        trk.trk_batch_create([b], [L])


def test_autotune_leaves_bunches_untouched_and_returns_valid_schedule():
    vs = variants(6)
    lats, bunches, _ = make(vs)
    before = [result(b) for b in bunches]
    sched, ms = trk.trk_autotune(bunches, lats, 4)
    assert sched["block"] in (64, 128, 256) and sched["per_thread"] in (1, 2, 4) and ms > 0
    for b, r in zip(bunches, before):
        a = result(b)
        assert np.array_equal(a["z"], r["z"]) and a["n_alive"] == r["n_alive"]
    # the chosen schedule runs and gives the same coordinates as the default one
    B = trk.trk_batch_create(bunches, lats)
    trk.trk_batch_set_schedule(B, **sched)
    trk.trk_batch_track(B, 6)
    lats2, bunches2, _ = make(vs)
    trk.trk_track_batch(bunches2, lats2, 6, {"block": 128, "per_thread": 1, "chunk_turns": 6})
    for b1, b2 in zip(bunches, bunches2):
        z1, _, _, _ = by_id(result(b1), b1.n)
        z2, _, _, _ = by_id(result(b2), b2.n)
        assert np.array_equal(z1, z2)
