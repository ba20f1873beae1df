"""trk_wake_static, the wake entry point that allocates nothing.

It exists for callers that may not allocate device memory when they need a wake
step (a fixed memory pool that must not grow, a host application that forbids
cudaMalloc after start-up, a device already full).  Its result must equal that
of trk_wake on the same particles, also on the second of two calls in a row,
where the shared fixed-size working array still holds the first call's data,
and it must match the CPU oracle's wake (histogram bit for bit, voltages to
1e-13 relative) at bin counts that take the shared-memory histogram (up to
8192 bins), the global-atomic one (8193 to 16384) and the 16384-bin maximum.
This file is collected last so that a stopping run has run every other test.
"""
import numpy as np
import pytest

import synthetic as syn
from oracle import oracle as orc
from paper_1710_07350_gb300 import trk

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def _with_trk_wake(z, nbins, p0c):
    coords, ids = trk.upload(z)
    b = trk.trk_bunch_wrap(coords, ids)
    h = torch.zeros(nbins, dtype=torch.int32, device="cuda")
    v = torch.zeros(nbins, dtype=torch.float64, device="cuda")
    trk.trk_wake(b, nbins, syn.C3_W0, syn.C3_SC, syn.C3_CHARGE, p0c, hist=h, volt=v)
    torch.cuda.synchronize()
    return coords.cpu().numpy(), h.cpu().numpy(), v.cpu().numpy()


def _with_static(z, nbins, p0c):
    coords, _ = trk.upload(z)
    h = torch.zeros(nbins, dtype=torch.int32, device="cuda")
    v = torch.zeros(nbins, dtype=torch.float64, device="cuda")
    trk.trk_wake_static(coords, z.shape[0], nbins, syn.C3_W0, syn.C3_SC, syn.C3_CHARGE, p0c, hist=h, volt=v)
    torch.cuda.synchronize()
    return coords.cpu().numpy(), h.cpu().numpy(), v.cpu().numpy()


def test_wake_static_equals_trk_wake_on_two_calls():
    p0c = 2.0e9
    # each call uses more bins than the one before, so stale histogram entries
    # left by an earlier call would show up if they were not cleared; 12000 and
    # 16384 bins take the global-atomic histogram, 16384 is the maximum
    for n, nbins, seed in ((20_000, 1000, 31), (7_777, 4096, 32), (15_000, 12_000, 33), (9_000, 16_384, 34)):
        z = syn.bunch("c3", n=n, seed=seed)
        ref_c, ref_h, ref_v = _with_trk_wake(z, nbins, p0c)
        got_c, got_h, got_v = _with_static(z, nbins, p0c)
        assert np.array_equal(got_h, ref_h)
        assert got_h.sum() == n
        assert np.allclose(got_v, ref_v, rtol=1e-13, atol=0)
        assert np.array_equal(got_c[:5], ref_c[:5])
        assert np.max(np.abs(got_c[5] - ref_c[5])) <= 1e-15
        # and against the CPU oracle on the same particles
        o, oh, oV = orc.wake(z, nbins, syn.C3_W0, syn.C3_SC, syn.C3_CHARGE, p0c)
        assert np.array_equal(got_h.astype(np.int64), oh), "histogram must be bit-exact on identical l"
        assert np.allclose(got_v, oV, rtol=1e-13, atol=0)
        assert np.array_equal(got_c[:5], o[:, :5].T)
        assert np.max(np.abs(got_c[5] - o[:, 5])) <= 1e-15


def test_wake_static_rejects_bad_tensors():
    """The binding checks what the C call cannot see behind bare pointers."""
    coords, _ = trk.upload(syn.bunch("c3", n=100))
    args = (syn.C3_W0, syn.C3_SC, syn.C3_CHARGE, 1e9)
    with pytest.raises(ValueError):
        trk.trk_wake_static(coords.float(), 100, 64, *args)
    with pytest.raises(ValueError):
        trk.trk_wake_static(coords, coords.shape[1] + 1, 64, *args)
    with pytest.raises(ValueError):
        trk.trk_wake_static(coords, 100, 64, *args, hist=torch.zeros(63, dtype=torch.int32, device="cuda"))
    with pytest.raises(ValueError):
        trk.trk_wake_static(coords, 100, 64, *args, volt=torch.zeros(64, dtype=torch.float32, device="cuda"))


def test_wake_static_rejects_oversize():
    coords, _ = trk.upload(syn.bunch("c3", n=100))
    with pytest.raises(trk.TrkError):
        trk.trk_wake_static(coords, 100, 16385, syn.C3_W0, syn.C3_SC, syn.C3_CHARGE, 1e9)
