"""GPU parity of the patch correlation (ba_patch_correlation, Eq. 4) with the
FP64 oracle.

Tolerance, from the arithmetic: each output is a bilinear combination of four
dot products of length D, each accumulated in FP32 by one thread (one
rounding per fused multiply-add), then combined with float weights; its error
is at most about (D + 8) u times the same sum taken over |g||f|, which the
oracle returns (u = 2^-24).  That worst-case bound is the test's tolerance.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2408_01654_b300 import capi, scenes  # noqa: E402
from paper_2408_01654_b300.ba import DPVBA  # noqa: E402

U = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_01654_b300 import build
    build.build()
    oracle.build()


def case(seed, Nf=3, H=24, W=30, D=64, P=6, p=3, E=40, spread=6.0, step=1.0):
    rng = np.random.default_rng(seed)
    fmap = rng.normal(size=(Nf, H, W, D)).astype(np.float32)
    gmap = rng.normal(size=(P, p, p, D)).astype(np.float32)
    kk = rng.integers(0, P, size=E).astype(np.int32)
    jj = rng.integers(0, Nf, size=E).astype(np.int32)
    centre = np.stack([rng.uniform(-spread, W - 1 + spread, E), rng.uniform(-spread, H - 1 + spread, E)], 1)
    off = (np.arange(p) - (p - 1) / 2) * step
    coords = np.empty((E, p, p, 2), np.float32)
    coords[..., 0] = centre[:, None, None, 0] + off[None, None, :] + rng.normal(0, 0.3, (E, p, p))
    coords[..., 1] = centre[:, None, None, 1] + off[None, :, None] + rng.normal(0, 0.3, (E, p, p))
    return fmap, gmap, kk, jj, coords


def gpu(ba, fmap, gmap, kk, jj, coords, R):
    dev = "cuda"
    out = ba.patch_correlation(torch.tensor(fmap, device=dev), torch.tensor(gmap, device=dev),
                               torch.tensor(kk, device=dev), torch.tensor(jj, device=dev),
                               torch.tensor(coords, device=dev), R)
    ba.sync()
    return out.cpu().numpy().astype(np.float64)


def check(got, want, bound, D):
    err = np.abs(got - want)
    assert np.all(err <= (D + 8) * U * bound + 1e-30), (err.max(), (err / (bound + 1e-30)).max() / U)


@pytest.mark.parametrize("D,p,R", [(64, 3, 3), (32, 3, 0), (128, 3, 4), (96, 2, 3), (32, 1, 2), (224, 3, 3),
                                   (256, 3, 2)])
def test_matches_oracle(D, p, R):
    fmap, gmap, kk, jj, coords = case(D + 10 * p + R, D=D, p=p)
    want, bound = oracle.patch_correlation(fmap, gmap, kk, jj, coords, R, bound=True)
    got = gpu(DPVBA(), fmap, gmap, kk, jj, coords, R)
    check(got, want, bound, D)


def test_integer_and_far_coordinates():
    fmap, gmap, kk, jj, coords = case(7)
    coords[:10] = np.round(coords[:10])          # exact taps
    coords[10:14] += 5000.0                     # far outside: zeros
    coords[14:16] -= 3.0e7                      # beyond the clamp
    coords[16] = np.float32(-0.5)               # straddling the border
    want, bound = oracle.patch_correlation(fmap, gmap, kk, jj, coords, 3, bound=True)
    got = gpu(DPVBA(), fmap, gmap, kk, jj, coords, 3)
    check(got, want, bound, 64)
    assert np.all(got[10:16] == 0.0)


@pytest.mark.parametrize("step", [2.5, 15.0])
def test_spread_patch_falls_back_to_rows_and_pixels(step):
    # pixels 2.5 map pixels apart: the union box exceeds the staging capacity
    # but a patch row fits; 15 apart: neither does, one block per pixel
    fmap, gmap, kk, jj, coords = case(8, H=64, W=80, D=128, spread=-10.0, step=step)
    want, bound = oracle.patch_correlation(fmap, gmap, kk, jj, coords, 3, bound=True)
    got = gpu(DPVBA(), fmap, gmap, kk, jj, coords, 3)
    check(got, want, bound, 128)


def test_odometry_window_workload():
    # the bench's shape: 22 frames of 120x160x128 maps, 27,456 edges
    s = scenes.odometry(0)
    ci = scenes.correlation_inputs(s)
    want, bound = oracle.patch_correlation(ci["fmap"], ci["gmap"], s.kk, s.jj, ci["coords"], 3, bound=True)
    ba = DPVBA()
    got = gpu(ba, ci["fmap"], ci["gmap"], s.kk, s.jj, ci["coords"], 3)
    check(got, want, bound, 128)
    assert np.count_nonzero(want) > 0.5 * want.size
    # a second call on the same handle (scratch reused) gives the same volume
    again = gpu(ba, ci["fmap"], ci["gmap"], s.kk, s.jj, ci["coords"], 3)
    assert np.array_equal(again, got)


def test_empty_and_invalid():
    ba = DPVBA()
    fmap, gmap, kk, jj, coords = case(9, E=0)
    assert gpu(ba, fmap, gmap, kk, jj, coords, 3).shape == (0, 3, 3, 7, 7)
    fmap, gmap, kk, jj, coords = case(10, E=8)
    kk[3] = 99
    jj[5] = -2
    dev = "cuda"
    out = ba.patch_correlation(torch.tensor(fmap, device=dev), torch.tensor(gmap, device=dev),
                               torch.tensor(kk, device=dev), torch.tensor(jj, device=dev),
                               torch.tensor(coords, device=dev), 3)
    with pytest.raises(capi.BAError) as e:
        ba.sync()
    assert e.value.status == capi.BA_ERR_INVALID_ARG
    assert torch.all(out[3] == 0) and torch.all(out[5] == 0)
    with pytest.raises(capi.BAError) as e:  # D not a multiple of 32
        fmap, gmap, kk, jj, coords = case(11, D=48)
        gpu(DPVBA(), fmap, gmap, kk, jj, coords, 3)
    assert e.value.status == capi.BA_ERR_INVALID_ARG
    with pytest.raises(capi.BAError) as e:  # too wide for the staging buffer
        fmap, gmap, kk, jj, coords = case(12, D=512)
        gpu(DPVBA(), fmap, gmap, kk, jj, coords, 4)
    assert e.value.status == capi.BA_ERR_UNSUPPORTED
