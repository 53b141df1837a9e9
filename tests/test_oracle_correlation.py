"""Pins for the oracle's patch correlation (Sec. 3.1 "Patch correlation",
Eq. 4): a library bilinear sampler (scipy.ndimage.map_coordinates, linear,
zero outside the map), integer coordinates (one tap per offset), feature maps
affine in the pixel position (bilinear sampling reproduces them exactly), a
patch far outside the map (zero), and linearity in the patch features.  A
swapped row/column offset, a wrong bilinear weight or corner, a missing zero
padding or a transposed feature index fails one of them.
"""
import numpy as np
from scipy import ndimage

import oracle


def rand_case(seed, Nf=3, H=12, W=15, D=8, P=5, p=3, E=7, spread=2.0):
    rng = np.random.default_rng(seed)
    fmap = rng.normal(size=(Nf, H, W, D)).astype(np.float32)
    gmap = rng.normal(size=(P, p, p, D)).astype(np.float32)
    kk = rng.integers(0, P, size=E).astype(np.int32)
    jj = rng.integers(0, Nf, size=E).astype(np.int32)
    centre = np.stack([rng.uniform(-spread, W - 1 + spread, E), rng.uniform(-spread, H - 1 + spread, E)], 1)
    off = np.arange(p) - p // 2
    coords = np.empty((E, p, p, 2), np.float32)
    coords[..., 0] = centre[:, None, None, 0] + off[None, None, :] + rng.normal(0, 0.2, (E, p, p))
    coords[..., 1] = centre[:, None, None, 1] + off[None, :, None] + rng.normal(0, 0.2, (E, p, p))
    return fmap, gmap, kk, jj, coords


def test_matches_library_bilinear_sampler():
    R = 3
    fmap, gmap, kk, jj, coords = rand_case(0)
    C = oracle.patch_correlation(fmap, gmap, kk, jj, coords, R)
    E, p = coords.shape[0], coords.shape[1]
    G = 2 * R + 1
    want = np.zeros_like(C)
    for e in range(E):
        F = fmap[jj[e]].astype(np.float64)
        for v in range(p):
            for u in range(p):
                x, y = float(coords[e, v, u, 0]), float(coords[e, v, u, 1])
                ys = (y + np.arange(G)[:, None] - R) * np.ones((1, G))
                xs = (x + np.arange(G)[None, :] - R) * np.ones((G, 1))
                samp = np.stack([ndimage.map_coordinates(F[..., d], [ys.ravel(), xs.ravel()], order=1,
                                                         mode="grid-constant", cval=0.0)
                                 for d in range(F.shape[-1])], -1).reshape(G, G, -1)
                want[e, v, u] = samp @ gmap[kk[e], v, u].astype(np.float64)
    assert np.abs(C - want).max() < 1e-9


def test_integer_coordinates_pick_single_taps():
    fmap, gmap, kk, jj, coords = rand_case(1, spread=-4.0)
    coords = np.round(coords).astype(np.float32)
    R = 2
    C = oracle.patch_correlation(fmap, gmap, kk, jj, coords, R)
    H, W = fmap.shape[1], fmap.shape[2]
    for e in range(len(kk)):
        for v in range(3):
            for u in range(3):
                x, y = int(coords[e, v, u, 0]), int(coords[e, v, u, 1])
                for a in range(2 * R + 1):
                    for b in range(2 * R + 1):
                        yy, xx = y + a - R, x + b - R
                        want = 0.0
                        if 0 <= yy < H and 0 <= xx < W:
                            want = float(np.dot(gmap[kk[e], v, u].astype(np.float64),
                                                fmap[jj[e], yy, xx].astype(np.float64)))
                        assert abs(C[e, v, u, a, b] - want) < 1e-9


def test_affine_feature_map_is_reproduced_exactly():
    # f_d(x, y) = A_d x + B_d y + K_d: bilinear sampling is exact, so
    # C = sum_d g_d (A_d sx + B_d sy + K_d) wherever all four taps are inside
    H, W, D = 20, 24, 4
    rng = np.random.default_rng(2)
    A, B, K = rng.normal(size=D), rng.normal(size=D), rng.normal(size=D)
    yy, xx = np.mgrid[0:H, 0:W]
    fmap = (xx[..., None] * A + yy[..., None] * B + K)[None].astype(np.float32)
    gmap = rng.normal(size=(1, 3, 3, D)).astype(np.float32)
    coords = np.empty((1, 3, 3, 2), np.float32)
    coords[..., 0] = 11.37 + np.arange(3)[None, None, :]
    coords[..., 1] = 9.61 + np.arange(3)[None, :, None]
    R = 3
    C = oracle.patch_correlation(fmap, gmap, [0], [0], coords, R)
    for v in range(3):
        for u in range(3):
            g = gmap[0, v, u].astype(np.float64)
            for a in range(7):
                for b in range(7):
                    sx = float(coords[0, v, u, 0]) + b - R
                    sy = float(coords[0, v, u, 1]) + a - R
                    want = float(np.dot(g, A * sx + B * sy + K))
                    assert abs(C[0, v, u, a, b] - want) < 1e-4 * (1 + abs(want)), (a, b)


def test_far_outside_is_zero_and_bound_dominates():
    fmap, gmap, kk, jj, coords = rand_case(3)
    coords[2] += 1000.0
    coords[4] -= 1000.0
    C, Bd = oracle.patch_correlation(fmap, gmap, kk, jj, coords, 3, bound=True)
    assert np.all(C[2] == 0.0) and np.all(C[4] == 0.0)
    assert np.all(np.abs(C) <= Bd + 1e-12) and Bd.max() > 0


def test_linear_in_patch_features():
    fmap, gmap, kk, jj, coords = rand_case(4)
    rng = np.random.default_rng(5)
    g2 = rng.normal(size=gmap.shape).astype(np.float32)
    c1 = oracle.patch_correlation(fmap, gmap, kk, jj, coords)
    c2 = oracle.patch_correlation(fmap, g2, kk, jj, coords)
    c3 = oracle.patch_correlation(fmap, (gmap.astype(np.float64) + 2 * g2.astype(np.float64)).astype(np.float32),
                                  kk, jj, coords)
    assert np.abs(c3 - (c1 + 2 * c2)).max() < 1e-5
