"""Pins for the oracle's proximity loop-edge construction (Sec. 3.2
"Proximity Loop Closure" and "Constructing the Patch Graph").

The rule (nearest older camera centre with b - a > gap, within a radius; the
old frame's patches become edges to the query frame where their Eq. 2
reprojection lies in front of the camera and inside the image) is tied to
closed forms: hand-placed camera centres under random rotations (the centre is
-R^T t, not t), exact ties and exact threshold distances (lowest index wins;
both the gap and the radius are strict), reprojections under a pure
translation (u' = fx (x/d + dx) / (1/d + dz) + cx), invariance under a rigid
change of world frame, and the loop edges the synthetic-scene generator builds
by its own numpy code from ground-truth camera positions.
"""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from paper_2408_01654_b300 import scenes

K = np.array([320.0, 320.0, 320.0, 240.0])


def poses_from(R, C):
    """world->camera poses (t, q xyzw) of cameras with rotation R (world->camera)
    placed at world positions C: t = -R C."""
    R = np.asarray(R, np.float64).reshape(-1, 3, 3)
    C = np.asarray(C, np.float64).reshape(-1, 3)
    t = -np.einsum("nij,nj->ni", R, C)
    return np.concatenate([t, Rotation.from_matrix(R).as_quat()], 1)


def flat_patches(uvd):
    """[P,3,3,3] patches from centre pixels and inverse depths [P,3]."""
    uvd = np.asarray(uvd, np.float64)
    p = np.zeros((len(uvd), 3, 3, 3))
    off = np.array([-1.0, 0.0, 1.0])
    p[:, 0] = uvd[:, 0, None, None] + off[None, None, :]
    p[:, 1] = uvd[:, 1, None, None] + off[None, :, None]
    p[:, 2] = uvd[:, 2, None, None]
    return p


def identity_poses(C):
    C = np.asarray(C, np.float64).reshape(-1, 3)
    q = np.tile([0.0, 0.0, 0.0, 1.0], (len(C), 1))
    return np.concatenate([-C, q], 1)


def test_line_out_and_back_closed_form():
    # outbound along x at integer positions, back at x + 0.3 and y = 0.2
    # (far off for the last frames); rotations random, so the centre must be
    # recovered as -R^T t
    n, gap, radius = 40, 10, 1.0
    C = [(float(i), 0.0, 0.0) for i in range(n)]
    C += [(n - 1 - j + 0.3, 0.2 if j < 25 else 5.0, 0.0) for j in range(n)]
    rng = np.random.default_rng(3)
    R = Rotation.random(2 * n, random_state=rng).as_matrix()
    poses = poses_from(R, C)
    patches = flat_patches([(320.0, 240.0, 1.0)] * (2 * n))
    r = oracle.proximity_edges(poses, patches, K, 1, 0, 2 * n, gap=gap, radius=radius)
    for b in range(2 * n):
        if b < n:
            want_a, want_d = -1, (11.0 if b > gap else -1.0)
        else:
            j = b - n
            if j < 5:  # the matching outbound frame is not yet older than the gap
                want_a, want_d = -1, np.hypot(10.3 - 2 * j, 0.2)
            elif j < 25:
                want_a, want_d = n - 1 - j, np.hypot(0.3, 0.2)
            else:
                want_a, want_d = -1, np.hypot(0.3, 5.0)
        assert r["match"][b] == want_a, (b, r["match"][b], want_a)
        assert abs(r["dist"][b] - want_d) < 1e-12, (b, r["dist"][b], want_d)


def test_ties_and_strict_thresholds():
    far = [(100.0 + 10 * i, 0.0, 0.0) for i in range(4)]
    C = [(0.0, 0.0, 0.0), (0.5, 0.0, 0.0)] + far + [(0.5, 0.2, 0.0), (0.25, 0.0, 0.0), (1.0, 0.0, 0.0)]
    poses = identity_poses(C)
    patches = flat_patches([(320.0, 240.0, 1.0)] * len(C))
    r = oracle.proximity_edges(poses, patches, K, 1, 6, 9, gap=5, radius=0.5)
    # b = 6: only a = 0 is older than the gap (a = 1, with b - a = 5, is not,
    # although it is nearer); 0.539 > radius
    assert r["match"][0] == -1 and abs(r["dist"][0] - np.hypot(0.5, 0.2)) < 1e-15
    # b = 7: a = 0 and a = 1 both at exactly 0.25: the lower index
    assert r["match"][1] == 0 and r["dist"][1] == 0.25
    # b = 8: a = 1 at exactly the radius is not taken
    assert r["match"][2] == -1 and r["dist"][2] == 0.5
    r = oracle.proximity_edges(poses, patches, K, 1, 6, 9, gap=5, radius=0.5 + 1e-9)
    assert list(r["match"]) == [-1, 0, 1]
    r = oracle.proximity_edges(poses, patches, K, 1, 6, 9, gap=5, radius=0.6)
    assert list(r["match"]) == [0, 0, 1]
    assert list(r["ii"]) == [0, 0, 1] and list(r["jj"]) == [6, 7, 8] and list(r["kk"]) == [0, 0, 1]


def test_reprojection_under_translation_closed_form():
    gap, M = 4, 64
    rng = np.random.default_rng(11)
    delta = np.array([0.3, -0.2, -0.5])  # t_b = t_a + delta (identity rotations)
    C = [(0.0, 0.0, 0.0)] + [(100.0 * i, 0.0, 0.0) for i in range(1, gap + 1)] + [tuple(-delta)]
    poses = identity_poses(C)
    N = len(C)
    uvd = np.zeros((N * M, 3))
    uvd[:, 0] = rng.uniform(-40.0, 680.0, N * M)
    uvd[:, 1] = rng.uniform(-40.0, 520.0, N * M)
    uvd[:, 2] = rng.uniform(0.3, 5.0, N * M)
    r = oracle.proximity_edges(poses, flat_patches(uvd), K, M, N - 1, N, gap=gap, radius=2.0)
    assert r["match"][0] == 0
    fx, fy, cx, cy = K
    u, v, d = uvd[:M, 0], uvd[:M, 1], uvd[:M, 2]
    X = (u - cx) / fx / d + delta[0]
    Y = (v - cy) / fy / d + delta[1]
    Z = 1.0 / d + delta[2]
    up, vp = fx * X / Z + cx, fy * Y / Z + cy
    keep = (Z > 0.1) & (up >= 0) & (up < 640) & (vp >= 0) & (vp < 480)
    assert 0 < keep.sum() < M and (Z <= 0.1).any()
    assert list(r["kk"]) == list(np.nonzero(keep)[0])
    assert np.all(r["ii"] == 0) and np.all(r["jj"] == N - 1)
    assert np.allclose(r["coords"][:, 0], up[keep], rtol=0, atol=1e-9)
    assert np.allclose(r["coords"][:, 1], vp[keep], rtol=0, atol=1e-9)


def _loop_scene(N, seed):
    return scenes._build("proximity", seed, N, lambda i, m: scenes._clipped_window(i, m, 6), 2, 1, loop=True)


def test_invariant_under_rigid_world_change():
    s = _loop_scene(160, 4)
    M = scenes.PATCHES_PER_FRAME
    base = oracle.proximity_edges(s.poses, s.patches, s.intrinsics, M, 0, s.N)
    assert base["n"] > 0 and (base["match"] >= 0).sum() > 10
    Rw = Rotation.from_rotvec([0.4, -1.1, 0.7]).as_matrix()
    tw = np.array([3.0, -7.5, 12.25])
    R = Rotation.from_quat(s.poses[:, 3:]).as_matrix()
    # new world coordinates X' = Rw X + tw: T_i' = T_i W^-1
    Rn = R @ Rw.T
    tn = s.poses[:, :3] - np.einsum("nij,j->ni", Rn, tw)
    moved = np.concatenate([tn, Rotation.from_matrix(Rn).as_quat()], 1)
    r = oracle.proximity_edges(moved, s.patches, s.intrinsics, M, 0, s.N)
    assert np.array_equal(r["match"], base["match"])
    assert np.array_equal(r["ii"], base["ii"]) and np.array_equal(r["jj"], base["jj"])
    assert np.array_equal(r["kk"], base["kk"])
    assert np.allclose(r["dist"], base["dist"], rtol=0, atol=1e-9)
    assert np.allclose(r["coords"], base["coords"], rtol=0, atol=1e-8)


@pytest.mark.parametrize("N,seed", [(200, 0), (260, 7)])
def test_matches_scene_generator_on_ground_truth(N, seed):
    s = _loop_scene(N, seed)
    M = scenes.PATCHES_PER_FRAME
    pt = s.patches.astype(np.float64)
    pt[:, 2] = s.depth_gt[:, None, None]
    r = oracle.proximity_edges(s.poses_gt, pt, s.intrinsics, M, 0, s.N)
    assert r["margin"].min() > 1e-7  # no decision within rounding of its threshold
    loop = (s.jj - s.ii) > 30
    assert r["n"] == loop.sum() == s.info["loop_edges"] > 0
    got = {t: e for e, t in enumerate(zip(r["ii"].tolist(), r["jj"].tolist(), r["kk"].tolist()))}
    want = list(zip(s.ii[loop].tolist(), s.jj[loop].tolist(), s.kk[loop].tolist()))
    assert set(got) == set(want)
    sel = [got[t] for t in want]
    assert np.allclose(r["coords"][sel], s.proj_gt[loop], rtol=0, atol=1e-8)


def test_query_window_and_capacity():
    s = _loop_scene(160, 4)
    M = scenes.PATCHES_PER_FRAME
    full = oracle.proximity_edges(s.poses, s.patches, s.intrinsics, M, 0, s.N)
    b0, b1 = 90, 130
    part = oracle.proximity_edges(s.poses, s.patches, s.intrinsics, M, b0, b1)
    sel = (full["jj"] >= b0) & (full["jj"] < b1)
    assert np.array_equal(part["match"], full["match"][b0:b1])
    assert np.array_equal(part["kk"], full["kk"][sel]) and np.array_equal(part["jj"], full["jj"][sel])
    cut = oracle.proximity_edges(s.poses, s.patches, s.intrinsics, M, 0, s.N, cap=17)
    assert cut["n"] == full["n"] and np.array_equal(cut["kk"], full["kk"][:17])
    empty = oracle.proximity_edges(s.poses, s.patches, s.intrinsics, M, 50, 50)
    assert empty["n"] == 0 and len(empty["match"]) == 0
    none = oracle.proximity_edges(s.poses, s.patches, s.intrinsics, M, 0, s.N, gap=s.N)
    assert none["n"] == 0 and np.all(none["match"] == -1) and np.all(none["dist"] == -1)
