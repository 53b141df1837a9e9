"""Pins for the FP64 oracle against facts fixed by the paper and by mathematics.

Each test ties one part of the oracle to something other than itself:
closed-form reprojections (Eq. 2), a library matrix exponential (SE(3)
retraction), central finite differences (the Jacobians of Eq. 3), a library
dense solve (Schur elimination, Cholesky, back-substitution), the seven gauge
directions of monocular BA (invariance of Eq. 3 under a world similarity),
world-frame equivariance of the step, and convergence to ground truth on
noise-free scenes.  A dropped term, a wrong sign or index, or a transposed
operand in the oracle fails at least one of them.
"""
import json
import os
import types

import numpy as np
import pytest
import scipy.linalg
from scipy.spatial.transform import Rotation

import oracle
from paper_2408_01654_b300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
NOPT = (0.0, 0.0, 0.1, 1e-3)  # no damping


def mini_scene(poses, uvd, edges, targets=None, weights=None, K=(320.0, 320.0, 320.0, 240.0), fixed=0):
    """A hand-made graph: poses [N,7], uvd [P,3] patch centre + inverse depth,
    edges list of (i, k, j)."""
    poses = np.asarray(poses, np.float64)
    uvd = np.asarray(uvd, np.float64)
    P = len(uvd)
    patches = np.zeros((P, 3, 3, 3))
    off = np.array([-1.0, 0.0, 1.0])
    patches[:, 0] = uvd[:, 0, None, None] + off[None, None, :]
    patches[:, 1] = uvd[:, 1, None, None] + off[None, :, None]
    patches[:, 2] = uvd[:, 2, None, None]
    ed = np.asarray(edges, np.int32).reshape(-1, 3)
    E = len(ed)
    return types.SimpleNamespace(
        N=len(poses), P=P, E=E, fixed=fixed, iters=1, poses=poses, patches=patches,
        ii=ed[:, 0].copy(), kk=ed[:, 1].copy(), jj=ed[:, 2].copy(),
        targets=np.zeros((E, 2)) if targets is None else np.asarray(targets, np.float64),
        weights=np.ones((E, 2)) if weights is None else np.asarray(weights, np.float64),
        intrinsics=np.asarray(K, np.float64))


def hat(w):
    return np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])


def pose_matrix(p):
    T = np.eye(4)
    T[:3, :3] = Rotation.from_quat(p[3:]).as_matrix()
    T[:3, 3] = p[:3]
    return T


def matrix_pose(T):
    q = Rotation.from_matrix(T[:3, :3]).as_quat()
    return np.concatenate([T[:3, 3], q])


def pose_err(a, b):
    """(rotation rad, translation m) between two [N,7] pose arrays."""
    rot = (Rotation.from_quat(a[:, 3:]) * Rotation.from_quat(b[:, 3:]).inv()).magnitude()
    return rot.max(), np.abs(a[:, :3] - b[:, :3]).max()


# --------------------------------------------------------------------------- #
# Eq. 2 closed forms
# --------------------------------------------------------------------------- #
def test_reprojection_closed_forms(oracle_lib):
    g = json.load(open(os.path.join(GOLDEN, "reprojection_closed_forms.json")))
    for c in g["cases"]:
        s = mini_scene([c["pose_i"], c["pose_j"]], [c["uv"] + [c["d"]]], [(0, 0, 1)], K=g["intrinsics"])
        proj, res, *_, valid = oracle.edge_terms(s)
        np.testing.assert_allclose(proj[0], c["proj"], atol=1e-9, err_msg=c["what"])
        np.testing.assert_allclose(res[0], -np.asarray(c["proj"]), atol=1e-9)  # r = I - proj, I = 0
        assert valid[0]


def test_masking_rules(oracle_lib):
    # self edge, a point behind frame j, and a point 5 cm in front of frame j
    poses = [[0, 0, 0, 0, 0, 0, 1], [0, 0, -2.0, 0, 0, 0, 1], [0, 0, -0.95, 0, 0, 0, 1]]
    s = mini_scene(poses, [[320, 240, 1.0]], [(0, 0, 0), (0, 0, 1), (0, 0, 2)])
    *_, valid = oracle.edge_terms(s)
    assert valid.tolist() == [False, False, False]
    s = mini_scene(poses, [[320, 240, 1.0]], [(0, 0, 2)])
    *_, valid = oracle.edge_terms(s, z_min=0.01)
    assert valid.tolist() == [True]


# --------------------------------------------------------------------------- #
# SE(3) retraction against the library matrix exponential
# --------------------------------------------------------------------------- #
@pytest.mark.parametrize("scale", [0.0, 1e-9, 1e-5, 9e-4, 1.1e-3, 0.05, 1.0, 3.0])
def test_retraction_matches_expm(oracle_lib, scale):
    rng = np.random.default_rng(int(scale * 1e9) % 1000)
    for _ in range(5):
        rho = rng.normal(size=3) * 0.3
        phi = rng.normal(size=3)
        phi *= scale / max(np.linalg.norm(phi), 1e-300)
        xi = np.concatenate([rho, phi])
        twist = np.zeros((4, 4))
        twist[:3, :3] = hat(phi)
        twist[:3, 3] = rho
        q0 = Rotation.random(random_state=rng).as_quat()
        pose = np.concatenate([rng.normal(size=3), q0])
        want = scipy.linalg.expm(twist) @ pose_matrix(pose)
        got = oracle.se3_retract(xi, pose)
        np.testing.assert_allclose(pose_matrix(got), want, atol=2e-14)
        assert abs(np.linalg.norm(got[3:]) - 1) < 1e-15


def test_quat_to_rot_matches_library(oracle_lib):
    rng = np.random.default_rng(3)
    for q in Rotation.random(20, random_state=rng).as_quat():
        np.testing.assert_allclose(oracle.quat_to_rot(q), Rotation.from_quat(q).as_matrix(), atol=1e-15)


# --------------------------------------------------------------------------- #
# Jacobians of Eq. 3 residuals against central finite differences
# --------------------------------------------------------------------------- #
def test_jacobians_central_fd(oracle_lib):
    s = scenes.tiny(seed=5)
    sel = np.random.default_rng(0).choice(s.E, 40, replace=False)
    sub = mini_scene(s.poses, np.c_[s.patches[:, 0, 1, 1], s.patches[:, 1, 1, 1], s.patches[:, 2, 1, 1]],
                     np.c_[s.ii[sel], s.kk[sel], s.jj[sel]])
    proj, _, Ji, Jj, Jd, valid = oracle.edge_terms(sub)
    assert valid.all()
    h = 1e-6
    for e in range(len(sel)):
        i, j, k = sub.ii[e], sub.jj[e], sub.kk[e]
        for which, J in ((i, Ji), (j, Jj)):
            for m in range(6):
                xi = np.zeros(6)
                xi[m] = h
                pp, pm = sub.poses.copy(), sub.poses.copy()
                pp[which] = oracle.se3_retract(xi, sub.poses[which])
                pm[which] = oracle.se3_retract(-xi, sub.poses[which])
                fd = (oracle.edge_terms(sub, poses=pp)[0][e] - oracle.edge_terms(sub, poses=pm)[0][e]) / (2 * h)
                np.testing.assert_allclose(J[e, :, m], fd, rtol=1e-6, atol=1e-5 * np.abs(fd).max() + 1e-7)
        hd = 1e-7
        pp, pm = sub.patches.copy(), sub.patches.copy()
        pp[k, 2] += hd
        pm[k, 2] -= hd
        fd = (oracle.edge_terms(sub, patches=pp)[0][e] - oracle.edge_terms(sub, patches=pm)[0][e]) / (2 * hd)
        np.testing.assert_allclose(Jd[e], fd, rtol=1e-6, atol=1e-6 * np.abs(fd).max() + 1e-7)


# --------------------------------------------------------------------------- #
# Schur + Cholesky + back-substitution against a library dense solve
# --------------------------------------------------------------------------- #
def dense_system(s, fixed, lam_p, lam_d):
    """Full (6 Nf + P) normal equations from the oracle's per-edge terms."""
    _, r, Ji, Jj, Jd, valid = oracle.edge_terms(s)
    nf = s.N - fixed
    n = 6 * nf + s.P
    H, g = np.zeros((n, n)), np.zeros(n)
    for e in np.nonzero(valid)[0]:
        J = np.zeros((2, n))
        i, j, k = s.ii[e], s.jj[e], s.kk[e]
        if i >= fixed:
            J[:, 6 * (i - fixed):6 * (i - fixed) + 6] += Ji[e]
        if j >= fixed:
            J[:, 6 * (j - fixed):6 * (j - fixed) + 6] += Jj[e]
        J[:, 6 * nf + k] = Jd[e]
        W = np.diag(s.weights[e])
        H += J.T @ W @ J
        g += J.T @ W @ r[e]
    H[np.arange(6 * nf), np.arange(6 * nf)] += lam_p
    H[np.arange(6 * nf, n), np.arange(6 * nf, n)] += lam_d
    return H, g


def small_graph(seed=1, N=5, M=6):
    s = scenes.tiny(seed=seed)
    keep = (s.kk % 96 < M) & (s.ii < N) & (s.jj < N)
    sub = mini_scene(s.poses[:N], np.c_[s.patches[:, 0, 1, 1], s.patches[:, 1, 1, 1], s.patches[:, 2, 1, 1]][
        np.r_[[np.arange(f * 96, f * 96 + M) for f in range(N)]].ravel()],
        [])
    # renumber patches frame-major 0..N*M-1
    kmap = {f * 96 + m: f * M + m for f in range(N) for m in range(M)}
    sub.ii = s.ii[keep].copy()
    sub.jj = s.jj[keep].copy()
    sub.kk = np.array([kmap[k] for k in s.kk[keep]], np.int32)
    sub.targets = s.targets[keep].astype(np.float64)
    sub.weights = s.weights[keep].astype(np.float64)
    sub.E = len(sub.kk)
    sub.fixed = 2
    return sub


@pytest.mark.parametrize("fixed", [1, 2])
def test_step_matches_dense_library_solve(oracle_lib, fixed):
    s = small_graph()
    opts = (1e-4, 1e-4, 0.1, 1e-3)
    H, g = dense_system(s, fixed, opts[0], opts[1])
    want = np.linalg.solve(H, g)
    nf6 = 6 * (s.N - fixed)
    r = oracle.gn(s, iters=1, fixed=fixed, opts=opts)
    x = np.r_[r["dxi"][0], r["dd"][0]]
    # backward error: the oracle's step solves the dense system to rounding
    assert np.abs(H @ x - g).max() < 1e-12 * (np.abs(H).max() * np.abs(x).max() + np.abs(g).max())
    # forward error within condition number x unit roundoff
    kappa = np.linalg.cond(H)
    assert np.abs(x - want).max() <= 10 * kappa * 2.2e-16 * np.abs(want).max(), kappa
    # the reduced system itself equals the library Schur complement of H
    S, y, Ct, w, _ = oracle.schur_system(s, fixed=fixed, opts=opts)
    Hpp, Hpd, Hdd = H[:nf6, :nf6], H[:nf6, nf6:], H[nf6:, nf6:]
    np.testing.assert_allclose(S, Hpp - Hpd @ np.linalg.solve(Hdd, Hpd.T), rtol=1e-9, atol=1e-9 * np.abs(S).max())
    np.testing.assert_allclose(y, g[:nf6] - Hpd @ np.linalg.solve(Hdd, g[nf6:]), rtol=1e-9,
                               atol=1e-9 * np.abs(y).max())
    np.testing.assert_allclose(Ct, np.diag(Hdd), rtol=1e-12)


def test_cholesky_rejects_indefinite(oracle_lib):
    s = small_graph()
    with pytest.raises(np.linalg.LinAlgError):
        oracle.gn(s, iters=1, fixed=s.fixed, opts=(-1e6, 1e-4, 0.1, 1e-3))


# --------------------------------------------------------------------------- #
# Gauge: Eq. 3 is invariant to a world SE(3) transform and to a global scale
# --------------------------------------------------------------------------- #
def gauge_directions(s):
    """7 tangent directions (poses, depths) of x -> world transform / scale."""
    dirs = []
    for m in range(6):
        zeta = np.zeros(6)
        zeta[m] = 1.0
        v = np.zeros(6 * s.N + s.P)
        for a in range(s.N):
            R = Rotation.from_quat(s.poses[a, 3:]).as_matrix()
            t = s.poses[a, :3]
            Ad = np.zeros((6, 6))
            Ad[:3, :3] = R
            Ad[:3, 3:] = hat(t) @ R
            Ad[3:, 3:] = R
            v[6 * a:6 * a + 6] = -Ad @ zeta
        dirs.append(v)
    v = np.zeros(6 * s.N + s.P)
    for a in range(s.N):
        v[6 * a:6 * a + 3] = s.poses[a, :3]
    v[6 * s.N:] = -s.patches[:, 2, 1, 1]
    dirs.append(v)
    return np.array(dirs)


def test_gauge_null_space(oracle_lib):
    s = small_graph()
    H, _ = dense_system(s, 0, 0.0, 0.0)
    D = gauge_directions(s)
    scale = np.abs(H).max()
    for v in D:
        assert np.abs(H @ v).max() < 1e-9 * scale * np.abs(v).max()
    # the reduced system carries the same null directions (pose parts)
    S, *_ = oracle.schur_system(s, fixed=0, opts=NOPT)
    for v in D:
        assert np.abs(S @ v[:6 * s.N]).max() < 1e-8 * np.abs(S).max() * np.abs(v).max()
    # and H is otherwise non-degenerate: exactly 7 near-zero eigenvalues
    ev = np.linalg.eigvalsh(H)
    assert np.sum(ev < 1e-9 * ev.max()) == 7


def test_world_frame_equivariance(oracle_lib):
    s = scenes.tiny(seed=2)
    r0 = oracle.gn(s, iters=1)
    X = np.eye(4)
    X[:3, :3] = Rotation.from_rotvec([0.3, -1.1, 0.4]).as_matrix()
    X[:3, 3] = [2.0, -1.0, 0.5]
    poses = np.array([matrix_pose(pose_matrix(p) @ np.linalg.inv(X)) for p in s.poses])
    r1 = oracle.gn(s, iters=1, poses=poses)
    np.testing.assert_allclose(r1["dxi"], r0["dxi"], rtol=1e-7, atol=1e-10)
    np.testing.assert_allclose(r1["dd"], r0["dd"], rtol=1e-7, atol=1e-10)
    # global scale: translations x2, inverse depths /2 -> translation steps x2, depth steps /2
    poses = s.poses.copy()
    poses[:, :3] *= 2.0
    patches = s.patches.astype(np.float64).copy()
    patches[:, 2] /= 2.0
    r2 = oracle.gn(s, iters=1, poses=poses, patches=patches, opts=(1e-12, 1e-12, 0.1, 1e-6))
    r0 = oracle.gn(s, iters=1, opts=(1e-12, 1e-12, 0.1, 1e-6))
    d0, d2 = r0["dxi"][0].reshape(-1, 6), r2["dxi"][0].reshape(-1, 6)
    np.testing.assert_allclose(d2[:, 3:], d0[:, 3:], rtol=1e-6, atol=1e-10)
    np.testing.assert_allclose(d2[:, :3], 2 * d0[:, :3], rtol=1e-6, atol=1e-10)
    np.testing.assert_allclose(r2["dd"][0], r0["dd"][0] / 2, rtol=1e-6, atol=1e-10)


# --------------------------------------------------------------------------- #
# whole GN: fixed point at ground truth, fixed poses untouched
# --------------------------------------------------------------------------- #
@pytest.mark.parametrize("make", [scenes.tiny, scenes.odometry])
def test_noise_free_convergence(oracle_lib, make):
    s = scenes.noise_free(make(seed=4))
    r = oracle.gn(s, iters=10)
    rot, tr = pose_err(r["poses"], s.poses_gt)
    assert rot < 1e-9 and tr < 1e-9, (rot, tr)
    assert np.abs(r["patches"][:, 2, 1, 1] / s.depth_gt - 1).max() < 1e-9
    assert r["cost"][-1] < 1e-12 * r["cost"][0]


def test_fixed_poses_bitwise_unchanged(oracle_lib):
    s = scenes.tiny(seed=7)
    r = oracle.gn(s, iters=2)
    assert np.array_equal(r["poses"][:s.fixed], s.poses[:s.fixed])
    assert not np.array_equal(r["poses"][s.fixed:], s.poses[s.fixed:])
    # all nine pixels of a patch carry the same updated inverse depth
    d = r["patches"][:, 2]
    assert np.array_equal(d, np.broadcast_to(d[:, 1:2, 1:2], d.shape))


def test_noisy_cost_decreases(oracle_lib):
    s = scenes.odometry(seed=1)
    r = oracle.gn(s, iters=4)
    assert np.all(np.diff(r["cost"]) < 0)


# --------------------------------------------------------------------------- #
# exact unrolled gradient (dual numbers) against central finite differences
# --------------------------------------------------------------------------- #
def test_dual_gradient_matches_central_fd(oracle_lib):
    s = small_graph(seed=3, N=6, M=8)
    s.iters = 2
    rng = np.random.default_rng(0)
    a = rng.normal(size=(s.N, 7))
    b = rng.normal(size=s.P)

    def L(targets=None, weights=None):
        r = oracle.gn(s, targets=targets, weights=weights)
        return (a * r["poses"]).sum() + (b * r["patches"][:, 2, 1, 1]).sum()

    kind = np.r_[np.zeros(12, int), np.ones(12, int)]
    index = rng.choice(2 * s.E, 24, replace=False)
    g = oracle.grad_fwd(s, a, b, kind, index)
    eps = 1e-3
    for c in range(24):
        base = (s.targets if kind[c] == 0 else s.weights).copy()
        p, m = base.copy(), base.copy()
        p.reshape(-1)[index[c]] += eps
        m.reshape(-1)[index[c]] -= eps
        if kind[c] == 0:
            fd = (L(targets=p) - L(targets=m)) / (2 * eps)
        else:
            fd = (L(weights=p) - L(weights=m)) / (2 * eps)
        assert abs(g[c] - fd) <= 1e-5 * max(1.0, abs(fd)), (c, g[c], fd)


def _pose_matrix(p):
    T = np.eye(4)
    T[:3, :3] = Rotation.from_quat(p[3:]).as_matrix()
    T[:3, 3] = p[:3]
    return T


def _pose_vector(T):
    q = Rotation.from_matrix(T[:3, :3]).as_quat()
    return np.r_[T[:3, 3], q]


def _se3_hat(xi):
    rho, phi = xi[:3], xi[3:]
    H = np.zeros((4, 4))
    H[:3, :3] = [[0, -phi[2], phi[1]], [phi[2], 0, -phi[0]], [-phi[1], phi[0], 0]]
    H[:3, 3] = rho
    return H


def test_dual_gradient_of_initial_state_matches_central_fd(oracle_lib):
    """Derivatives with respect to the initial inverse depths and to left
    perturbations of the initial poses (kinds 2 and 3) against central
    differences; the perturbed pose is formed with the library matrix
    exponential, independent of the oracle's own perturbation formula."""
    s = small_graph(seed=5, N=6, M=8)
    s.iters = 2
    rng = np.random.default_rng(1)
    a = rng.normal(size=(s.N, 7))
    b = rng.normal(size=s.P)

    def L(poses, patches):
        r = oracle.gn(s, poses=poses, patches=patches)
        return (a * r["poses"]).sum() + (b * r["patches"][:, 2, 1, 1]).sum()

    kpatch = rng.choice(s.P, 8, replace=False)
    kpose = rng.choice(np.arange(6 * s.fixed, 6 * s.N), 12, replace=False)
    kind = np.r_[np.full(8, 2), np.full(12, 3)]
    index = np.r_[kpatch, kpose]
    g = oracle.grad_fwd(s, a, b, kind, index)
    eps = 1e-4
    for c in range(len(kind)):
        if kind[c] == 2:
            pp, pm = s.patches.copy(), s.patches.copy()
            pp[index[c], 2] += eps
            pm[index[c], 2] -= eps
            fd = (L(s.poses, pp) - L(s.poses, pm)) / (2 * eps)
        else:
            q, m = divmod(int(index[c]), 6)
            xi = np.zeros(6)
            xi[m] = eps
            Pp, Pm = s.poses.copy(), s.poses.copy()
            T = _pose_matrix(s.poses[q])
            Pp[q] = _pose_vector(scipy.linalg.expm(_se3_hat(xi)) @ T)
            Pm[q] = _pose_vector(scipy.linalg.expm(_se3_hat(-xi)) @ T)
            # keep the quaternion hemisphere of the input
            for Pq in (Pp, Pm):
                if np.dot(Pq[q, 3:], s.poses[q, 3:]) < 0:
                    Pq[q, 3:] *= -1
            fd = (L(Pp, s.patches) - L(Pm, s.patches)) / (2 * eps)
        assert abs(g[c] - fd) <= 1e-5 * max(1.0, abs(fd)), (c, kind[c], g[c], fd)


# --------------------------------------------------------------------------- #
# graph indexing: canonical block keys on a hand-made graph
# --------------------------------------------------------------------------- #
def test_block_keys_hand_made():
    # edges (i, j): (0,1) (2,1) (3,3 self) (1,4) (4,0)
    ii = np.array([0, 2, 3, 1, 4])
    jj = np.array([1, 1, 3, 4, 0])
    want_all = [(0, 0), (0, 1), (0, 4), (1, 1), (1, 2), (1, 4), (2, 2), (4, 4)]
    assert [tuple(k) for k in oracle.block_keys(ii, jj, 0)] == want_all
    want_fixed2 = [(2, 2), (4, 4)]
    assert [tuple(k) for k in oracle.block_keys(ii, jj, 2)] == want_fixed2
