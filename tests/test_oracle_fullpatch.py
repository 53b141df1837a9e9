"""Pins for the oracle's whole-patch residual (Eq. 3 summed over all nine
pixels of each patch, 18 residual rows per edge, one weight pair per edge
shared by its pixels).

* One GN step equals the library dense solve of the full (6 Nf + P) normal
  equations built here from central-difference Jacobians of a plain pinhole
  model (left perturbations T <- Exp(xi) T formed with scipy's matrix
  exponential), independent of the oracle's analytic Jacobians.
* The reduced system is the library Schur complement of that matrix.
* The whole-patch cost is the sum of nine centre-only costs, each with one
  pixel moved into the centre slot (patch and target).
* Noise-free whole-patch targets are reached from the perturbed start
  (ground truth to the float32 rounding of the targets).
"""
import numpy as np
import scipy.linalg
from scipy.spatial.transform import Rotation

import oracle
from paper_2408_01654_b300 import scenes
from test_oracle_pins import pose_err, small_graph

K = (320.0, 320.0, 320.0, 240.0)


def twist(xi):
    A = np.zeros((4, 4))
    A[:3, :3] = [[0, -xi[5], xi[4]], [xi[5], 0, -xi[3]], [-xi[4], xi[3], 0]]
    A[:3, 3] = xi[:3]
    return scipy.linalg.expm(A)


def mat(p):
    T = np.eye(4)
    T[:3, :3] = Rotation.from_quat(p[3:]).as_matrix()
    T[:3, 3] = p[:3]
    return T


def pixel_projections(Ts, s, d):
    """[E,9,2] projections and [E,9] depths of every patch pixel, from the
    world->camera matrices Ts [N,4,4] and inverse depths d [P]."""
    fx, fy, cx, cy = K
    u = s.patches[:, 0].reshape(-1, 9)[s.kk]
    v = s.patches[:, 1].reshape(-1, 9)[s.kk]
    z = np.broadcast_to(1.0 / d[s.kk][:, None], u.shape)
    pc = np.stack([(u - cx) / fx * z, (v - cy) / fy * z, z, np.ones_like(u)], -1)
    rel = np.einsum("eij,ejk->eik", Ts[s.jj], np.linalg.inv(Ts[s.ii]))
    q = np.einsum("eij,epj->epi", rel, pc)
    return np.stack([fx * q[..., 0] / q[..., 2] + cx, fy * q[..., 1] / q[..., 2] + cy], -1), q[..., 2]


def dense_full_patch_system(s, targets, fixed, lam_p, lam_d, h=1e-6):
    Ts = np.stack([mat(p) for p in s.poses])
    d = s.patches[:, 2, 1, 1].astype(np.float64)
    nf = s.N - fixed
    n = 6 * nf + s.P
    proj, z = pixel_projections(Ts, s, d)
    assert np.all(z > 0.1)  # no pixel masked
    r = (targets - proj).reshape(len(s.kk), 18)
    J = np.zeros((len(s.kk), 18, n))
    for a in range(nf):
        for m in range(6):
            xi = np.zeros(6)
            xi[m] = h
            Tp, Tm = Ts.copy(), Ts.copy()
            Tp[fixed + a] = twist(xi) @ Ts[fixed + a]
            Tm[fixed + a] = twist(-xi) @ Ts[fixed + a]
            J[:, :, 6 * a + m] = ((pixel_projections(Tp, s, d)[0] - pixel_projections(Tm, s, d)[0]) /
                                  (2 * h)).reshape(-1, 18)
    for k in range(s.P):
        dp, dm = d.copy(), d.copy()
        dp[k] += h
        dm[k] -= h
        J[:, :, 6 * nf + k] = ((pixel_projections(Ts, s, dp)[0] - pixel_projections(Ts, s, dm)[0]) /
                               (2 * h)).reshape(-1, 18)
    w = np.tile(s.weights, 9)  # [E,18]: the edge's (wx, wy) for every pixel
    H = np.einsum("eri,er,erj->ij", J, w, J)
    g = np.einsum("eri,er,er->i", J, w, r)
    H[np.arange(6 * nf), np.arange(6 * nf)] += lam_p
    H[np.arange(6 * nf, n), np.arange(6 * nf, n)] += lam_d
    return H, g


def noisy_targets(s, seed):
    Ts = np.stack([mat(p) for p in s.poses])
    proj, _ = pixel_projections(Ts, s, s.patches[:, 2, 1, 1].astype(np.float64))
    rng = np.random.default_rng(seed)
    # a shared flow correction per edge plus a little per-pixel noise
    return proj + rng.normal(0, 1.5, (len(s.kk), 1, 2)) + rng.normal(0, 0.2, proj.shape)


def test_step_matches_dense_library_solve_of_fd_system():
    s = small_graph(seed=3)
    fixed = 2
    opts = (1e-4, 1e-4, 0.1, 1e-3)
    t9 = noisy_targets(s, 0)
    H, g = dense_full_patch_system(s, t9, fixed, opts[0], opts[1])
    want = np.linalg.solve(H, g)
    r = oracle.gn(s, iters=1, fixed=fixed, opts=opts, targets=t9.reshape(-1, 3, 3, 2), pixels=9)
    got = np.r_[r["dxi"][0], r["dd"][0]]
    assert np.abs(got - want).max() < 1e-5 * np.abs(want).max(), np.abs(got - want).max()
    # the reduced pose system is the Schur complement of the full one
    nf6 = 6 * (s.N - fixed)
    S, y, Ct, w, cost = oracle.schur_system(s, fixed=fixed, opts=opts, targets=t9, pixels=9)
    Hpp, Hpd, Hdd = H[:nf6, :nf6], H[:nf6, nf6:], H[nf6:, nf6:]
    Sw = Hpp - Hpd @ np.linalg.solve(Hdd, Hpd.T)
    assert np.abs(S - Sw).max() < 1e-6 * np.abs(Sw).max()
    assert np.abs(Ct - np.diag(Hdd)).max() < 1e-6 * np.abs(Ct).max()
    Ts = np.stack([mat(p) for p in s.poses])
    proj, _ = pixel_projections(Ts, s, s.patches[:, 2, 1, 1].astype(np.float64))
    want_cost = np.sum(np.tile(s.weights, 9).reshape(-1, 9, 2) * (t9 - proj) ** 2)
    assert abs(cost - want_cost) < 1e-10 * want_cost


def test_cost_is_the_sum_of_the_pixels_centre_only_costs():
    # moving pixel q to the centre slot (patch and target) gives a centre-only
    # problem whose cost is that pixel's share of the whole-patch cost
    s = small_graph(seed=4)
    t9 = noisy_targets(s, 1)
    total = oracle.schur_system(s, fixed=2, targets=t9, pixels=9)[4]
    parts = 0.0
    for q in range(9):
        sq = small_graph(seed=4)
        pt = sq.patches.copy()
        pt[:, 0, 1, 1] = sq.patches[:, 0].reshape(-1, 9)[:, q]
        pt[:, 1, 1, 1] = sq.patches[:, 1].reshape(-1, 9)[:, q]
        parts += oracle.schur_system(sq, fixed=2, patches=pt, targets=t9[:, q])[4]
    assert abs(total - parts) < 1e-12 * total


def test_noise_free_whole_patch_targets_are_reached():
    s = scenes.noise_free(scenes.tiny(seed=4))
    t9 = scenes.full_patch_targets(s)
    r = oracle.gn(s, iters=10, targets=t9, pixels=9)
    rot, tr = pose_err(r["poses"], s.poses_gt)
    # float32 targets: the fixed point is ground truth to float32 rounding
    assert rot < 1e-6 and tr < 1e-6, (rot, tr)
    assert np.abs(r["patches"][:, 2, 1, 1] / s.depth_gt - 1).max() < 1e-5
    assert r["cost"][-1] < 1e-6 * r["cost"][0]


def test_dual_gradient_matches_central_fd():
    # exact derivatives of the unrolled whole-patch iterations with respect to
    # single pixel targets and edge weights, against central differences
    s = small_graph(seed=3, N=6, M=8)
    s.iters = 2
    s.targets = noisy_targets(s, 2)
    rng = np.random.default_rng(0)
    a = rng.normal(size=(s.N, 7))
    b = rng.normal(size=s.P)

    def L(targets=None, weights=None):
        r = oracle.gn(s, targets=targets, weights=weights, pixels=9)
        return (a * r["poses"]).sum() + (b * r["patches"][:, 2, 1, 1]).sum()

    kind = np.r_[np.zeros(10, int), np.ones(6, int)]
    index = np.r_[rng.choice(18 * s.E, 10, replace=False), rng.choice(2 * s.E, 6, replace=False)]
    g = oracle.grad_fwd(s, a, b, kind, index, pixels=9)
    eps = 1e-3
    for c in range(len(kind)):
        base = (s.targets if kind[c] == 0 else s.weights).copy()
        p, m = base.copy(), base.copy()
        p.reshape(-1)[index[c]] += eps
        m.reshape(-1)[index[c]] -= eps
        if kind[c] == 0:
            fd = (L(targets=p) - L(targets=m)) / (2 * eps)
        else:
            fd = (L(weights=p) - L(weights=m)) / (2 * eps)
        assert abs(g[c] - fd) <= 1e-5 * max(1.0, abs(fd)), (c, g[c], fd)
