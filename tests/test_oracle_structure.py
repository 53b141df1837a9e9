"""Pins for structure-only bundle adjustment (Sec. 3.3: with the poses held,
Eq. 3 is minimised over the patches' inverse depths only; here the oracle's
GN iteration with every pose fixed, fixed_poses = N).

* Under pure camera translations the reprojection is affine in the inverse
  depth (u' = u + fx tx d, v' = v + fy ty d, Eq. 2 with R = I and tz = 0), so
  an undamped GN step lands exactly on the depth the targets were made with,
  from any start, in one iteration.
* With rotations the step is the 1-D normal equation of each patch: checked
  against a central-difference Jacobian of a plain pinhole model written out
  here, and against the weighted least-squares closed form.
* The poses never move.
"""
import numpy as np
from scipy.spatial.transform import Rotation

import oracle
from test_oracle_pins import NOPT, mini_scene

K = (320.0, 320.0, 320.0, 240.0)


def project(pose_i, pose_j, u, v, d):
    """pinhole reprojection of pixel (u, v) at inverse depth d from frame i
    (world->camera pose (t, q)) into frame j"""
    fx, fy, cx, cy = K
    Ri, Rj = Rotation.from_quat(pose_i[3:]).as_matrix(), Rotation.from_quat(pose_j[3:]).as_matrix()
    pc = np.array([(u - cx) / fx, (v - cy) / fy, 1.0]) / d
    pw = Ri.T @ (pc - pose_i[:3])
    q = Rj @ pw + pose_j[:3]
    return np.array([fx * q[0] / q[2] + cx, fy * q[1] / q[2] + cy])


def test_translation_only_converges_in_one_undamped_step():
    ident = [0.0, 0.0, 0.0, 1.0]
    poses = [[0.0, 0.0, 0.0] + ident, [0.4, -0.1, 0.0] + ident, [-0.3, 0.25, 0.0] + ident]
    rng = np.random.default_rng(0)
    P = 6
    uvd = np.stack([rng.uniform(50, 590, P), rng.uniform(40, 440, P), rng.uniform(0.3, 2.0, P)], 1)
    d_true = rng.uniform(0.3, 2.0, P)
    edges, targets = [], []
    for k in range(P):
        for j in (1, 2):
            edges.append((0, k, j))
            targets.append(project(np.array(poses[0]), np.array(poses[j]), uvd[k, 0], uvd[k, 1], d_true[k]))
    s = mini_scene(poses, uvd, edges, targets=targets, fixed=3)
    r = oracle.gn(s, iters=1, fixed=3, opts=NOPT)
    assert np.allclose(r["patches"][:, 2, 1, 1], d_true, rtol=0, atol=1e-12)
    assert np.array_equal(r["poses"], np.asarray(poses))


def test_general_step_is_the_per_patch_normal_equation():
    rng = np.random.default_rng(1)
    N, P = 4, 5
    C = rng.normal(0, 0.3, (N, 3))
    # rotations small enough that the points stay in front of every camera
    R = Rotation.from_rotvec(rng.normal(0, 0.05, (N, 3))).as_matrix()
    R[0] = np.eye(3)
    poses = np.concatenate([-np.einsum("nij,nj->ni", R, C), Rotation.from_matrix(R).as_quat()], 1)
    uvd = np.stack([rng.uniform(200, 440, P), rng.uniform(150, 330, P), rng.uniform(0.3, 0.8, P)], 1)
    edges = [(0, k, j) for k in range(P) for j in range(1, N)]
    targets = np.array([project(poses[i], poses[j], uvd[k, 0], uvd[k, 1], uvd[k, 2]) for i, k, j in edges])
    targets += rng.normal(0, 2.0, targets.shape)
    weights = rng.uniform(0.5, 1.0, targets.shape)
    s = mini_scene(poses, uvd, edges, targets=targets, weights=weights, fixed=N)
    lam = 1e-4
    opts = (0.0, lam, 0.1, 1e-3)
    r = oracle.gn(s, iters=1, fixed=N, opts=opts)
    got = r["patches"][:, 2, 1, 1] - uvd[:, 2]
    for k in range(P):
        num = den = 0.0
        for e, (i, kk, j) in enumerate(edges):
            if kk != k:
                continue
            h = 1e-6
            jd = (project(poses[i], poses[j], uvd[k, 0], uvd[k, 1], uvd[k, 2] + h)
                  - project(poses[i], poses[j], uvd[k, 0], uvd[k, 1], uvd[k, 2] - h)) / (2 * h)
            res = targets[e] - project(poses[i], poses[j], uvd[k, 0], uvd[k, 1], uvd[k, 2])
            num += np.sum(weights[e] * jd * res)
            den += np.sum(weights[e] * jd * jd)
        assert abs(got[k] - num / (den + lam)) < 1e-6 * (1 + abs(num / den)), (k, got[k], num / (den + lam))
    assert np.array_equal(r["poses"], poses)
