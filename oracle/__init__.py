"""FP64 CPU oracle for patch-graph Gauss-Newton bundle adjustment.

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only ``tests/``, the smoke check in
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package.  The CUDA path never calls it and shares no code with it.

The numerical work lives in ``ba_oracle.cpp`` (plain C++, FP64, templated so
the same code runs on forward-mode dual numbers); this module only marshals
numpy arrays through ctypes.  What each entry point computes, with the passage
of arxiv 2408.01654 it follows:

* ``edge_terms``   Eq. 2 reprojection of each patch centre, residual against the
                   target and the analytic Jacobians in both poses and the
                   inverse depth (Sec. 3.1).
* ``schur_system`` the Gauss-Newton normal equations of Eq. 3 with the inverse
                   depths eliminated (Sec. 3.2 "Efficient Global Optimization",
                   appendix "Bundle-Adjustment Efficiency").
* ``gn``           whole Gauss-Newton iterations: linearise, Schur-eliminate,
                   Cholesky-solve the pose system, back-substitute the depths,
                   retract the poses on SE(3); with ``pixels=9`` every pixel
                   of the patch contributes its own 2-D residual (Eq. 3 over
                   the whole patch, 18 rows per edge).
* ``proximity_edges`` loop edges from camera proximity (Sec. 3.2 "Proximity
                   Loop Closure"): for each query frame the nearest older
                   camera centre within a radius, then uni-directional edges
                   from that frame's patches to the query frame, kept where
                   the Eq. 2 reprojection lies in front of the camera and
                   inside the image.
* ``patch_correlation`` Eq. 4 (Sec. 3.1 "Patch correlation"): for every edge
                   and patch pixel, dot products of the patch's correlation
                   features with the target frame's feature map bilinearly
                   sampled on a 7x7 grid of integer offsets around the
                   reprojected pixel (zero outside the map).
* ``pgo_lm``       Sim(3) pose-graph optimisation (Sec. 3.3 "Optimization",
                   Eqs. 5-7): smoothness factors log(dS^-1 Sa^-1 Sb) and loop
                   factors log(dS Sa^-1 Sb), Levenberg-Marquardt with
                   central-difference Jacobians and a dense Cholesky solve,
                   the first similarity held; with ``sim3_exp``/``sim3_log``
                   and ``pgo_residuals``.
* ``grad_fwd``     exact derivatives of a linear functional of the final state
                   with respect to single targets/weights (dual numbers through
                   the unrolled iterations).

Parity pins: every routine here is checked in ``tests/test_oracle_*.py``
against closed forms, finite differences, a library dense solve, the gauge
null space, world-frame equivariance and noise-free convergence; the paper
prints no worked example, so nothing is pinned to printed values.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ba_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")

# damping and clamps: lambda_p, lambda_d, z_min, d_min
DEFAULT_OPTS = (1e-4, 1e-4, 0.1, 1e-3)


def build(force: bool = False) -> str:
    """Compile the oracle (single-threaded, -O2, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", _LIB, _SRC])
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
    return _lib


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(st):
    if st == 1:
        raise ValueError("oracle: edge index out of range or patch with two source frames")
    if st == 4:
        raise np.linalg.LinAlgError("oracle: reduced pose system is not positive definite")
    if st:
        raise RuntimeError(f"oracle: status {st}")


def se3_retract(xi, pose):
    """T <- Exp(xi) T for one pose (t, q[x,y,z,w]), xi = (rho, phi)."""
    xi, pose = _d(xi), _d(pose)
    out = np.empty(7)
    lib().oracle_se3_retract(_p(xi), _p(pose), _p(out))
    return out


def quat_to_rot(q):
    q = _d(q)
    R = np.empty(9)
    lib().oracle_quat_to_rot(_p(q), _p(R))
    return R.reshape(3, 3)


def edge_terms(s, poses=None, patches=None, targets=None, z_min=DEFAULT_OPTS[2]):
    """Per-edge (proj [E,2], r [E,2], Ji [E,2,6], Jj [E,2,6], Jd [E,2], valid [E])."""
    poses = _d(s.poses if poses is None else poses)
    patches = _d(s.patches if patches is None else patches)
    targets = _d(s.targets if targets is None else targets)
    E = len(s.kk)
    proj, res = np.empty((E, 2)), np.empty((E, 2))
    Ji, Jj, Jd = np.empty((E, 2, 6)), np.empty((E, 2, 6)), np.empty((E, 2))
    valid = np.empty(E, np.int32)
    ii, jj, kk = _i(s.ii), _i(s.jj), _i(s.kk)
    _check(lib().oracle_edge_terms(
        s.N, s.P, E, _p(poses), _p(patches), _p(ii), _p(jj), _p(kk), _p(targets),
        _p(_d(s.intrinsics)), ctypes.c_double(z_min), _p(proj), _p(res), _p(Ji), _p(Jj), _p(Jd), _p(valid)))
    return proj, res, Ji, Jj, Jd, valid.astype(bool)


def schur_system(s, fixed=None, opts=DEFAULT_OPTS, poses=None, patches=None, targets=None, weights=None,
                 pixels=1):
    """Reduced pose system at the given state: (S [n,n], y [n], Ct [P], w [P], cost).
    pixels = 9: one residual per patch pixel, targets [E,9,2]."""
    fixed = s.fixed if fixed is None else fixed
    poses = _d(s.poses if poses is None else poses)
    patches = _d(s.patches if patches is None else patches)
    targets = _d(s.targets if targets is None else targets)
    weights = _d(s.weights if weights is None else weights)
    n = 6 * (s.N - fixed)
    S, y = np.empty((n, n)), np.empty(n)
    Ct, w = np.empty(s.P), np.empty(s.P)
    cost = ctypes.c_double()
    ii, jj, kk = _i(s.ii), _i(s.jj), _i(s.kk)
    if targets.size != 2 * pixels * len(s.kk):
        raise ValueError("targets: [E,2] for pixels = 1, [E,9,2] for pixels = 9")
    _check(lib().oracle_schur_system_px(
        s.N, s.P, len(s.kk), _p(poses), _p(patches), _p(ii), _p(jj), _p(kk), _p(targets), _p(weights),
        _p(_d(s.intrinsics)), fixed, _p(_d(opts)), pixels, _p(S), _p(y), _p(Ct), _p(w), ctypes.byref(cost)))
    return S, y, Ct, w, cost.value


def gn(s, iters=None, fixed=None, opts=DEFAULT_OPTS, poses=None, patches=None, targets=None, weights=None,
       pixels=1):
    """Run GN iterations from the scene's state.  Returns a dict with the final
    poses [N,7], patches [P,3,3,3], the per-iteration steps dxi [iters,n] and
    dd [iters,P], and the cost before each iteration plus after the last.
    pixels = 9: one residual per patch pixel (Eq. 3 over the whole patch),
    targets [E,9,2], the edge's weights shared by its nine residuals."""
    iters = s.iters if iters is None else iters
    fixed = s.fixed if fixed is None else fixed
    poses = _d(s.poses if poses is None else poses).copy()
    patches = _d(s.patches if patches is None else patches).copy()
    targets = _d(s.targets if targets is None else targets)
    weights = _d(s.weights if weights is None else weights)
    n = 6 * (s.N - fixed)
    dxi, dd, cost = np.empty((iters, n)), np.empty((iters, s.P)), np.empty(iters + 1)
    ii, jj, kk = _i(s.ii), _i(s.jj), _i(s.kk)
    if targets.size != 2 * pixels * len(s.kk):
        raise ValueError("targets: [E,2] for pixels = 1, [E,9,2] for pixels = 9")
    _check(lib().oracle_gn_px(
        s.N, s.P, len(s.kk), _p(poses), _p(patches), _p(ii), _p(jj), _p(kk), _p(targets), _p(weights),
        _p(_d(s.intrinsics)), iters, fixed, _p(_d(opts)), pixels, _p(dxi), _p(dd), _p(cost)))
    return {"poses": poses, "patches": patches, "dxi": dxi, "dd": dd, "cost": cost}


def gn_steps(s, iters=None, fixed=None, opts=DEFAULT_OPTS, pixels=1):
    """States after each GN iteration: list of (poses, depths) of length iters."""
    iters = s.iters if iters is None else iters
    out, poses, patches = [], s.poses, s.patches
    for _ in range(iters):
        r = gn(s, 1, fixed, opts, poses=poses, patches=patches, pixels=pixels)
        poses, patches = r["poses"], r["patches"]
        out.append((poses.copy(), patches[:, 2, 1, 1].copy()))
    return out


def grad_fwd(s, a, b, kind, index, iters=None, fixed=None, opts=DEFAULT_OPTS, pixels=1):
    """d/d(input coordinate) of <a, poses_final> + <b, depths_final>, one value
    per coordinate; kind 0 = target, 1 = weight (index into the flat [E,2]),
    2 = initial inverse depth (index = patch), 3 = left perturbation
    T <- Exp(xi) T of an initial pose (index = 6 * pose + component of
    xi = (rho, phi))."""
    iters = s.iters if iters is None else iters
    fixed = s.fixed if fixed is None else fixed
    kind = _i(kind)
    index = np.ascontiguousarray(index, dtype=np.int64)
    out = np.empty(len(kind))
    ii, jj, kk = _i(s.ii), _i(s.jj), _i(s.kk)
    _check(lib().oracle_grad_fwd_px(
        s.N, s.P, len(s.kk), _p(_d(s.poses)), _p(_d(s.patches)), _p(ii), _p(jj), _p(kk), _p(_d(s.targets)),
        _p(_d(s.weights)), _p(_d(s.intrinsics)), iters, fixed, _p(_d(opts)), pixels, _p(_d(a)), _p(_d(b)),
        len(kind), _p(kind), _p(index), _p(out)))
    return out


def block_keys(ii, jj, fixed):
    """Canonical pose-pose block keys of the reduced system's B part: the sorted
    unique (a, b), a <= b, over (i,i), (j,j), (min, max) of every non-self edge,
    both poses free (index >= fixed).  Plain Python, for bit-exact checks."""
    keys = set()
    for i, j in zip(np.asarray(ii).tolist(), np.asarray(jj).tolist()):
        if i == j:
            continue
        for a, b in ((i, i), (j, j), (min(i, j), max(i, j))):
            if a >= fixed and b >= fixed:
                keys.add((a, b))
    return np.array(sorted(keys), dtype=np.int32).reshape(-1, 2)


def proximity_edges(poses, patches, intrinsics, M, b0, b1, gap=30, radius=2.0, z_min=DEFAULT_OPTS[2],
                    width=640.0, height=480.0, cap=None):
    """Proximity loop edges for the query frames b0 <= b < b1 (the rule is
    stated beside ``oracle_proximity_edges`` in ba_oracle.cpp).  poses [N,7]
    world->camera, patches [N*M,3,3,3] (patch a*M + m belongs to frame a).
    Returns a dict: match [Q] (selected old frame or -1), dist [Q] (nearest
    candidate distance or -1), margin [Q] (scaled distance of the query's
    closest decision from its threshold), ii, jj, kk [n] int32 and coords
    [n,2] float64, ordered by query frame then patch."""
    poses = _d(poses)
    patches = _d(patches)
    N = len(poses)
    if patches.shape[0] != N * M:
        raise ValueError("patches must hold M patches per frame")
    Q = max(0, b1 - b0)
    cap = Q * M if cap is None else cap
    match, dist, margin = np.empty(Q, np.int32), np.empty(Q), np.empty(Q)
    ii, jj, kk = np.empty(cap, np.int32), np.empty(cap, np.int32), np.empty(cap, np.int32)
    coords = np.empty((cap, 2))
    n = ctypes.c_longlong()
    _check(lib().oracle_proximity_edges(
        N, M, _p(poses), _p(patches), _p(_d(intrinsics)), b0, b1, gap, ctypes.c_double(radius),
        ctypes.c_double(z_min), ctypes.c_double(width), ctypes.c_double(height), _p(match), _p(dist),
        _p(margin), _p(ii), _p(jj), _p(kk), _p(coords), ctypes.c_longlong(cap), ctypes.byref(n)))
    m = min(n.value, cap)
    return {"match": match, "dist": dist, "margin": margin, "ii": ii[:m], "jj": jj[:m], "kk": kk[:m],
            "coords": coords[:m], "n": n.value}


def patch_correlation(fmap, gmap, kk, jj, coords, radius=3, bound=False):
    """Eq. 4 correlation volume: fmap [Nf,H,W,D] and gmap [P,p,p,D] float32
    (channels last), kk/jj [E] (patch, target frame), coords [E,p,p,2] float32
    (x, y) in feature-map pixels.  Returns C [E,p,p,2R+1,2R+1] float64 (row
    offset, then column offset), and with ``bound`` also the same sums of
    |g||f| (the scale of any summation order's rounding error)."""
    fmap = np.ascontiguousarray(fmap, dtype=np.float32)
    gmap = np.ascontiguousarray(gmap, dtype=np.float32)
    coords = np.ascontiguousarray(coords, dtype=np.float32)
    kk, jj = _i(kk), _i(jj)
    Nf, H, W, D = fmap.shape
    P, p = gmap.shape[0], gmap.shape[1]
    E = len(kk)
    G = 2 * radius + 1
    out = np.empty((E, p, p, G, G))
    bnd = np.empty((E, p, p, G, G)) if bound else None
    _check(lib().oracle_patch_correlation(
        Nf, H, W, D, P, p, E, _p(fmap), _p(gmap), _p(kk), _p(jj), _p(coords), radius, _p(out),
        _p(bnd) if bound else None))
    return (out, bnd) if bound else out


def sim3_exp(xi):
    """Exp of a Sim(3) tangent vector (rho, phi, sigma) [7] -> (t, q xyzw, s) [8]."""
    out = np.empty(8)
    lib().oracle_sim3_exp(_p(_d(xi)), _p(out))
    return out


def sim3_log(S):
    """Log of a similarity (t, q xyzw, s) [8] -> (rho, phi, sigma) [7]."""
    out = np.empty(7)
    lib().oracle_sim3_log(_p(_d(S)), _p(out))
    return out


def pgo_residuals(S, dS, fa, fb, loop):
    """[F,7] factor residuals (Eq. 5 for loop = 0, Eq. 6 for loop = 1) at the
    similarities S [N,8], measurements dS [F,8], factor endpoints fa/fb [F]."""
    S, dS = _d(S), _d(dS)
    fa, fb, loop = _i(fa), _i(fb), _i(loop)
    r = np.empty((len(fa), 7))
    lib().oracle_pgo_residuals(len(S), len(fa), _p(S), _p(dS), _p(fa), _p(fb), _p(loop), _p(r))
    return r


def pgo_lm(S, dS, fa, fb, loop, iters=20, lambda0=1e-4, h=1e-6):
    """Levenberg-Marquardt on Eq. 7 from the similarities S [N,8] (S[0] held).
    Returns dict(S [N,8], cost [iters+1], accepted [iters])."""
    S = _d(S).copy()
    dS = _d(dS)
    fa, fb, loop = _i(fa), _i(fb), _i(loop)
    cost = np.empty(iters + 1)
    acc = np.empty(iters, np.int32)
    _check(lib().oracle_pgo_lm(len(S), len(fa), _p(S), _p(dS), _p(fa), _p(fb), _p(loop), iters,
                               ctypes.c_double(lambda0), ctypes.c_double(h), _p(cost), _p(acc)))
    return dict(S=S, cost=cost, accepted=acc.astype(bool))
