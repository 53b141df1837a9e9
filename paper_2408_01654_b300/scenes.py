"""Seeded synthetic patch-graph scenes shaped like the paper's workloads.

This module only *synthesises inputs*.  It holds none of the bundle-adjustment
arithmetic (no residual, Jacobian, normal equation, Schur step or SE(3)
retraction): ground-truth targets come from a plain 4x4-matrix camera model
(camera-to-world matrices, world points, pinhole projection) and every rotation
goes through ``scipy.spatial.transform.Rotation``.  Both the CUDA path and the
FP64 oracle consume what it returns, so it is the only code they share.

Conventions of the returned arrays (the library's input layout):

* ``poses``   float64 [N,7]  world->camera (tx,ty,tz,qx,qy,qz,qw)
* ``patches`` float32 [P,3,3,3]  channels (x, y, inverse depth), 3x3 pixels;
  the centre pixel is ``[:, :, 1, 1]`` and all nine pixels share one inverse
  depth (the paper's patch, Sec. 3.1 Eq. 1, with p = 3)
* ``ii, jj, kk`` int32 [E]  edge (i,k,j): patch ``kk`` of frame ``ii`` seen in
  frame ``jj`` (Sec. 3.1, the patch graph)
* ``targets`` float32 [E,2] pixels, ``weights`` float32 [E,2] (Eq. 3)
* ``intrinsics`` float32 [4] (fx, fy, cx, cy)

Workloads (patches per frame, patch size, camera and noise model as the paper's
DPVO setting: 96 random patches per frame, Sec. 3.1 and Sec. 3.3):

* ``tiny``      8 frames, each patch -> the 6 nearest other frames
* ``odometry``  22 frames, each patch -> the 13 nearest other frames
                ("patch lifetime 13"), 8% outliers
* ``global``    1000 frames, local edges within +-6 frames plus proximity loop
                edges (old patches -> recent frame, Sec. 3.2)
* ``batched``   many problems with log-uniform frame counts in [8, 400] and the
                ``global`` edge rules
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy.spatial.transform import Rotation

WIDTH, HEIGHT = 640, 480
FX = FY = 320.0
CX, CY = 320.0, 240.0
PATCHES_PER_FRAME = 96


@dataclass
class Scene:
    name: str
    seed: int
    N: int
    P: int
    E: int
    fixed: int
    iters: int
    poses: np.ndarray          # float64 [N,7] initial (perturbed) poses
    patches: np.ndarray        # float32 [P,3,3,3] initial patches
    ii: np.ndarray             # int32 [E]
    jj: np.ndarray             # int32 [E]
    kk: np.ndarray             # int32 [E]
    targets: np.ndarray        # float32 [E,2]
    weights: np.ndarray        # float32 [E,2]
    intrinsics: np.ndarray     # float32 [4]
    poses_gt: np.ndarray       # float64 [N,7]
    depth_gt: np.ndarray       # float64 [P]  ground-truth inverse depth
    proj_gt: np.ndarray        # float64 [E,2] noise-free ground-truth projections
    info: dict = field(default_factory=dict)


# --------------------------------------------------------------------------- #
# small helpers (input synthesis only)
# --------------------------------------------------------------------------- #
def _unit(rng: np.random.Generator, n: int) -> np.ndarray:
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _random_walk(rng: np.random.Generator, n: int, step_m=0.1, step_deg=2.0):
    """Camera-to-world 4x4 matrices: G_0 = I, G_{i+1} = G_i * D_i, where D_i
    rotates 2 degrees about a uniformly random axis and translates 0.1 m along
    a uniformly random direction."""
    G = np.zeros((n, 4, 4))
    G[0] = np.eye(4)
    axes = _unit(rng, n)
    dirs = _unit(rng, n)
    for i in range(1, n):
        D = np.eye(4)
        D[:3, :3] = Rotation.from_rotvec(math.radians(step_deg) * axes[i]).as_matrix()
        D[:3, 3] = step_m * dirs[i]
        G[i] = G[i - 1] @ D
    return G


def _world_to_camera(G: np.ndarray):
    """Invert camera-to-world matrices; return (R [n,3,3], t [n,3])."""
    R = np.transpose(G[:, :3, :3], (0, 2, 1))
    t = -np.einsum("nij,nj->ni", R, G[:, :3, 3])
    return R, t


def _pose_vec(R: np.ndarray, t: np.ndarray) -> np.ndarray:
    q = Rotation.from_matrix(R).as_quat()  # (x, y, z, w)
    q = np.where(q[:, 3:4] < 0, -q, q)
    return np.concatenate([t, q], axis=1).astype(np.float64)


def _camera_points(u, v, d):
    """Points in the source camera for pixels (u,v) at inverse depth d."""
    z = 1.0 / d
    return np.stack([(u - CX) / FX * z, (v - CY) / FY * z, z], axis=-1)


def _project(Rw2c, tw2c, pw):
    """Pinhole projection of world points pw [E,3] with per-edge world->camera
    (R [E,3,3], t [E,3]).  Returns (uv [E,2], z [E])."""
    pc = np.einsum("eij,ej->ei", Rw2c, pw) + tw2c
    z = pc[:, 2]
    with np.errstate(divide="ignore", invalid="ignore"):
        uv = np.stack([FX * pc[:, 0] / z + CX, FY * pc[:, 1] / z + CY], axis=1)
    return uv, z


def _shifted_window(i: int, n: int, size: int) -> list[int]:
    """The `size`-frame window around i, shifted to stay inside [0, n),
    without i itself (the `size`-1 nearest other frames)."""
    size = min(size, n)
    lo = min(max(i - (size - 1) // 2, 0), n - size)
    return [j for j in range(lo, lo + size) if j != i]


def _clipped_window(i: int, n: int, radius: int) -> list[int]:
    return [j for j in range(max(0, i - radius), min(n, i + radius + 1)) if j != i]


# --------------------------------------------------------------------------- #
# scene assembly
# --------------------------------------------------------------------------- #
def _build(name, seed, N, neighbours, fixed, iters, outlier_frac=0.0,
           loop=False, rng=None) -> Scene:
    rng = np.random.default_rng(seed) if rng is None else rng
    M = PATCHES_PER_FRAME
    P = N * M

    G = _random_walk(rng, N)
    Rgt, tgt = _world_to_camera(G)
    poses_gt = _pose_vec(Rgt, tgt)

    # patch centres are rounded to float32 first so that the stored patches
    # and the ground-truth geometry agree exactly
    u = rng.uniform(1.0, WIDTH - 1.0, size=P).astype(np.float32).astype(np.float64)
    v = rng.uniform(1.0, HEIGHT - 1.0, size=P).astype(np.float32).astype(np.float64)
    dgt = rng.uniform(0.2, 2.0, size=P)
    src = np.repeat(np.arange(N), M)
    pcam = _camera_points(u, v, dgt)
    pw = np.einsum("pij,pj->pi", G[src, :3, :3], pcam) + G[src, :3, 3]

    # local edges: patch-major, targets ascending within a patch
    kk_l, jj_l = [], []
    for i in range(N):
        js = neighbours(i, N)
        ks = np.arange(i * M, (i + 1) * M)
        kk_l.append(np.repeat(ks, len(js)))
        jj_l.append(np.tile(np.asarray(js, dtype=np.int64), M))
    kk = np.concatenate(kk_l) if kk_l else np.zeros(0, np.int64)
    jj = np.concatenate(jj_l) if jj_l else np.zeros(0, np.int64)
    n_local = len(kk)

    if loop:
        # proximity loop edges (Sec. 3.2): for each frame b, the nearest
        # (ground-truth camera centre) frame a with b - a > 30 closer than
        # 2 m; all patches of a get a uni-directional edge a -> b.
        centres = G[:, :3, 3]
        lk, lj = [], []
        for b in range(N):
            cand = np.arange(0, max(0, b - 30))
            if len(cand) == 0:
                continue
            dist = np.linalg.norm(centres[cand] - centres[b], axis=1)
            a = int(cand[np.argmin(dist)])
            if dist.min() >= 2.0:
                continue
            lk.append(np.arange(a * M, (a + 1) * M))
            lj.append(np.full(M, b))
        if lk:
            kk = np.concatenate([kk] + lk)
            jj = np.concatenate([jj] + lj)
    ii = src[kk]

    uv, z = _project(Rgt[jj], tgt[jj], pw[kk])
    keep = z > 0.1
    if loop:
        inside = (uv[:, 0] >= 0) & (uv[:, 0] < WIDTH) & (uv[:, 1] >= 0) & (uv[:, 1] < HEIGHT)
        is_loop = np.arange(len(kk)) >= n_local
        keep &= ~is_loop | inside
    ii, jj, kk, uv = ii[keep], jj[keep], kk[keep], uv[keep]
    n_loop = int(np.count_nonzero(np.arange(len(keep))[keep] >= n_local))

    # sort edges by (kk, jj): the natural patch-major order of a patch graph
    order = np.lexsort((jj, kk))
    ii, jj, kk, uv = ii[order], jj[order], kk[order], uv[order]
    E = len(kk)

    targets = uv + rng.normal(0.0, 0.5, size=(E, 2))
    weights = rng.uniform(0.5, 1.0, size=(E, 2))
    n_out = 0
    if outlier_frac > 0:
        out = rng.random(E) < outlier_frac
        n_out = int(out.sum())
        ang = rng.uniform(0, 2 * np.pi, size=n_out)
        mag = rng.uniform(5.0, 30.0, size=n_out)
        targets[out] += np.stack([np.cos(ang), np.sin(ang)], 1) * mag[:, None]
        weights[out] = 0.05

    # initial state: free poses perturbed 0.05 rad / 0.05 m, depths log-normal
    Rin, tin = Rgt.copy(), tgt.copy()
    free = np.arange(fixed, N)
    if len(free):
        rot = Rotation.from_rotvec(0.05 * _unit(rng, len(free))).as_matrix()
        Rin[free] = rot @ Rgt[free]
        tin[free] = tgt[free] + 0.05 * _unit(rng, len(free))
    poses = _pose_vec(Rin, tin)
    poses[:fixed] = poses_gt[:fixed]
    d0 = dgt * np.exp(rng.normal(0.0, 0.1, size=P))

    patches = np.empty((P, 3, 3, 3), np.float32)
    off = np.array([-1.0, 0.0, 1.0])
    patches[:, 0] = (u[:, None, None] + off[None, None, :]).astype(np.float32)
    patches[:, 1] = (v[:, None, None] + off[None, :, None]).astype(np.float32)
    patches[:, 2] = d0[:, None, None].astype(np.float32)

    return Scene(
        name=name, seed=seed, N=N, P=P, E=E, fixed=fixed, iters=iters,
        poses=poses, patches=patches,
        ii=ii.astype(np.int32), jj=jj.astype(np.int32), kk=kk.astype(np.int32),
        targets=targets.astype(np.float32), weights=weights.astype(np.float32),
        intrinsics=np.array([FX, FY, CX, CY], np.float32),
        poses_gt=poses_gt, depth_gt=dgt, proj_gt=uv,
        info={"local_edges": E - n_loop, "loop_edges": n_loop, "outliers": n_out},
    )


def tiny(seed: int = 0) -> Scene:
    """8 frames, 96 patches/frame, each patch -> 6 nearest other frames
    (about 4.6k edges), first 2 poses fixed, 2 GN iterations."""
    return _build("tiny", seed, 8, lambda i, n: _shifted_window(i, n, 7), 2, 2)


def odometry(seed: int = 0) -> Scene:
    """Odometry window: 22 keyframes, patch lifetime 13 (about 27k edges),
    8% outlier targets offset U[5,30] px with weight 0.05, 2 GN iterations."""
    return _build("odometry", seed, 22, lambda i, n: _shifted_window(i, n, 14),
                  2, 2, outlier_frac=0.08)


def window(seed: int = 0, N: int = 22) -> Scene:
    """Odometry-style window of N keyframes: patch lifetime 13 (each patch
    linked to the 13 frames of a 14-frame window around its source), no
    outliers, 2 GN iterations, 2 fixed poses (the graph-size sweep of the
    dense and block-sparse forms)."""
    return _build("window", seed, N, lambda i, n: _shifted_window(i, n, 14), 2, 2)


def global_ba(seed: int = 0, N: int = 1000) -> Scene:
    """Global loop-closure BA: 1000 keyframes, local edges within +-6 frames
    plus proximity loop edges, 4 GN iterations."""
    return _build("global", seed, N, lambda i, n: _clipped_window(i, n, 6),
                  2, 4, loop=True)


def batched(seed: int = 0, B: int = 64, lo: int = 8, hi: int = 400) -> list[Scene]:
    """Independent problems with frame counts round(exp(U[ln lo, ln hi])) and
    the global edge rules, 4 GN iterations each."""
    rng = np.random.default_rng(seed)
    Ns = np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), size=B))).astype(int)
    return [_build("batched", seed * 1000 + b, int(n), lambda i, m: _clipped_window(i, m, 6),
                   2, 4, loop=True) for b, n in enumerate(Ns)]


def noise_free(scene: Scene) -> Scene:
    """Copy of a scene whose targets are the exact ground-truth projections
    (float64; a float32 cast of them is the GPU input) and whose first `fixed`
    poses sit at ground truth."""
    s = Scene(**{k: getattr(scene, k) for k in scene.__dataclass_fields__})
    s.targets = scene.proj_gt.copy()
    s.info = dict(scene.info, noise_free=True)
    return s


WORKLOADS = {"tiny": tiny, "odometry": odometry, "global": global_ba}


def correlation_inputs(scene: Scene, D: int = 128, scale: int = 4, noise_px: float = 1.0, seed: int = 0) -> dict:
    """Inputs of the patch correlation (Eq. 4) for a scene's edges, at the
    feature maps' 1/``scale`` resolution (DPVO's maps are 1/4 of the frame,
    Sec. 3.1 "Patch extraction"):

    * ``fmap``   float32 [N, HEIGHT/scale, WIDTH/scale, D]: random N(0, 1/D)
      feature maps (channels last), one per frame;
    * ``gmap``   float32 [P, 3, 3, D]: random patch features, same scale;
    * ``coords`` float32 [E, 3, 3, 2]: where each of the nine pixels of the
      edge's patch (the 3x3 grid one feature-map pixel apart around the patch
      centre) lands in the target frame (ground-truth camera model at the
      ground-truth inverse depth, as ``proj_gt`` for the centre), divided by
      ``scale``, plus N(0, (noise_px/scale)^2) per axis -- the estimate's
      drift.

    D = 128 float32 channels is the size that matches the paper's storage
    figure for patch features (~0.6 GB per 1000 frames with 96 patches of
    3x3 pixels, plus the context features)."""
    rng = np.random.default_rng(seed)
    N, P, E = scene.N, scene.P, scene.E
    Hf, Wf = HEIGHT // scale, WIDTH // scale
    fmap = rng.standard_normal((N, Hf, Wf, D), dtype=np.float32) / np.float32(math.sqrt(D))
    gmap = rng.standard_normal((P, 3, 3, D), dtype=np.float32) / np.float32(math.sqrt(D))
    Rq = Rotation.from_quat(scene.poses_gt[:, 3:]).as_matrix()  # world -> camera
    t = scene.poses_gt[:, :3]
    ii, jj, kk = scene.ii.astype(np.int64), scene.jj.astype(np.int64), scene.kk.astype(np.int64)
    uc = scene.patches[kk, 0, 1, 1].astype(np.float64)
    vc = scene.patches[kk, 1, 1, 1].astype(np.float64)
    d = scene.depth_gt[kk]
    off = np.array([-1.0, 0.0, 1.0]) * scale  # the patch's pixels are one feature-map pixel apart
    u = np.broadcast_to(uc[:, None, None] + off[None, None, :], (E, 3, 3))
    v = np.broadcast_to(vc[:, None, None] + off[None, :, None], (E, 3, 3))
    pc = _camera_points(u, v, np.broadcast_to(d[:, None, None], (E, 3, 3)))       # [E,3,3,3] in frame i
    pw = np.einsum("eji,evuj->evui", Rq[ii], pc - t[ii][:, None, None, :])           # R_i^T (p - t_i)
    pcj = np.einsum("eij,evuj->evui", Rq[jj], pw) + t[jj][:, None, None, :]
    z = pcj[..., 2]
    with np.errstate(divide="ignore", invalid="ignore"):
        x = FX * pcj[..., 0] / z + CX
        y = FY * pcj[..., 1] / z + CY
    coords = np.stack([x, y], -1) / scale + rng.normal(0.0, noise_px / scale, size=(E, 3, 3, 2))
    coords = np.where(np.isfinite(coords), coords, -1.0e4).astype(np.float32)
    return {"fmap": fmap, "gmap": gmap, "coords": coords}


def _sim_matrix(R: np.ndarray, t: np.ndarray, s: float) -> np.ndarray:
    M = np.eye(4)
    M[:3, :3] = s * R
    M[:3, 3] = t
    return M


def _sim_vec(M: np.ndarray) -> np.ndarray:
    """4x4 similarity matrix -> (t, q xyzw, s)."""
    s = float(np.cbrt(np.linalg.det(M[:3, :3])))
    return np.concatenate([M[:3, 3], Rotation.from_matrix(M[:3, :3] / s).as_quat(), [s]])


def pose_graph(seed: int = 0, N: int = 1000, laps: float = 2.0, loop_every: int = 40, loop_noise: float = 0.0,
               drift_scale: float = 0.3, odo_rot_deg: float = 0.1, odo_trans: float = 0.01) -> dict:
    """A Sim(3) pose graph shaped like the classical backend's (Sec. 3.3
    "Optimization"): N keyframes along a trajectory that circles the same
    ground `laps` times, a smoothness factor between consecutive keyframes
    and loop factors between keyframes one lap apart.

    The true similarities S*_i carry a slowly varying scale (the odometry's
    scale drift, exp(drift_scale sin(2 pi i / N))).  The odometry estimate
    composes the true relative motions with the scale ratio removed and small
    rotation / relative-translation noise, and starts every keyframe at scale
    1 (the paper's initialisation).  Smoothness measurements are the
    estimate's own relative motions; loop measurements the inverse true
    relative similarity (the Eq. 6 convention) with optional noise.

    Plain 4x4 matrices and scipy rotations only.  Returns dict(S [N,8] the
    start, gt [N,8] the true similarities, dS [F,8], fa, fb, loop int32 [F]);
    similarities are (tx, ty, tz, qx, qy, qz, qw, s) mapping x to s R x + t."""
    rng = np.random.default_rng(seed)
    u = np.arange(N) / N
    ang = 2 * np.pi * laps * u
    pos = np.stack([20 * np.cos(ang), 20 * np.sin(ang), 0.5 * np.sin(3 * ang)], 1)
    rot = Rotation.from_euler("zyx", np.stack([ang + np.pi / 2, 0.05 * np.sin(5 * ang), 0.03 * np.cos(7 * ang)], 1))
    scale = np.exp(drift_scale * np.sin(2 * np.pi * u))
    gt = np.stack([_sim_matrix(rot[i].as_matrix(), pos[i], scale[i]) for i in range(N)])
    est = [_sim_matrix(gt[0][:3, :3] / scale[0], gt[0][:3, 3], 1.0)]
    for i in range(N - 1):
        rel = np.linalg.inv(gt[i]) @ gt[i + 1]
        s = np.cbrt(np.linalg.det(rel[:3, :3]))
        R = Rotation.from_rotvec(np.deg2rad(odo_rot_deg) * rng.normal(size=3)).as_matrix() @ (rel[:3, :3] / s)
        t = rel[:3, 3] * (1 + odo_trans * rng.normal()) + odo_trans * np.linalg.norm(rel[:3, 3]) * rng.normal(size=3)
        est.append(est[-1] @ _sim_matrix(R, t, 1.0))
    fa, fb, loop, dS = [], [], [], []
    for i in range(N - 1):
        fa.append(i), fb.append(i + 1), loop.append(0)
        dS.append(_sim_vec(np.linalg.inv(est[i]) @ est[i + 1]))
    lap = int(round(N / laps)) if laps > 1 else N - 1
    for j in range(0, N - lap, max(1, loop_every)):
        k = j + lap
        meas = np.linalg.inv(np.linalg.inv(gt[j]) @ gt[k])
        if loop_noise:
            R = Rotation.from_rotvec(loop_noise * rng.normal(size=3)).as_matrix()
            meas = _sim_matrix(R, loop_noise * rng.normal(size=3), float(np.exp(loop_noise * rng.normal()))) @ meas
        fa.append(j), fb.append(k), loop.append(1), dS.append(_sim_vec(meas))
    i32 = lambda a: np.asarray(a, np.int32)  # noqa: E731
    return dict(S=np.stack([_sim_vec(M) for M in est]), gt=np.stack([_sim_vec(M) for M in gt]),
                dS=np.asarray(dS), fa=i32(fa), fb=i32(fb), loop=i32(loop))


def full_patch_targets(scene: Scene) -> np.ndarray:
    """Targets for the whole-patch residual (Eq. 3 summed over all nine
    pixels of each patch): float32 [E,3,3,2], pixel (v, u) of edge e's
    patch at its ground-truth inverse depth projected into frame jj with
    the ground-truth poses, plus the edge's own centre offset (noise and
    outlier displacement, targets - proj_gt), which the nine pixels share as
    they share the update operator's flow correction."""
    R = Rotation.from_quat(scene.poses_gt[:, 3:]).as_matrix()
    t = scene.poses_gt[:, :3]
    px = scene.patches[:, 0].reshape(-1, 9).astype(np.float64)[scene.kk]  # [E,9]
    py = scene.patches[:, 1].reshape(-1, 9).astype(np.float64)[scene.kk]
    d = np.broadcast_to(scene.depth_gt[scene.kk][:, None], px.shape)
    pc = _camera_points(px, py, d)                                          # [E,9,3] in frame ii
    Ri, ti, Rj, tj = R[scene.ii], t[scene.ii], R[scene.jj], t[scene.jj]
    pw = np.einsum("eji,epj->epi", Ri, pc - ti[:, None, :])                 # R_i^T (pc - t_i)
    q = np.einsum("eij,epj->epi", Rj, pw) + tj[:, None, :]
    with np.errstate(divide="ignore", invalid="ignore"):
        uv = np.stack([FX * q[..., 0] / q[..., 2] + CX, FY * q[..., 1] / q[..., 2] + CY], -1)
    off = scene.targets.astype(np.float64) - scene.proj_gt
    return (uv + off[:, None, :]).reshape(-1, 3, 3, 2).astype(np.float32)
