"""GPU parity: the CUDA path against the FP64 oracle, element by element.

Floating point is compared at the FP32 path's stated tolerance (1e-5 relative
on poses and depths per GN step; rotation in radians, translation relative to
max(1, |t|)); graph indexing is compared bit-exactly against its definition.
All inputs come from the seeded scene generator; nothing here reads values
produced by the CUDA path into the oracle.
"""
import copy

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2408_01654_b300 import capi, scenes  # noqa: E402
from paper_2408_01654_b300.ba import DPVBA, scene_tensors  # noqa: E402

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_01654_b300 import build
    build.build()
    oracle.build()


def pose_error(a, b):
    """max rotation error (rad) and translation error relative to max(1, |t|)."""
    rot = (Rotation.from_quat(a[:, 3:]) * Rotation.from_quat(b[:, 3:]).inv()).magnitude()
    tr = np.linalg.norm(a[:, :3] - b[:, :3], axis=1) / np.maximum(1.0, np.linalg.norm(b[:, :3], axis=1))
    return rot.max(), tr.max()


def depth_error(a, b):
    return np.max(np.abs(a - b) / np.abs(b))


def bind(scene, **opts):
    T = scene_tensors(scene)
    ba = DPVBA(**opts)
    ba.set_graph(**T)
    return ba, T


def sizes_case(name):
    if name == "tiny":
        return scenes.tiny(seed=0)
    if name == "odometry":
        return scenes.odometry(seed=0)
    raise KeyError(name)


# --------------------------------------------------------------------------- #
# graph indexing: bit-exact
# --------------------------------------------------------------------------- #
@pytest.mark.parametrize("case", ["tiny", "odometry"])
@pytest.mark.parametrize("G", [0, 8, 32])
@pytest.mark.parametrize("shuffle", [False, True])
def test_indexing_bit_exact(case, G, shuffle):
    # these graphs fit one co-resident wave: the fused binding kernel
    check_indexing(sizes_case(case), G, shuffle)


@pytest.mark.parametrize("shuffle", [False, True])
def test_indexing_bit_exact_separate_launches(shuffle):
    # 200 keyframes with loop edges: ~240k edges in 600 groups of 32, more
    # than one co-resident wave of the fused kernel, so one launch per step
    s = scenes.global_ba(0, N=200)
    assert s.E > 256 * 600
    check_indexing(s, 32, shuffle, keys=False)


def check_indexing(s, G, shuffle, keys=True):
    if shuffle:  # unsorted input takes the device-side kk sort
        order = np.random.default_rng(1).permutation(s.E)
        for f in ("ii", "jj", "kk", "targets", "weights"):
            setattr(s, f, getattr(s, f)[order].copy())
    ba, T = bind(s, patches_per_group=G)
    inf = ba.info()
    Gr = inf["G"]
    perm = ba.export(capi.EXPORT_PERM).cpu().numpy()
    want = np.lexsort((s.kk % Gr, s.jj, s.ii, s.kk // Gr))  # stable sort by (group, ii, jj, patch-in-group)
    assert np.array_equal(perm, want)
    ng = inf["groups"]
    gptr = ba.export(capi.EXPORT_GPTR).cpu().numpy()
    assert np.array_equal(gptr, np.searchsorted(s.kk[want] // Gr, np.arange(ng + 1)))
    win = ba.export(capi.EXPORT_WIN).cpu().numpy().reshape(ng, capi.WMAX)
    slots = ba.export(capi.EXPORT_SLOTS).cpu().numpy().view(np.uint32)
    for g in range(ng):
        e = want[gptr[g]:gptr[g + 1]]
        frames = np.unique(np.r_[s.ii[e], s.jj[e]])
        assert np.array_equal(win[g, :len(frames)], frames)
        assert np.all(win[g, len(frames):] == -1)
        sw = slots[gptr[g]:gptr[g + 1]]
        assert np.array_equal(frames[sw & 0xff], s.ii[e])
        assert np.array_equal(frames[(sw >> 8) & 0xff], s.jj[e])
        assert np.array_equal(sw >> 16, s.kk[e] % Gr)
    # patch-major order: the stable sort of the input by kk; CSR per patch
    pm = ba.export(capi.EXPORT_PMPOS).cpu().numpy()
    pos_kk = np.empty(s.E, np.int64)
    pos_kk[np.argsort(s.kk, kind="stable")] = np.arange(s.E)
    assert np.array_equal(pm, pos_kk[want])
    pptr = ba.export(capi.EXPORT_PPTR).cpu().numpy()
    assert np.array_equal(pptr, np.searchsorted(np.sort(s.kk), np.arange(s.P + 1)))
    # runs: one per distinct (group, ii, jj)
    key = np.c_[s.kk[want] // Gr, s.ii[want], s.jj[want]]
    assert inf["runs"] == 1 + np.count_nonzero(np.any(key[1:] != key[:-1], axis=1))
    for fixed in (0, 2) if keys else ():
        got = ba.block_keys(fixed).cpu().numpy()
        assert np.array_equal(got, oracle.block_keys(s.ii, s.jj, fixed))


# --------------------------------------------------------------------------- #
# linear system at the initial state
# --------------------------------------------------------------------------- #
@pytest.mark.parametrize("case", ["tiny", "odometry"])
def test_reduced_system_matches_oracle(case):
    s = sizes_case(case)
    ba, T = bind(s)
    ba.linearize(s.fixed)
    S = ba.export(capi.EXPORT_S).cpu().numpy().astype(np.float64)
    y = ba.export(capi.EXPORT_Y).cpu().numpy().astype(np.float64)
    Ct = ba.export(capi.EXPORT_CT).cpu().numpy()
    w = ba.export(capi.EXPORT_W).cpu().numpy()
    cost = ba.export(capi.EXPORT_COST).cpu().numpy()[0]
    So, yo, Cto, wo, costo = oracle.schur_system(s)
    L = np.tril(So)
    scale = np.abs(np.diag(So))
    # entrywise, relative to the geometric mean of the two diagonals
    ref = np.sqrt(np.outer(scale, scale))
    err_S = np.abs(np.tril(S) - L) / ref
    assert err_S.max() < 2e-5, err_S.max()
    assert np.abs(y - yo).max() < 2e-5 * np.abs(yo).max()
    assert np.abs(Ct / Cto - 1).max() < 2e-5
    assert np.abs(w - wo).max() < 2e-5 * np.abs(wo).max()
    assert abs(cost / costo - 1) < 1e-5


# --------------------------------------------------------------------------- #
# whole GN steps: 1e-5 per step on poses and depths
# --------------------------------------------------------------------------- #
@pytest.mark.parametrize("case", ["tiny", "odometry"])
@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_gn_steps_match_oracle(case, precision):
    s = sizes_case(case)
    ba, T = bind(s, precision=precision)
    want = oracle.gn_steps(s, iters=s.iters)
    for it in range(s.iters):
        ba.step(1, s.fixed)
        ba.sync()
        poses = T["poses"].cpu().numpy()
        depths = T["patches"][:, 2, 1, 1].cpu().numpy().astype(np.float64)
        rot, tr = pose_error(poses, want[it][0])
        dep = depth_error(depths, want[it][1])
        assert rot < TOL and tr < TOL and dep < TOL, (it, rot, tr, dep)
    # all nine pixels of every patch carry the same inverse depth
    d = T["patches"][:, 2].cpu().numpy()
    assert np.array_equal(d, np.broadcast_to(d[:, 1:2, 1:2], d.shape))


@pytest.mark.parametrize("frames", [3, 12, 30, 44])
def test_gn_step_across_pose_system_sizes(frames):
    # 6 (frames - 2) unknowns: one-CTA solver layouts from 32 up to 256 rows
    # FP32-only factorisation holds 1e-5 up to the odometry window (n = 120);
    # above it, BA_MIXED's FP64 refinement is what keeps depths within 1e-5
    s = scenes._build("sized", 11, frames, lambda i, n: scenes._shifted_window(i, n, 14), 2, 1)
    for precision in (("fp32", "mixed") if frames <= 22 else ("mixed",)):
        ba, T = bind(s, precision=precision)
        ba.step(1, s.fixed)
        ba.sync()
        want = oracle.gn_steps(s, iters=1)[0]
        rot, tr = pose_error(T["poses"].cpu().numpy(), want[0])
        dep = depth_error(T["patches"][:, 2, 1, 1].cpu().numpy().astype(np.float64), want[1])
        assert rot < TOL and tr < TOL and dep < TOL, (frames, precision, rot, tr, dep)


@pytest.mark.parametrize("frames", [60, 120])
def test_gn_step_blocked_solver(frames):
    # 6 (frames - 2) = 348 / 708 unknowns: the blocked large-system solver
    s = scenes._build("sized", 13, frames, lambda i, n: scenes._clipped_window(i, n, 6), 2, 1)
    for precision in ("fp32", "mixed"):
        ba, T = bind(s, precision=precision)
        ba.step(1, s.fixed)
        ba.sync()
        want = oracle.gn_steps(s, iters=1)[0]
        rot, tr = pose_error(T["poses"].cpu().numpy(), want[0])
        dep = depth_error(T["patches"][:, 2, 1, 1].cpu().numpy().astype(np.float64), want[1])
        assert rot < TOL and tr < TOL and dep < TOL, (frames, precision, rot, tr, dep)


@pytest.mark.parametrize("frames", [60, 120])
@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_large_solver_matches_exact_solve_of_its_system(frames, precision):
    # the persistent factorisation + preconditioned CG against an exact FP64
    # solve (LAPACK) of the pose system the GPU assembled: the solver alone
    s = scenes._build("sized", 17, frames, lambda i, n: scenes._clipped_window(i, n, 6), 2, 1, loop=True)
    ba, T = bind(s, precision=precision)
    ba.linearize(s.fixed)
    ba.sync()
    n = ba.info()["n"]
    S = ba.export(capi.EXPORT_S).cpu().numpy().reshape(n, n)
    S = np.tril(S) + np.tril(S, -1).T
    y = ba.export(capi.EXPORT_Y).cpu().numpy()
    ba2, T2 = bind(s, precision=precision)
    ba2.step(1, s.fixed)
    ba2.sync()
    dx = ba2.export(capi.EXPORT_DX).cpu().numpy()
    x = np.linalg.solve(S, y)
    assert np.abs(dx - x).max() <= 1e-6 * np.abs(x).max(), (np.abs(dx - x).max(), np.abs(x).max())


def test_gn_step_independent_of_input_edge_order():
    s = scenes.odometry(seed=2)
    order = np.random.default_rng(5).permutation(s.E)
    for f in ("ii", "jj", "kk", "targets", "weights"):
        setattr(s, f, getattr(s, f)[order].copy())
    ba, T = bind(s)
    ba.step(1, s.fixed)
    ba.sync()
    want = oracle.gn_steps(s, iters=1)[0]
    rot, tr = pose_error(T["poses"].cpu().numpy(), want[0])
    dep = depth_error(T["patches"][:, 2, 1, 1].cpu().numpy().astype(np.float64), want[1])
    assert rot < TOL and tr < TOL and dep < TOL, (rot, tr, dep)


def test_multi_iteration_call_equals_single_steps():
    s = scenes.odometry(seed=3)
    ba1, T1 = bind(s)
    ba1.step(2, s.fixed)
    ba1.sync()
    ba2, T2 = bind(s)
    ba2.step(1, s.fixed)
    ba2.step(1, s.fixed)
    ba2.sync()
    rot, tr = pose_error(T1["poses"].cpu().numpy(), T2["poses"].cpu().numpy())
    assert rot < 1e-6 and tr < 1e-6


def test_fixed_poses_bitwise_unchanged_and_steps_recorded():
    s = scenes.tiny(seed=7)
    ba, T = bind(s)
    p0 = T["poses"].clone()
    ba.step(2, 3)
    ba.sync()
    assert torch.equal(T["poses"][:3], p0[:3])
    assert not torch.equal(T["poses"][3:], p0[3:])
    dx = ba.export(capi.EXPORT_DX).cpu().numpy()
    assert dx.shape == (6 * (s.N - 3),) and np.isfinite(dx).all()


def test_noise_free_scene_converges_to_ground_truth():
    s = scenes.noise_free(scenes.odometry(seed=4))
    ba, T = bind(s, precision="mixed")
    ba.step(6, s.fixed)
    ba.sync()
    rot, tr = pose_error(T["poses"].cpu().numpy(), s.poses_gt)
    dep = depth_error(T["patches"][:, 2, 1, 1].cpu().numpy().astype(np.float64), s.depth_gt)
    assert rot < 1e-5 and tr < 1e-5 and dep < 1e-4, (rot, tr, dep)


# --------------------------------------------------------------------------- #
# edge cases and errors
# --------------------------------------------------------------------------- #
def test_ragged_groups_self_edges_and_patches_without_edges():
    s = scenes.tiny(seed=9)
    # drop every edge of some patches, add self edges, and cut P to a ragged size
    P = 700
    keep = s.kk < P
    keep &= (s.kk % 13) != 0
    for f in ("ii", "jj", "kk", "targets", "weights"):
        setattr(s, f, getattr(s, f)[keep].copy())
    selfk = np.arange(1, P, 97)
    s.ii = np.r_[s.ii, selfk // 96].astype(np.int32)
    s.jj = np.r_[s.jj, selfk // 96].astype(np.int32)
    s.kk = np.r_[s.kk, selfk].astype(np.int32)
    s.targets = np.r_[s.targets, np.full((len(selfk), 2), 100.0, np.float32)]
    s.weights = np.r_[s.weights, np.ones((len(selfk), 2), np.float32)]
    s.patches = s.patches[:P].copy()
    s.P, s.E = P, len(s.kk)
    for G in (8, 24):
        ba, T = bind(s, patches_per_group=G)
        ba.step(1, s.fixed)
        ba.sync()
        want = oracle.gn_steps(s, iters=1)[0]
        rot, tr = pose_error(T["poses"].cpu().numpy(), want[0])
        dep = depth_error(T["patches"][:, 2, 1, 1].cpu().numpy().astype(np.float64), want[1])
        assert rot < TOL and tr < TOL and dep < TOL, (G, rot, tr, dep)
        dd = ba.export(capi.EXPORT_DD).cpu().numpy()
        assert np.all(dd[np.setdiff1d(np.arange(P), s.kk)] == 0)


def test_long_runs_of_patches_without_edges():
    # runs of 300 patches without edges at the start, in the middle and at the
    # end: longer than the span the fused binding writes speculatively, so it
    # takes its exact CSR pass (sorted input) or the sort's (shuffled)
    s = scenes.tiny(seed=3)
    gap, half = 300, s.P // 2
    old = s.kk.copy()
    s.kk = (old + gap + np.where(old >= half, gap, 0)).astype(np.int32)
    filler = np.repeat(s.patches[:1], gap, axis=0)
    s.patches = np.concatenate([filler, s.patches[:half], filler, s.patches[half:], filler]).copy()
    s.P += 3 * gap
    ba, T = bind(s)
    ba.step(1, s.fixed)
    ba.sync()
    want = oracle.gn_steps(s, iters=1)[0]
    rot, tr = pose_error(T["poses"].cpu().numpy(), want[0])
    dep = depth_error(T["patches"][:, 2, 1, 1].cpu().numpy().astype(np.float64), want[1])
    assert rot < TOL and tr < TOL and dep < TOL, (rot, tr, dep)
    for shuffle in (False, True):
        check_indexing(copy.deepcopy(s), 8, shuffle, keys=False)


def test_graph_without_edges_leaves_state_unchanged():
    s = scenes.tiny(seed=1)
    T = scene_tensors(s)
    p0, q0 = T["poses"].clone(), T["patches"].clone()
    ba = DPVBA()
    e = T["ii"][:0]
    ba.set_graph(T["poses"], T["patches"], e, e, e, T["targets"][:0], T["weights"][:0], T["intrinsics"])
    ba.step(2, 2)
    ba.sync()
    # zero step: poses change only by the quaternion renormalisation rounding
    assert torch.allclose(T["poses"], p0, rtol=0, atol=1e-15) and torch.equal(T["patches"], q0)


def test_bad_index_reported_not_faulted():
    s = scenes.tiny(seed=1)
    T = scene_tensors(s)
    T["jj"][5] = s.N + 3
    ba = DPVBA()
    ba.set_graph(**T)
    p0 = T["poses"].clone()
    ba.step(1, 2)
    with pytest.raises(capi.BAError) as ei:
        ba.sync()
    assert ei.value.status == capi.BA_ERR_INVALID_ARG
    assert torch.equal(T["poses"], p0)


def test_patch_with_two_source_frames_rejected():
    s = scenes.tiny(seed=1)
    T = scene_tensors(s)
    T["ii"][0] = (int(T["ii"][0]) + 1) % s.N
    ba = DPVBA()
    ba.set_graph(**T)
    with pytest.raises(capi.BAError) as ei:
        ba.sync()
    assert ei.value.status == capi.BA_ERR_INVALID_ARG


def test_indefinite_system_reports_not_spd_and_keeps_state():
    s = scenes.tiny(seed=1)
    ba, T = bind(s, lambda_pose=-1e7)
    p0, q0 = T["poses"].clone(), T["patches"].clone()
    ba.step(1, 2)
    with pytest.raises(capi.BAError) as ei:
        ba.sync()
    assert ei.value.status == capi.BA_ERR_NOT_SPD
    assert torch.equal(T["poses"], p0) and torch.equal(T["patches"], q0)


def test_host_checked_errors():
    s = scenes.tiny(seed=1)
    ba = DPVBA()
    with pytest.raises(capi.BAError) as ei:
        ba.step(1, 0)
    assert ei.value.status == capi.BA_ERR_STATE
    ba2, T = bind(s)
    with pytest.raises(capi.BAError) as ei:
        ba2.step(1, s.N + 1)
    assert ei.value.status == capi.BA_ERR_INVALID_ARG
