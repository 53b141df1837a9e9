"""GPU parity of the batched binding (ba_set_graph_batched): independent
problems of uneven sizes solved together must each match the FP64 oracle run
on that problem alone (1e-5 relative per step, as for a single problem) and
the same library run on each problem separately."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2408_01654_b300 import capi, scenes  # noqa: E402
from paper_2408_01654_b300.ba import DPVBA, batch_tensors, scene_tensors  # noqa: E402

from test_gpu_parity import depth_error, pose_error  # noqa: E402

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_01654_b300 import build
    build.build()
    oracle.build()


def problems(frames, seed=0, iters=1):
    # the global-BA edge rules (+-6 frames and loop edges), per problem
    return [scenes._build("batched", seed * 100 + b, n, lambda i, m: scenes._clipped_window(i, m, 6), 2, iters,
                          loop=True) for b, n in enumerate(frames)]


def run_batched(probs, iters, fixed=2, **opts):
    T, offs = batch_tensors(probs)
    ba = DPVBA(**opts)
    ba.set_graph_batched(**T, **offs)
    ba.step(iters, fixed)
    ba.sync()
    return T, offs, ba


def split(T, offs, b):
    f0, f1 = offs["frame_off"][b], offs["frame_off"][b + 1]
    p0, p1 = offs["patch_off"][b], offs["patch_off"][b + 1]
    return T["poses"][f0:f1].cpu().numpy(), T["patches"][p0:p1, 2, 1, 1].cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_batched_step_matches_oracle_per_problem(precision):
    # 36 .. 288 unknowns: one-CTA systems of several block counts and one large system
    frames = [8, 30, 13, 50, 21]
    probs = problems(frames, seed=1)
    T, offs, ba = run_batched(probs, 1, precision=precision)
    for b, sc in enumerate(probs):
        want = oracle.gn_steps(sc, iters=1)[0]
        poses, d = split(T, offs, b)
        rot, tr = pose_error(poses, want[0])
        dep = depth_error(d, want[1])
        assert rot < TOL and tr < TOL and dep < TOL, (b, frames[b], precision, rot, tr, dep)


def test_batched_several_large_systems():
    # three systems above 256 unknowns factored in one launch, beside small ones
    frames = [46, 70, 12, 52]
    probs = problems(frames, seed=5)
    T, offs, ba = run_batched(probs, 1, precision="mixed")
    for b, sc in enumerate(probs):
        want = oracle.gn_steps(sc, iters=1)[0]
        poses, d = split(T, offs, b)
        rot, tr = pose_error(poses, want[0])
        dep = depth_error(d, want[1])
        assert rot < TOL and tr < TOL and dep < TOL, (b, frames[b], rot, tr, dep)


def test_batched_equals_separate_handles():
    frames = [9, 27, 46, 15]
    probs = problems(frames, seed=2, iters=2)
    # the same group size on both sides: the same groups and summation order,
    # up to the order of the FP64 atomics
    T, offs, ba = run_batched(probs, 2, precision="mixed", patches_per_group=16)
    for b, sc in enumerate(probs):
        Ts = scene_tensors(sc)
        one = DPVBA(precision="mixed", patches_per_group=16)
        one.set_graph(**Ts)
        one.step(2, sc.fixed)
        one.sync()
        poses, d = split(T, offs, b)
        # equal up to the order of the FP64 atomic sums into the pose systems
        assert np.allclose(poses, Ts["poses"].cpu().numpy(), rtol=0, atol=1e-9), b
        assert np.allclose(d, Ts["patches"][:, 2, 1, 1].cpu().numpy(), rtol=1e-6, atol=0), b


def test_batched_more_row_blocks_than_solver_ctas():
    # eight 400-frame systems: 8 x 38 = 304 row blocks, more than the solve
    # kernel's resident CTAs, so CTAs own row blocks of several systems (the
    # chain-ordered path); each problem must match its own handle
    frames = [400] * 8
    probs = problems(frames, seed=6)
    T, offs, ba = run_batched(probs, 1, precision="mixed", patches_per_group=32)
    for b, sc in enumerate(probs):
        Ts = scene_tensors(sc)
        one = DPVBA(precision="mixed", patches_per_group=32)
        one.set_graph(**Ts)
        one.step(1, sc.fixed)
        one.sync()
        poses, d = split(T, offs, b)
        assert np.allclose(poses, Ts["poses"].cpu().numpy(), rtol=0, atol=1e-7), b
        assert np.allclose(d, Ts["patches"][:, 2, 1, 1].cpu().numpy(), rtol=1e-5, atol=0), b


def test_batched_padded_patch_counts_and_intrinsics():
    # patch counts that are not multiples of the group size (the padded copy)
    # and a different camera per problem
    probs = problems([10, 14, 12], seed=3)
    for b, sc in enumerate(probs):
        keep = sc.P - 5 * (b + 1)
        sel = sc.kk < keep
        sc.patches = sc.patches[:keep].copy()
        sc.P = keep
        sc.ii, sc.jj, sc.kk = sc.ii[sel].copy(), sc.jj[sel].copy(), sc.kk[sel].copy()
        sc.targets, sc.weights = sc.targets[sel].copy(), sc.weights[sel].copy()
        sc.E = int(sel.sum())
    probs[1].intrinsics = (probs[1].intrinsics * np.float32(1.1)).astype(np.float32)
    T, offs, ba = run_batched(probs, 1, patches_per_group=8)
    for b, sc in enumerate(probs):
        want = oracle.gn_steps(sc, iters=1)[0]
        poses, d = split(T, offs, b)
        rot, tr = pose_error(poses, want[0])
        dep = depth_error(d, want[1])
        assert rot < TOL and tr < TOL and dep < TOL, (b, rot, tr, dep)
    # the caller's patch array holds the updated depths (written back from the copy)
    d_all = T["patches"][:, 2].cpu().numpy()
    assert np.array_equal(d_all, np.broadcast_to(d_all[:, 1:2, 1:2], d_all.shape))


def test_batched_errors():
    probs = problems([8, 9], seed=4)
    T, offs = batch_tensors(probs)
    ba = DPVBA()
    bad = dict(offs)
    bad["frame_off"] = offs["frame_off"] + 1
    with pytest.raises(capi.BAError) as e:
        ba.set_graph_batched(**T, **bad)
    assert e.value.status == capi.BA_ERR_INVALID_ARG
    empty = dict(offs)
    empty["frame_off"] = np.array([0, 0, offs["frame_off"][-1]])
    with pytest.raises(capi.BAError):
        ba.set_graph_batched(**T, **empty)
    # a local index outside its problem is reported by ba_sync, without a fault
    T2 = {k: v.clone() for k, v in T.items()}
    T2["ii"][-1] = 9  # problem 1 has 9 frames: local indices 0..8
    ba.set_graph_batched(**T2, **offs)
    ba.step(1, 2)
    with pytest.raises(capi.BAError) as e:
        ba.sync()
    assert e.value.status == capi.BA_ERR_INVALID_ARG
    ba2 = DPVBA()
    ba2.set_graph_batched(**T, **offs)
    with pytest.raises(capi.BAError):
        ba2.step(1, 9)  # more fixed poses than the smallest problem has frames
