"""GPU parity of structure-only bundle adjustment (Sec. 3.3): ba_step with
every pose held (fixed_poses = N) minimises Eq. 3 over the inverse depths
only.  The poses must come back bit for bit; the depths match the FP64
oracle at the per-step tolerance of the other parity tests.

The scenes hold their poses at the ground truth (structure-only BA
triangulates depths for known cameras).  Held at the perturbed starting
poses instead, the targets cannot be met and some depth steps run into the
d_min clamp, where FP32 and FP64 clamp different patches: a property of that
problem, not a parity target."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2408_01654_b300 import scenes  # noqa: E402
from paper_2408_01654_b300.ba import DPVBA, batch_tensors, scene_tensors  # noqa: E402
import dataclasses  # noqa: E402

from test_gpu_parity import depth_error, pose_error  # noqa: E402

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_01654_b300 import build
    build.build()
    oracle.build()


def known_poses(s):
    return dataclasses.replace(s, poses=s.poses_gt.copy())


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_odometry_window_structure_only(precision):
    s = known_poses(scenes.odometry(seed=2))
    T = scene_tensors(s)
    before = T["poses"].clone()
    ba = DPVBA(precision=precision)
    ba.set_graph(**T)
    want = oracle.gn_steps(s, iters=2, fixed=s.N)
    for it in range(2):
        ba.step(1, s.N)
        ba.sync()
        assert torch.equal(T["poses"], before)
        dep = depth_error(T["patches"][:, 2, 1, 1].cpu().numpy().astype(np.float64), want[it][1])
        assert dep < TOL, (it, dep)


def test_loop_graph_structure_only():
    s = known_poses(scenes._build("structure", 11, 120, lambda i, m: scenes._clipped_window(i, m, 6), 2, 1,
                                  loop=True))
    T = scene_tensors(s)
    ba = DPVBA()
    ba.set_graph(**T)
    ba.step(1, s.N)
    ba.sync()
    want = oracle.gn_steps(s, iters=1, fixed=s.N)[0]
    assert np.array_equal(T["poses"].cpu().numpy(), s.poses)
    dep = depth_error(T["patches"][:, 2, 1, 1].cpu().numpy().astype(np.float64), want[1])
    assert dep < TOL, dep


def test_batched_mix_of_structure_only_and_full():
    # fixed_poses = 9 holds every pose of the 9-frame problem and the first 9
    # of the 14-frame one
    probs = [known_poses(scenes._build("batched", 40 + b, n, lambda i, m: scenes._clipped_window(i, m, 6), 2, 1,
                                       loop=True)) for b, n in enumerate([14, 9])]
    T, offs = batch_tensors(probs)
    ba = DPVBA(precision="mixed")
    ba.set_graph_batched(**T, **offs)
    ba.step(1, 9)
    ba.sync()
    for b, sc in enumerate(probs):
        want = oracle.gn_steps(sc, iters=1, fixed=9)[0]
        f0, f1 = offs["frame_off"][b], offs["frame_off"][b + 1]
        p0, p1 = offs["patch_off"][b], offs["patch_off"][b + 1]
        rot, tr = pose_error(T["poses"][f0:f1].cpu().numpy(), want[0])
        dep = depth_error(T["patches"][p0:p1, 2, 1, 1].cpu().numpy().astype(np.float64), want[1])
        assert rot < TOL and tr < TOL and dep < TOL, (b, rot, tr, dep)
    assert np.array_equal(T["poses"][offs["frame_off"][1]:].cpu().numpy(), probs[1].poses)
