"""The dense form of an iteration (small graphs) and the automatic switch.

The appendix "Bundle-Adjustment Efficiency" compares DPVO's dense bundle
adjustment with the block-sparse one and switches between them by graph
size.  The dense form scatters every edge's products into dense arrays (the
pose system, the pose-depth matrix with one column per patch, C and w) and
forms the Schur complement as one dense product.  Bar: the same as the
block-sparse path's (poses and depths within 1e-5 of the FP64 oracle per GN
step), and agreement with the block-sparse path run on the same handle type.
"""
import ctypes

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


def sized(frames, seed=11):
    return scenes._build("sized", seed, frames, lambda i, n: scenes._shifted_window(i, n, 14), 2, 2)


def run(s, iters, **opts):
    T = scene_tensors(s)
    ba = DPVBA(**opts)
    ba.set_graph(**T)
    out = []
    for _ in range(iters):
        ba.step(1, s.fixed)
        ba.sync()
        out.append((T["poses"].cpu().numpy().copy(), T["patches"][:, 2, 1, 1].cpu().numpy().astype(np.float64)))
    return out, ba


@pytest.mark.parametrize("case", ["tiny", "odometry", "44"])
def test_dense_steps_match_oracle(case):
    s = {"tiny": lambda: scenes.tiny(seed=0), "odometry": lambda: scenes.odometry(seed=0),
         "44": lambda: sized(44)}[case]()
    got, ba = run(s, s.iters, dense="always")
    assert ba.info()["dense"] == 1
    want = oracle.gn_steps(s, iters=s.iters)
    for it in range(s.iters):
        rot, tr = pose_error(got[it][0], want[it][0])
        dep = depth_error(got[it][1], want[it][1])
        assert rot < TOL and tr < TOL and dep < TOL, (case, it, rot, tr, dep)


def test_dense_agrees_with_block_sparse_and_exports():
    s = scenes.odometry(seed=3)
    dense, bd = run(s, 2, dense="always")
    sparse, bs = run(s, 2, dense="never")
    assert bd.info()["dense"] == 1 and bs.info()["dense"] == 0
    for (pd, dd), (ps, ds) in zip(dense, sparse):
        rot, tr = pose_error(pd, ps)
        assert rot < TOL and tr < TOL and depth_error(dd, ds) < TOL  # each is within ~3e-6 of the oracle
    # the reduced system of both forms at the same state
    sys = []
    for dense_policy in ("always", "never"):
        T = scene_tensors(s)
        ba = DPVBA(dense=dense_policy)
        ba.set_graph(**T)
        ba.linearize(s.fixed)
        sys.append([ba.export(w).cpu().numpy().astype(np.float64)
                    for w in (capi.EXPORT_S, capi.EXPORT_Y, capi.EXPORT_CT, capi.EXPORT_W)])
    (S1, y1, c1, w1), (S2, y2, c2, w2) = sys
    ref = np.sqrt(np.outer(np.abs(np.diag(S2)), np.abs(np.diag(S2))))
    assert np.abs(S1 - S2).max() <= 2e-5 * ref.max()
    assert np.abs(y1 - y2).max() <= 2e-5 * np.abs(y2).max()
    assert np.allclose(c1, c2, rtol=1e-5) and np.abs(w1 - w2).max() <= 1e-5 * np.abs(w2).max()


def test_automatic_switch():
    # the automatic policy follows the measured crossover (block-sparse at
    # every size on this part); the dense form applies only to single FP32
    # problems of at most 256 unknowns with the centre residual and no tape
    for make in (lambda: scenes.tiny(seed=1), lambda: scenes.odometry(seed=1)):
        _, b = run(make(), 1)
        assert b.info()["dense"] == 0
        _, b = run(make(), 1, dense="always")
        assert b.info()["dense"] == 1
    _, b = run(sized(60), 1, dense="always")  # 348 unknowns
    assert b.info()["dense"] == 0
    _, b = run(scenes.odometry(seed=1), 1, precision="mixed", dense="always")
    assert b.info()["dense"] == 0
    probs = [scenes.tiny(seed=2), scenes.tiny(seed=3)]
    T, offs = batch_tensors(probs)
    bb = DPVBA(dense="always")
    bb.set_graph_batched(**T, **offs)
    bb.step(1, 2)
    bb.sync()
    assert bb.info()["dense"] == 0
    # a recorded step runs block-sparse, and its adjoint is the usual one
    s = scenes.tiny(seed=4)
    T = scene_tensors(s)
    ba = DPVBA(dense="always")
    ba.set_graph(**T)
    ba.set_record(True)
    ba.step(s.iters, s.fixed)
    assert ba.info()["dense"] == 0
    gT, gW = ba.backward(torch.ones((s.N, 7), dtype=torch.float64).cuda(), torch.ones(s.P).cuda())
    ba.sync()
    assert torch.isfinite(gT).all() and torch.isfinite(gW).all()
    ba.set_record(False)
    ba.step(1, s.fixed)  # dense again once nothing is recorded
    assert ba.info()["dense"] == 1


def test_dense_graph_replay_equals_eager():
    s = scenes.odometry(seed=5)
    T0 = scene_tensors(s)
    eager = DPVBA(dense="always")
    Te = {k: v.clone() for k, v in T0.items()}
    eager.set_graph(**Te)
    eager.step(s.iters, s.fixed)
    eager.sync()
    cap = DPVBA(dense="always", capture=True)
    Tc = {k: v.clone() for k, v in T0.items()}
    for _ in range(3):  # eager, capture, replay (the same buffers: a graph is keyed by the binding's pointers)
        Tc["poses"].copy_(T0["poses"])
        Tc["patches"].copy_(T0["patches"])
        cap.set_graph(**Tc)
        cap.step(s.iters, s.fixed)
        cap.sync()
    assert cap.info()["graph_replays"] >= 1
    rot, tr = pose_error(Tc["poses"].cpu().numpy(), Te["poses"].cpu().numpy())
    assert rot < 1e-7 and tr < 1e-7


def test_dense_policy_checked():
    h = ctypes.c_void_p()
    assert capi.lib().ba_create(ctypes.byref(h), ctypes.byref(capi.default_options(dense_policy=3))) == \
        capi.BA_ERR_INVALID_ARG
