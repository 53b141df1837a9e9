"""GPU parity of the Sim(3) pose-graph Levenberg-Marquardt (ba_pgo_lm, Sec. 3.3
"Optimization", Eqs. 5-7) with the FP64 oracle.

Tolerances, from the arithmetic: both sides take central differences of step
h = 1e-6 of the same FP64 residual, so their Jacobians differ by about
eps |r| / h ~ 1e-10 relative, and the GPU's solve (FP32 factor with FP64
refinement under the mixed precision option) by its refinement tolerance.
Each LM step therefore agrees to ~1e-9 relative; accepted iterations move the
costs by far more, so the cost curves agree to 1e-6 relative and the
accept/reject decisions agree wherever the cost changed by more than that
(at convergence both sides reject steps whose gain is rounding noise, in
either order).  The final similarities agree to 1e-7 (their matrices,
relative to the largest entry: the solvers stop once the error left in a step
is below 1e-7 of it).
"""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2408_01654_b300 import capi, scenes  # noqa: E402
from paper_2408_01654_b300.ba import DPVBA, scene_tensors  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_01654_b300 import build
    build.build()
    oracle.build()


def as_matrix(S):
    M = np.eye(4)
    M[:3, :3] = S[7] * Rotation.from_quat(S[3:7]).as_matrix()
    M[:3, 3] = S[:3]
    return M


def gpu(ba, g, iters, lambda0=1e-4):
    dev = "cuda"
    S = torch.tensor(g["S"], device=dev)
    args = [torch.tensor(g[k], device=dev) for k in ("dS", "fa", "fb", "loop")]
    cost, acc = ba.pgo_lm(S, *args, iters=iters, lambda0=lambda0)
    ba.sync()
    return S.cpu().numpy(), cost.cpu().numpy(), acc.cpu().numpy().astype(bool)


def compare(got, want, tol=1e-7):
    S, cost, acc = got
    assert np.allclose(cost, want["cost"], rtol=1e-6, atol=1e-12), (cost, want["cost"])
    decisive = np.abs(np.diff(want["cost"])) > 1e-6 * want["cost"][1:]
    assert np.array_equal(acc[decisive], want["accepted"][decisive])
    # relative to the matrix's largest entry (translations reach 20 m here)
    err = max(np.abs(as_matrix(a) - as_matrix(b)).max() / max(1.0, np.abs(as_matrix(b)).max())
              for a, b in zip(S, want["S"]))
    assert err < tol, err
    assert np.array_equal(S[0], want["S"][0])


@pytest.mark.parametrize("N,loop_every,precision", [(24, 3, "mixed"), (37, 4, "mixed"), (24, 3, "fp32")])
def test_small_system_matches_oracle(N, loop_every, precision):
    # 7 (N - 1) <= 256 unknowns: the one-CTA solver
    g = scenes.pose_graph(N, N=N, loop_every=loop_every, loop_noise=0.01)
    want = oracle.pgo_lm(g["S"], g["dS"], g["fa"], g["fb"], g["loop"], iters=12)
    got = gpu(DPVBA(precision=precision), g, 12)
    compare(got, want, 1e-7 if precision == "mixed" else 1e-5)
    assert got[1][-1] < 1e-2 * got[1][0]


def test_large_system_matches_oracle():
    # 7 * 199 = 1393 unknowns: the tiled factorisation with FP64 refinement
    g = scenes.pose_graph(5, N=200, loop_every=10, loop_noise=0.005)
    want = oracle.pgo_lm(g["S"], g["dS"], g["fa"], g["fb"], g["loop"], iters=10)
    got = gpu(DPVBA(precision="mixed"), g, 10)
    compare(got, want)


def test_noise_free_loop_reaches_truth_up_to_gauge():
    # consistent loops and smoothness measurements taken from the truth:
    # the optimum is the truth moved by the similarity that maps S*_0 to S_0
    g = scenes.pose_graph(3, N=30, loop_every=2, odo_rot_deg=0.0, odo_trans=0.0, drift_scale=0.0)
    gt = np.stack([as_matrix(x) for x in g["gt"]])
    g["dS"][:len(g["fa"]) - g["loop"].sum()] = [
        scenes._sim_vec(np.linalg.inv(gt[a]) @ gt[b]) for a, b in zip(g["fa"], g["fb"]) if b == a + 1]
    S = g["S"].copy()
    rng = np.random.default_rng(0)
    for i in range(1, len(S)):  # start away from the solution
        S[i, :3] += rng.normal(0, 0.3, 3)
        S[i, 7] *= np.exp(rng.normal(0, 0.05))
    g["S"] = S
    Sg, cost, acc = gpu(DPVBA(precision="mixed"), g, 30)
    assert cost[-1] < 1e-16
    T = as_matrix(S[0]) @ np.linalg.inv(gt[0])
    err = max(np.abs(as_matrix(a) - T @ b).max() for a, b in zip(Sg, gt))
    assert err < 1e-6, err


def test_edge_cases_and_errors():
    ba = DPVBA(precision="mixed")
    dev = "cuda"
    # one keyframe: no unknowns, nothing moves, every step rejected
    g = scenes.pose_graph(1, N=24, loop_every=3)
    one = dict(S=g["S"][:1], dS=np.zeros((0, 8)), fa=np.zeros(0, np.int32), fb=np.zeros(0, np.int32),
               loop=np.zeros(0, np.int32))
    S, cost, acc = gpu(ba, one, 3)
    assert np.array_equal(S, g["S"][:1]) and np.all(cost == 0) and not acc.any()
    # an invalid endpoint: the device status
    bad = dict(g)
    bad["fb"] = g["fb"].copy()
    bad["fb"][2] = 99
    with pytest.raises(capi.BAError) as e:
        gpu(ba, bad, 2)
    assert e.value.status == capi.BA_ERR_INVALID_ARG
    # a keyframe that no factor touches: the damped system is singular
    ba = DPVBA(precision="mixed")
    cut = dict(g)
    keep = (g["fa"] != 5) & (g["fb"] != 5)
    for k in ("dS", "fa", "fb", "loop"):
        cut[k] = g[k][keep]
    with pytest.raises(capi.BAError) as e:
        gpu(ba, cut, 2)
    assert e.value.status == capi.BA_ERR_NOT_SPD
    # parameters checked at once
    ba = DPVBA(precision="mixed")
    S = torch.tensor(g["S"], device=dev)
    args = [torch.tensor(g[k], device=dev) for k in ("dS", "fa", "fb", "loop")]
    for kw in (dict(lambda0=0.0), dict(fd_step=0.0), dict(fd_step=0.1)):
        with pytest.raises(capi.BAError) as e:
            ba.pgo_lm(S, *args, iters=2, **kw)
        assert e.value.status == capi.BA_ERR_INVALID_ARG


def test_bundle_adjustment_after_pgo_on_the_same_handle():
    # the pose-graph call borrows the handle's pose-system buffers; a later
    # ba_step lays its own system out again and gives the same result as a
    # fresh handle
    s = scenes.tiny(0)
    fresh = DPVBA(precision="mixed")
    t = scene_tensors(s)
    fresh.set_graph(**t)
    fresh.step(2, s.fixed)
    fresh.sync()
    want = t["poses"].cpu().numpy()
    ba = DPVBA(precision="mixed")
    t2 = scene_tensors(s)
    ba.set_graph(**t2)
    ba.step(1, s.fixed)
    ba.sync()
    t2["poses"].copy_(torch.tensor(s.poses, device="cuda"))
    t2["patches"].copy_(torch.tensor(s.patches, device="cuda"))
    gpu(ba, scenes.pose_graph(2, N=60, loop_every=5), 3)  # n = 413: the large solver's layout
    ba.step(2, s.fixed)
    ba.sync()
    # (the assembly's floating-point atomics make repeated runs agree to
    # rounding, not bit for bit)
    assert np.abs(t2["poses"].cpu().numpy() - want).max() < 1e-6
