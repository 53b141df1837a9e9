"""GPU parity of the adjoint (ba_backward) against the FP64 oracle.

The oracle differentiates the unrolled Gauss-Newton iterations in forward
mode (dual numbers, one run per input coordinate, pinned against central
differences in test_oracle_pins.py).  The CUDA path runs reverse mode through
the same iterations.  Both give d L / d(coordinate) for
L = <a, poses_final> + <b, inverse_depths_final> with seeded a, b; sampled
coordinates are compared against the sample's largest magnitude.

Tolerance: the forward path holds each step to 1e-5 relative (FP32 per-edge
arithmetic with compensated sums, FP32 factorisation with refinement).  The
adjoint has no compensated sums in its per-edge FP32 dual arithmetic and
accumulates one rank of rounding per iteration, so it is held to 1e-4 of the
sample's largest gradient (ADJ_TOL) and 1e-3 relative on the sample's 2-norm.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2408_01654_b300 import capi, scenes  # noqa: E402
from paper_2408_01654_b300.ba import DPVBA, bundle_adjust, scene_tensors  # noqa: E402

ADJ_TOL = 1e-4
NORM_TOL = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_01654_b300 import build
    build.build()
    oracle.build()


def loss_weights(s, seed=0):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(s.N, 7)), rng.normal(size=s.P)


def gpu_backward(s, a, b, precision="fp32", iters=None, initial=False):
    T = scene_tensors(s)
    ba = DPVBA(precision=precision)
    ba.set_graph(**T)
    ba.set_record(True)
    ba.step(s.iters if iters is None else iters, s.fixed)
    out = ba.backward(torch.as_tensor(a, dtype=torch.float64).cuda(), torch.as_tensor(b, dtype=torch.float32).cuda(),
                      initial=initial)
    ba.sync()
    return [None if o is None else o.cpu().numpy().astype(np.float64) for o in out], ba, T


def sample_coords(s, n, seed=1):
    rng = np.random.default_rng(seed)
    kind = np.r_[np.zeros(n // 2, int), np.ones(n - n // 2, int)]
    index = rng.choice(2 * s.E, n, replace=False)
    return kind, index


def compare(got, want, label):
    scale = np.abs(want).max()
    err = np.abs(got - want).max() / scale
    nerr = np.linalg.norm(got - want) / np.linalg.norm(want)
    print(f"{label}: max err {err:.2e} of max |g| {scale:.3e}, norm err {nerr:.2e}")
    assert err < ADJ_TOL and nerr < NORM_TOL, (label, err, nerr)


def picked(gT, gW, kind, index):
    return np.where(kind == 0, gT.reshape(-1)[index], gW.reshape(-1)[index])


@pytest.mark.parametrize("case,n", [("tiny", 200), ("odometry", 40)])
@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_backward_matches_oracle(case, n, precision):
    s = scenes.tiny(seed=0) if case == "tiny" else scenes.odometry(seed=0)
    a, b = loss_weights(s)
    (gT, gW), _, _ = gpu_backward(s, a, b, precision)
    kind, index = sample_coords(s, n)
    want = oracle.grad_fwd(s, a, b, kind, index)
    compare(picked(gT, gW, kind, index), want, f"{case}/{precision}")


def test_backward_initial_state_matches_oracle():
    s = scenes.tiny(seed=1)
    a, b = loss_weights(s, 2)
    (gT, gW, x0, d0), _, _ = gpu_backward(s, a, b, "mixed", initial=True)
    rng = np.random.default_rng(3)
    kp = rng.choice(s.P, 24, replace=False)
    kx = rng.choice(np.arange(6 * s.fixed, 6 * s.N), 24, replace=False)
    want_d = oracle.grad_fwd(s, a, b, np.full(24, 2), kp)
    want_x = oracle.grad_fwd(s, a, b, np.full(24, 3), kx)
    compare(d0[kp], want_d, "initial depths")
    compare(x0.reshape(-1)[kx], want_x, "initial pose tangents")
    assert np.all(x0[: s.fixed] == 0.0)


@pytest.mark.parametrize("frames", [30, 60])
def test_backward_across_solver_sizes(frames):
    # 168 unknowns (one-CTA solver) and 348 (blocked solver)
    s = scenes._build("sized", 13, frames, lambda i, n: scenes._clipped_window(i, n, 6), 2, 2)
    a, b = loss_weights(s, 4)
    (gT, gW), _, _ = gpu_backward(s, a, b, "mixed")
    kind, index = sample_coords(s, 20, seed=5)
    want = oracle.grad_fwd(s, a, b, kind, index)
    compare(picked(gT, gW, kind, index), want, f"{frames} frames")


def test_autograd_function_matches_backward():
    s = scenes.tiny(seed=2)
    T = scene_tensors(s)
    a, b = loss_weights(s, 6)
    tg = T["targets"].clone().requires_grad_(True)
    wt = T["weights"].clone().requires_grad_(True)
    poses, depths = bundle_adjust(tg, wt, T["poses"], T["patches"], T["ii"], T["jj"], T["kk"], T["intrinsics"],
                                  s.iters, s.fixed)
    L = (torch.as_tensor(a).cuda() * poses).sum() + (torch.as_tensor(b, dtype=torch.float32).cuda() * depths).sum()
    L.backward()
    (gT, gW), _, _ = gpu_backward(s, a, b)
    assert np.allclose(tg.grad.cpu().numpy(), gT, rtol=1e-5, atol=1e-6 * np.abs(gT).max())
    assert np.allclose(wt.grad.cpu().numpy(), gW, rtol=1e-5, atol=1e-6 * np.abs(gW).max())
    # the forward values are the plain step's
    ref = DPVBA()
    T2 = scene_tensors(s)
    ref.set_graph(**T2)
    ref.step(s.iters, s.fixed)
    ref.sync()
    # (equal up to the order of the FP64 atomic sums into the pose system)
    assert torch.allclose(poses.detach(), T2["poses"], rtol=0, atol=1e-9)
    assert torch.allclose(depths.detach(), T2["patches"][:, 2, 1, 1], rtol=1e-6, atol=0)


def test_backward_against_gpu_central_differences():
    # an independent check of the adjoint against the CUDA forward path itself
    s = scenes.tiny(seed=3)
    a, b = loss_weights(s, 7)
    (gT, gW), _, _ = gpu_backward(s, a, b, "mixed")
    at = torch.as_tensor(a).cuda()
    bt = torch.as_tensor(b).cuda()

    def L(targets, weights):
        T = scene_tensors(s)
        T["targets"], T["weights"] = targets, weights
        ba = DPVBA(precision="mixed")
        ba.set_graph(**T)
        ba.step(s.iters, s.fixed)
        ba.sync()
        return float((at * T["poses"]).sum() + (bt * T["patches"][:, 2, 1, 1].double()).sum())

    base = scene_tensors(s)
    rng = np.random.default_rng(8)
    # the largest target gradients, with a central difference of 0.1 px (the
    # residual noise is 0.5 px): the FP32 rounding of the ~800 state values in
    # L stays ~1e-3 of L(+) - L(-), the O(eps^2) truncation below that
    idx = np.argsort(-np.abs(gT.reshape(-1)))[:6]
    idx = np.r_[idx, rng.choice(2 * s.E, 2, replace=False)]
    eps = 1e-1
    for q in idx:
        tp, tm = base["targets"].clone(), base["targets"].clone()
        tp.view(-1)[q] += eps
        tm.view(-1)[q] -= eps
        fd = (L(tp, base["weights"]) - L(tm, base["weights"])) / (2 * eps)
        assert abs(fd - gT.reshape(-1)[q]) <= 1e-2 * np.abs(gT).max(), (q, fd, gT.reshape(-1)[q])


def test_backward_masked_edges_and_fixed_poses():
    # self edges and points behind z_min contribute nothing
    s = scenes.tiny(seed=4)
    extra_i = np.arange(s.N, dtype=np.int32)
    extra_k = (extra_i * 96 + 5).astype(np.int32)
    s.ii = np.r_[s.ii, extra_i]
    s.jj = np.r_[s.jj, extra_i]
    s.kk = np.r_[s.kk, extra_k]
    s.targets = np.r_[s.targets, np.full((s.N, 2), 100.0, np.float32)]
    s.weights = np.r_[s.weights, np.ones((s.N, 2), np.float32)]
    s.E = len(s.kk)
    a, b = loss_weights(s, 9)
    (gT, gW, x0, d0), _, _ = gpu_backward(s, a, b, initial=True)
    assert np.all(gT[-s.N:] == 0.0) and np.all(gW[-s.N:] == 0.0)
    assert np.all(x0[: s.fixed] == 0.0)
    kind, index = sample_coords(s, 60, seed=10)
    want = oracle.grad_fwd(s, a, b, kind, index)
    compare(picked(gT, gW, kind, index), want, "with self edges")


def test_zero_iteration_tape_and_missing_tape():
    s = scenes.tiny(seed=5)
    a, b = loss_weights(s, 11)
    (gT, gW, x0, d0), ba, T = gpu_backward(s, a, b, iters=0, initial=True)
    assert np.all(gT == 0.0) and np.all(gW == 0.0)
    assert np.array_equal(d0, np.asarray(b, np.float32).astype(np.float64))
    ba2 = DPVBA()
    ba2.set_graph(**scene_tensors(s))
    with pytest.raises(capi.BAError) as e:
        ba2.backward()
    assert e.value.status == capi.BA_ERR_STATE
    # a new graph discards the tape
    ba.set_graph(**scene_tensors(s))
    with pytest.raises(capi.BAError):
        ba.backward()


def test_backward_twice_gives_the_same_result():
    s = scenes.odometry(seed=1)
    a, b = loss_weights(s, 12)
    T = scene_tensors(s)
    ba = DPVBA()
    ba.set_graph(**T)
    ba.set_record(True)
    ba.step(s.iters, s.fixed)
    g1 = [t.clone() for t in ba.backward(torch.as_tensor(a).cuda(), torch.as_tensor(b, dtype=torch.float32).cuda())]
    g2 = ba.backward(torch.as_tensor(a).cuda(), torch.as_tensor(b, dtype=torch.float32).cuda())
    ba.sync()
    for x, y in zip(g1, g2):
        # pose cotangents are summed with FP64 atomics in arbitrary order
        assert torch.allclose(x, y, rtol=1e-5, atol=1e-6 * float(x.abs().max()))
