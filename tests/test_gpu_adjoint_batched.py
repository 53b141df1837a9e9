"""The differentiable layer over a batch of independent windows (the
differentiable-BA workload: 16 odometry windows of 22 keyframes, 96 patches
per frame, ~27k edges each, two unrolled GN steps, bound to one handle).

``ba_backward`` on a handle bound by ``ba_set_graph_batched`` against the
FP64 oracle's forward-mode (dual-number) derivatives of each window, 13
sampled coordinates per window (208 in all, targets and weights), at the
tolerance of the single-problem adjoint tests (1e-4 of the sample's largest
gradient, 1e-3 on its 2-norm); and the autograd function over the batch
against per-window handles.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2408_01654_b300 import scenes  # noqa: E402
from paper_2408_01654_b300.ba import DPVBA, batch_tensors, bundle_adjust_batched, scene_tensors  # noqa: E402

ADJ_TOL, NORM_TOL = 1e-4, 1e-3
B = 16


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_01654_b300 import build
    build.build()
    oracle.build()


@pytest.fixture(scope="module")
def windows():
    return [scenes.odometry(seed=b) for b in range(B)]


def loss_weights(probs, seed=0):
    rng = np.random.default_rng(seed)
    return [rng.normal(size=(p.N, 7)) for p in probs], [rng.normal(size=p.P) for p in probs]


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_batched_backward_matches_oracle(windows, precision):
    probs = windows
    A, Bd = loss_weights(probs)
    T, offs = batch_tensors(probs)
    ba = DPVBA(precision=precision)
    ba.set_graph_batched(**T, **offs)
    ba.set_record(True)
    ba.step(probs[0].iters, probs[0].fixed)
    gT, gW = ba.backward(torch.as_tensor(np.concatenate(A), dtype=torch.float64).cuda(),
                         torch.as_tensor(np.concatenate(Bd), dtype=torch.float32).cuda())
    ba.sync()
    gT, gW = gT.cpu().numpy().astype(np.float64), gW.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(1)
    got_all, want_all = [], []
    for b, p in enumerate(probs):
        e0, e1 = offs["edge_off"][b], offs["edge_off"][b + 1]
        kind = np.r_[np.zeros(7, int), np.ones(6, int)]
        index = rng.choice(2 * p.E, 13, replace=False)
        want = oracle.grad_fwd(p, A[b], Bd[b], kind, index)
        got = np.where(kind == 0, gT[e0:e1].reshape(-1)[index], gW[e0:e1].reshape(-1)[index])
        got_all.append(got)
        want_all.append(want)
    got, want = np.concatenate(got_all), np.concatenate(want_all)
    err = np.abs(got - want).max() / np.abs(want).max()
    nerr = np.linalg.norm(got - want) / np.linalg.norm(want)
    print(f"batched adjoint ({precision}): max err {err:.2e}, norm err {nerr:.2e} over {len(got)} coordinates")
    assert err < ADJ_TOL and nerr < NORM_TOL, (err, nerr)


def test_batched_autograd_matches_per_window_handles(windows):
    probs = windows[:4]
    A, Bd = loss_weights(probs, 2)
    T, offs = batch_tensors(probs)
    tg = T["targets"].clone().requires_grad_(True)
    wt = T["weights"].clone().requires_grad_(True)
    poses, depths = bundle_adjust_batched(tg, wt, T["poses"], T["patches"], T["ii"], T["jj"], T["kk"],
                                          T["intrinsics"], offs["frame_off"], offs["patch_off"], offs["edge_off"],
                                          probs[0].iters, probs[0].fixed)
    L = (torch.as_tensor(np.concatenate(A)).cuda() * poses).sum() + \
        (torch.as_tensor(np.concatenate(Bd), dtype=torch.float32).cuda() * depths).sum()
    L.backward()
    for b, p in enumerate(probs):
        Tp = scene_tensors(p)
        h = DPVBA()
        h.set_graph(**Tp)
        h.set_record(True)
        h.step(p.iters, p.fixed)
        gT, gW = h.backward(torch.as_tensor(A[b], dtype=torch.float64).cuda(),
                            torch.as_tensor(Bd[b], dtype=torch.float32).cuda())
        h.sync()
        e0, e1 = offs["edge_off"][b], offs["edge_off"][b + 1]
        f0, f1 = offs["frame_off"][b], offs["frame_off"][b + 1]
        # the same arithmetic up to the order of the FP64 atomic sums
        assert torch.allclose(tg.grad[e0:e1], gT, rtol=1e-4, atol=1e-5 * float(gT.abs().max()))
        assert torch.allclose(wt.grad[e0:e1], gW, rtol=1e-4, atol=1e-5 * float(gW.abs().max()))
        assert torch.allclose(poses.detach()[f0:f1], Tp["poses"], rtol=0, atol=1e-8)
