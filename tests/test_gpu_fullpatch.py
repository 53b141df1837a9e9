"""GPU parity of the whole-patch residual (residual_pixels = 9: Eq. 3 summed
over the nine pixels of each patch, 18 rows per edge) with the FP64 oracle.

Same bar as the centre-only parity tests: the reduced system entrywise within
2e-5 of the geometric mean of its diagonals, and poses and depths within 1e-5
per GN step (FP32 linearisation and compensated sums; nine times the rows per
edge does not change the per-entry error model, each run and patch sum being
compensated).  The centre-only path on the same handle type is unchanged
(checked bit for bit against a handle built without the option).
"""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2408_01654_b300 import capi, scenes  # noqa: E402
from paper_2408_01654_b300.ba import DPVBA, batch_tensors, bundle_adjust, scene_tensors  # noqa: E402

from test_gpu_parity import depth_error, pose_error  # noqa: E402

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_01654_b300 import build
    build.build()
    oracle.build()


def full(s):
    return dataclasses.replace(s, targets=scenes.full_patch_targets(s))


def bind(s, **opts):
    T = scene_tensors(s)
    ba = DPVBA(residual_pixels=9, **opts)
    ba.set_graph(**T)
    return ba, T


@pytest.mark.parametrize("make", [scenes.tiny, scenes.odometry])
def test_reduced_system_matches_oracle(make):
    s = full(make(seed=0))
    ba, T = bind(s)
    ba.linearize(s.fixed)
    S = ba.export(capi.EXPORT_S).cpu().numpy().astype(np.float64)
    y = ba.export(capi.EXPORT_Y).cpu().numpy().astype(np.float64)
    Ct = ba.export(capi.EXPORT_CT).cpu().numpy()
    w = ba.export(capi.EXPORT_W).cpu().numpy()
    cost = ba.export(capi.EXPORT_COST).cpu().numpy()[0]
    So, yo, Cto, wo, costo = oracle.schur_system(s, pixels=9)
    ref = np.sqrt(np.outer(np.abs(np.diag(So)), np.abs(np.diag(So))))
    assert (np.abs(np.tril(S) - np.tril(So)) / ref).max() < 2e-5
    assert np.abs(y - yo).max() < 2e-5 * np.abs(yo).max()
    assert np.abs(Ct / Cto - 1).max() < 2e-5
    assert np.abs(w - wo).max() < 2e-5 * np.abs(wo).max()
    assert abs(cost / costo - 1) < 1e-5


@pytest.mark.parametrize("make", [scenes.tiny, scenes.odometry])
@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_gn_steps_match_oracle(make, precision):
    s = full(make(seed=1))
    ba, T = bind(s, precision=precision)
    poses, patches = s.poses, s.patches
    for it in range(s.iters):
        ba.step(1, s.fixed)
        ba.sync()
        r = oracle.gn(s, iters=1, poses=poses, patches=patches, pixels=9)
        poses, patches = r["poses"], r["patches"]
        rot, tr = pose_error(T["poses"].cpu().numpy(), poses)
        dep = depth_error(T["patches"][:, 2, 1, 1].cpu().numpy().astype(np.float64), patches[:, 2, 1, 1])
        assert rot < TOL and tr < TOL and dep < TOL, (it, rot, tr, dep)


def test_large_solver_and_loop_edges():
    # 6 * 58 = 348 unknowns (the blocked solver), local and loop edges
    s = full(scenes._build("sized", 13, 60, lambda i, n: scenes._clipped_window(i, n, 6), 2, 1, loop=True))
    ba, T = bind(s, precision="mixed")
    ba.step(1, s.fixed)
    ba.sync()
    r = oracle.gn(s, iters=1, pixels=9)
    rot, tr = pose_error(T["poses"].cpu().numpy(), r["poses"])
    dep = depth_error(T["patches"][:, 2, 1, 1].cpu().numpy().astype(np.float64), r["patches"][:, 2, 1, 1])
    assert rot < TOL and tr < TOL and dep < TOL, (rot, tr, dep)


def test_noise_free_converges_and_batched_matches():
    s = full(scenes.noise_free(scenes.tiny(seed=4)))
    ba, T = bind(s, precision="mixed")
    ba.step(8, s.fixed)
    ba.sync()
    rot, tr = pose_error(T["poses"].cpu().numpy(), s.poses_gt)
    assert rot < 1e-5 and tr < 1e-5
    # two problems bound together: each matches its own oracle run
    probs = [full(scenes.tiny(seed=5)), full(scenes.odometry(seed=6))]
    Tb, offs = batch_tensors(probs)
    bb = DPVBA(residual_pixels=9, precision="mixed")
    bb.set_graph_batched(**Tb, **offs)
    bb.step(1, 2)
    bb.sync()
    f0 = 0
    for p in probs:
        r = oracle.gn(p, iters=1, pixels=9)
        got = Tb["poses"][f0:f0 + p.N].cpu().numpy()
        rot, tr = pose_error(got, r["poses"])
        assert rot < TOL and tr < TOL, (rot, tr)
        f0 += p.N


def test_centre_only_unchanged_and_errors():
    s = scenes.tiny(seed=2)
    a, Ta = DPVBA(), scene_tensors(s)
    a.set_graph(**Ta)
    a.step(2, s.fixed)
    a.sync()
    b, Tb = DPVBA(residual_pixels=1), scene_tensors(s)
    b.set_graph(**Tb)
    b.step(2, s.fixed)
    b.sync()
    assert np.abs(Ta["poses"].cpu().numpy() - Tb["poses"].cpu().numpy()).max() < 1e-9
    with pytest.raises(ValueError):  # [E,2] targets on a whole-patch handle
        DPVBA(residual_pixels=9).set_graph(**scene_tensors(s))
    with pytest.raises(capi.BAError) as e:
        DPVBA(residual_pixels=4)
    assert e.value.status == capi.BA_ERR_INVALID_ARG


@pytest.mark.parametrize("make,precision", [(scenes.tiny, "fp32"), (scenes.tiny, "mixed"), (scenes.odometry, "mixed")])
def test_backward_matches_oracle(make, precision):
    # ba_backward over recorded whole-patch iterations against the oracle's
    # dual-number derivatives of single pixel targets and edge weights; the
    # tolerance of the centre-only adjoint tests (1e-4 of the sample's
    # largest gradient, 1e-3 on its 2-norm)
    s = full(make(seed=0))
    rng = np.random.default_rng(0)
    a, b = rng.normal(size=(s.N, 7)), rng.normal(size=s.P)
    ba, T = bind(s, precision=precision)
    ba.set_record(True)
    ba.step(s.iters, s.fixed)
    gT, gW = ba.backward(torch.as_tensor(a, dtype=torch.float64).cuda(),
                         torch.as_tensor(b, dtype=torch.float32).cuda())
    ba.sync()
    assert gT.shape == (s.E, 3, 3, 2)
    n = 40 if s.E > 10000 else 120
    kind = np.r_[np.zeros(n // 2, int), np.ones(n - n // 2, int)]
    index = np.r_[rng.choice(18 * s.E, n // 2, replace=False), rng.choice(2 * s.E, n - n // 2, replace=False)]
    want = oracle.grad_fwd(s, a, b, kind, index, pixels=9)
    gTn, gWn = gT.cpu().numpy().astype(np.float64), gW.cpu().numpy().astype(np.float64)
    got = np.r_[gTn.reshape(-1)[index[:n // 2]], gWn.reshape(-1)[index[n // 2:]]]
    err = np.abs(got - want).max() / np.abs(want).max()
    nerr = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert err < 1e-4 and nerr < 1e-3, (err, nerr)


def test_backward_initial_state_matches_oracle():
    # cotangents of the initial state through the whole-patch iterations: the
    # pose tangents (through the retraction's adjoint and every edge's nine
    # pixels) and the inverse depths (nine pixels per edge summed), against
    # the oracle's dual numbers of kinds 2 (initial depth) and 3 (initial
    # left pose perturbation) in the whole-patch mode
    s = full(scenes.tiny(seed=1))
    rng = np.random.default_rng(2)
    a, b = rng.normal(size=(s.N, 7)), rng.normal(size=s.P)
    ba, T = bind(s, precision="mixed")
    ba.set_record(True)
    ba.step(s.iters, s.fixed)
    gT, gW, x0, d0 = ba.backward(torch.as_tensor(a, dtype=torch.float64).cuda(),
                                 torch.as_tensor(b, dtype=torch.float32).cuda(), initial=True)
    ba.sync()
    kp = rng.choice(s.P, 24, replace=False)
    kx = rng.choice(np.arange(6 * s.fixed, 6 * s.N), 24, replace=False)
    want_d = oracle.grad_fwd(s, a, b, np.full(24, 2), kp, pixels=9)
    want_x = oracle.grad_fwd(s, a, b, np.full(24, 3), kx, pixels=9)
    for got, want in ((d0.cpu().numpy().astype(np.float64)[kp], want_d),
                      (x0.cpu().numpy().reshape(-1)[kx], want_x)):
        err = np.abs(got - want).max() / np.abs(want).max()
        nerr = np.linalg.norm(got - want) / np.linalg.norm(want)
        assert err < 1e-4 and nerr < 1e-3, (err, nerr)
    assert np.all(x0.cpu().numpy()[: s.fixed] == 0.0)


@pytest.mark.parametrize("layout", ["E92", "E332"])
def test_autograd_function_keeps_the_target_layout(layout):
    # the differentiable layer returns target gradients in the layout of the
    # targets it was given ([E,9,2] or [E,3,3,2]) and equal to ba_backward's
    s = full(scenes.tiny(seed=3))
    T = scene_tensors(s)
    shape = (s.E, 9, 2) if layout == "E92" else (s.E, 3, 3, 2)
    tg = T["targets"].reshape(shape).clone().requires_grad_(True)
    wt = T["weights"].clone().requires_grad_(True)
    rng = np.random.default_rng(4)
    a, b = rng.normal(size=(s.N, 7)), rng.normal(size=s.P)
    poses, depths = bundle_adjust(tg, wt, T["poses"], T["patches"], T["ii"], T["jj"], T["kk"], T["intrinsics"],
                                  s.iters, s.fixed, residual_pixels=9)
    L = (torch.as_tensor(a).cuda() * poses).sum() + (torch.as_tensor(b, dtype=torch.float32).cuda() * depths).sum()
    L.backward()
    assert tg.grad.shape == shape and wt.grad.shape == (s.E, 2)
    ba, T2 = bind(s)
    ba.set_record(True)
    ba.step(s.iters, s.fixed)
    gT, gW = ba.backward(torch.as_tensor(a, dtype=torch.float64).cuda(), torch.as_tensor(b, dtype=torch.float32).cuda())
    ba.sync()
    gTn = gT.reshape(shape)
    assert torch.allclose(tg.grad, gTn, rtol=1e-5, atol=1e-6 * float(gTn.abs().max()))
    assert torch.allclose(wt.grad, gW, rtol=1e-5, atol=1e-6 * float(gW.abs().max()))
