"""GPU tests of the batched-execution patterns: ba_step replayed from a
captured CUDA graph (ba_set_capture) and the group-size autotuner
(ba_autotune).  A replayed step runs the same kernels in the same order as
the eager step, so results agree up to the order of the FP64 atomics; the
batched case is also held to the FP64 oracle at the per-step tolerance."""
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
    yield
    capi.lib().ba_autotune_clear()  # later tests see the fixed automatic rule


def close(a, b):
    """equal up to the order of the FP64 atomic sums"""
    assert np.allclose(a["poses"].cpu().numpy(), b["poses"].cpu().numpy(), rtol=0, atol=1e-9)
    da = a["patches"][:, 2, 1, 1].cpu().numpy()
    db = b["patches"][:, 2, 1, 1].cpu().numpy()
    assert np.allclose(da, db, rtol=1e-6, atol=0)


def steady(ba, before, step=True):
    """one more call replayed both graphs (the step's only if `step`) and captured nothing"""
    now = ba.info()
    assert now["bind_replays"] == before["bind_replays"] + 1, (before, now)
    assert now["graph_replays"] == before["graph_replays"] + (1 if step else 0), (before, now)
    assert now["bind_captures"] == before["bind_captures"] and now["graph_captures"] == before["graph_captures"]
    return now


def run_calls(ba, T, pristine, calls, iters, fixed, batched_offs=None):
    """`calls` times: restore the state, rebind the same buffers, step."""
    for _ in range(calls):
        T["poses"].copy_(pristine["poses"])
        T["patches"].copy_(pristine["patches"])
        if batched_offs is None:
            ba.set_graph(**T)
        else:
            ba.set_graph_batched(**T, **batched_offs)
        ba.step(iters, fixed)
    ba.sync()


def test_capture_odometry_matches_eager():
    s = scenes.odometry(seed=0)
    T0 = scene_tensors(s)
    pristine = {k: v.clone() for k, v in T0.items()}
    Te = {k: v.clone() for k, v in T0.items()}
    eager = DPVBA()
    run_calls(eager, Te, pristine, 1, s.iters, s.fixed)
    g = DPVBA(capture=True)
    run_calls(g, T0, pristine, 4, s.iters, s.fixed)
    before = g.info()
    run_calls(g, T0, pristine, 1, s.iters, s.fixed)
    inf = steady(g, before)
    assert inf["graph_captures"] == 1 and inf["bind_captures"] == 1, inf
    assert inf["graph_kernels"] > 0 and inf["bind_kernels"] > 0
    close(T0, Te)
    # the replayed step against the oracle
    want = oracle.gn_steps(s, iters=s.iters)[-1]
    rot, tr = pose_error(T0["poses"].cpu().numpy(), want[0])
    dep = depth_error(T0["patches"][:, 2, 1, 1].cpu().numpy().astype(np.float64), want[1])
    assert rot < TOL * s.iters and tr < TOL * s.iters and dep < TOL * s.iters, (rot, tr, dep)


def test_capture_batched_with_large_systems_matches_oracle():
    # small one-CTA systems and two large systems (the persistent cooperative
    # factorisation and solve kernels inside the graph)
    frames = [12, 50, 9, 46]
    probs = [scenes._build("batched", 700 + b, n, lambda i, m: scenes._clipped_window(i, m, 6), 2, 1, loop=True)
             for b, n in enumerate(frames)]
    T, offs = batch_tensors(probs)
    pristine = {k: v.clone() for k, v in T.items()}
    Te = {k: v.clone() for k, v in T.items()}
    eager = DPVBA(precision="mixed")
    run_calls(eager, Te, pristine, 1, 1, 2, offs)
    g = DPVBA(precision="mixed", capture=True)
    run_calls(g, T, pristine, 3, 1, 2, offs)
    before = g.info()
    run_calls(g, T, pristine, 1, 1, 2, offs)
    steady(g, before)
    close(T, Te)
    for b, sc in enumerate(probs):
        want = oracle.gn_steps(sc, iters=1)[0]
        f0, f1 = offs["frame_off"][b], offs["frame_off"][b + 1]
        p0, p1 = offs["patch_off"][b], offs["patch_off"][b + 1]
        rot, tr = pose_error(T["poses"][f0:f1].cpu().numpy(), want[0])
        dep = depth_error(T["patches"][p0:p1, 2, 1, 1].cpu().numpy().astype(np.float64), want[1])
        assert rot < TOL and tr < TOL and dep < TOL, (b, rot, tr, dep)


def test_capture_follows_new_contents_and_rekeys():
    s = scenes.odometry(seed=3)
    T = scene_tensors(s)
    pristine = {k: v.clone() for k, v in T.items()}
    g = DPVBA(capture=True)
    run_calls(g, T, pristine, 4, s.iters, s.fixed)
    before = g.info()
    # new contents in the same buffers: the graph is kept and follows them
    gen = torch.Generator(device="cpu").manual_seed(5)
    new = {k: v.clone() for k, v in pristine.items()}
    new["targets"] += (0.3 * torch.randn(new["targets"].shape, generator=gen)).to(new["targets"].device)
    new["poses"][s.fixed:, :3] += 0.01
    for k in T:
        pristine[k].copy_(new[k])
        T[k].copy_(new[k])
    run_calls(g, T, pristine, 1, s.iters, s.fixed)
    steady(g, before)
    Te = {k: v.clone() for k, v in new.items()}
    e = DPVBA()
    run_calls(e, Te, {k: v.clone() for k, v in new.items()}, 1, s.iters, s.fixed)
    close(T, Te)
    # another iteration count is another step graph (eager first, then captured)
    run_calls(g, T, pristine, 2, 1, s.fixed)
    assert g.info()["graph_captures"] == 2
    # recording a tape runs the step eagerly (the binding still replays)
    g.set_record(True)
    before = g.info()
    run_calls(g, T, pristine, 1, 1, s.fixed)
    steady(g, before, step=False)
    g.set_record(False)
    g.set_capture(False)
    before = g.info()
    run_calls(g, T, pristine, 1, 1, s.fixed)
    now = g.info()
    assert now["graph_replays"] == before["graph_replays"] and now["bind_replays"] == before["bind_replays"]


def test_capture_profiling_reads_every_replay():
    s = scenes.odometry(seed=0)
    T = scene_tensors(s)
    pristine = {k: v.clone() for k, v in T.items()}
    g = DPVBA(capture=True)
    g.profile(True)
    run_calls(g, T, pristine, 6, s.iters, s.fixed)  # eager runs, captures, then replays
    prof = g.profile_read()
    assert g.info()["graph_replays"] >= 3 and g.info()["bind_replays"] >= 3
    # one solve and one back-substitution per iteration in each of the 6 steps, one
    # preprocessing pass per binding, whether eager, captured or replayed
    assert prof["solve"][1] == 6 * s.iters and prof["backsub"][1] == 6 * s.iters, prof
    assert prof["preprocess"][1] == 6, prof
    assert prof["solve"][0] > 0 and prof["assemble"][0] > 0 and prof["preprocess"][0] > 0


def test_profile_classes_records_only_the_chosen_class():
    s = scenes.odometry(seed=0)
    T = scene_tensors(s)
    pristine = {k: v.clone() for k, v in T.items()}
    g = DPVBA(capture=True)
    g.profile(True, classes=["solve"])
    run_calls(g, T, pristine, 5, s.iters, s.fixed)
    prof = g.profile_read()
    assert prof["solve"][1] == 5 * s.iters and prof["solve"][0] > 0, prof
    assert all(v == (0.0, 0) for k, v in prof.items() if k != "solve"), prof
    # switching to every class re-captures the step: the replays record all classes again
    g.profile(True)
    run_calls(g, T, pristine, 4, s.iters, s.fixed)
    prof = g.profile_read()
    assert prof["backsub"][1] == 4 * s.iters and prof["preprocess"][1] == 4, prof
    # the poses after the masked replays match an unprofiled handle's
    T2 = {k: v.clone() for k, v in pristine.items()}
    ref = DPVBA(capture=True)
    run_calls(ref, T2, pristine, 1, s.iters, s.fixed)
    close(T, T2)
    # a bit beyond the last class is refused
    assert g._lib.ba_profile_classes(g._h, 1 << len(capi.KERNEL_CLASSES)) == capi.BA_ERR_INVALID_ARG


def test_autotune_keeps_state_and_fills_table():
    s = scenes.odometry(seed=0)
    T = scene_tensors(s)
    before = {k: v.clone() for k, v in T.items()}
    ba = DPVBA()
    ba.set_graph(**T)
    res = ba.autotune(s.iters, s.fixed, reps=2)
    assert res["G"] in (8, 16, 24, 32, 48, 64)
    assert res["candidates"][res["G"]] == min(v for v in res["candidates"].values() if v >= 0)
    assert ba.info()["G"] == res["G"]
    for k in T:
        assert torch.equal(T[k], before[k]), k
    # the tuned handle steps like a handle created with that size
    ba.step(s.iters, s.fixed)
    ba.sync()
    T2 = {k: v.clone() for k, v in before.items()}
    ref = DPVBA(patches_per_group=res["G"])
    ref.set_graph(**T2)
    ref.step(s.iters, s.fixed)
    ref.sync()
    close(T, T2)
    # a new automatic handle of the same shape class takes the tuned size
    auto = DPVBA()
    auto.set_graph(**scene_tensors(scenes.odometry(seed=1)))
    assert auto.info()["G"] == res["G"]


def test_autotune_batched_with_capture():
    probs = [scenes._build("batched", 900 + b, n, lambda i, m: scenes._clipped_window(i, m, 6), 2, 1, loop=True)
             for b, n in enumerate([10, 30, 17])]
    T, offs = batch_tensors(probs)
    before = {k: v.clone() for k, v in T.items()}
    ba = DPVBA(precision="mixed", capture=True, patches_per_group=8)
    ba.set_graph_batched(**T, **offs)
    res = ba.autotune(1, 2, reps=2)
    assert ba.info()["G"] == res["G"]  # explicit size: the handle keeps the best one
    for k in T:
        assert torch.equal(T[k], before[k]), k
    ba.step(1, 2)
    ba.sync()
    for b, sc in enumerate(probs):
        want = oracle.gn_steps(sc, iters=1)[0]
        f0, f1 = offs["frame_off"][b], offs["frame_off"][b + 1]
        p0, p1 = offs["patch_off"][b], offs["patch_off"][b + 1]
        rot, tr = pose_error(T["poses"][f0:f1].cpu().numpy(), want[0])
        dep = depth_error(T["patches"][p0:p1, 2, 1, 1].cpu().numpy().astype(np.float64), want[1])
        assert rot < TOL and tr < TOL and dep < TOL, (b, rot, tr, dep)


def test_autotune_errors():
    ba = DPVBA()
    with pytest.raises(capi.BAError) as e:
        ba.autotune(1, 0)
    assert e.value.status == capi.BA_ERR_STATE
