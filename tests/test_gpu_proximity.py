"""GPU parity of the proximity loop-edge construction (ba_proximity_edges,
Sec. 3.2 "Proximity Loop Closure") against the FP64 oracle.

Selections and edge indices are compared bit for bit; every comparison first
checks that the oracle's decisions are not within rounding of a threshold
(margin), which is what makes bit equality the right bar.  Reprojected pixels
are FP64 rounded to float32 on both sides: equal to one float32 ulp.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2408_01654_b300 import capi, scenes  # noqa: E402
from paper_2408_01654_b300.ba import DPVBA, scene_tensors  # noqa: E402

from test_gpu_parity import depth_error, pose_error  # noqa: E402

Z_MIN = float(np.float32(0.1))  # the handle keeps z_min in float32
PIX_TOL = 2e-4                  # one float32 ulp at 640 px is 6.1e-5
MARGIN = 1e-9


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_01654_b300 import build
    build.build()
    oracle.build()


def problem(N, M, seed, step_m=0.1):
    """Random-walk trajectory (the global workload's) with M random patches
    per frame; poses perturbed like the scenes' initial estimates."""
    rng = np.random.default_rng(seed)
    G = scenes._random_walk(rng, N, step_m=step_m)
    R, t = scenes._world_to_camera(G)
    poses = scenes._pose_vec(R, t)
    poses[:, :3] += rng.normal(0.0, 0.02, size=(N, 3))
    patches = np.zeros((N * M, 3, 3, 3), np.float32)
    u = rng.uniform(-20.0, 660.0, N * M)
    v = rng.uniform(-20.0, 500.0, N * M)
    d = rng.uniform(0.2, 2.0, N * M)
    off = np.array([-1.0, 0.0, 1.0])
    patches[:, 0] = (u[:, None, None] + off[None, None, :]).astype(np.float32)
    patches[:, 1] = (v[:, None, None] + off[None, :, None]).astype(np.float32)
    patches[:, 2] = d[:, None, None].astype(np.float32)
    return poses, patches, np.array([scenes.FX, scenes.FY, scenes.CX, scenes.CY], np.float32)


def run_both(poses, patches, intr, M, b0=0, b1=None, gap=30, radius=2.0, ba=None):
    N = len(poses)
    b1 = N if b1 is None else b1
    want = oracle.proximity_edges(poses, patches.astype(np.float64), intr.astype(np.float64), M, b0, b1, gap=gap,
                                  radius=radius, z_min=Z_MIN)
    ba = ba or DPVBA()
    got = ba.proximity_edges(torch.tensor(poses, device="cuda"), torch.tensor(patches, device="cuda"), intr, M,
                             b0, b1, gap=gap, radius=radius)
    return want, got


def assert_same(want, got):
    assert want["margin"].min() > MARGIN, want["margin"].min()
    assert got["n"] == want["n"]
    assert np.array_equal(got["match"].cpu().numpy(), want["match"])
    for k in ("ii", "jj", "kk"):
        assert np.array_equal(got[k].cpu().numpy(), want[k]), k
    assert np.abs(got["coords"].cpu().numpy().astype(np.float64) - want["coords"]).max(initial=0.0) < PIX_TOL


@pytest.mark.parametrize("N,M,seed", [(150, 96, 0), (230, 70, 1), (97, 33, 2), (120, 1, 3), (60, 1024, 4)])
def test_matches_oracle(N, M, seed):
    # M = 70, 33: a ragged last mask word; M = 1: one patch; M = 1024: the limit
    poses, patches, intr = problem(N, M, seed)
    gap = 30 if N > 80 else 10
    want, got = run_both(poses, patches, intr, M, gap=gap)
    assert (want["match"] >= 0).sum() > 5 and want["n"] > 0
    assert_same(want, got)


def test_full_size_loop_graph():
    # the global workload's shape: 1000 frames, 96 patches per frame, every frame queried
    poses, patches, intr = problem(1000, 96, 0)
    want, got = run_both(poses, patches, intr, 96)
    assert want["n"] > 20000
    assert_same(want, got)


def test_scene_generator_loop_edges_from_ground_truth():
    s = scenes._build("proximity", 5, 300, lambda i, m: scenes._clipped_window(i, m, 6), 2, 1, loop=True)
    M = scenes.PATCHES_PER_FRAME
    pt = s.patches.copy()
    pt[:, 2] = s.depth_gt[:, None, None].astype(np.float32)
    want, got = run_both(s.poses_gt, pt, s.intrinsics, M)
    assert_same(want, got)


def test_query_window_appended_after_local_edges():
    poses, patches, intr = problem(400, 96, 6)
    M, b0, b1, E_local = 96, 380, 400, 12345
    want = oracle.proximity_edges(poses, patches.astype(np.float64), intr.astype(np.float64), M, b0, b1,
                                  z_min=Z_MIN)
    cap = (b1 - b0) * M
    ii = torch.full((E_local + cap,), -7, dtype=torch.int32, device="cuda")
    jj, kk = ii.clone(), ii.clone()
    out = {"ii": ii[E_local:], "jj": jj[E_local:], "kk": kk[E_local:]}
    got = DPVBA().proximity_edges(torch.tensor(poses, device="cuda"), torch.tensor(patches, device="cuda"), intr,
                                  M, b0, b1, out=out)
    assert got["n"] == want["n"] > 0
    assert torch.all(ii[:E_local] == -7)
    n = want["n"]
    assert np.array_equal(ii[E_local:E_local + n].cpu().numpy(), want["ii"])
    assert np.array_equal(kk[E_local:E_local + n].cpu().numpy(), want["kk"])
    assert np.array_equal(got["match"].cpu().numpy(), want["match"])


def test_capacity_and_device_count():
    poses, patches, intr = problem(200, 96, 7)
    want = oracle.proximity_edges(poses, patches.astype(np.float64), intr.astype(np.float64), 96, 0, 200,
                                  z_min=Z_MIN)
    cap = want["n"] // 2
    out = {k: torch.full((cap,), -1, dtype=torch.int32, device="cuda") for k in ("ii", "jj", "kk")}
    out["count"] = torch.zeros(1, dtype=torch.int32, device="cuda")
    ba = DPVBA()
    P, T = torch.tensor(poses, device="cuda"), torch.tensor(patches, device="cuda")
    with pytest.raises(capi.BAError) as e:
        ba.proximity_edges(P, T, intr, 96, out=out)
    assert e.value.status == capi.BA_ERR_INVALID_ARG
    assert int(out["count"].item()) == want["n"]
    assert np.array_equal(out["kk"].cpu().numpy(), want["kk"][:cap])
    # queued only: the count stays on the device
    res = ba.proximity_edges(P, T, intr, 96, sync=False)
    torch.cuda.synchronize()
    n = int(res["count"].item())
    assert n == want["n"] and np.array_equal(res["jj"][:n].cpu().numpy(), want["jj"])


def test_degenerate_queries():
    poses, patches, intr = problem(90, 40, 8)
    ba = DPVBA()
    P, T = torch.tensor(poses, device="cuda"), torch.tensor(patches, device="cuda")
    assert ba.proximity_edges(P, T, intr, 40, 50, 50)["n"] == 0           # no query
    r = ba.proximity_edges(P, T, intr, 40, gap=90)                        # no candidate
    assert r["n"] == 0 and torch.all(r["match"] == -1)
    r = ba.proximity_edges(P, T, intr, 40, gap=0, radius=0.0)             # nothing closer than 0
    assert r["n"] == 0 and torch.all(r["match"] == -1)
    one = ba.proximity_edges(P[:1], T[:40], intr, 40)                     # a single frame
    assert one["n"] == 0 and int(one["match"][0]) == -1
    # duplicated poses: equal distances, the lowest index wins
    dup = np.repeat(poses[:1], 40, axis=0)
    want, got = run_both(dup, patches[:40 * 40], intr, 40, gap=5, radius=1.0)
    assert np.array_equal(want["match"][6:], np.zeros(34, np.int32))
    assert np.array_equal(got["match"].cpu().numpy(), want["match"]) and got["n"] == want["n"]
    assert np.array_equal(got["kk"].cpu().numpy(), want["kk"])


@pytest.mark.parametrize("kw", [dict(M=0), dict(M=1025), dict(b1=91), dict(b0=5, b1=4), dict(gap=-1),
                                dict(radius=-1.0), dict(radius=float("nan")), dict(width=0.0)])
def test_invalid_arguments(kw):
    poses, patches, intr = problem(90, 40, 8)
    P, T = torch.tensor(poses, device="cuda"), torch.tensor(patches, device="cuda")
    args = dict(M=40, b0=0, b1=None, gap=30, radius=2.0, width=640.0, height=480.0)
    args.update(kw)
    M = args.pop("M")
    out = None
    if M < 1 or M > 1024:
        out = {k: torch.zeros(8, dtype=torch.int32, device="cuda") for k in ("ii", "jj", "kk")}
        if M > 1024:  # patches enough for the size, so the library itself refuses it
            P, T = P[:2], torch.zeros((2 * M, 3, 3, 3), dtype=torch.float32, device="cuda")
            args["b1"] = 2
    with pytest.raises(capi.BAError) as e:
        DPVBA().proximity_edges(P, T, intr, M, out=out, **args)
    assert e.value.status == capi.BA_ERR_INVALID_ARG


def test_loop_edges_feed_global_bundle_adjustment():
    # local edges of a 90-frame graph, loop edges built on the GPU from the
    # current estimate, targets at the oracle's reprojections plus noise; one
    # GN step on the combined graph against the oracle's
    s = scenes._build("proximity_ba", 9, 90, lambda i, m: scenes._clipped_window(i, m, 4), 2, 1)
    M = scenes.PATCHES_PER_FRAME
    want = oracle.proximity_edges(s.poses, s.patches.astype(np.float64), s.intrinsics.astype(np.float64), M, 0,
                                  s.N, z_min=Z_MIN)
    assert want["margin"].min() > MARGIN and want["n"] > 500
    rng = np.random.default_rng(19)
    n = want["n"]
    lt = (want["coords"] + rng.normal(0.0, 0.5, size=(n, 2))).astype(np.float32)
    lw = rng.uniform(0.5, 1.0, size=(n, 2)).astype(np.float32)
    E0 = s.E
    T = scene_tensors(s)
    cap = s.N * M
    ii = torch.empty(E0 + cap, dtype=torch.int32, device="cuda")
    jj, kk = torch.empty_like(ii), torch.empty_like(ii)
    ii[:E0], jj[:E0], kk[:E0] = T["ii"], T["jj"], T["kk"]
    ba = DPVBA()
    got = ba.proximity_edges(T["poses"], T["patches"], s.intrinsics, M,
                             out={"ii": ii[E0:], "jj": jj[E0:], "kk": kk[E0:]})
    assert got["n"] == n
    assert np.array_equal(kk[E0:E0 + n].cpu().numpy(), want["kk"])
    assert np.array_equal(jj[E0:E0 + n].cpu().numpy(), want["jj"])
    E = E0 + n
    targets = torch.cat([T["targets"], torch.tensor(lt, device="cuda")]).contiguous()
    weights = torch.cat([T["weights"], torch.tensor(lw, device="cuda")]).contiguous()
    ba.set_graph(T["poses"], T["patches"], ii[:E].contiguous(), jj[:E].contiguous(), kk[:E].contiguous(),
                 targets, weights, T["intrinsics"])
    ba.step(1, s.fixed)
    ba.sync()
    import dataclasses
    g = dataclasses.replace(s, E=E, ii=np.concatenate([s.ii, want["ii"]]), jj=np.concatenate([s.jj, want["jj"]]),
                            kk=np.concatenate([s.kk, want["kk"]]), targets=np.concatenate([s.targets, lt]),
                            weights=np.concatenate([s.weights, lw]))
    ref = oracle.gn_steps(g, iters=1)[0]
    rot, tr = pose_error(T["poses"].cpu().numpy(), ref[0])
    dep = depth_error(T["patches"][:, 2, 1, 1].cpu().numpy().astype(np.float64), ref[1])
    assert rot < 1e-5 and tr < 1e-5 and dep < 1e-5, (rot, tr, dep)
