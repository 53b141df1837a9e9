"""The row envelope of the large pose systems (Sec. 3.2, the block-sparse
structure of the reduced system) and the factorisation restricted to it.

The factor L of an LDL^T without pivoting is zero left of each row's first
nonzero, so the persistent factorisation and the preconditioned solves visit
only the 64 x 64 tiles of the envelope.  The envelope is found on the GPU
from the values of S; here it must equal the one that the graph fixes (tile
rows of the free poses that share a patch: the pose-pose blocks and the
Schur fill of every patch's frames), and the steps it produces must match
the FP64 oracle (the loop-closure and parity tests cover the sizes).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2408_01654_b300 import scenes  # noqa: E402
from paper_2408_01654_b300.ba import DPVBA, batch_tensors, scene_tensors  # noqa: E402

from test_gpu_parity import depth_error, pose_error  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_01654_b300 import build
    build.build()
    oracle.build()


def graph_envelope(s, tile=64):
    """First tile column of each tile row of S from the graph alone."""
    M = s.P // s.N
    n = 6 * (s.N - s.fixed)
    T = (n + tile - 1) // tile
    env = np.arange(T)
    frames = [set() for _ in range(s.P)]
    for k, j in zip(np.asarray(s.kk), np.asarray(s.jj)):
        frames[int(k)].add(int(j))
    for k in range(s.P):
        f = [x - s.fixed for x in frames[k] | {k // M} if x >= s.fixed]
        if not f:
            continue
        tiles = sorted({6 * x // tile for x in f} | {(6 * x + 5) // tile for x in f})
        for t in tiles:
            env[t] = min(env[t], tiles[0])
    return env


def test_envelope_of_the_loop_closure_system():
    s = scenes.global_ba(seed=0, N=400)
    ba = DPVBA(precision="mixed")
    ba.set_graph(**scene_tensors(s))
    ba.step(1, s.fixed)
    ba.sync()
    (env,) = ba.envelope()
    want = graph_envelope(s)
    assert np.array_equal(env, want)
    assert (env < np.arange(len(env))).sum() > 0 and env.min() == 0


def test_envelope_of_a_batch():
    probs = [scenes.global_ba(seed=3, N=120), scenes.tiny(seed=1), scenes.global_ba(seed=4, N=90)]
    T, offs = batch_tensors(probs)
    ba = DPVBA(precision="mixed")
    ba.set_graph_batched(**T, **offs)
    ba.step(1, probs[0].fixed)
    ba.sync()
    envs = ba.envelope()
    assert len(envs) == 2  # the two systems above 256 unknowns
    assert np.array_equal(envs[0], graph_envelope(probs[0]))
    assert np.array_equal(envs[1], graph_envelope(probs[2]))


def two_passes(seed=21, Na=34):
    """The same 34-frame trajectory twice (frames Na..2Na-1 repeat frames
    0..Na-1, patches and observations included), the second pass also
    observed in the two fixed frames 0 and 1 (the first pass's edges into
    them, copied): in the pose system (fixed poses eliminated) the passes are
    uncoupled, the second pass's gauge is fixed through the fixed frames, and
    with 6 (Na - 2) = 192 unknowns the second pass begins on a tile row of
    its own."""
    import dataclasses
    a = scenes._build("two passes", seed, Na, lambda i, n: scenes._clipped_window(i, n, 6), 2, 2)
    M = a.P // a.N
    cp = np.nonzero(np.asarray(a.jj) < a.fixed)[0]  # first-pass edges into the fixed frames
    cat = np.concatenate
    return dataclasses.replace(
        a, N=2 * a.N, P=2 * a.P, E=2 * a.E + len(cp),
        poses=cat([a.poses, a.poses]), patches=cat([a.patches, a.patches]),
        ii=cat([a.ii, a.ii + a.N, a.ii[cp] + a.N]), jj=cat([a.jj, a.jj + a.N, a.jj[cp]]),
        kk=cat([a.kk, a.kk + a.P, a.kk[cp] + a.P]), targets=cat([a.targets, a.targets, a.targets[cp]]),
        weights=cat([a.weights, a.weights, a.weights[cp]]), poses_gt=cat([a.poses_gt, a.poses_gt]),
        depth_gt=cat([a.depth_gt, a.depth_gt]), proj_gt=cat([a.proj_gt, a.proj_gt, a.proj_gt[cp]]))


def test_uncoupled_blocks_factor_without_coupling():
    """A pose system with two uncoupled diagonal blocks: the tile rows of the
    second start their own envelope (env[a] = a: the factorisation's
    diagonal step takes no panel and no update there) and the steps match
    the oracle's."""
    s = two_passes()
    ba = DPVBA(precision="mixed")
    T = scene_tensors(s)
    ba.set_graph(**T)
    want = oracle.gn_steps(s, iters=2)
    for it in range(2):
        ba.step(1, s.fixed)
        ba.sync()
        rot, tr = pose_error(T["poses"].cpu().numpy(), want[it][0])
        dep = depth_error(T["patches"][:, 2, 1, 1].cpu().numpy().astype(np.float64), want[it][1])
        assert rot < 1e-5 and tr < 1e-5 and dep < 1e-5, (it, rot, tr, dep)
    (env,) = ba.envelope()
    assert np.array_equal(env, graph_envelope(s))
    assert env[3] == 3  # the second pass's first tile row
