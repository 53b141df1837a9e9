"""The multi-rank path on the CPU: world size 2 over gloo (no GPU).  Each
rank works on its own independent problem (no collective on the data path);
the only exchange is the max over ranks of the timed region, and the job's
throughput is all ranks' work over that slowest time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2408_01654_b300 import multi, scenes  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = multi.rank_info()
        # each rank its own problem: a different seeded scene
        s = scenes.tiny(seed=multi.problem_seed(r))
        local_ms = 10.0 + 5.0 * r  # this rank's timed region
        mx = multi.max_over_ranks(local_ms)
        out[r] = (r, w, local, float(s.targets.sum()), mx, multi.job_throughput(3 * s.iters, w, mx))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_gloo_ranks_time_by_their_slowest_and_solve_their_own_problems():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
        res = dict(out)
    assert sorted(res) == [0, 1]
    for r in (0, 1):
        rr, w, local, tsum, mx, thr = res[r]
        assert (rr, w, local) == (r, world, r)
        assert mx == 15.0  # the slower rank's 15 ms on both ranks
        assert thr == pytest.approx(world * 3 * 2 / 0.015)  # 3 steps x 2 iterations per rank
    assert res[0][3] != res[1][3]  # independent problems


def test_single_process_needs_no_group():
    assert multi.max_over_ranks(3.5) == 3.5
    assert multi.job_throughput(100, 1, 1000.0) == 100.0


def test_shard_problems_balances_cubic_cost_and_covers_every_problem():
    rng = __import__("numpy").random.default_rng(0)
    frames = [int(v) for v in rng.integers(8, 400, size=64)]
    for world in (1, 2, 3, 8):
        parts = multi.shard_problems(frames, world)
        assert len(parts) == world
        flat = sorted(b for p in parts for b in p)
        assert flat == list(range(len(frames)))
        loads = [sum(frames[b] ** 3 for b in p) for p in parts]
        # greedy LPT: no rank exceeds the mean by more than the largest single problem
        assert max(loads) <= sum(loads) / world + max(f ** 3 for f in frames)
    assert multi.shard_problems([5, 9, 7], 2) == [[1], [0, 2]]
    with pytest.raises(ValueError):
        multi.shard_problems([1], 0)
