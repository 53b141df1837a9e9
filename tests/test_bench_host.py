"""Host-side arithmetic of bench.py, on the CPU: the envelope flop count that
the factorisation's roofline divides by, the choice of the dominant kernel
class, and the committed DRAM-traffic records the bench line reports."""
import importlib.util
import json
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_factor_flops_full_envelope_is_the_dense_count(bench):
    # every tile row reaching column 0: step k has m = T - 1 - k rows below, so the
    # sum is b^3 (T/3 + T(T-1)/2 + (T-1)T(2T-1)/6) = b^3 T^3 / 3: exactly n^3 / 3
    # for n = T b (the diagonal tiles' b^3/3 and the m^2 update term absorb the
    # lower-order terms of the dense count)
    b3 = 64.0 ** 3
    for T in (1, 2, 7, 94):
        got = bench.factor_flops([np.zeros(T, dtype=np.int64)])
        want = b3 * (T / 3 + T * (T - 1) / 2 + (T - 1) * T * (2 * T - 1) / 6)
        assert got == pytest.approx(want, rel=1e-12)
        assert got == pytest.approx((64.0 * T) ** 3 / 3, rel=1e-12)


def test_factor_flops_block_diagonal_and_sums_over_systems(bench):
    b3 = 64.0 ** 3
    diag = np.arange(5)  # env[a] = a: no tile below the diagonal anywhere
    assert bench.factor_flops([diag]) == pytest.approx(5 * b3 / 3)
    # a banded envelope: every row reaches one tile left of the diagonal
    band = np.maximum(np.arange(6) - 1, 0)
    m = [int(np.count_nonzero(band[k + 1:] <= k)) for k in range(6)]
    assert m == [1, 1, 1, 1, 1, 0]
    assert bench.factor_flops([band]) == pytest.approx(b3 * sum(1 / 3 + x + x * x for x in m))
    # several systems: the counts add
    assert bench.factor_flops([diag, band]) == pytest.approx(bench.factor_flops([diag]) +
                                                             bench.factor_flops([band]))


def test_dominant_class_takes_the_largest_time_with_launches(bench):
    prof = {"assemble": (2.5, 4), "solve": (3.5, 8), "factor": (9.0, 0), "backsub": (0.4, 4)}
    assert bench.dominant_class(prof) == "solve"  # a class without launches never dominates


def test_committed_traffic_records_point_at_profiles_and_follow_the_source(bench):
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        records = json.load(f)
    for key, rec in records.items():
        if key.startswith("_"):
            continue
        kind, workload = key.split(":")
        assert os.path.exists(os.path.join(ROOT, "profiles", rec["profile"])), key
        assert rec["dram_bytes_per_launch"] > 0, key
        assert len(rec["source_sha"]) == 16 and int(rec["source_sha"], 16) >= 0, key
        # reported while the kernel's source file is the one the counters were taken on
        current = bench.kernel_hash(kind) == rec["source_sha"]
        assert (bench.committed_traffic(kind, workload) == rec["dram_bytes_per_launch"]) == current, key
    assert bench.committed_traffic("assemble", "no-such-workload") is None
