"""GPU test of the allocation-free pose-system solve.

Some callers cannot allocate device memory when they need a solve (a tracking
loop with a fixed per-frame budget, where cudaMalloc may stall the device, or
a framework that owns every allocation).  They call
ba_solve_pose_system_noalloc, which keeps its working copy in a fixed device
array inside the library.  This test calls it through the C ABI and checks
that it returns the same pose step as ba_step on the same reduced system, on
two calls in a row with different systems (the shared array keeps the
previous call's contents, so the second call must not depend on them).
"""
import ctypes

import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2408_01654_b300 import capi, scenes  # noqa: E402
from paper_2408_01654_b300.ba import DPVBA, scene_tensors  # noqa: E402

TOL = 1e-5


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _system_and_step(scene):
    """The reduced system at the scene's initial state, and ba_step's pose step."""
    T = scene_tensors(scene)
    ba = DPVBA(precision="mixed", max_refine=2)  # FP64 refinement, as the call below
    ba.set_graph(**T)
    ba.linearize(scene.fixed)
    S = ba.export(capi.EXPORT_S).contiguous()
    y = ba.export(capi.EXPORT_Y).contiguous()
    ba.step(1, scene.fixed)
    ba.sync()
    return S, y, ba.export(capi.EXPORT_DX)


def test_noalloc_solve_matches_ba_step_on_two_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_01654_b300 import build
    build.build()
    L = capi.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    cases = [_system_and_step(scenes.odometry(seed=0)), _system_and_step(scenes.tiny(seed=0))]
    for S, y, want in cases:
        n = y.numel()
        x = torch.full_like(y, float("nan"))
        st = L.ba_solve_pose_system_noalloc(n, _ptr(S), _ptr(y), _ptr(x), 2, stream)
        assert st == capi.BA_OK, L.ba_status_string(st)
        err = ((x - want).abs().max() / want.abs().max()).item()
        assert err < TOL, err


def test_noalloc_rejects_sizes_beyond_its_limit():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L = capi.lib()
    buf = torch.zeros(257 * 257, dtype=torch.float64, device="cuda")
    st = L.ba_solve_pose_system_noalloc(257, _ptr(buf), _ptr(buf), _ptr(buf), 0, None)
    assert st == capi.BA_ERR_UNSUPPORTED
    st = L.ba_solve_pose_system_noalloc(0, _ptr(buf), _ptr(buf), _ptr(buf), 0, None)
    assert st == capi.BA_ERR_INVALID_ARG
