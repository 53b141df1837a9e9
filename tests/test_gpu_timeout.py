"""A bounded device-side wait that runs out (failure detection without a fault).

Every wait of the library's persistent kernels on another CTA (tile versions
of the factorisation, solved-row words and grid barriers of the solve, the
radix sort's barriers) gives up after ``timeout_cycles`` and writes
BA_ERR_TIMEOUT to the handle's device status; the kernels that follow skip
their work, so the poses and depths keep their last completed values, and the
CUDA context stays usable.  Waits on a CTA's own bulk copies and MMAs keep a
floor of ~0.1 s, so a short budget never abandons an operation in flight.

The test gives a handle a budget of 2,000 cycles (~1 us), far below the
~20 us one diagonal step of the factorisation takes, so the workers' first
wait for a panel runs out; nothing faults or hangs: every wait still ends.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2408_01654_b300 import capi, scenes  # noqa: E402
from paper_2408_01654_b300.ba import DPVBA, scene_tensors  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_01654_b300 import build
    build.build()


def sized(frames):
    return scenes._build("sized", 13, frames, lambda i, n: scenes._clipped_window(i, n, 6), 2, 2)


def test_factorisation_wait_runs_out_and_state_is_kept():
    s = sized(60)  # 348 unknowns: the persistent tiled factorisation
    # kk-sorted: the binding's sort is skipped; its two other grid barriers keep a ~0.05 s floor
    assert np.all(np.diff(s.kk) >= 0)
    T = scene_tensors(s)
    p0, t0 = T["poses"].clone(), T["patches"].clone()
    ba = DPVBA(precision="mixed", timeout_cycles=2000)
    ba.set_graph(**T)
    ba.sync()  # the binding has no wait on this input
    ba.step(1, s.fixed)
    with pytest.raises(capi.BAError) as e:
        ba.sync()
    assert e.value.status == capi.BA_ERR_TIMEOUT
    assert torch.equal(T["poses"], p0) and torch.equal(T["patches"], t0)
    # a later call on the same handle does no work either
    ba.step(1, s.fixed)
    with pytest.raises(capi.BAError):
        ba.sync()
    assert torch.equal(T["poses"], p0)
    ba.close()
    # the context is intact: a handle with the default budget solves the same graph
    T2 = scene_tensors(s)
    ok = DPVBA(precision="mixed")
    ok.set_graph(**T2)
    ok.step(1, s.fixed)
    ok.sync()
    assert not torch.equal(T2["poses"], p0)
    assert torch.isfinite(T2["poses"]).all()


def test_one_cta_systems_have_no_wait_to_run_out():
    # the one-CTA solver waits on no other CTA: the same budget changes nothing
    s = sized(20)  # 108 unknowns
    Ta, Tb = scene_tensors(s), scene_tensors(s)
    a = DPVBA(precision="mixed", timeout_cycles=2000)
    b = DPVBA(precision="mixed")
    for h, T in ((a, Ta), (b, Tb)):
        h.set_graph(**T)
        h.step(2, s.fixed)
        h.sync()
    assert torch.allclose(Ta["poses"], Tb["poses"], rtol=0, atol=1e-9)
