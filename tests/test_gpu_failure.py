"""Failure detection without faulting the GPU: every device-side wait of the
pair kernel is bounded.  A test hook (HSMA_TEST_STALL_WAIT=1 when the plan is
created) makes the kernel wait on an mbarrier that nothing arrives at; the
wait runs out after ~1e6 cycles, the kernel records a timeout and returns,
the call reports HSMA_E_TIMEOUT, and the context stays usable."""
import numpy as np
import pytest

from gpu_common import to_dev
from paper_1806_04801_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_context_survives(monkeypatch):
    import torch
    from paper_1806_04801_gb300 import build, hsma
    assert torch.cuda.is_available()
    build.build()
    w = I.SMALL_PERIODIC
    xyz, q = I.small_periodic()
    dx, dq = to_dev(xyz, q)
    monkeypatch.setenv("HSMA_TEST_STALL_WAIT", "1")
    stalled = hsma.Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon)
    monkeypatch.delenv("HSMA_TEST_STALL_WAIT")
    with pytest.raises(hsma.HsmaError) as ei:
        stalled.energy_forces(dx, dq)
    assert ei.value.code == -6
    stalled.close()
    with hsma.Plan(w.box, w.bc, w.p, w.R, w.Q, w.Kmon) as plan:
        U, F, _, _ = plan.energy_forces(dx, dq)
        U2, F2, _, _ = plan.energy_forces(dx, dq)
    assert np.isfinite(U) and U == U2 and bool((F == F2).all())
    torch.cuda.synchronize()
