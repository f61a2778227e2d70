"""Failure detection without a GPU fault: a kernel whose mbarrier is never
completed gives up after its bounded wait, reports DCFLOW_ERR_TIMEOUT through
the error word, and the context keeps working."""
import numpy as np
import pytest

import oracle
from paper_2501_17529_b300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2501_17529_b300.csrc import build
    build.build()


def test_bounded_wait_expires_and_context_survives():
    from paper_2501_17529_b300.dcflow import DeviceBatch, Solver, dcflow_selftest_bounded_wait
    w = synth.workload(1)
    lim = oracle.thermal_limits(w.grid, w.inj)
    s = Solver(w.grid, precision="fp64")
    s.set_study(w.mon, w.cont, lim, split_bus=w.subs)
    assert dcflow_selftest_bounded_wait(s.ctx) == -5  # DCFLOW_ERR_TIMEOUT, as designed
    out = s.solve(DeviceBatch(w.topo, w.inj)).to_host()  # the context is still usable
    ref = oracle.evaluate(w.grid, w.topo, w.inj, w.mon, w.cont, lim)
    np.testing.assert_array_equal(out["status"], ref["status"])
    ok = ref["status"] == 0
    np.testing.assert_allclose(out["n1_max"][ok], ref["n1_max"][ok], rtol=1e-10, atol=1e-10)
    s.close()
