"""The allocation-free base-PTDF entry point matches dcflow_base_ptdf and the oracle.

dcflow_base_ptdf_noalloc serves callers that cannot allocate device memory
(an arena they do not own, allocator-free real-time loops): its workspace is a
fixed array inside the library.  This file is collected last so that a run
stopping at the first failure has run every other test before it.
"""
import numpy as np
import pytest

import oracle
from paper_2501_17529_b300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_noalloc_matches_base_ptdf_twice():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2501_17529_b300.csrc import build
    build.build()
    from paper_2501_17529_b300 import dcflow

    g = synth.make_grid(300, 420, 61)
    # the base PTDF by its definition (Def. 2 / Eq. (1)), FP64 on the CPU
    pt_ref = oracle.ptdf(g.n_bus, g.f, g.t, g.b, g.slack)
    ctx = dcflow.dcflow_setup(g.n_bus, g.f, g.t, g.b, g.slack, precision="fp64")
    try:
        # two calls in a row with different row sets: the second must not see the first's contents
        for rows in (np.array([0, 7, 33, 419, 200, 5], np.int32), np.arange(0, 420, 3, dtype=np.int32)):
            ref = torch.empty((rows.size, g.n_bus), dtype=torch.float64, device="cuda")
            got = torch.full((rows.size, g.n_bus), np.nan, dtype=torch.float64, device="cuda")
            dcflow.dcflow_base_ptdf(ctx, rows, ref)
            dcflow.dcflow_base_ptdf_noalloc(ctx, rows, got)
            torch.cuda.synchronize()
            err = (got - ref).abs().max().item()
            assert err <= 1e-12, err
            assert torch.all(got[:, g.slack] == 0)
            err_o = np.abs(got.cpu().numpy() - pt_ref[rows]).max()
            assert err_o <= 1e-11 * max(1.0, np.abs(pt_ref).max()), err_o
        # a request larger than the fixed workspace is refused, not attempted
        big = np.arange(420, dtype=np.int32).repeat(40)
        out = torch.empty((big.size, g.n_bus), dtype=torch.float64, device="cuda")
        with pytest.raises(dcflow.DCFlowError) as e:
            dcflow.dcflow_base_ptdf_noalloc(ctx, big, out)
        assert e.value.code == -1
    finally:
        dcflow.dcflow_destroy(ctx)
