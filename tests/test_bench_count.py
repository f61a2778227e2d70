"""The benchmark's loadflow count (its metric's numerator) against the oracle's.

bench.py counts the solved N-1 cases from the solver's own outputs (status,
islanding-contingency counts) and the batch's outages; oracle.loadflow_count
counts them from the refactorising oracle.  On the same batch the two agree.
"""
import numpy as np

import bench
import oracle
from paper_2501_17529_b300 import synth


def test_bench_count_matches_oracle_count_grid500_sample():
    w = synth.workload(2, n_topo=24)
    lim = oracle.thermal_limits(w.grid, w.inj)
    r = oracle.evaluate(w.grid, w.topo, w.inj, w.mon, w.cont, lim)
    T = w.inj.shape[0]
    assert (r["status"] != 0).any() and (r["status"] == 0).any()
    assert bench._loadflows(w.topo, r["status"], r["n_island_cont"], w.cont, T) == oracle.loadflow_count(r, T)


def test_bench_count_matches_oracle_count_subset_contingencies():
    """Outaged branches inside and outside a contingency subset."""
    w = synth.workload(2, n_topo=16)
    rng = np.random.default_rng(3)
    cont = np.sort(rng.choice(w.grid.n_branch, 200, replace=False)).astype(np.int32)
    cont = np.union1d(cont, w.topo.out_branch[:20]).astype(np.int32)
    lim = oracle.thermal_limits(w.grid, w.inj[:2])
    r = oracle.evaluate(w.grid, w.topo, w.inj[:2], w.mon, cont, lim)
    assert bench._loadflows(w.topo, r["status"], r["n_island_cont"], cont, 2) == oracle.loadflow_count(r, 2)
