"""CUDA path vs the FP64 oracle, element by element, through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_2501_17529_b300 import synth

from .parity import BAND, TOL, compare

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2501_17529_b300.csrc import build
    build.build()


def _solver(w, lim, precision, chunk=0, split_bus="subs", outage_cand=None):
    from paper_2501_17529_b300.dcflow import Solver
    s = Solver(w.grid, precision=precision, chunk_topo=chunk)
    s.set_study(w.mon, w.cont, lim, split_bus=(w.subs if split_bus == "subs" else split_bus),
                outage_cand=outage_cand)
    return s


def _gpu(w, lim, precision, topo=None, chunk=0, want_flows=True, outage_cand=None):
    from paper_2501_17529_b300.dcflow import DeviceBatch
    s = _solver(w, lim, precision, chunk, outage_cand=outage_cand)
    topo = w.topo if topo is None else topo
    res = s.solve(DeviceBatch(topo, w.inj), want_flows=want_flows, want_cont_max=want_flows)
    torch.cuda.synchronize()
    out = res.to_host()
    s.close()
    return out


def _ref(w, lim, topo=None, precision=None):
    """The oracle's outputs; with a precision, its reported indices use that form's tie band."""
    topo = w.topo if topo is None else topo
    return oracle.evaluate(w.grid, topo, w.inj, w.mon, w.cont, lim, want_flows=True, want_cmax=True,
                           tie_eps=BAND[precision] if precision else 0.0)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16x3"])
def test_tiny_grid_all_topologies(precision):
    """14-bus grid, 64 single splits (slack included), full N-1: every output."""
    w = synth.workload(1)
    lim = oracle.thermal_limits(w.grid, w.inj)
    compare(_gpu(w, lim, precision), _ref(w, lim, precision=precision), w, w.topo, lim, TOL[precision])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_tiny_grid_every_mask(precision):
    """Every busbar assignment of every substation (islanding ones included)."""
    w = synth.workload(1)
    g = w.grid
    inc = oracle.incident_lists(g.n_bus, g.f, g.t)
    sp, ss, sm = [0], [], []
    for A in range(g.n_bus):
        for m in range(1, 2 ** len(inc[A]) - 1):
            ss.append(A)
            sm.append(m)
            sp.append(len(ss))
    topo = synth.Topologies(np.array(sp, np.int32), np.array(ss, np.int32), np.array(sm, np.uint64),
                            np.zeros(len(ss) + 1, np.int32), np.zeros(0, np.int32))
    w.subs = np.arange(g.n_bus, dtype=np.int32)
    lim = oracle.thermal_limits(g, w.inj)
    ref = _ref(w, lim, topo, precision)
    assert (ref["status"] == 1).sum() > 0
    compare(_gpu(w, lim, precision, topo), ref, w, topo, lim, TOL[precision])


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16x3"])
def test_grid500_sample(precision):
    """500-bus grid, 1-4 splits + 0-3 outages, 24 timesteps: 48 topologies."""
    w = synth.workload(2, n_topo=48)
    lim = oracle.thermal_limits(w.grid, w.inj)
    compare(_gpu(w, lim, precision), _ref(w, lim, precision=precision), w, w.topo, lim, TOL[precision])


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
@pytest.mark.parametrize("scale", [0.35, 0.8, 3.0])
def test_grid500_overloaded_rows(precision, scale):
    """Limits scaled so that rows overloaded already in N-0 are everywhere
    (0.35: most tiles hold more of them than the FP32 kernel evaluates apart),
    common (0.8) or rare (3.0): maxima, overload sums and indices against
    the oracle, 24 topologies of the 500-bus study."""
    w = synth.workload(2, n_topo=24)
    lim = oracle.thermal_limits(w.grid, w.inj) * scale
    ref = _ref(w, lim, precision=precision)
    ok = ref["status"] == 0
    n0 = ref["n0_max"][ok]
    assert (n0 > 1).mean() > 0.9 if scale < 1 else (n0 > 1).mean() < 0.05
    compare(_gpu(w, lim, precision), ref, w, w.topo, lim, TOL[precision])


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16x3"])
def test_grid500_row_restricted_study(precision):
    """The benchmark's study: only the rows of the monitored, contingency,
    split-bus and outage-candidate branches, the candidates being exactly the
    batch's outaged branches (PTDF row restriction of Sec. II).  48 topologies
    of the 500-bus study against the oracle, plus the loadflow count the
    benchmark reports from these outputs against the oracle's count."""
    import bench
    w = synth.workload(2, n_topo=48)
    lim = oracle.thermal_limits(w.grid, w.inj)
    ocand = np.unique(np.asarray(w.topo.out_branch, np.int32))
    ref = oracle.evaluate(w.grid, w.topo, w.inj, w.mon, w.cont, lim, want_flows=True, want_cmax=True,
                          split_bus=w.subs, outage_cand=ocand, tie_eps=BAND[precision])
    gpu = _gpu(w, lim, precision, outage_cand=ocand)
    compare(gpu, ref, w, w.topo, lim, TOL[precision])
    T = w.inj.shape[0]
    assert bench._loadflows(w.topo, gpu["status"], gpu["n_island_cont"], w.cont, T) == oracle.loadflow_count(ref, T)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_switching_outside_the_study_is_invalid(precision):
    """A topology that takes out a branch outside the study's outage candidates,
    or splits a substation outside its split buses, is invalid (flag 2) on both
    sides; the rest of the batch is unaffected."""
    w = synth.workload(2, n_topo=12)
    g = w.grid
    lim = oracle.thermal_limits(g, w.inj[:4])
    w.inj = w.inj[:4]
    ocand = np.unique(np.asarray(w.topo.out_branch, np.int32))
    other = int(np.setdiff1d(np.arange(g.n_branch), ocand)[0])
    not_split = int(np.setdiff1d(np.arange(g.n_bus), w.subs)[0])
    sp = list(w.topo.split_ptr)
    ss, sm = list(w.topo.split_sub), list(w.topo.split_mask)
    op, ob = list(w.topo.out_ptr), list(w.topo.out_branch)
    # topology 12: one outage outside the candidates; topology 13: a split outside the split buses
    ob.append(other)
    op.append(len(ob))
    sp.append(len(ss))
    ss.append(not_split)
    sm.append(1)
    sp.append(len(ss))
    op.append(len(ob))
    topo = synth.Topologies(np.array(sp, np.int32), np.array(ss, np.int32), np.array(sm, np.uint64),
                            np.array(op, np.int32), np.array(ob, np.int32))
    ref = oracle.evaluate(g, topo, w.inj, w.mon, w.cont, lim, want_flows=True, want_cmax=True,
                          split_bus=w.subs, outage_cand=ocand, tie_eps=BAND[precision])
    assert ref["status"][12] == oracle.INVALID and ref["status"][13] == oracle.INVALID
    gpu = _gpu(w, lim, precision, topo=topo, outage_cand=ocand)
    compare(gpu, ref, w, topo, lim, TOL[precision])


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16x3"])
@pytest.mark.parametrize("rem", [1, 3, 4, 5])
def test_contingency_remainder_columns(precision, rem):
    """A contingency range of 64 + rem columns: a remainder of at most 4 is
    evaluated by the final pass instead of an N-1 block of its own (5 takes
    the block); every output, per-contingency maxima included, against the oracle."""
    g = synth.make_grid(200, 300, 81)
    subs = synth.split_capable(g, 30, 81)
    br = oracle.bridges(g.n_bus, g.f, g.t, np.ones(g.n_branch, bool))
    nonbridge = np.nonzero(~br)[0]
    rng = np.random.default_rng(82 + rem)
    cont = np.sort(rng.choice(nonbridge, 64 + rem, replace=False)).astype(np.int32)
    mon = np.sort(rng.choice(g.n_branch, 150, replace=False)).astype(np.int32)
    topo = synth.make_topologies(g, subs, 24, 83, (1, 3), (0, 2))
    inj = synth.make_injections(g, 5, 84, daily=True)
    w = synth.Workload("rem", g, topo, inj, mon, cont, subs)
    lim = oracle.thermal_limits(g, inj)
    compare(_gpu(w, lim, precision), _ref(w, lim, precision=precision), w, topo, lim, TOL[precision])


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16x3"])
def test_ragged_chunks_times_and_sets(precision):
    """Small chunks across rank classes, T beyond one pass, ragged mon / cont subsets."""
    g = synth.make_grid(120, 170, 31)
    subs = synth.split_capable(g, 30, 31)
    rng = np.random.default_rng(32)
    topo = synth.make_topologies(g, subs, 40, 33, (0, 9), (0, 7))
    T = 37 if precision != "fp64" else 19
    inj = synth.make_injections(g, T, 34, daily=True)
    mon = np.sort(rng.choice(g.n_branch, 101, replace=False)).astype(np.int32)
    cont = np.sort(rng.choice(g.n_branch, 77, replace=False)).astype(np.int32)
    w = synth.Workload("ragged", g, topo, inj, mon, cont, subs)
    lim = oracle.thermal_limits(g, inj)
    compare(_gpu(w, lim, precision, chunk=7), _ref(w, lim, precision=precision), w, topo, lim, TOL[precision])


def test_edge_cases_and_invalid_inputs():
    """Empty batch, no-op masks, base topology, outaged monitored / contingency branches,
    islanding outages, rank 16 and invalid topology inputs (flag 2, never a fault)."""
    g = synth.make_grid(40, 60, 41)
    subs = synth.split_capable(g, None, 41, min_degree=2)
    inc = oracle.incident_lists(g.n_bus, g.f, g.t)
    deg = np.array([len(x) for x in inc])
    A = int(subs[0])
    full = (1 << int(deg[A])) - 1
    br = oracle.bridges(g.n_bus, g.f, g.t, np.ones(g.n_branch, bool))
    bridge = int(np.nonzero(br)[0][0]) if br.any() else -1
    many = [int(x) for x in subs[:16]]
    cases = [
        ([], []),                                   # base topology
        ([(A, 0)], []),                             # empty busbar B: no-op
        ([(A, full)], []),                          # empty busbar A: no-op
        ([(A, 1)], [5]),                            # split + outage
        ([], [3, 4]),                               # outages of monitored and contingency branches
        ([], [bridge] if bridge >= 0 else [0]),     # islanding outage
        ([(s, 1) for s in many[:10]], [7, 8, 9, 10, 11, 12]),  # rank 16
        ([(A, 1), (A, 2)], []),                     # invalid: same substation twice
        ([(A, 1 << int(deg[A]))], []),              # invalid: mask bit beyond the degree
        ([], [g.n_branch]),                         # invalid: outage out of range
        ([], [2, 2]),                               # invalid: duplicate outage
        ([(s, 1) for s in many[:12]], [7, 8, 9, 10, 11]),  # invalid: rank 17
    ]
    sp, ss, sm, op, ob = [0], [], [], [0], []
    for splits, outs in cases:
        for s, m in splits:
            ss.append(s)
            sm.append(m)
        sp.append(len(ss))
        ob.extend(outs)
        op.append(len(ob))
    topo = synth.Topologies(np.array(sp, np.int32), np.array(ss, np.int32), np.array(sm, np.uint64),
                            np.array(op, np.int32), np.array(ob, np.int32))
    inj = synth.make_injections(g, 3, 42, daily=False)
    mon = np.arange(g.n_branch, dtype=np.int32)
    w = synth.Workload("edge", g, topo, inj, mon, mon.copy(), subs)
    lim = oracle.thermal_limits(g, inj)
    for precision in ("fp64", "fp32"):
        gpu = _gpu(w, lim, precision)
        ref = _ref(w, lim, precision=precision)
        assert list(ref["status"][7:]) == [2, 2, 2, 2, 2]
        compare(gpu, ref, w, topo, lim, TOL[precision])
    # empty batch is a no-op
    from paper_2501_17529_b300.dcflow import DeviceBatch
    s = _solver(w, lim, "fp32")
    empty = topo.subset([])
    s.solve(DeviceBatch(empty, inj))
    torch.cuda.synchronize()
    s.close()


def test_base_ptdf_matches_oracle():
    g = synth.make_grid(300, 420, 51)
    from paper_2501_17529_b300.dcflow import Solver
    s = Solver(g, precision="fp64")
    rows = np.array([0, 5, 17, 419, 200], np.int32)
    out = s.base_ptdf(rows).cpu().numpy()
    torch.cuda.synchronize()
    ref = oracle.ptdf(g.n_bus, g.f, g.t, g.b, g.slack)[rows]
    assert np.abs(out - ref).max() < 1e-11
    assert np.all(out[:, g.slack] == 0.0)
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_grid500_full_batch_sampled(precision):
    """The 10,000-topology batch in the benchmark's launch configuration; 24
    sampled topologies checked against the oracle, invariants on all."""
    w = synth.workload(2)
    lim = oracle.thermal_limits(w.grid, w.inj)
    gpu = _gpu(w, lim, precision, want_flows=False)
    N = w.topo.n_topo
    assert gpu["status"].shape == (N,)
    ok = gpu["status"] == 0
    assert np.all(gpu["n1_max"][ok] > 0) and np.all(gpu["ovl"][ok] >= 0)
    assert np.all(gpu["worst_cont"][ok] >= 0) and np.all(gpu["worst_cont"][~ok] == -1)
    idx = np.random.default_rng(7).choice(N, 24, replace=False)
    sub = w.topo.subset(idx)
    ref = _ref(w, lim, sub, precision)
    g2 = {k: v[idx] for k, v in gpu.items()}
    compare(g2, ref, w, sub, lim, TOL[precision])


def _check_candidates(w, lim, precision):
    """Run the candidate brute force on the GPU and check it against the oracle:
    the pick must be the oracle's pick under the same tie band (the lowest
    candidate within the band of the smallest maximum loading), exactly, and
    every output must match the oracle evaluated for that candidate."""
    from paper_2501_17529_b300.dcflow import DeviceBatch
    g, var, inj = w.grid, w.var, w.inj
    s = _solver(w, lim, precision)
    out = s.solve(DeviceBatch(w.topo, inj, var), want_flows=True).to_host()
    torch.cuda.synchronize()
    s.close()
    T, U = inj.shape[0], var.n_var
    # every (timestep, candidate) as its own timestep of the oracle
    per_u = oracle.evaluate(g, w.topo, np.repeat(inj, U, axis=0) + _cand_matrix(g, var, T), w.mon, w.cont, lim,
                            want_flows=True, want_cmax=True, tie_eps=BAND[precision])
    tol = TOL[precision]
    np.testing.assert_array_equal(out["status"], per_u["status"])
    ok = per_u["status"] == 0
    assert ok.sum() >= 2
    assert np.all(out["best_var"][~ok] == -1)
    ref = {k: per_u[k] for k in ("status", "n_island_cont", "n_valid_cont")}
    cols = np.zeros((w.topo.n_topo, T), np.int64)
    for i in range(w.topo.n_topo):
        for t in range(T):
            vals = per_u["n1_max"][i, t * U:(t + 1) * U]
            gu = int(out["best_var"][i, t])
            if not ok[i]:
                continue
            assert gu == oracle.first_in_band(vals, BAND[precision], lowest=True), (i, t, gu)
            cols[i, t] = t * U + gu
    rows = np.arange(w.topo.n_topo)[:, None]
    for k in ("n0_max", "n1_max", "ovl", "worst_cont", "worst_mon", "cmax", "n0_flow"):
        ref[k] = per_u[k][rows, cols]
    ref["tie_eps"] = per_u["tie_eps"]
    inj_pick = np.repeat(inj, U, axis=0) + _cand_matrix(g, var, T)
    return out, ref, inj_pick, cols


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16x3"])
def test_injection_candidates_bruteforce(precision):
    """Injection candidates (Eq. (8), metric-first): argmin over candidates of the
    maximum loading, ties to the lowest index, and that candidate's outputs."""
    g = synth.make_grid(150, 220, 71)
    subs = synth.split_capable(g, 30, 71)
    topo = synth.make_topologies(g, subs, 20, 72, (1, 3), (0, 2))
    inj = synth.make_injections(g, 3, 73, daily=True)
    var = synth.make_variations(g, 37, 9, 74)
    rng = np.random.default_rng(75)
    mon = np.arange(g.n_branch, dtype=np.int32)
    cont = np.sort(rng.choice(g.n_branch, 90, replace=False)).astype(np.int32)
    w = synth.Workload("cand", g, topo, inj, mon, cont, subs, var)
    lim = oracle.thermal_limits(g, inj)
    out, ref, inj_pick, cols = _check_candidates(w, lim, precision)
    _compare_picked(out, ref, w, lim, precision, inj_pick, cols)


def _compare_picked(out, ref, w, lim, precision, inj_pick, cols):
    """compare() against the oracle rows of the picked candidates (the worst
    monitored branch near-tie check needs the picked injections per timestep)."""
    class _W:
        pass
    w2 = _W()
    w2.grid, w2.mon, w2.cont = w.grid, w.mon, w.cont
    ok = ref["status"] == 0
    for i in np.nonzero(ok)[0]:
        w2.inj = inj_pick[cols[i]]
        sub = {k: v[[i]] for k, v in out.items()}
        r = {k: (v[[i]] if hasattr(v, "shape") else v) for k, v in ref.items()}
        compare(sub, r, w2, w.topo.subset([i]), lim, TOL[precision])


def _cand_matrix(g, var, T):
    """[T*U, V] injection deltas of every candidate, repeated per timestep."""
    U = var.n_var
    D = np.zeros((U, g.n_bus))
    for u in range(U):
        for k in range(var.var_ptr[u], var.var_ptr[u + 1]):
            D[u, var.var_bus[k]] += var.var_delta[k]
    return np.tile(D, (T, 1))


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16x3"])
def test_grid2000_candidates_sample(precision):
    """Full 2000-bus / 3000-branch grid, 1000 random contingencies, uneven k
    (geometric splits and outages), 8 injection candidates, 2 timesteps."""
    w = synth.workload(3, n_topo=4, T=2, n_var=8)
    lim = oracle.thermal_limits(w.grid, w.inj)
    out, ref, inj_pick, cols = _check_candidates(w, lim, precision)
    _compare_picked(out, ref, w, lim, precision, inj_pick, cols)


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_grid10000_sample(precision):
    """Full 10,000-bus / 15,000-branch grid, 5000 monitored x 2000 contingencies,
    1-6 splits, 16 timesteps: three topologies."""
    w = synth.workload(4, n_topo=3)
    lim = oracle.thermal_limits(w.grid, w.inj)
    compare(_gpu(w, lim, precision), _ref(w, lim, precision=precision), w, w.topo, lim, TOL[precision])


@pytest.mark.parametrize("precision,T,compact", [("fp64", 3, False), ("fp32", 3, False), ("fp32", 40, False),
                                                ("fp32", 3, True), ("bf16x3", 3, False)])
def test_top_cases_match_oracle(precision, T, compact):
    """agg_i: the k worst N-1 cases per (topology, timestep) with their most loaded branch.
    FP32 dense: the tracking N-1 pass and 16 rows per case (T = 40: two timestep
    passes); compacted FP32, BF16x3 and FP64: each distinct case column rebuilt."""
    from paper_2501_17529_b300.dcflow import DeviceBatch
    w = synth.workload(2, n_topo=16, T=T)
    lim = oracle.thermal_limits(w.grid, w.inj)
    k = 5
    s = _solver(w, lim, precision)
    if compact:
        s.set_schedule({"compact_n1": 1})
    res = s.solve(DeviceBatch(w.topo, w.inj), top_k=k)
    torch.cuda.synchronize()
    g = res.to_host()
    s.close()
    ref = oracle.evaluate(w.grid, w.topo, w.inj, w.mon, w.cont, lim, want_cmax=True)
    rc, rm, rl = oracle.top_cases(ref["cmax"], ref["cargmax"], k)
    tol = max(TOL[precision], 2e-7)  # the loadings are float32 outputs in both forms
    mon = np.asarray(w.mon)
    for i in range(w.topo.n_topo):
        if ref["status"][i] != 0:
            assert (g["top_cont"][i] == -1).all() and (g["top_mon"][i] == -1).all()
            continue
        for t in range(T):
            np.testing.assert_allclose(g["top_loading"][i, t], rl[i, t], rtol=0, atol=tol * max(1.0, rl[i, t, 0]))
            for j in range(k):
                c, l = g["top_cont"][i, t, j], g["top_mon"][i, t, j]
                if rc[i, t, j] < 0:
                    assert c == -1 and l == -1
                    continue
                # the pick is a case of (near) the same loading, and l its (near) most loaded branch
                assert abs(ref["cmax"][i, t, c] - rl[i, t, j]) <= 2 * tol * max(1.0, rl[i, t, j])
                if c == rc[i, t, j]:
                    if l != rm[i, t, j]:
                        a, b = w.topo.split_ptr[i], w.topo.split_ptr[i + 1]
                        splits = list(zip(w.topo.split_sub[a:b], w.topo.split_mask[a:b]))
                        a, b = w.topo.out_ptr[i], w.topo.out_ptr[i + 1]
                        col = oracle.n1_loading_column(w.grid, splits, list(w.topo.out_branch[a:b]), w.inj[t],
                                                       w.mon, w.cont[c], lim).copy()
                        col[mon == w.cont[c]] = 0.0
                        assert col[l] >= col.max() - 2 * tol * max(1.0, col.max())


def test_top_cases_tracking_matches_full_columns():
    """The FP32 top-k cases from the tracking N-1 pass (each maximum's 16-row tile)
    against the same batch with the N-1 over compacted lists (no tracking: every
    case's column rebuilt over all rows): the same cases and loadings, and the same
    most loaded branch wherever no other row of the column is within 1e-6 of it.
    Invariant of the tracking: the row of a case's maximum lies in the recorded tile."""
    from paper_2501_17529_b300.dcflow import DeviceBatch
    w = synth.workload(2, n_topo=48, T=24)
    lim = oracle.thermal_limits(w.grid, w.inj)
    k = 8
    out = []
    for compact in (False, True):
        s = _solver(w, lim, "fp32")
        s.set_schedule({"compact_n1": 1 if compact else 0})
        out.append(s.solve(DeviceBatch(w.topo, w.inj), top_k=k).to_host())
        s.close()
    a, b = out
    # the dense run leaves its one-column contingency remainder to the final pass, whose
    # arithmetic differs in the last bits: loadings agree to 1e-6, the order almost everywhere
    np.testing.assert_allclose(a["top_loading"], b["top_loading"], rtol=1e-6, atol=1e-6)
    same = a["top_cont"] == b["top_cont"]
    assert same.mean() > 0.999, same.mean()
    diff = same & (a["top_mon"] != b["top_mon"])
    assert diff.mean() < 1e-3, diff.mean()
    ok = a["status"] == 0
    for i, t, j in zip(*np.nonzero(diff)):  # a near tie: both rows reach the case's loading
        assert ok[i]
        c = int(a["top_cont"][i, t, j])
        a2, b2 = w.topo.split_ptr[i], w.topo.split_ptr[i + 1]
        splits = list(zip(w.topo.split_sub[a2:b2], w.topo.split_mask[a2:b2]))
        a2, b2 = w.topo.out_ptr[i], w.topo.out_ptr[i + 1]
        col = oracle.n1_loading_column(w.grid, splits, list(w.topo.out_branch[a2:b2]), w.inj[t], w.mon,
                                       w.cont[c], lim).copy()
        col[np.asarray(w.mon) == w.cont[c]] = 0.0
        for l in (a["top_mon"][i, t, j], b["top_mon"][i, t, j]):
            assert col[l] >= col.max() - 1e-6 * max(1.0, col.max())


def _candidate_workloads(kind):
    if kind == "ti":
        w = synth.workload(2, n_topo=12, T=3)
        return w, dict(ti=synth.make_injection_topologies(w.grid, w.subs, w.topo, w.inj, 5, 91))
    g = synth.make_grid(150, 220, 71)
    subs = synth.split_capable(g, 30, 71)
    topo = synth.make_topologies(g, subs, 20, 72, (1, 3), (0, 2))
    inj = synth.make_injections(g, 3, 73, daily=True)
    var = synth.make_variations(g, 37, 9, 74)
    rng = np.random.default_rng(75)
    mon = np.arange(g.n_branch, dtype=np.int32)
    cont = np.sort(rng.choice(g.n_branch, 90, replace=False)).astype(np.int32)
    return synth.Workload("cand", g, topo, inj, mon, cont, subs, var), dict(var=var)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("kind", ["ti", "var"])
def test_output_first_matches_metric_first(precision, kind):
    """Injection candidates with the top-k cases: output-first (agg_i of every
    (timestep, candidate) inside the candidate loop, the chosen one's kept) and
    metric-first (agg_i of the chosen candidate only) report the same outputs:
    the same pick, maxima, overload sums, indices and cases.  The FP32
    metric-first cases come from the tracking pass, so their most loaded branch
    may differ from the output-first column rebuild on a near tie only."""
    from paper_2501_17529_b300.dcflow import DeviceBatch, Solver
    w, extra = _candidate_workloads(kind)
    lim = oracle.thermal_limits(w.grid, w.inj)
    k = 5
    out = []
    for of in (False, True):
        s = Solver(w.grid, precision=precision, output_first=of)
        s.set_study(w.mon, w.cont, lim, split_bus=w.subs)
        batch = DeviceBatch(w.topo, w.inj, **extra)
        out.append(s.solve(batch, top_k=k).to_host())
        torch.cuda.synchronize()
        s.close()
    mf, of_ = out
    assert (mf["status"] == 0).sum() >= 8
    for key in ("status", "n_island_cont", "best_var", "worst_cont", "worst_mon", "top_cont"):
        np.testing.assert_array_equal(mf[key], of_[key], err_msg=key)
    for key in ("n1_max", "ovl", "top_loading"):
        np.testing.assert_array_equal(mf[key], of_[key], err_msg=key)
    diff = mf["top_mon"] != of_["top_mon"]
    if precision == "fp64":
        assert not diff.any()
    else:
        assert diff.mean() < 0.01, diff.mean()
        assert (mf["top_cont"][diff] >= 0).all()


def _top_k_of(cmax, k):
    """Per (topology, timestep) the top k of the per-contingency maxima by
    (value descending, position ascending); -1 / 0 where the value is below 0."""
    n, T, C = cmax.shape
    kk = min(k, C)
    cont = np.full((n, T, k), -1, np.int64)
    load = np.zeros((n, T, k), np.float32)
    for i in range(n):
        for t in range(T):
            v = cmax[i, t]
            order = np.lexsort((np.arange(C), -v.astype(np.float64)))[:kk]
            ok = v[order] >= 0
            cont[i, t, :kk] = np.where(ok, order, -1)
            load[i, t, :kk] = np.where(ok, v[order], 0.0)
    return cont, load


@pytest.mark.parametrize("k,cset", [(1, "all"), (5, "all"), (32, "all"), (33, "all"), (64, "all"),
                                    (8, "bridges+20"), (32, "bridges+20")])
def test_top_cases_exact_selection(k, cset):
    """The k worst cases are exactly the top k of the kernel's own per-contingency
    maxima (ties to the lower position), for the small-k candidate select and the
    radix select (k > 32, or more than 64 keys tied at the threshold)."""
    from paper_2501_17529_b300.dcflow import DeviceBatch
    w = synth.workload(2, n_topo=24, T=3)
    lim = oracle.thermal_limits(w.grid, w.inj)
    if cset == "bridges+20":  # 100 bridges (maxima -1) first, then 20 ordinary branches
        br = np.nonzero(oracle.bridges(w.grid.n_bus, w.grid.f, w.grid.t, np.ones(w.grid.n_branch, bool)))[0]
        rest = np.setdiff1d(np.asarray(w.cont), br)[:20]
        w.cont = np.concatenate([br[:100], rest]).astype(np.int32)
    s = _solver(w, lim, "fp32")
    res = s.solve(DeviceBatch(w.topo, w.inj), want_cont_max=True, top_k=k)
    torch.cuda.synchronize()
    g = res.to_host()
    s.close()
    cont, load = _top_k_of(g["cont_max"], k)
    okq = g["status"] == 0
    assert okq.any()
    np.testing.assert_array_equal(g["top_cont"][okq], cont[okq])
    np.testing.assert_array_equal(g["top_loading"][okq], load[okq])
    assert (g["top_cont"][~okq] == -1).all()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("which", ["bridges_only", "empty"])
def test_degenerate_contingency_sets(precision, which):
    """Contingencies that are all base-grid bridges (no N-1 launch at all) and
    an empty contingency set: N-0 outputs as usual, no valid N-1 case."""
    from paper_2501_17529_b300.dcflow import DeviceBatch
    w = synth.workload(2, n_topo=12, T=2)
    lim = oracle.thermal_limits(w.grid, w.inj)
    br = oracle.bridges(w.grid.n_bus, w.grid.f, w.grid.t, np.ones(w.grid.n_branch, bool))
    cont = np.nonzero(br)[0].astype(np.int32)[:40] if which == "bridges_only" else np.zeros(0, np.int32)
    w.cont = cont
    s = _solver(w, lim, precision)
    res = s.solve(DeviceBatch(w.topo, w.inj), want_flows=True, want_cont_max=cont.size > 0,
                  top_k=3 if cont.size else 0)
    torch.cuda.synchronize()
    g = res.to_host()
    s.close()
    ref = oracle.evaluate(w.grid, w.topo, w.inj, w.mon, cont, lim, want_flows=True, want_cmax=cont.size > 0)
    np.testing.assert_array_equal(g["status"], ref["status"])
    ok = ref["status"] == 0
    np.testing.assert_array_equal(g["n_island_cont"][ok], ref["n_island_cont"][ok])
    assert (g["worst_cont"][ok] == -1).all() and (g["n1_max"][ok] == 0).all() and (g["ovl"][ok] == 0).all()
    tol = TOL[precision]
    np.testing.assert_allclose(g["n0_max"][ok], ref["n0_max"][ok], rtol=tol, atol=tol)
    if cont.size:
        assert (g["cont_max"] == -1).all()
        assert (g["top_cont"] == -1).all() and (g["top_mon"] == -1).all()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_generator_failures_match_oracle(precision):
    """Generator-failure N-1 against refactorisation with each generator's output removed."""
    from paper_2501_17529_b300.dcflow import DeviceBatch
    w = synth.workload(2, n_topo=14, T=3)
    lim = oracle.thermal_limits(w.grid, w.inj)
    rng = np.random.default_rng(61)
    gb = np.sort(rng.choice(np.arange(1, w.grid.n_bus), 9, replace=False)).astype(np.int32)
    gp = np.abs(rng.normal(1.0, 0.5, (3, 9)))
    s = _solver(w, lim, precision)
    g = s.solve(DeviceBatch(w.topo, w.inj, gen_bus=gb, gen_p=gp)).to_host()
    s.close()
    ref = oracle.generator_n1(w.grid, w.topo, w.inj, gb, gp, w.mon, lim)
    tol = TOL[precision]
    ok = ref["status"] == 0
    np.testing.assert_array_equal(g["status"], ref["status"])
    np.testing.assert_allclose(g["gen_max"][ok], ref["gen_max"][ok], rtol=tol, atol=tol)
    d = np.abs(g["gen_ovl"][ok] - ref["gen_ovl"][ok]) / np.maximum(ref["gen_ovl"][ok], 1.0)
    assert d.max() <= tol
    for i in np.nonzero(ok)[0]:
        for t in range(3):
            wg = g["worst_gen"][i, t]
            assert wg == ref["worst_gen"][i, t] or \
                ref["gen_each"][i, t, wg] >= ref["gen_max"][i, t] - 2 * tol * max(1.0, ref["gen_max"][i, t])
    assert (g["worst_gen"][~ok] == -1).all()


def _multi_sets(w, rng):
    """Sets of 1-4 branches: random ones, ones holding a branch some topology already lost, the
    single branch of a degree-1 bus and every branch of a degree-3 bus (both island)."""
    g = w.grid
    E = len(g.f)
    deg = np.bincount(np.concatenate([g.f, g.t]), minlength=g.n_bus)
    pool = np.nonzero(~oracle.bridges(g.n_bus, g.f, g.t, np.ones(E, bool)))[0]
    sets = [[int(b) for b in rng.choice(pool, k, replace=False)] for k in (1, 2, 2, 3, 4, 4, 1, 3)]
    lost = [int(b) for b in w.topo.out_branch[:3]]
    sets += [[lost[0]], [lost[1], int((lost[1] + 7) % E)], [int((lost[2] + 11) % E), lost[2], 3]]
    leaf = int(np.nonzero(deg == 1)[0][0])
    sets.append([int(np.nonzero((g.f == leaf) | (g.t == leaf))[0][0])])
    v3 = int([v for v in np.nonzero(deg == 3)[0] if v != g.slack][0])
    sets.append([int(b) for b in np.nonzero((g.f == v3) | (g.t == v3))[0]])
    return sets


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_multi_outages_match_oracle(precision):
    """Multi-outage N-1 (MODF) against refactorisation of each topology without each set."""
    from paper_2501_17529_b300.dcflow import DeviceBatch, Solver
    w = synth.workload(2, n_topo=14, T=11)
    lim = oracle.thermal_limits(w.grid, w.inj)
    sets = _multi_sets(w, np.random.default_rng(71))
    s = Solver(w.grid, precision=precision)
    s.set_study(w.mon, w.cont, lim, split_bus=w.subs, multi=sets)
    g = s.solve(DeviceBatch(w.topo, w.inj)).to_host()
    s.close()
    ref = oracle.multi_outage_n1(w.grid, w.topo, w.inj, sets, w.mon, lim)
    tol = TOL[precision]
    ok = ref["status"] == 0
    np.testing.assert_array_equal(g["status"], ref["status"])
    np.testing.assert_array_equal(g["n_island_multi"][ok], ref["n_island_multi"][ok])
    assert (ref["n_island_multi"][ok] >= 1).all()  # the leaf branch islands every topology
    np.testing.assert_allclose(g["multi_max"][ok], ref["multi_max"][ok], rtol=tol, atol=tol)
    d = np.abs(g["multi_ovl"][ok] - ref["multi_ovl"][ok]) / np.maximum(ref["multi_ovl"][ok], 1.0)
    assert d.max() <= tol
    for i in np.nonzero(ok)[0]:
        for t in range(w.inj.shape[0]):
            wm = g["worst_multi"][i, t]
            assert wm == ref["worst_multi"][i, t] or \
                ref["multi_each"][i, t, wm] >= ref["multi_max"][i, t] - 2 * tol * max(1.0, ref["multi_max"][i, t])
    assert (g["worst_multi"][~ok] == -1).all()
    assert (g["n_island_multi"][~ok] == 0).all()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_generator_and_multi_groups_and_passes(precision):
    """37 generators (groups of 16, 16 and 5) and 75 sets of 1-4 branches (groups of 32, 32 and
    11) in one solve over 29 timesteps (two passes of the FP32 kernels, the second ragged): the
    group and pass boundaries of the generator and multi-outage kernels against the oracle."""
    from paper_2501_17529_b300.dcflow import DeviceBatch, Solver
    T, G = 29, 37
    w = synth.workload(2, n_topo=10, T=T)
    lim = oracle.thermal_limits(w.grid, w.inj)
    rng = np.random.default_rng(83)
    gb = np.sort(rng.choice(np.arange(1, w.grid.n_bus), G, replace=False)).astype(np.int32)
    gp = np.abs(rng.normal(1.0, 0.5, (T, G)))
    E = len(w.grid.f)
    pool = np.nonzero(~oracle.bridges(w.grid.n_bus, w.grid.f, w.grid.t, np.ones(E, bool)))[0]
    sets = [[int(b) for b in rng.choice(pool, 1 + k % 4, replace=False)] for k in range(75)]
    s = Solver(w.grid, precision=precision)
    s.set_study(w.mon, w.cont, lim, split_bus=w.subs, multi=sets)
    g = s.solve(DeviceBatch(w.topo, w.inj, gen_bus=gb, gen_p=gp)).to_host()
    s.close()
    tol = TOL[precision]
    rg = oracle.generator_n1(w.grid, w.topo, w.inj, gb, gp, w.mon, lim)
    rm = oracle.multi_outage_n1(w.grid, w.topo, w.inj, sets, w.mon, lim)
    ok = rg["status"] == 0
    assert ok.sum() >= 3
    np.testing.assert_array_equal(g["status"], rg["status"])
    np.testing.assert_allclose(g["gen_max"][ok], rg["gen_max"][ok], rtol=tol, atol=tol)
    d = np.abs(g["gen_ovl"][ok] - rg["gen_ovl"][ok]) / np.maximum(rg["gen_ovl"][ok], 1.0)
    assert d.max() <= tol
    np.testing.assert_array_equal(g["n_island_multi"][ok], rm["n_island_multi"][ok])
    np.testing.assert_allclose(g["multi_max"][ok], rm["multi_max"][ok], rtol=tol, atol=tol)
    d = np.abs(g["multi_ovl"][ok] - rm["multi_ovl"][ok]) / np.maximum(rm["multi_ovl"][ok], 1.0)
    assert d.max() <= tol
    for i in np.nonzero(ok)[0]:
        for t in range(T):
            wg, wm = g["worst_gen"][i, t], g["worst_multi"][i, t]
            assert wg == rg["worst_gen"][i, t] or \
                rg["gen_each"][i, t, wg] >= rg["gen_max"][i, t] - 2 * tol * max(1.0, rg["gen_max"][i, t])
            assert wm == rm["worst_multi"][i, t] or \
                rm["multi_each"][i, t, wm] >= rm["multi_max"][i, t] - 2 * tol * max(1.0, rm["multi_max"][i, t])
    assert (g["worst_gen"][~ok] == -1).all() and (g["worst_multi"][~ok] == -1).all()
    # the last groups hold worst cases here (so a dropped or misplaced group fails above)
    assert (rg["worst_gen"][ok] >= 32).any() and (rm["worst_multi"][ok] >= 64).any()
    assert (g["worst_gen"][ok] >= 32).any() and (g["worst_multi"][ok] >= 64).any()


def test_multi_outages_rejected_forms():
    """Multi-outage outputs need a study with sets, all four arrays and no injection candidates;
    a set has 1-4 distinct in-range branches."""
    from paper_2501_17529_b300.dcflow import DCFlowError, DeviceBatch, DeviceResults, Solver
    w = synth.workload(1)
    lim = oracle.thermal_limits(w.grid, w.inj)
    s = Solver(w.grid, precision="fp32")
    E = len(w.grid.f)
    for bad in ([[]], [[0, 1, 2, 3, 4]], [[2, 2]], [[E]], [[-1]], [[0]] * (4 * 65535 + 1)):
        with pytest.raises(DCFlowError):
            s.set_study(w.mon, w.cont, lim, split_bus=w.subs, multi=bad)
    s.set_study(w.mon, w.cont, lim, split_bus=w.subs)
    db = DeviceBatch(w.topo, w.inj)
    with pytest.raises(DCFlowError):  # no sets in the study
        s.solve(db, results=DeviceResults(w.topo.n_topo, w.inj.shape[0], len(w.mon), want_multi=True))
    s.set_study(w.mon, w.cont, lim, split_bus=w.subs, multi=[[0, 1]])
    r = DeviceResults(w.topo.n_topo, w.inj.shape[0], len(w.mon), want_multi=True)
    r.n_island_multi = None
    with pytest.raises(DCFlowError):  # not all four arrays
        s.solve(db, results=r)
    out = s.solve(db).to_host()
    assert out["worst_multi"].shape == (w.topo.n_topo, w.inj.shape[0])
    s.close()


def _ti_lists(ti, topo, u):
    """Candidate u of every topology as one-candidate lists (oracle input)."""
    tp = np.arange(topo.n_topo + 1, dtype=np.int32)
    tm = np.array([ti.ti_mask[ti.ti_ptr[i] + u] for i in range(topo.n_topo)], dtype=np.uint64)
    return (tp, tm, ti.inj_bus, ti.inj_p)


def _ti_moved(w, ti, i, u):
    """[(effective split position, power [T])] that candidate u of topology i puts on busbar B."""
    inc = oracle.incident_lists(w.grid.n_bus, w.grid.f, w.grid.t)
    a, c = w.topo.split_ptr[i], w.topo.split_ptr[i + 1]
    el, _ = oracle.eligible_injections(inc, list(zip(w.topo.split_sub[a:c], w.topo.split_mask[a:c])), ti.inj_bus)
    m = int(ti.ti_mask[ti.ti_ptr[i] + u])
    return [(pos, ti.inj_p[:, e]) for j, (e, pos) in enumerate(el) if (m >> j) & 1]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_injection_topologies_match_oracle(precision):
    """Injection topologies t_i (Sec. III-A): per (topology, timestep) the argmin over the topology's
    busbar assignments of agg_m (exact where the runner-up is clear, within tolerance on near-ties),
    and every output equal to the oracle's for the GPU's pick."""
    from paper_2501_17529_b300.dcflow import DeviceBatch
    w = synth.workload(2, n_topo=12, T=3)
    U = 5
    ti = synth.make_injection_topologies(w.grid, w.subs, w.topo, w.inj, U, 91)
    lim = oracle.thermal_limits(w.grid, w.inj)
    s = _solver(w, lim, precision)
    out = s.solve(DeviceBatch(w.topo, w.inj, ti=ti), want_flows=True, want_cont_max=True).to_host()
    torch.cuda.synchronize()
    s.close()
    per_u = [oracle.evaluate(w.grid, w.topo, w.inj, w.mon, w.cont, lim, want_flows=True, want_cmax=True,
                             ti=_ti_lists(ti, w.topo, u), tie_eps=BAND[precision]) for u in range(U)]
    tol = TOL[precision]
    np.testing.assert_array_equal(out["status"], per_u[0]["status"])
    ok = per_u[0]["status"] == 0
    assert ok.sum() >= 8
    assert np.all(out["best_var"][~ok] == -1)
    N, T = w.topo.n_topo, w.inj.shape[0]
    vals = np.stack([p["n1_max"] for p in per_u], axis=2)  # [N, T, U]
    pick = out["best_var"]
    moved_any = 0
    for i in np.nonzero(ok)[0]:
        for t in range(T):
            gu = int(pick[i, t])
            assert 0 <= gu < U
            assert gu == oracle.first_in_band(vals[i, t], BAND[precision], lowest=True), (i, t, gu)
            moved_any += int(gu != 0)
    ref = {k: per_u[0][k] for k in ("status", "n_island_cont", "n_valid_cont")}
    for k in ("n0_max", "n1_max", "ovl", "worst_cont", "worst_mon", "cmax", "n0_flow"):
        ref[k] = np.stack([np.stack([per_u[max(int(pick[i, t]), 0)][k][i, t] for t in range(T)])
                           for i in range(N)])
    ref["tie_eps"] = per_u[0]["tie_eps"]

    def column(i, t, c):
        a, b = w.topo.split_ptr[i], w.topo.split_ptr[i + 1]
        splits = list(zip(w.topo.split_sub[a:b], w.topo.split_mask[a:b]))
        a, b = w.topo.out_ptr[i], w.topo.out_ptr[i + 1]
        mv = [(p, pw[t]) for p, pw in _ti_moved(w, ti, i, int(pick[i, t]))]
        return oracle.n1_loading_column(w.grid, splits, list(w.topo.out_branch[a:b]), w.inj[t], w.mon,
                                        w.cont[c], lim, moved=mv)

    compare(out, ref, w, w.topo, lim, tol, column=column)
    assert moved_any > 0  # some picks move injections to busbar B


def test_injection_topologies_uneven_and_invalid_lists():
    """Lists of different lengths (shorter ones are padded on the device and never pick the pad),
    an empty list and a mask bit beyond the eligible injections (both invalid, flag 2)."""
    from paper_2501_17529_b300.dcflow import DeviceBatch
    g = synth.make_grid(120, 170, 95)
    subs = synth.split_capable(g, 30, 95)
    topo = synth.make_topologies(g, subs, 14, 96, (1, 3), (0, 2))
    inj = synth.make_injections(g, 2, 97, daily=False)
    mon = np.arange(g.n_branch, dtype=np.int32)
    w = synth.Workload("ti", g, topo, inj, mon, mon.copy(), subs)
    full = synth.make_injection_topologies(g, subs, topo, inj, 6, 98)
    inc = oracle.incident_lists(g.n_bus, g.f, g.t)
    tp, tm = [0], []
    for i in range(topo.n_topo):
        lst = [int(x) for x in full.ti_mask[full.ti_ptr[i]:full.ti_ptr[i + 1]]][:1 + i % 6]
        if i == 0:
            lst = []
        if i == 1:
            a, c = topo.split_ptr[1], topo.split_ptr[2]
            el, _ = oracle.eligible_injections(inc, list(zip(topo.split_sub[a:c], topo.split_mask[a:c])), full.inj_bus)
            lst = [0, 1 << len(el)]
        tm.extend(lst)
        tp.append(len(tm))
    ti = synth.InjectionTopologies(full.inj_bus, full.inj_p, np.array(tp, np.int32), np.array(tm, dtype=np.uint64))
    lim = oracle.thermal_limits(g, inj)
    ref = oracle.evaluate(g, topo, inj, mon, mon, lim, ti=(ti.ti_ptr, ti.ti_mask, ti.inj_bus, ti.inj_p))
    assert ref["status"][0] == 2 and ref["status"][1] == 2
    for precision in ("fp64", "fp32"):
        s = _solver(w, lim, precision)
        out = s.solve(DeviceBatch(topo, inj, ti=ti)).to_host()
        torch.cuda.synchronize()
        s.close()
        np.testing.assert_array_equal(out["status"], ref["status"])
        ok = ref["status"] == 0
        tol = TOL[precision]
        np.testing.assert_allclose(out["n1_max"][ok], ref["n1_max"][ok], rtol=tol, atol=tol)
        cnt = np.diff(ti.ti_ptr)
        assert np.all(out["best_var"][ok] < cnt[ok][:, None])
        assert np.all(out["best_var"][~ok] == -1)


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
@pytest.mark.parametrize("compact", [False, True])
def test_grid500_dense_and_compacted_n1(compact, precision):
    """FP32 N-1 over every contingency column and over each topology's compacted valid contingencies
    (compact_n1): the same outputs as the oracle, per-contingency maxima (-1 where skipped) included;
    with the FFMA2 and the tensor-core (split BF16x3) Phi_f build."""
    from paper_2501_17529_b300.dcflow import DeviceBatch, Solver
    w = synth.workload(2, n_topo=40)
    lim = oracle.thermal_limits(w.grid, w.inj)
    s = Solver(w.grid, precision=precision, compact_n1=compact)
    s.set_study(w.mon, w.cont, lim, split_bus=w.subs)
    out = s.solve(DeviceBatch(w.topo, w.inj), want_flows=True, want_cont_max=True).to_host()
    torch.cuda.synchronize()
    s.close()
    compare(out, _ref(w, lim, precision=precision), w, w.topo, lim, TOL[precision])
