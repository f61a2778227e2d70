"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

None of these re-types an oracle formula: each check goes through an
independent route (hand-worked values, the Moore-Penrose pseudo-inverse of the
full Laplacian, networkx, brute-force union-find, refactorisation).
"""
import json
import os
import itertools

import networkx as nx
import numpy as np
import pytest

import oracle
from paper_2501_17529_b300 import synth


def _grid(V, E, seed):
    return synth.make_grid(V, E, seed)


def _incidence(g):
    C = np.zeros((g.n_branch, g.n_bus))
    C[np.arange(g.n_branch), g.f] = 1.0
    C[np.arange(g.n_branch), g.t] = -1.0
    return C


# --------------------------------------------------------------------------
# hand-worked examples (tests/golden)
# --------------------------------------------------------------------------

def test_three_bus_golden(golden_dir):
    d = json.load(open(os.path.join(golden_dir, "three_bus.json")))
    f, t, b = np.array(d["from"]), np.array(d["to"]), np.array(d["b"])
    PT = oracle.ptdf(d["n_bus"], f, t, b, d["slack"])
    np.testing.assert_allclose(PT, np.array(d["ptdf"]), atol=1e-15)
    p = oracle.n0_flows(PT, np.array(d["P"]))
    np.testing.assert_allclose(p, d["n0_flows"], atol=1e-15)
    k = d["outage"]
    col = oracle.lodf_column(PT, f, t, k)
    np.testing.assert_allclose(col, d["lodf_column"], atol=1e-15)
    num = PT[:, f[k]] - PT[:, t[k]]
    assert abs((1 - num[k]) - d["lodf_denominator"]) < 1e-15
    np.testing.assert_allclose(oracle.n1_flows(p, col, k), d["n1_flows"], atol=1e-15)


def test_three_bus_batch_evaluator(golden_dir):
    """The batch evaluator reproduces the worked N-1 of the 3-bus example."""
    d = json.load(open(os.path.join(golden_dir, "three_bus.json")))
    g = synth.Grid(3, np.array(d["from"], np.int32), np.array(d["to"], np.int32),
                   np.array(d["b"]), 0)
    topo = synth.Topologies(np.array([0, 0], np.int32), np.zeros(0, np.int32),
                            np.zeros(0, np.uint64), np.array([0, 0], np.int32), np.zeros(0, np.int32))
    lim = np.ones(3)
    r = oracle.evaluate(g, topo, np.array([d["P"]]), np.arange(3), np.array([1]), lim)
    # only contingency 1 (branch 1); its N-1 flows are (-1, 0, 0) -> max loading 1 on branch 0
    assert r["status"][0] == 0 and r["n_island_cont"][0] == 0
    assert abs(r["n1_max"][0, 0] - 1.0) < 1e-15
    assert r["worst_cont"][0, 0] == 0 and r["worst_mon"][0, 0] == 0
    assert abs(r["n0_max"][0, 0] - 2.0 / 3.0) < 1e-15
    assert r["ovl"][0, 0] < 1e-15


def test_split_examples_golden(golden_dir):
    d = json.load(open(os.path.join(golden_dir, "split_examples.json")))
    for case in d["cases"]:
        g = synth.Grid(case["n_bus"], np.array(case["from"], np.int32),
                       np.array(case["to"], np.int32), np.array(case["b"]), case["slack"])
        P = np.array(case["P"])
        fl0, _ = oracle.topology_flows(g, [], [], P)
        np.testing.assert_allclose(fl0, case["unsplit_flows"], atol=1e-14, err_msg=case["name"])
        splits = [tuple(s) for s in case["splits"]]
        fl, info = oracle.topology_flows(g, splits, case["outages"], P)
        np.testing.assert_allclose(fl, case["flows"], atol=1e-14, err_msg=case["name"])
        if "islanding_outage" in case:
            fl2, info2 = oracle.topology_flows(g, splits, [case["islanding_outage"]], P)
            assert fl2 is None and info2[0] == oracle.ISLANDED


# --------------------------------------------------------------------------
# closed forms and invariants
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", [1, 2, 3])
def test_slack_column_zero_and_pinv(seed):
    """Zero slack column (Def. 2); flows equal diag(b) C L^+ P for any slack (pseudo-inverse)."""
    g = _grid(25, 40, seed)
    rng = np.random.default_rng(seed)
    for slack in (0, 7):
        PT = oracle.ptdf(g.n_bus, g.f, g.t, g.b, slack)
        assert np.all(PT[:, slack] == 0.0)
        P = rng.normal(size=g.n_bus)
        P -= P.mean()
        C = _incidence(g)
        L = C.T @ np.diag(g.b) @ C
        ref = np.diag(g.b) @ C @ np.linalg.pinv(L) @ P
        np.testing.assert_allclose(PT @ P, ref, atol=1e-11)


def test_kcl_on_split_topologies():
    """Kirchhoff: net branch outflow equals the injection at every bus of the rebuilt graph."""
    w = synth.workload(2, n_topo=30, T=3)
    g = w.grid
    inc = oracle.incident_lists(g.n_bus, g.f, g.t)
    checked = 0
    for i in range(w.topo.n_topo):
        a, c = w.topo.split_ptr[i], w.topo.split_ptr[i + 1]
        splits = list(zip(w.topo.split_sub[a:c], w.topo.split_mask[a:c]))
        a, c = w.topo.out_ptr[i], w.topo.out_ptr[i + 1]
        outs = list(w.topo.out_branch[a:c])
        fl, (st, n, f2, t2, alive) = oracle.topology_flows(g, splits, outs, w.inj.T)
        if fl is None:
            continue
        net = np.zeros((n, fl.shape[1]))
        np.add.at(net, f2, fl)
        np.subtract.at(net, t2, fl)
        Pn = np.zeros((n, fl.shape[1]))
        Pn[:g.n_bus] = w.inj.T
        keep = np.arange(n) != g.slack
        np.testing.assert_allclose(net[keep], Pn[keep], atol=1e-9)
        assert np.all(fl[~alive] == 0.0)
        checked += 1
    assert checked > 10


@pytest.mark.parametrize("seed", [4, 5])
def test_lodf_diagonal_and_outaged_flow(seed):
    """Def. 3: LODF[k,k] = -1, so the outaged branch carries nothing after Eq. (5)."""
    g = _grid(20, 32, seed)
    PT = oracle.ptdf(g.n_bus, g.f, g.t, g.b, 0)
    P = np.random.default_rng(seed).normal(size=g.n_bus)
    p = PT @ P
    br = oracle.bridges(g.n_bus, g.f, g.t, np.ones(g.n_branch, bool))
    for k in range(g.n_branch):
        if br[k]:
            continue
        col = oracle.lodf_column(PT, g.f, g.t, k)
        assert col[k] == -1.0
        assert abs(oracle.n1_flows(p, col, k)[k]) < 1e-12


@pytest.mark.parametrize("seed", [6, 7])
def test_reciprocity_and_phi_range(seed):
    """Phi[l,c]/b_l = Phi[c,l]/b_c; 0 <= Phi_cc <= 1 with Phi_cc = 1 exactly at bridges."""
    g = _grid(30, 38, seed)
    PT = oracle.ptdf(g.n_bus, g.f, g.t, g.b, 0)
    C = _incidence(g)
    Phi = PT @ C.T
    np.testing.assert_allclose(Phi / g.b[:, None], (Phi / g.b[:, None]).T, atol=1e-13)
    d = np.diag(Phi)
    assert np.all(d > -1e-13) and np.all(d < 1 + 1e-13)
    G = nx.Graph()
    G.add_nodes_from(range(g.n_bus))
    G.add_edges_from(zip(g.f.tolist(), g.t.tolist()))
    nxb = {tuple(sorted(e)) for e in nx.bridges(G)}
    is_bridge = np.array([tuple(sorted((int(g.f[l]), int(g.t[l])))) in nxb for l in range(g.n_branch)])
    assert is_bridge.any() and (~is_bridge).any()
    assert np.all(np.abs(d[is_bridge] - 1.0) < 1e-12)
    assert np.all(d[~is_bridge] < 1.0 - 1e-6)


def test_bridges_bruteforce_multigraph():
    """Tarjan bridges equal 'removal disconnects' (union-find per branch), parallel branches included."""
    rng = np.random.default_rng(9)
    for trial in range(30):
        n = int(rng.integers(2, 12))
        E = int(rng.integers(1, 18))
        f = rng.integers(0, n, E)
        t = rng.integers(0, n, E)
        keep = f != t
        f, t = f[keep], t[keep]
        if f.size == 0:
            continue
        alive = rng.random(f.size) < 0.9
        br = oracle.bridges(n, f, t, alive)
        base = oracle.components(n, f, t, alive)
        for l in range(f.size):
            if not alive[l]:
                assert not br[l]
                continue
            a2 = alive.copy()
            a2[l] = False
            assert br[l] == (oracle.components(n, f, t, a2) > base)


def test_components_against_networkx():
    rng = np.random.default_rng(10)
    for _ in range(30):
        n = int(rng.integers(1, 15))
        E = int(rng.integers(0, 20))
        f = rng.integers(0, n, E)
        t = rng.integers(0, n, E)
        alive = rng.random(E) < 0.8
        G = nx.MultiGraph()
        G.add_nodes_from(range(n))
        G.add_edges_from((int(a), int(c)) for a, c, al in zip(f, t, alive) if al)
        assert oracle.components(n, f, t, alive) == nx.number_connected_components(G)


def test_cholesky_solve_matches_numpy_solve():
    """Library special case: the factor-solve equals numpy.linalg.solve on B'."""
    g = _grid(12, 18, 11)
    keep = np.arange(1, g.n_bus)
    B = oracle.nodal_susceptance(g.n_bus, g.f, g.t, g.b)
    Cw = oracle.weighted_connectivity(g.n_bus, g.f, g.t, g.b)
    X = np.linalg.solve(B[np.ix_(keep, keep)], Cw[:, keep].T)
    PT = oracle.ptdf(g.n_bus, g.f, g.t, g.b, 0)
    np.testing.assert_allclose(PT[:, keep], X.T, atol=1e-13)


def test_laplacian_parallel_branches_sum():
    """Def. 1 with parallel branches: B equals C^T diag(b) C (sums the pair)."""
    f = np.array([0, 0, 1])
    t = np.array([1, 1, 2])
    b = np.array([2.0, 3.0, 4.0])
    B = oracle.nodal_susceptance(3, f, t, b)
    C = np.zeros((3, 3))
    C[np.arange(3), f] = 1
    C[np.arange(3), t] = -1
    np.testing.assert_array_equal(B, C.T @ np.diag(b) @ C)
    assert B[0, 1] == -5.0


# --------------------------------------------------------------------------
# the paper's update formulas against refactorisation
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", [12, 13, 14])
def test_lodf_equals_refactorisation(seed):
    """Eq. (5) with Def. 3 equals the flows of the grid refactored without k."""
    g = _grid(24, 36, seed)
    P = np.random.default_rng(seed).normal(size=g.n_bus)
    P -= P.mean()
    PT = oracle.ptdf(g.n_bus, g.f, g.t, g.b, 0)
    p = PT @ P
    br = oracle.bridges(g.n_bus, g.f, g.t, np.ones(g.n_branch, bool))
    for k in range(g.n_branch):
        if br[k]:
            continue
        fl, _ = oracle.topology_flows(g, [], [k], P)
        np.testing.assert_allclose(oracle.n1_flows(p, oracle.lodf_column(PT, g.f, g.t, k), k), fl, atol=1e-11)


@pytest.mark.parametrize("seed", [15, 16])
def test_modf_equals_refactorisation(seed):
    """Def. 4: MODF flows equal refactorisation; a single outage gives the LODF."""
    g = _grid(30, 50, seed)
    rng = np.random.default_rng(seed)
    P = rng.normal(size=g.n_bus)
    P -= P.mean()
    PT = oracle.ptdf(g.n_bus, g.f, g.t, g.b, 0)
    p = PT @ P
    done = 0
    for trial in range(40):
        k = int(rng.integers(1, 5))
        O = [int(x) for x in rng.choice(g.n_branch, k, replace=False)]
        fl, info = oracle.topology_flows(g, [], O, P)
        if fl is None:
            continue
        M = oracle.modf(PT, g.f, g.t, O)
        np.testing.assert_allclose(oracle.apply_modf(p, M, O), fl, atol=1e-10)
        if k == 1:
            np.testing.assert_allclose(M[:, 0], oracle.lodf_column(PT, g.f, g.t, O[0]), atol=1e-12)
        done += 1
    assert done > 20


def _split_moved(g, A, mask):
    inc = oracle.incident_lists(g.n_bus, g.f, g.t)[A]
    return [l for j, l in enumerate(inc) if (mask >> j) & 1]


@pytest.mark.parametrize("seed", [17, 18])
def test_bsdf_sequential_equals_refactorisation(seed):
    """Def. 5-6 and Eq. (7), applied once per split, equal the refactored split grid
    (slack splits and branches shared by two split substations included)."""
    g = _grid(20, 34, seed)
    rng = np.random.default_rng(seed)
    P = rng.normal(size=g.n_bus)
    P -= P.mean()
    deg = g.degree()
    cand = [n for n in range(g.n_bus) if deg[n] >= 2]
    checked = 0
    for trial in range(60):
        ks = int(rng.integers(1, 4))
        subs = [int(x) for x in rng.choice(cand, ks, replace=False)]
        if trial % 7 == 0 and 0 not in subs and deg[0] >= 2:
            subs[0] = 0  # slack split
        splits = []
        for A in subs:
            while True:
                m = int(rng.integers(1, 2 ** int(deg[A]) - 1))
                if 0 < bin(m).count("1") < deg[A]:
                    break
            splits.append((A, m))
        fl, info = oracle.topology_flows(g, splits, [], P)
        if fl is None:
            continue
        # sequential application on an ever-growing PTDF
        f = g.f.astype(np.int64).copy()
        t = g.t.astype(np.int64).copy()
        PT = oracle.ptdf(g.n_bus, g.f, g.t, g.b, 0)
        Vc = g.n_bus
        for i, (A, m) in enumerate(splits):
            moved = _split_moved(g, A, m)
            vec, bbc, ext = oracle.bsdf(PT, f, t, g.b, A, moved, Vc)
            PT = ext + np.outer(vec, bbc)  # Eq. (7)
            for l in moved:
                if f[l] == A:
                    f[l] = Vc
                if t[l] == A:
                    t[l] = Vc
            Vc += 1
        Pn = np.concatenate([P, np.zeros(Vc - g.n_bus)])
        np.testing.assert_allclose(PT @ Pn, fl, atol=1e-10)
        checked += 1
    assert checked > 20


def test_split_with_one_moved_branch_is_its_outage():
    """A split moving a single branch leaves it dangling: same flows as its outage."""
    g = _grid(20, 34, 19)
    P = np.random.default_rng(19).normal(size=g.n_bus)
    P -= P.mean()
    inc = oracle.incident_lists(g.n_bus, g.f, g.t)
    n = 0
    for A in range(g.n_bus):
        if len(inc[A]) < 2:
            continue
        for j, l in enumerate(inc[A]):
            fs, _ = oracle.topology_flows(g, [(A, 1 << j)], [], P)
            fo, _ = oracle.topology_flows(g, [], [l], P)
            assert (fs is None) == (fo is None)
            if fs is not None:
                np.testing.assert_allclose(fs, fo, atol=1e-11)
                n += 1
    assert n > 20


def test_split_order_invariance():
    """Permuting the splits of a topology changes no output."""
    w = synth.workload(2, n_topo=12, T=2)
    g = w.grid
    lim = oracle.thermal_limits(g, w.inj)
    r0 = oracle.evaluate(g, w.topo, w.inj, w.mon, w.cont, lim)
    # reverse the split order of every topology
    sp, ss, sm = [0], [], []
    for i in range(w.topo.n_topo):
        a, c = w.topo.split_ptr[i], w.topo.split_ptr[i + 1]
        ss.extend(w.topo.split_sub[a:c][::-1])
        sm.extend(w.topo.split_mask[a:c][::-1])
        sp.append(len(ss))
    topo2 = synth.Topologies(np.array(sp, np.int32), np.array(ss, np.int32), np.array(sm, np.uint64),
                             w.topo.out_ptr, w.topo.out_branch)
    r1 = oracle.evaluate(g, topo2, w.inj, w.mon, w.cont, lim)
    for k in ("n0_max", "n1_max", "ovl"):
        np.testing.assert_allclose(r0[k], r1[k], atol=1e-12)
    for k in ("worst_cont", "worst_mon", "status", "n_island_cont"):
        np.testing.assert_array_equal(r0[k], r1[k])


# --------------------------------------------------------------------------
# brute force on the 14-bus shape
# --------------------------------------------------------------------------

def test_bruteforce_every_mask_tiny_grid():
    """Every busbar assignment of every substation of the 14-bus grid: islanding
    equals networkx connectivity of the rebuilt multigraph, and the LODF-based
    N-1 equals refactorisation per contingency."""
    w = synth.workload(1)
    g = w.grid
    lim = oracle.thermal_limits(g, w.inj)
    inc = oracle.incident_lists(g.n_bus, g.f, g.t)
    sp, ss, sm = [0], [], []
    for A in range(g.n_bus):
        deg = len(inc[A])
        for m in range(1, 2 ** deg - 1):
            ss.append(A)
            sm.append(m)
            sp.append(len(ss))
    N = len(ss)
    topo = synth.Topologies(np.array(sp, np.int32), np.array(ss, np.int32), np.array(sm, np.uint64),
                            np.zeros(N + 1, np.int32), np.zeros(0, np.int32))
    r = oracle.evaluate(g, topo, w.inj, w.mon, w.cont, lim)
    n_island = 0
    for i in range(N):
        st, n, f2, t2, alive, _ = oracle.build_topology(g.n_bus, g.f, g.t, inc, [(ss[i], sm[i])], [])
        G = nx.MultiGraph()
        G.add_nodes_from(range(n))
        G.add_edges_from((int(a), int(c)) for a, c in zip(f2, t2))
        isl = not nx.is_connected(G)
        assert (r["status"][i] == oracle.ISLANDED) == isl
        n_island += isl
        if not isl:
            # bridge contingencies: networkx on the multigraph, via edge removal
            cnt = 0
            for l in range(g.n_branch):
                H = G.copy()
                H.remove_edge(int(f2[l]), int(t2[l]))
                cnt += not nx.is_connected(H)
            assert r["n_island_cont"][i] == cnt
    assert n_island > 0
    idx = [i for i in range(N) if r["status"][i] == 0][::7]
    r1 = oracle.evaluate(g, topo, w.inj, w.mon, w.cont, lim, mode="refactor", idx=idx)
    for k in ("n0_max", "n1_max", "ovl"):
        np.testing.assert_allclose(r[k][idx], r1[k], atol=1e-11)
    np.testing.assert_array_equal(r["worst_cont"][idx], r1["worst_cont"])


def test_modes_agree_with_outages_and_splits():
    """LODF-of-own-PTDF N-1 equals refactorisation per contingency with splits + outages."""
    g = _grid(40, 60, 20)
    subs = synth.split_capable(g, None, 20)
    topo = synth.make_topologies(g, subs, 16, 21, (1, 3), (0, 3))
    P = synth.make_injections(g, 2, 22, daily=True)
    lim = oracle.thermal_limits(g, P)
    mon = np.arange(g.n_branch)
    cont = np.arange(0, g.n_branch, 2)
    r2 = oracle.evaluate(g, topo, P, mon, cont, lim, want_flows=True)
    r1 = oracle.evaluate(g, topo, P, mon, cont, lim, mode="refactor", want_flows=True)
    for k in ("n0_max", "n1_max", "ovl", "n0_flow"):
        np.testing.assert_allclose(r2[k], r1[k], atol=1e-11)
    for k in ("worst_cont", "worst_mon", "status", "n_island_cont"):
        np.testing.assert_array_equal(r2[k], r1[k])


def test_variation_argmin_is_bruteforce():
    """Eq. (8): the reported candidate is argmin over T_i of agg_m, ties to the lowest index,
    and its outputs equal evaluating that candidate's injections directly."""
    g = _grid(30, 45, 23)
    subs = synth.split_capable(g, None, 23)
    topo = synth.make_topologies(g, subs, 6, 24, (1, 2), (0, 1))
    P = synth.make_injections(g, 2, 25, daily=False)
    var = synth.make_variations(g, 9, 6, 26)
    # duplicate variation 3 as 9: a tie that must resolve to 3
    vp = list(var.var_ptr)
    vb = list(var.var_bus) + list(var.var_bus[vp[3]:vp[4]])
    vd = list(var.var_delta) + list(var.var_delta[vp[3]:vp[4]])
    vp.append(len(vb))
    var = synth.Variations(np.array(vp, np.int32), np.array(vb, np.int32), np.array(vd))
    lim = oracle.thermal_limits(g, P)
    mon, cont = np.arange(g.n_branch), np.arange(g.n_branch)
    r = oracle.evaluate(g, topo, P, mon, cont, lim, var=var)
    # brute force: every (t, u) as its own timestep
    U = var.n_var
    Pu = np.zeros((P.shape[0] * U, g.n_bus))
    for ti in range(P.shape[0]):
        for u in range(U):
            Pu[ti * U + u] = P[ti]
            for k in range(vp[u], vp[u + 1]):
                Pu[ti * U + u, vb[k]] += vd[k]
    rb = oracle.evaluate(g, topo, Pu, mon, cont, lim)
    exact = 0
    for i in range(topo.n_topo):
        if r["status"][i] != 0:
            continue
        for ti in range(P.shape[0]):
            vals = rb["n1_max"][i, ti * U:(ti + 1) * U]
            ub = int(r["best_var"][i, ti])
            assert ub != 9  # exact duplicate of candidate 3: the tie goes to the lower index
            # Eq. (3) (base + PTDF dP) vs a direct solve of P + dP agree up to rounding,
            # so the pick is exact wherever the runner-up is not a near-tie
            assert abs(r["n1_max"][i, ti] - vals.min()) < 1e-12
            assert abs(vals[ub] - vals.min()) < 1e-12
            srt = np.sort(np.unique(np.round(vals, 9)))
            if srt.size > 1 and srt[1] - srt[0] > 1e-9:
                u = int(np.argmin(vals))
                assert ub == u
                assert abs(r["ovl"][i, ti] - rb["ovl"][i, ti * U + ub]) < 1e-11
                assert r["worst_cont"][i, ti] == rb["worst_cont"][i, ti * U + ub]
                exact += 1
    assert exact > 0


def test_top_cases_k1_is_the_worst_case_and_k3_matches_refactorisation():
    """agg_i (Sec. III-A): top 1 per N-1 case, then top k over the cases."""
    from paper_2501_17529_b300 import synth
    w = synth.workload(2, n_topo=6, T=2)
    lim = oracle.thermal_limits(w.grid, w.inj)
    r = oracle.evaluate(w.grid, w.topo, w.inj, w.mon, w.cont, lim, want_cmax=True)
    c1, m1, l1 = oracle.top_cases(r["cmax"], r["cargmax"], 1)
    ok = r["status"] == 0
    np.testing.assert_array_equal(c1[ok, :, 0], r["worst_cont"][ok])
    np.testing.assert_array_equal(m1[ok, :, 0], r["worst_mon"][ok])
    np.testing.assert_allclose(l1[ok, :, 0], r["n1_max"][ok], rtol=1e-12)
    c3, m3, l3 = oracle.top_cases(r["cmax"], r["cargmax"], 3)
    for i in np.nonzero(ok)[0][:3]:
        a, b = w.topo.split_ptr[i], w.topo.split_ptr[i + 1]
        splits = list(zip(w.topo.split_sub[a:b], w.topo.split_mask[a:b]))
        a, b = w.topo.out_ptr[i], w.topo.out_ptr[i + 1]
        outs = list(w.topo.out_branch[a:b])
        for t in range(2):
            assert np.all(np.diff(l3[i, t]) <= 0)
            for j in range(3):
                col = oracle.n1_loading_column(w.grid, splits, outs, w.inj[t], w.mon, w.cont[c3[i, t, j]], lim)
                col = col.copy()
                mon_pos = np.nonzero(np.asarray(w.mon) == w.cont[c3[i, t, j]])[0]
                col[mon_pos] = 0.0  # the outaged branch itself carries nothing
                assert l3[i, t, j] == pytest.approx(col.max(), rel=1e-9)
                assert col[m3[i, t, j]] == pytest.approx(col.max(), rel=1e-9)


def test_generator_n1_closed_forms():
    """Generator-failure N-1: a generator with zero output changes nothing (the
    maximum is the N-0 loading), and on the unsplit grid the flows follow
    p0 - P_g PTDF[:, b] (Eq. (3), the slack column being zero)."""
    from paper_2501_17529_b300 import synth
    w = synth.workload(2, n_topo=4, T=2)
    lim = oracle.thermal_limits(w.grid, w.inj)
    gb = np.array([3, 17, 40])
    r0 = oracle.generator_n1(w.grid, w.topo, w.inj, gb, np.zeros((2, 3)), w.mon, lim)
    ev = oracle.evaluate(w.grid, w.topo, w.inj, w.mon, w.cont, lim)
    ok = ev["status"] == 0
    np.testing.assert_allclose(r0["gen_max"][ok], ev["n0_max"][ok], rtol=1e-12)
    assert (r0["worst_gen"][ok] == 0).all()  # all equal: the lowest index
    empty = synth.Topologies(np.zeros(2, np.int32), np.zeros(0, np.int32), np.zeros(0, np.uint64),
                             np.zeros(2, np.int32), np.zeros(0, np.int32))
    gp = np.array([[0.7, 1.3, 0.4], [0.9, 1.1, 0.2]])
    r = oracle.generator_n1(w.grid, empty, w.inj, gb, gp, w.mon, lim)
    ptdf = oracle.ptdf(w.grid.n_bus, w.grid.f, w.grid.t, w.grid.b, w.grid.slack)
    p0 = w.inj @ ptdf.T  # [T, E]
    for t in range(2):
        rho = np.abs(p0[t][:, None] - gp[t][None, :] * ptdf[:, gb]) / lim[:, None]
        assert r["gen_max"][0, t] == pytest.approx(rho.max(), rel=1e-10)
        assert r["worst_gen"][0, t] == int(np.argmax(rho.max(axis=0)))
        assert r["gen_ovl"][0, t] == pytest.approx(np.maximum(rho - 1, 0).sum(), rel=1e-9, abs=1e-12)


def test_multi_outage_reduces_to_lodf_and_modf():
    """A one-branch set is the LODF case of Def. 3 (the evaluator's per-contingency
    maxima); a two-branch set on the unsplit grid follows the MODF of Def. 4."""
    from paper_2501_17529_b300 import synth
    w = synth.workload(2, n_topo=5, T=2)
    lim = oracle.thermal_limits(w.grid, w.inj)
    single = [[int(c)] for c in w.cont[:12]]
    r = oracle.multi_outage_n1(w.grid, w.topo, w.inj, single, w.mon, lim)
    ev = oracle.evaluate(w.grid, w.topo, w.inj, w.mon, w.cont[:12], lim, want_cmax=True)
    ok = ev["status"] == 0
    np.testing.assert_allclose(r["multi_each"][ok], ev["cmax"][ok], rtol=1e-9, atol=1e-12)
    np.testing.assert_array_equal(r["n_island_multi"][ok], ev["n_island_cont"][ok])
    empty = synth.Topologies(np.zeros(2, np.int32), np.zeros(0, np.int32), np.zeros(0, np.uint64),
                             np.zeros(2, np.int32), np.zeros(0, np.int32))
    br = oracle.bridges(w.grid.n_bus, w.grid.f, w.grid.t, np.ones(w.grid.n_branch, bool))
    pair = [int(b) for b in np.nonzero(~br)[0][:2]]
    r2 = oracle.multi_outage_n1(w.grid, empty, w.inj, [pair], w.mon, lim)
    ptdf = oracle.ptdf(w.grid.n_bus, w.grid.f, w.grid.t, w.grid.b, w.grid.slack)
    p0 = w.inj @ ptdf.T
    modf = oracle.modf(ptdf, w.grid.f, w.grid.t, pair)
    for t in range(2):
        n1 = oracle.apply_modf(p0[t], modf, pair)
        rho = np.abs(n1[w.mon]) / lim[w.mon]
        if r2["n_island_multi"][0] == 0:
            assert r2["multi_each"][0, t, 0] == pytest.approx(rho.max(), rel=1e-9)


# --------------------------------------------------------------------------
# injection topologies t_i (Sec. III-A): busbar choice of the injections at
# split substations
# --------------------------------------------------------------------------

def _split_graph_by_hand(g, splits, outages):
    """The split topology written out directly: busbar B of the i-th split with both busbars
    non-empty is bus V + i and takes the masked incident branches (ascending branch id)."""
    f2, t2 = g.f.astype(np.int64).copy(), g.t.astype(np.int64).copy()
    inc = [sorted(np.nonzero((g.f == v) | (g.t == v))[0]) for v in range(g.n_bus)]
    buses = []
    for A, m in splits:
        A, m = int(A), int(m)
        moved = [l for j, l in enumerate(inc[A]) if (m >> j) & 1]
        if not moved or len(moved) == len(inc[A]):
            continue
        nb = g.n_bus + len(buses)
        buses.append(A)
        for l in moved:
            if g.f[l] == A:
                f2[l] = nb
            if g.t[l] == A:
                t2[l] = nb
    alive = np.ones(g.n_branch, bool)
    alive[list(outages)] = False
    return g.n_bus + len(buses), f2, t2, alive, buses


def _ti_case(n_cand=5, T=3, seed=81):
    g = _grid(80, 120, seed)
    subs = synth.split_capable(g, 24, seed)
    topo = synth.make_topologies(g, subs, 12, seed + 1, (1, 3), (0, 2))
    P = synth.make_injections(g, T, seed + 2, daily=False)
    mon = np.arange(g.n_branch)
    w = synth.Workload("ti", g, topo, P, mon, mon.copy(), subs)
    ti = synth.make_injection_topologies(g, subs, topo, P, n_cand, seed + 3)
    lim = oracle.thermal_limits(g, P)
    return w, ti, lim, mon


def _one_candidate(ti, topo, u):
    """The same injection topologies with only candidate u of every topology."""
    tp = np.arange(topo.n_topo + 1, dtype=np.int32)
    tm = np.array([ti.ti_mask[ti.ti_ptr[i] + u] for i in range(topo.n_topo)], dtype=np.uint64)
    return (tp, tm, ti.inj_bus, ti.inj_p)


def test_injection_topology_flows_match_the_split_grid_by_hand():
    """A candidate's N-0 flows equal the PTDF of the hand-built split graph (Def. 2) applied to the
    nodal injections with the chosen injections moved from bus A to busbar B; Kirchhoff holds at
    busbar B with exactly the moved injections; candidate 0 (all on A) equals the plain evaluation."""
    w, ti, lim, mon = _ti_case()
    g = w.grid
    plain = oracle.evaluate(g, w.topo, w.inj, mon, w.cont, lim, want_flows=True)
    checked = 0
    for u in range(4):
        r = oracle.evaluate(g, w.topo, w.inj, mon, w.cont, lim, want_flows=True, ti=_one_candidate(ti, w.topo, u))
        for i in range(w.topo.n_topo):
            if r["status"][i] != 0:
                continue
            a, c = w.topo.split_ptr[i], w.topo.split_ptr[i + 1]
            splits = list(zip(w.topo.split_sub[a:c], w.topo.split_mask[a:c]))
            a, c = w.topo.out_ptr[i], w.topo.out_ptr[i + 1]
            n, f2, t2, alive, buses = _split_graph_by_hand(g, splits, list(w.topo.out_branch[a:c]))
            elig = [e for e in range(ti.n_inj) if int(ti.inj_bus[e]) in buses][:64]
            m = int(ti.ti_mask[ti.ti_ptr[i] + u])
            Pn = np.zeros((w.inj.shape[0], n))
            Pn[:, :g.n_bus] = w.inj
            moved = np.zeros((w.inj.shape[0], len(buses)))
            for j, e in enumerate(elig):
                if (m >> j) & 1:
                    k = buses.index(int(ti.inj_bus[e]))
                    Pn[:, g.n_bus + k] += ti.inj_p[:, e]
                    Pn[:, buses[k]] -= ti.inj_p[:, e]
                    moved[:, k] += ti.inj_p[:, e]
            H = oracle.ptdf(n, f2[alive], t2[alive], g.b[alive], g.slack)
            fl = np.zeros((w.inj.shape[0], g.n_branch))
            fl[:, alive] = Pn @ H.T
            np.testing.assert_allclose(r["n0_flow"][i], fl[:, mon], atol=1e-9)
            mv = [(buses.index(int(ti.inj_bus[e])), ti.inj_p[:, e]) for j, e in enumerate(elig) if (m >> j) & 1]
            fl2, _ = oracle.topology_flows(g, splits, list(w.topo.out_branch[a:c]), w.inj.T, moved=mv)
            np.testing.assert_allclose(fl2.T, fl, atol=1e-9)
            for k in range(len(buses)):  # Kirchhoff at busbar B
                out = fl[:, f2 == g.n_bus + k].sum(axis=1) - fl[:, t2 == g.n_bus + k].sum(axis=1)
                np.testing.assert_allclose(out, moved[:, k], atol=1e-9)
            if u == 0:
                np.testing.assert_allclose(r["n0_flow"][i], plain["n0_flow"][i], atol=1e-12)
                np.testing.assert_allclose(r["n1_max"][i], plain["n1_max"][i], atol=1e-12)
            checked += int(m != 0)
    assert checked >= 10


def test_injection_topology_n1_equals_refactorisation():
    """The N-1 of every injection topology by Def. 3 (LODF of the topology's own PTDF) equals a
    fresh factorisation without each contingency under the moved injections."""
    w, ti, lim, mon = _ti_case(n_cand=3, T=2, seed=82)
    differs = 0
    for u in range(3):  # one candidate at a time: no argmin between near-equal candidates
        t = _one_candidate(ti, w.topo, u)
        a = oracle.evaluate(w.grid, w.topo, w.inj, mon, w.cont, lim, ti=t, idx=range(6))
        b = oracle.evaluate(w.grid, w.topo, w.inj, mon, w.cont, lim, ti=t, idx=range(6), mode="refactor")
        np.testing.assert_array_equal(a["status"], b["status"])
        np.testing.assert_allclose(a["n1_max"], b["n1_max"], atol=1e-9)
        np.testing.assert_allclose(a["ovl"], b["ovl"], rtol=1e-10, atol=1e-8)
        np.testing.assert_array_equal(a["worst_cont"], b["worst_cont"])
        if u == 0:
            ovl0 = a["ovl"]
        else:
            differs += int((np.abs(a["ovl"] - ovl0) > 1e-6).sum())
    assert differs > 0  # the candidates do change the N-1 flows


def test_injection_topology_argmin_and_invalid_lists():
    """t_i* is the argmin of agg_m over T_i, ties to the lowest index (a duplicated candidate never
    wins); an empty list or a mask bit beyond the eligible injections makes the topology invalid."""
    w, ti, lim, mon = _ti_case(n_cand=4, T=2, seed=83)
    N = w.topo.n_topo
    # append a copy of candidate 2 to every list
    tp, tm = [0], []
    for i in range(N):
        lst = list(ti.ti_mask[ti.ti_ptr[i]:ti.ti_ptr[i + 1]])
        tm.extend(lst + [lst[2]])
        tp.append(len(tm))
    t = (np.array(tp, np.int32), np.array(tm, dtype=np.uint64), ti.inj_bus, ti.inj_p)
    r = oracle.evaluate(w.grid, w.topo, w.inj, mon, w.cont, lim, ti=t)
    each = [oracle.evaluate(w.grid, w.topo, w.inj, mon, w.cont, lim, ti=_one_candidate(ti, w.topo, u))
            for u in range(4)]
    ok = r["status"] == 0
    assert ok.sum() >= 6
    vals = np.stack([e["n1_max"] for e in each], axis=2)  # [N, T, U]
    np.testing.assert_allclose(r["n1_max"][ok], vals[ok].min(axis=2), atol=1e-12)
    assert (r["best_var"][ok] != 4).all()
    for i in np.nonzero(ok)[0]:
        for tt in range(2):
            u = r["best_var"][i, tt]
            assert vals[i, tt, u] == pytest.approx(vals[i, tt].min(), abs=1e-12)
            assert r["ovl"][i, tt] == pytest.approx(each[u]["ovl"][i, tt], abs=1e-10)
    # invalid: topology 0 without candidates, topology 1 with a bit beyond its eligible injections
    inc = oracle.incident_lists(w.grid.n_bus, w.grid.f, w.grid.t)
    a, c = w.topo.split_ptr[1], w.topo.split_ptr[2]
    el, _ = oracle.eligible_injections(inc, list(zip(w.topo.split_sub[a:c], w.topo.split_mask[a:c])), ti.inj_bus)
    tp = np.array([0, 0] + [1 + k for k in range(N - 1)], np.int32)
    tm = np.array([1 << len(el)] + [0] * (N - 2), dtype=np.uint64)
    r2 = oracle.evaluate(w.grid, w.topo, w.inj, mon, w.cont, lim, ti=(tp, tm, ti.inj_bus, ti.inj_p))
    assert r2["status"][0] == 2 and r2["status"][1] == 2
    assert (r2["status"][2:] == r["status"][2:]).all()


# --------------------------------------------------------------------------
# the metric's numerator: N-1 cases actually solved (hand count)
# --------------------------------------------------------------------------

def _count_case(golden_dir):
    d = json.load(open(os.path.join(golden_dir, "loadflow_count.json")))
    g = synth.Grid(d["n_bus"], np.array(d["from"], np.int32), np.array(d["to"], np.int32),
                   np.full(len(d["from"]), 10.0), d["slack"])
    sp, ss, sm, op, ob = [0], [], [], [0], []
    for tp in d["topologies"]:
        for A, m in tp["splits"]:
            ss.append(A)
            sm.append(m)
        sp.append(len(ss))
        ob.extend(tp["outages"])
        op.append(len(ob))
    topo = synth.Topologies(np.array(sp, np.int32), np.array(ss, np.int32), np.array(sm, np.uint64),
                            np.array(op, np.int32), np.array(ob, np.int32))
    rng = np.random.default_rng(5)
    P = rng.normal(size=(d["timesteps"], d["n_bus"]))
    P -= P.mean(axis=1, keepdims=True)
    return d, g, topo, P


def test_loadflow_count_hand_counted(golden_dir):
    """Solved N-1 cases per topology and the metric's numerator against a hand
    count: outaged contingencies are not counted, bridges are counted as
    islanding only, islanded topologies contribute nothing, and the count
    multiplies by the timesteps and by the candidates when there are any."""
    d, g, topo, P = _count_case(golden_dir)
    assert oracle.incident_lists(g.n_bus, g.f, g.t) == d["incident_lists"]
    E = g.n_branch
    cont = np.arange(E, dtype=np.int32)
    r = oracle.evaluate(g, topo, P, cont, cont, np.ones(E))
    np.testing.assert_array_equal(r["status"], [x["status"] for x in d["topologies"]])
    np.testing.assert_array_equal(r["n_island_cont"], [x["n_island_cont"] for x in d["topologies"]])
    np.testing.assert_array_equal(r["n_valid_cont"], [x["n_valid_cont"] for x in d["topologies"]])
    assert oracle.loadflow_count(r, d["timesteps"]) == d["loadflows_all_contingencies"]
    assert oracle.loadflow_count(r, d["timesteps"], d["candidates"]) == \
        d["loadflows_all_contingencies_with_candidates"]
    rc = np.array(d["restricted_cont"], np.int32)
    r2 = oracle.evaluate(g, topo, P, cont, rc, np.ones(E))
    np.testing.assert_array_equal(r2["n_island_cont"], d["restricted_n_island_cont"])
    np.testing.assert_array_equal(r2["n_valid_cont"], d["restricted_n_valid_cont"])
    assert oracle.loadflow_count(r2, d["timesteps"]) == d["loadflows_restricted"]


def test_study_switching_sets_make_other_topologies_invalid(golden_dir):
    """A study names the substations its batches may split and the branches
    they may take out (PTDF row restriction of Sec. II); a topology that
    switches anything else is invalid (status 2), the others are unchanged."""
    d, g, topo, P = _count_case(golden_dir)
    E = g.n_branch
    cont = np.arange(E, dtype=np.int32)
    full = oracle.evaluate(g, topo, P, cont, cont, np.ones(E))
    r = oracle.evaluate(g, topo, P, cont, cont, np.ones(E), split_bus=[0, 3], outage_cand=[1, 4, 5])
    # topology 3 splits bus 2, topology 5 outages branch 3: not switchable in this study
    want = np.array(full["status"])
    want[[3, 5]] = oracle.INVALID
    np.testing.assert_array_equal(r["status"], want)
    same = want != oracle.INVALID
    np.testing.assert_array_equal(r["n_valid_cont"][same], full["n_valid_cont"][same])
    np.testing.assert_array_equal(r["n1_max"][same], full["n1_max"][same])


# --------------------------------------------------------------------------
# tie band of the reported indices (worst contingency, worst branch, candidate)
# --------------------------------------------------------------------------

def test_first_in_band_hand_values():
    f = oracle.first_in_band
    assert f([0.5, 0.99999, 1.0], 1e-4) == 1
    assert f([0.5, 0.99999, 1.0], 0.0) == 2
    assert f([0.5, 1.0, 0.7, 1.0], 0.0) == 1          # exact ties: the lowest index
    assert f([10.0, 9.9995, 3.0], 1e-4) == 0          # band scales with |best| above 1
    assert f([9.9995, 10.0, 3.0], 1e-4) == 0
    assert f([9.998, 10.0, 3.0], 1e-4) == 1
    assert f([1.0, 0.5, 0.50001, 0.5], 1e-4, lowest=True) == 1
    assert f([1.0, 0.50001, 0.5], 0.0, lowest=True) == 2


def test_series_branches_tie_goes_to_the_lowest_position(golden_dir):
    """On the 6-bus grid, branches 4 and 5 are in series through bus 4 (no
    injection there): their outages give identical N-1 flows.  With a small
    limit on the parallel branch 6, either outage is the worst case; inside the
    tie band the reported contingency is the lower position in the caller's
    contingency list, in either list order."""
    d, g, _, _ = _count_case(golden_dir)
    topo = synth.Topologies(np.array([0, 0], np.int32), np.zeros(0, np.int32), np.zeros(0, np.uint64),
                            np.array([0, 0], np.int32), np.zeros(0, np.int32))
    P = np.zeros((1, 6))
    P[0, 5], P[0, 1] = 1.0, -1.0
    lim = np.full(7, 10.0)
    lim[6] = 0.5
    mon = np.arange(7, dtype=np.int32)
    r = oracle.evaluate(g, topo, P, mon, np.arange(7, dtype=np.int32), lim, want_cmax=True, tie_eps=1e-9)
    assert abs(r["cmax"][0, 0, 4] - r["cmax"][0, 0, 5]) < 1e-12 and r["cmax"][0, 0, 4] > r["cmax"][0, 0, 6]
    assert r["worst_cont"][0, 0] == 4 and r["worst_mon"][0, 0] == 6
    rev = np.arange(7, dtype=np.int32)[::-1].copy()
    r2 = oracle.evaluate(g, topo, P, mon, rev, lim, tie_eps=1e-9)
    assert r2["worst_cont"][0, 0] == 1  # branch 5 sits at position 1 of the reversed list
