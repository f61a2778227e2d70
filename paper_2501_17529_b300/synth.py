"""Seeded synthetic inputs for batched DC loadflow studies.

This module only draws random numbers and builds graphs: it holds none of the
loadflow arithmetic (no PTDF, no flows, no limits), so the CUDA library and
the CPU oracle can both be fed from it without sharing any solver code.

The paper's benchmark grids (Table "grids": case300, ACTIVSg2000, pegase9421
and a TSO grid) are not available, so the inputs stand in for them by shape:

* grid: a random recursive spanning tree over a random bus permutation plus
  uniformly random extra edges (no self loops, no duplicate bus pairs), with
  random orientation; susceptances b ~ U(5, 50); bus 0 is the slack;
* topologies: two-way bus splits given as (substation, busbar-B mask over the
  substation's incident branches in ascending branch id) plus branch outages,
  the topology vectors t_b and t_d of Sec. III-A;
* injections: N(0,1) nodal powers, or a daily sinusoid per bus with noise,
  re-centred to sum zero per timestep (the slack balances them);
* injection variations: sparse redispatch deltas on 1-3 buses of a small pool,
  the injection candidates T_i brute-forced in the loop (Sec. III-A, Eq. for
  t_i^*).

Seeds follow the convention grid = 100 + cfg, topologies = 200 + cfg,
injections = 300 + cfg, variations = 400 + cfg.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Grid:
    n_bus: int
    f: np.ndarray  # int32 [E] from bus
    t: np.ndarray  # int32 [E] to bus
    b: np.ndarray  # float64 [E] susceptance
    slack: int = 0

    @property
    def n_branch(self) -> int:
        return int(self.f.shape[0])

    def incident(self) -> list[np.ndarray]:
        """Incident branch ids of every bus, ascending (the mask bit order)."""
        inc = [[] for _ in range(self.n_bus)]
        for l in range(self.n_branch):
            inc[int(self.f[l])].append(l)
            inc[int(self.t[l])].append(l)
        return [np.array(sorted(x), dtype=np.int32) for x in inc]

    def degree(self) -> np.ndarray:
        d = np.zeros(self.n_bus, dtype=np.int64)
        np.add.at(d, self.f, 1)
        np.add.at(d, self.t, 1)
        return d


@dataclass
class Topologies:
    """CSR lists of splits and outages, one entry per topology."""
    split_ptr: np.ndarray  # int32 [N+1]
    split_sub: np.ndarray  # int32 [S]
    split_mask: np.ndarray  # uint64 [S]; bit j = j-th incident branch goes to busbar B
    out_ptr: np.ndarray  # int32 [N+1]
    out_branch: np.ndarray  # int32 [O]

    @property
    def n_topo(self) -> int:
        return int(self.split_ptr.shape[0] - 1)

    def subset(self, idx) -> "Topologies":
        idx = np.asarray(idx, dtype=np.int64)
        sp, ss, sm, op, ob = [0], [], [], [0], []
        for i in idx:
            a, b = self.split_ptr[i], self.split_ptr[i + 1]
            ss.extend(self.split_sub[a:b]); sm.extend(self.split_mask[a:b]); sp.append(len(ss))
            a, b = self.out_ptr[i], self.out_ptr[i + 1]
            ob.extend(self.out_branch[a:b]); op.append(len(ob))
        return Topologies(np.array(sp, np.int32), np.array(ss, np.int32),
                          np.array(sm, np.uint64), np.array(op, np.int32),
                          np.array(ob, np.int32))


@dataclass
class Variations:
    """Sparse injection deltas shared by every (topology, timestep)."""
    var_ptr: np.ndarray  # int32 [U+1]
    var_bus: np.ndarray  # int32 [nnz]
    var_delta: np.ndarray  # float64 [nnz]
    pool: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))

    @property
    def n_var(self) -> int:
        return int(self.var_ptr.shape[0] - 1)


def make_grid(n_bus: int, n_branch: int, seed: int) -> Grid:
    """Random recursive spanning tree plus random extra edges, b ~ U(5, 50)."""
    if n_branch < n_bus - 1:
        raise ValueError("a connected grid needs n_branch >= n_bus - 1")
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n_bus)
    pairs = set()
    ends = []
    for i in range(1, n_bus):
        j = int(rng.integers(0, i))
        a, c = int(perm[j]), int(perm[i])
        pairs.add((min(a, c), max(a, c)))
        ends.append((a, c))
    max_pairs = n_bus * (n_bus - 1) // 2
    if n_branch > max_pairs:
        raise ValueError("too many branches for a simple graph")
    while len(ends) < n_branch:
        a, c = (int(x) for x in rng.integers(0, n_bus, 2))
        if a == c or (min(a, c), max(a, c)) in pairs:
            continue
        pairs.add((min(a, c), max(a, c)))
        ends.append((a, c))
    ends = np.array(ends, dtype=np.int64)
    order = rng.permutation(n_branch)  # branch ids not tied to the tree order
    ends = ends[order]
    flip = rng.random(n_branch) < 0.5
    f = np.where(flip, ends[:, 1], ends[:, 0]).astype(np.int32)
    t = np.where(flip, ends[:, 0], ends[:, 1]).astype(np.int32)
    b = rng.uniform(5.0, 50.0, n_branch)
    return Grid(n_bus, f, t, b, 0)


def split_capable(grid: Grid, n_sub: int | None, seed: int, min_degree: int = 3,
                  include_slack: bool = False) -> np.ndarray:
    """Substations that may be split: all of degree >= min_degree, or n_sub of them."""
    deg = grid.degree()
    cand = [n for n in range(grid.n_bus)
            if deg[n] >= min_degree and deg[n] <= 64 and (include_slack or n != grid.slack)]
    cand = np.array(cand, dtype=np.int32)
    if n_sub is None or n_sub >= cand.size:
        return cand
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(cand, n_sub, replace=False)).astype(np.int32)


def _random_mask(rng, deg: int) -> int:
    """Uniform busbar assignment with both busbars non-empty (resampled)."""
    while True:
        bits = rng.integers(0, 2, deg)
        if 0 < bits.sum() < deg:
            return int(sum(int(v) << j for j, v in enumerate(bits)))


def make_topologies(grid: Grid, subs: np.ndarray, n_topo: int, seed: int,
                    n_split, n_out, outage_pool: np.ndarray | None = None) -> Topologies:
    """n_split / n_out: callables rng -> count, or (lo, hi) inclusive uniform ranges."""
    rng = np.random.default_rng(seed)
    inc = grid.incident()
    pool = np.arange(grid.n_branch, dtype=np.int32) if outage_pool is None else np.asarray(outage_pool, np.int32)

    def draw(spec):
        if callable(spec):
            return int(spec(rng))
        lo, hi = spec
        return int(rng.integers(lo, hi + 1))

    sp, ss, sm, op, ob = [0], [], [], [0], []
    for _ in range(n_topo):
        ks = min(draw(n_split), subs.size)
        ko = min(draw(n_out), pool.size)
        chosen = rng.choice(subs, ks, replace=False) if ks else []
        for a in chosen:
            ss.append(int(a))
            sm.append(_random_mask(rng, int(inc[int(a)].size)))
        sp.append(len(ss))
        if ko:
            ob.extend(int(x) for x in rng.choice(pool, ko, replace=False))
        op.append(len(ob))
    return Topologies(np.array(sp, np.int32), np.array(ss, np.int32),
                      np.array(sm, dtype=np.uint64), np.array(op, np.int32),
                      np.array(ob, np.int32))


def geometric_count(p: float, lo: int, hi: int):
    """lo + Geom(p) failures, truncated to hi."""
    def f(rng):
        k = lo
        while k < hi and rng.random() >= p:
            k += 1
        return k
    return f


def make_injections(grid: Grid, T: int, seed: int, daily: bool) -> np.ndarray:
    """[T, n_bus] float64 nodal injections, each timestep summing to zero."""
    rng = np.random.default_rng(seed)
    V = grid.n_bus
    if not daily:
        P = rng.normal(0.0, 1.0, (T, V))
    else:
        P0 = rng.normal(0.0, 1.0, V)
        phi = rng.uniform(0.0, 2.0 * np.pi, V)
        tt = np.arange(T)[:, None]
        P = P0[None, :] * (1.0 + 0.5 * np.sin(2.0 * np.pi * tt / max(T, 1) + phi[None, :]))
        P = P + rng.normal(0.0, 0.2, (T, V))
    P = P - P.mean(axis=1, keepdims=True)
    return np.ascontiguousarray(P)


def make_variations(grid: Grid, n_var: int, n_pool: int, seed: int,
                    sigma: float = 0.5) -> Variations:
    """n_var redispatch deltas on 1-3 buses of an n_pool-bus pool (slack excluded)."""
    rng = np.random.default_rng(seed)
    cand = np.array([n for n in range(grid.n_bus) if n != grid.slack], np.int32)
    pool = np.sort(rng.choice(cand, min(n_pool, cand.size), replace=False)).astype(np.int32)
    vp, vb, vd = [0], [], []
    for _ in range(n_var):
        k = int(rng.integers(1, 4))
        buses = rng.choice(pool, min(k, pool.size), replace=False)
        vb.extend(int(x) for x in buses)
        vd.extend(float(x) for x in rng.normal(0.0, sigma, buses.size))
        vp.append(len(vb))
    return Variations(np.array(vp, np.int32), np.array(vb, np.int32),
                      np.array(vd, np.float64), pool)


@dataclass
class InjectionTopologies:
    """Injections whose busbar can be chosen and, per topology, its candidate
    injection topologies T_i.  inj_bus [n_inj] ascending; inj_p [T, n_inj];
    ti_ptr [n_topo + 1]; ti_mask: bit j puts the topology's j-th eligible
    injection (at one of its split buses, ascending index) on busbar B."""
    inj_bus: np.ndarray
    inj_p: np.ndarray
    ti_ptr: np.ndarray
    ti_mask: np.ndarray

    @property
    def n_inj(self) -> int:
        return int(self.inj_bus.size)


def make_injection_topologies(grid: Grid, subs: np.ndarray, topo: Topologies, P: np.ndarray, n_cand: int,
                              seed: int, per_bus: int = 3) -> InjectionTopologies:
    """per_bus injections at every split-capable bus: a generator / load pair
    and a remainder, summing to the bus injection P[t, bus] of every timestep;
    n_cand random busbar assignments per topology (the first keeps every
    injection on busbar A) over the injections at its split buses, counted per
    split entry (a split with an empty busbar has no busbar B, so a topology
    with one draws over fewer bits)."""
    rng = np.random.default_rng(seed)
    P = np.atleast_2d(P)
    subs = np.sort(np.asarray(subs, np.int32))
    inj_bus = np.repeat(subs, per_bus).astype(np.int32)
    T = P.shape[0]
    inj_p = np.zeros((T, inj_bus.size))
    for k, a in enumerate(subs):
        x = np.abs(rng.normal(0.5, 0.25, (T, per_bus - 1)))
        sgn = np.where(np.arange(per_bus - 1) % 2 == 0, 1.0, -1.0)
        inj_p[:, k * per_bus:k * per_bus + per_bus - 1] = x * sgn
        inj_p[:, k * per_bus + per_bus - 1] = P[:, a] - (x * sgn).sum(axis=1)
    per_sub = {int(a): per_bus for a in subs}
    tp, tm = [0], []
    inc = grid.incident()
    for i in range(topo.n_topo):
        a, c = topo.split_ptr[i], topo.split_ptr[i + 1]
        k = 0
        for A, m in zip(topo.split_sub[a:c], topo.split_mask[a:c]):
            nb = bin(int(m)).count("1")
            if 0 < nb < int(inc[int(A)].size):
                k += per_sub.get(int(A), 0)
        k = min(k, 64)
        tm.append(0)
        for _ in range(n_cand - 1):
            tm.append(int(rng.integers(0, 1 << k, dtype=np.uint64)) if k else 0)
        tp.append(len(tm))
    return InjectionTopologies(inj_bus, inj_p, np.array(tp, np.int32), np.array(tm, dtype=np.uint64))


@dataclass
class Workload:
    name: str
    grid: Grid
    topo: Topologies
    inj: np.ndarray
    mon: np.ndarray
    cont: np.ndarray
    subs: np.ndarray
    var: Variations | None = None


def workload(cfg: int, n_topo: int | None = None, T: int | None = None,
             n_var: int | None = None) -> Workload:
    """The five study shapes (tiny 14-bus, 500-bus, 2000-bus, 10000-bus, screener).

    n_topo / T / n_var override the batch sizes for reduced test cases; the
    grid itself is always the full-size one of that shape.
    """
    if cfg == 1:
        g = make_grid(14, 20, 101)
        subs = split_capable(g, None, 101, min_degree=2, include_slack=True)
        N = 64 if n_topo is None else n_topo
        topo = make_topologies(g, subs, N, 201, (1, 1), (0, 0))
        inj = make_injections(g, 1 if T is None else T, 301, daily=False)
        allb = np.arange(g.n_branch, dtype=np.int32)
        return Workload("tiny14", g, topo, inj, allb, allb.copy(), subs)
    if cfg == 2:
        g = make_grid(500, 700, 102)
        subs = split_capable(g, 50, 102)
        N = 10000 if n_topo is None else n_topo
        topo = make_topologies(g, subs, N, 202, (1, 4), (0, 3))
        inj = make_injections(g, 24 if T is None else T, 302, daily=True)
        allb = np.arange(g.n_branch, dtype=np.int32)
        return Workload("grid500", g, topo, inj, allb, allb.copy(), subs)
    if cfg in (3, 5):
        g = make_grid(2000, 3000, 103)
        subs = split_capable(g, 200, 103)
        N = (100000 if cfg == 3 else 200000) if n_topo is None else n_topo
        if cfg == 3:
            topo = make_topologies(g, subs, N, 200 + cfg, geometric_count(0.5, 1, 8),
                                   geometric_count(0.5, 0, 4))
        else:
            topo = make_topologies(g, subs, N, 200 + cfg, (1, 8), (0, 0))
        inj = make_injections(g, 8 if T is None else T, 300 + cfg, daily=True)
        rng = np.random.default_rng(500 + cfg)
        mon = np.arange(g.n_branch, dtype=np.int32)
        cont = np.sort(rng.choice(g.n_branch, 1000, replace=False)).astype(np.int32)
        var = None
        if cfg == 3:
            var = make_variations(g, 256 if n_var is None else n_var, 16, 400 + cfg)
        return Workload("grid2000" if cfg == 3 else "grid2000_screen", g, topo, inj, mon, cont, subs, var)
    if cfg == 4:
        g = make_grid(10000, 15000, 104)
        subs = split_capable(g, 500, 104)
        N = 50000 if n_topo is None else n_topo
        topo = make_topologies(g, subs, N, 204, (1, 6), (0, 0))
        inj = make_injections(g, 16 if T is None else T, 304, daily=True)
        rng = np.random.default_rng(504)
        mon = np.sort(rng.choice(g.n_branch, 5000, replace=False)).astype(np.int32)
        cont = np.sort(rng.choice(g.n_branch, 2000, replace=False)).astype(np.int32)
        return Workload("grid10000", g, topo, inj, mon, cont, subs)
    raise ValueError(f"unknown study shape {cfg}")
