"""Plain FP64 reference for DC loadflow under topology changes (test infrastructure).

Section, definition and equation numbers refer to the paper "Accelerated DC
loadflow solver for topology optimization" (arXiv 2501.17529):

* Sec. II, Def. 1: weighted connectivity matrix C_w and nodal susceptance B;
* Sec. II, Def. 2 / Eq. (1): PTDF' B' = C_w', slack column zero;
* Eq. (2): N-0 flows p_n0 = PTDF P_n;   Eq. (3): incremental injections;
* Def. 3: LODF;   Eq. (5): N-1 flows p_n1[k] = p_n0 + LODF[:,k] p_n0[k];
* Def. 4: MODF for several simultaneous outages;
* Def. 5 / Def. 6 / Eq. (7): BSDF for a bus split;
* Sec. III-A: topology vectors t_b (busbar assignment), t_d (disconnections),
  the injection candidate set T_i and t_i^* = argmin agg_m (Eq. (8)).

The batch evaluator (``evaluate``) is the plain definition: per topology the
split/outaged graph is rebuilt and its reduced susceptance matrix factored
from scratch (no low-rank update).  Its N-1 either uses the LODF of that
topology's own freshly computed PTDF (mode "lodf") or refactors once more per
contingency (mode "refactor").  Islanding is decided combinatorially
(union-find, Tarjan bridges), never by a floating-point threshold.

Readings of points the paper leaves open (each pinned by a test):

* the nodal susceptance matrix is C^T diag(b) C, which sums parallel branches;
* a split of substation A creates a new bus B = n_bus + i (0-based, i = split
  position within the topology); branches whose mask bit is 1 move their A end
  to B; injections and the slack stay on A; a mask with an empty side is a
  no-op; an isolated bus counts as an island;
* limits: rho = |flow| / limit; agg_m is the maximum rho over the monitored
  branches and the valid N-1 cases; the overload sum adds max(0, rho - 1);
  ties go to the lowest position in the contingency list, then the lowest
  monitored position;
* an outaged monitored branch reports flow 0; the outaged contingency itself
  is skipped; a contingency that islands the topology is skipped and counted.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

# status codes of a topology (island flag output)
OK, ISLANDED, INVALID = 0, 1, 2
MAX_MODIFICATIONS = 16  # largest number of effective splits + outages per topology
MAX_DEGREE = 64  # a split mask addresses at most 64 incident branches


# ---------------------------------------------------------------------------
# Sec. II definitions
# ---------------------------------------------------------------------------

def weighted_connectivity(n_bus, f, t, b):
    """Def. 1: C_w[l, f_l] = b_l, C_w[l, t_l] = -b_l (E x V, dense)."""
    E = len(f)
    Cw = np.zeros((E, n_bus))
    for l in range(E):
        Cw[l, f[l]] += b[l]
        Cw[l, t[l]] -= b[l]
    return Cw


def nodal_susceptance(n_bus, f, t, b):
    """Def. 1: B[n,n] = sum of incident b, B[n,m] = -b of the (n,m) branches.

    Parallel branches add up (the Laplacian C^T diag(b) C)."""
    B = np.zeros((n_bus, n_bus))
    for l in range(len(f)):
        i, j, w = f[l], t[l], b[l]
        B[i, i] += w
        B[j, j] += w
        B[i, j] -= w
        B[j, i] -= w
    return B


def ptdf(n_bus, f, t, b, slack):
    """Def. 2, Eq. (1): solve PTDF' B' = C_w' (prime = slack removed); slack column 0.

    B' is symmetric, so each row of PTDF' solves B' x = C_w'[l, :]^T."""
    keep = np.array([n for n in range(n_bus) if n != slack], dtype=np.int64)
    Bp = nodal_susceptance(n_bus, f, t, b)[np.ix_(keep, keep)]
    Cwp = weighted_connectivity(n_bus, f, t, b)[:, keep]
    fac = sla.cho_factor(Bp, lower=True)
    X = sla.cho_solve(fac, Cwp.T)  # (V-1) x E
    out = np.zeros((len(f), n_bus))
    out[:, keep] = X.T
    return out


def n0_flows(ptdf_m, P):
    """Eq. (2): p_n0 = PTDF . P_n  (P may be [V] or [V, T])."""
    return ptdf_m @ P


def lodf_column(ptdf_m, f, t, k):
    """Def. 3: LODF[l,k] = (PTDF[l,f_k]-PTDF[l,t_k]) / (1-(PTDF[k,f_k]-PTDF[k,t_k])), LODF[k,k] = -1."""
    num = ptdf_m[:, f[k]] - ptdf_m[:, t[k]]
    col = num / (1.0 - num[k])
    col[k] = -1.0
    return col


def n1_flows(p_n0, lodf_col, k):
    """Eq. (5): p_n1[k] = p_n0 + LODF[:,k] p_n0[k]."""
    return p_n0 + lodf_col * p_n0[k]


def modf(ptdf_m, f, t, outages):
    """Def. 4: MODF (I - (PTDF[O,fO] - PTDF[O,tO])) = PTDF[:,fO] - PTDF[:,tO]; rows O := -I."""
    O = list(outages)
    rhs = ptdf_m[:, [f[k] for k in O]] - ptdf_m[:, [t[k] for k in O]]  # E x |O|
    A = np.eye(len(O)) - rhs[O, :]
    M = np.linalg.solve(A.T, rhs.T).T  # M A = rhs
    for i, k in enumerate(O):
        M[k, :] = 0.0
        M[k, i] = -1.0
    return M


def apply_modf(p_n0, modf_m, outages):
    """Flows after the simultaneous outage of O: p + MODF p[O] (as for the LODF)."""
    return p_n0 + modf_m @ p_n0[list(outages)]


def bsdf(ptdf_m, f, t, b, A, moved, new_bus):
    """Def. 5 / Def. 6: BSDF vector and PTDF_bbc row for splitting bus A.

    ``moved`` are the branches going to the new busbar ``new_bus``; S (the set
    that stays on A) is every other branch incident to A.  The PTDF matrix is
    extended by a column for ``new_bus`` equal to column A.  Reading of the
    garbled definitions: P_shift[far end of l] += b_l / sum_S b for l in S and
    P_shift[B] = -1; P_corr is nonzero only on S (+b_l/sum_S b if f_l = A,
    -b_l/sum_S b if t_l = A); PTDF_bbc is the coupler flow A->B,
    sum_{m moved} sigma_m PTDF[m,:] with sigma_m = +1 if f_m = A else -1, and
    PTDF_bbc[B] = PTDF_bbc[A] - 1.

    Returns (bsdf [E], ptdf_bbc [V+1], ptdf_ext [E, V+1]); Eq. (7) then gives
    the split PTDF as ptdf_ext + outer(bsdf, ptdf_bbc).
    """
    E, V = ptdf_m.shape
    assert new_bus == V
    moved = set(int(m) for m in moved)
    inc = [l for l in range(E) if f[l] == A or t[l] == A]
    S = [l for l in inc if l not in moved]
    ext = np.concatenate([ptdf_m, ptdf_m[:, [A]]], axis=1)
    bS = sum(b[l] for l in S)
    shift = np.zeros(V + 1)
    shift[new_bus] = -1.0
    corr = np.zeros(E)
    for l in S:
        far = t[l] if f[l] == A else f[l]
        shift[far] += b[l] / bS
        corr[l] = b[l] / bS if f[l] == A else -b[l] / bS
    bbc = np.zeros(V + 1)
    for m in moved:
        bbc += (1.0 if f[m] == A else -1.0) * ext[m, :]
    bbc[new_bus] = bbc[A] - 1.0
    vec = (ext @ shift + corr) / (1.0 - bbc @ shift)
    return vec, bbc, ext


# ---------------------------------------------------------------------------
# graph helpers (combinatorial, exact)
# ---------------------------------------------------------------------------

def components(n, f, t, alive):
    """Union-find; returns the number of connected components over n buses."""
    parent = list(range(n))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    for l in range(len(f)):
        if alive[l]:
            a, c = find(int(f[l])), find(int(t[l]))
            if a != c:
                parent[a] = c
    return len({find(x) for x in range(n)})


def bridges(n, f, t, alive):
    """Tarjan's bridge finding on the multigraph of alive branches (bool [E]).

    A branch is a bridge iff removing it increases the number of components;
    parallel branches are never bridges (the parent edge is skipped by id)."""
    adj = [[] for _ in range(n)]
    for l in range(len(f)):
        if alive[l]:
            adj[int(f[l])].append((int(t[l]), l))
            adj[int(t[l])].append((int(f[l]), l))
    disc = [-1] * n
    low = [0] * n
    out = np.zeros(len(f), dtype=bool)
    timer = 0
    for root in range(n):
        if disc[root] != -1:
            continue
        disc[root] = low[root] = timer
        timer += 1
        stack = [(root, -1, iter(adj[root]))]
        while stack:
            u, pedge, it = stack[-1]
            advanced = False
            for v, l in it:
                if l == pedge:
                    continue
                if disc[v] == -1:
                    disc[v] = low[v] = timer
                    timer += 1
                    stack.append((v, l, iter(adj[v])))
                    advanced = True
                    break
                low[u] = min(low[u], disc[v])
            if not advanced:
                stack.pop()
                if stack:
                    p = stack[-1][0]
                    low[p] = min(low[p], low[u])
                    if low[u] > disc[p]:
                        out[pedge] = True
    return out


def incident_lists(n_bus, f, t):
    """Incident branch ids per bus, ascending: the split-mask bit order."""
    inc = [[] for _ in range(n_bus)]
    for l in range(len(f)):
        inc[int(f[l])].append(l)
        inc[int(t[l])].append(l)
    return [sorted(x) for x in inc]


# ---------------------------------------------------------------------------
# topology construction (Sec. III-A: t_b, t_d)
# ---------------------------------------------------------------------------

def build_topology(n_bus, f, t, inc, splits, outages, max_mod=MAX_MODIFICATIONS, split_bus=None,
                   outage_cand=None):
    """Rebuild the branch endpoints of one topology.

    splits: list of (substation, mask); outages: list of branch ids.
    split_bus / outage_cand: the study's switchable substations and the
    branches it may take out (None: every bus / branch).  A topology that
    splits another substation or outages another branch is not a topology of
    the study: INVALID (the PTDF row restriction of Sec. II keeps only the
    rows such a study needs).
    Returns (status, n_bus_new, f2, t2, alive, n_eff_splits)."""
    E = len(f)
    f2 = np.array(f, dtype=np.int64)
    t2 = np.array(t, dtype=np.int64)
    alive = np.ones(E, dtype=bool)
    seen = set()
    k_eff = 0
    for (A, mask) in splits:
        A = int(A)
        mask = int(mask)
        if A < 0 or A >= n_bus or A in seen or (split_bus is not None and A not in split_bus):
            return INVALID, n_bus, f2, t2, alive, 0
        seen.add(A)
        deg = len(inc[A])
        if deg > MAX_DEGREE or (deg < 64 and (mask >> deg) != 0):
            return INVALID, n_bus, f2, t2, alive, 0
        nb = bin(mask).count("1")
        if nb == 0 or nb == deg:
            continue  # one busbar empty: no split
        newb = n_bus + k_eff
        k_eff += 1
        for j, l in enumerate(inc[A]):
            if (mask >> j) & 1:
                if f[l] == A:
                    f2[l] = newb
                if t[l] == A:
                    t2[l] = newb
    outs = set()
    for c in outages:
        c = int(c)
        if c < 0 or c >= E or c in outs or (outage_cand is not None and c not in outage_cand):
            return INVALID, n_bus, f2, t2, alive, 0
        outs.add(c)
        alive[c] = False
    if k_eff + len(outs) > max_mod:
        return INVALID, n_bus, f2, t2, alive, 0
    return OK, n_bus + k_eff, f2, t2, alive, k_eff


class _Factor:
    """Factorisation of the reduced susceptance matrix B' of one topology."""

    def __init__(self, n, f2, t2, b, alive, slack):
        self.n = n
        self.slack = slack
        self.keep = np.array([x for x in range(n) if x != slack], dtype=np.int64)
        self.pos = -np.ones(n, dtype=np.int64)
        self.pos[self.keep] = np.arange(self.keep.size)
        idx = np.nonzero(alive)[0]
        if n <= 2500:
            B = nodal_susceptance(n, f2[idx], t2[idx], b[idx])
            Bp = B[np.ix_(self.keep, self.keep)]
            self._fac = sla.cho_factor(Bp, lower=True)
            self._solve = lambda r: sla.cho_solve(self._fac, r)
        else:
            rows, cols, vals = [], [], []
            for l in idx:
                i, j, w = int(f2[l]), int(t2[l]), float(b[l])
                rows += [i, j, i, j]
                cols += [i, j, j, i]
                vals += [w, w, -w, -w]
            B = sp.csc_matrix((vals, (rows, cols)), shape=(n, n))
            Bp = B[self.keep][:, self.keep].tocsc()
            lu = spla.splu(Bp)
            self._solve = lambda r: lu.solve(np.asarray(r, dtype=np.float64))

    def solve_full(self, rhs):
        """theta = B'^{-1} rhs with the slack angle 0; rhs [n, k] on all buses."""
        rhs = np.asarray(rhs, dtype=np.float64)
        one = rhs.ndim == 1
        r2 = rhs.reshape(self.n, -1)
        th = np.zeros_like(r2)
        th[self.keep] = np.asarray(self._solve(r2[self.keep])).reshape(self.keep.size, -1)
        return th[:, 0] if one else th


def _flows_from_angles(th, f2, t2, b, alive):
    """flow_l = b_l (theta_f - theta_t) (C_w theta, Eq. (1)-(2)); outaged branches 0."""
    fl = b[:, None] * (th[f2] - th[t2]) if th.ndim == 2 else b * (th[f2] - th[t2])
    if th.ndim == 2:
        fl[~alive, :] = 0.0
    else:
        fl[~alive] = 0.0
    return fl


# ---------------------------------------------------------------------------
# one topology, plain definition
# ---------------------------------------------------------------------------

def eligible_injections(inc, splits, inj_bus, cap=64):
    """Injections whose busbar an injection topology t_i chooses (Sec. III-A):
    those at the bus of one of the topology's effective splits, in ascending
    injection index, at most `cap` (one bit each of a candidate mask).
    Returns [(injection, position of its split among the effective splits)]
    and the effective split buses in that order."""
    buses = []
    for (A, mask) in splits:
        nb = bin(int(mask)).count("1")
        if nb == 0 or nb == len(inc[int(A)]):
            continue  # one busbar empty: no split, no busbar B
        buses.append(int(A))
    pos = {A: i for i, A in enumerate(buses)}
    el = [(e, pos[int(b)]) for e, b in enumerate(inj_bus) if int(b) in pos]
    return el[:cap], buses


def first_in_band(values, eps, lowest=False):
    """The reported index of an arg-max (or, lowest=True, an arg-min) with a tie
    band: the lowest index whose value lies within eps * max(|best|, 1) of the
    best value.  eps = 0 is the plain arg-max / arg-min with ties to the lowest
    index.  The band makes the reported index the same for two computations of
    the same values that differ by less than the band (rounding of one
    precision against another) whenever no value lies at the band's edge."""
    v = np.asarray(values, np.float64)
    if lowest:
        best = v.min()
        return int(np.nonzero(v <= best + eps * max(abs(best), 1.0))[0][0])
    best = v.max()
    return int(np.nonzero(v >= best - eps * max(abs(best), 1.0))[0][0])


def classify_contingencies(cont, alive, br):
    """Which N-1 cases of one topology are solved (Def. 3 / Eq. (5) need
    1 - Phi[c, c] != 0): a contingency branch in service that is not a bridge
    of the topology is solved; one that is a bridge would island the grid and
    is skipped and counted; an outaged branch is not a contingency of the
    topology (skipped, not counted).  Returns (solved mask over cont, number
    of islanding contingencies)."""
    valid = np.array([bool(alive[c]) and not bool(br[c]) for c in cont], dtype=bool)
    n_island = int(sum(1 for c in cont if alive[c] and br[c]))
    return valid, n_island


def evaluate_topology(grid, inc, splits, outages, P, mon, cont, limit,
                      var=None, mode="lodf", want_flows=False, want_cmax=False, ti=None,
                      split_bus=None, outage_cand=None, tie_eps=0.0):
    """Outputs of one topology for every timestep (and variation).

    P: [T, V] injections.  var: (var_ptr, var_bus, var_delta) or None.
    ti: injection topologies T_i of this topology (Sec. III-A) as
    (masks, inj_bus, inj_p [T, n_inj]) or None: candidate u moves the j-th
    eligible injection (eligible_injections) from bus A onto busbar B of its
    split when bit j of masks[u] is set; an empty candidate list or a bit
    beyond the eligible injections makes the topology invalid.
    Returns a dict with per-timestep arrays: n0_max, n1_max, ovl, worst_cont,
    worst_mon, best_var, plus island status and n_island_cont (and n0 flows
    of the monitored branches if want_flows).  split_bus / outage_cand: the
    study's switchable substations and outage candidates (build_topology).
    tie_eps: the tie band of the reported indices (first_in_band): the worst
    contingency is the lowest position whose maximum loading is within the
    band of the largest, its worst monitored branch likewise within its
    column, and the chosen candidate the lowest index within the band of the
    smallest maximum loading."""
    V, f, t, b, slack = grid.n_bus, grid.f, grid.t, grid.b, grid.slack
    T = P.shape[0]
    M, C = len(mon), len(cont)
    res = dict(status=OK, n_island_cont=0,
               n0_max=np.zeros(T), n1_max=np.zeros(T), ovl=np.zeros(T),
               worst_cont=-np.ones(T, np.int64), worst_mon=-np.ones(T, np.int64),
               best_var=-np.ones(T, np.int64), n_valid_cont=0)
    if want_flows:
        res["n0_flow"] = np.zeros((T, M))
    if want_cmax:
        res["cmax"] = -np.ones((T, C))  # per contingency: max_l rho (-1 if skipped)
        res["cargmax"] = -np.ones((T, C), np.int64)  # its monitored position (lowest on ties)
    st, n, f2, t2, alive, k_eff = build_topology(V, f, t, inc, splits, outages, split_bus=split_bus,
                                                 outage_cand=outage_cand)
    if st != OK:
        res["status"] = st
        return res
    if ti is not None:
        masks, inj_bus, inj_p = ti
        el, sbus = eligible_injections(inc, splits, inj_bus)
        if len(masks) == 0 or any(int(m) >> len(el) for m in masks):
            res["status"] = INVALID
            return res
    if components(n, f2, t2, alive) > 1:
        res["status"] = ISLANDED
        return res
    br = bridges(n, f2, t2, alive)
    mon = np.asarray(mon, np.int64)
    cont = np.asarray(cont, np.int64)
    lim_mon = np.asarray(limit, np.float64)[mon]
    valid, res["n_island_cont"] = classify_contingencies(cont, alive, br)
    res["n_valid_cont"] = int(valid.sum())
    vj = np.nonzero(valid)[0]
    vc = cont[vj]
    fac = _Factor(n, f2, t2, grid.b, alive, slack)

    # injections on the new topology: new buses carry none (they stay on A)
    Pn = np.zeros((n, T))
    Pn[:V, :] = P.T
    base_flows = _flows_from_angles(fac.solve_full(Pn), f2, t2, b, alive)  # [E, T]

    # candidate injection changes dP [n, T, U]: the same for every timestep for
    # the nodal candidates of Eq. (8); per timestep for the injection topologies
    nvar = 0
    if var is not None and len(var[0]) > 1:
        vp, vb, vd = var
        nvar = len(vp) - 1
        dP = np.zeros((n, T, nvar))
        for u in range(nvar):
            for k in range(vp[u], vp[u + 1]):
                dP[vb[k], :, u] += vd[k]
    elif ti is not None:
        nvar = len(masks)
        dP = np.zeros((n, T, nvar))
        inj_p = np.atleast_2d(np.asarray(inj_p, np.float64))
        for u, m in enumerate(masks):
            for j, (e, i) in enumerate(el):
                if (int(m) >> j) & 1:
                    dP[V + i, :, u] += inj_p[:, e]  # onto busbar B (new bus V + i)
                    dP[sbus[i], :, u] -= inj_p[:, e]  # off busbar A
    if nvar:
        dflow = _flows_from_angles(fac.solve_full(dP.reshape(n, T * nvar)), f2, t2, b, alive).reshape(-1, T, nvar)

    if mode == "lodf":
        # Phi_tau[l, c] = PTDF_tau[l, f'_c] - PTDF_tau[l, t'_c]: flows of a unit
        # transfer between the ends of c in this topology (Def. 3 numerator)
        rhs = np.zeros((n, vc.size))
        for j, c in enumerate(vc):
            rhs[f2[c], j] += 1.0
            rhs[t2[c], j] -= 1.0
        Phi = _flows_from_angles(fac.solve_full(rhs), f2, t2, b, alive)  # [E, Cv]
        den = 1.0 - Phi[vc, np.arange(vc.size)]
        lodf = Phi / den[None, :]  # Def. 3 (l != k)
        for j, c in enumerate(vc):
            lodf[c, j] = -1.0  # Def. 3 (l == k)
    diag_mask = mon[:, None] == vc[None, :]

    def n1_block(p, pinj):
        """N-1 flows of every valid contingency, M x Cv: Eq. (5) with the LODF of
        this topology's own PTDF, or a fresh factorisation without c."""
        if mode == "lodf":
            return p[mon][:, None] + lodf[mon, :] * p[vc][None, :]
        out = np.zeros((M, vc.size))
        for j, c in enumerate(vc):
            alive2 = alive.copy()
            alive2[c] = False
            fac2 = _Factor(n, f2, t2, grid.b, alive2, slack)
            out[:, j] = _flows_from_angles(fac2.solve_full(pinj), f2, t2, b, alive2)[mon]
        return out

    def metrics(p, pinj):
        n0r = np.abs(p[mon]) / lim_mon
        n0m = float(n0r.max()) if M else 0.0
        if vc.size == 0:
            return n0m, 0.0, 0.0, -1, -1, None
        n1 = n1_block(p, pinj)
        rho = np.abs(n1) / lim_mon[:, None]
        rho[diag_mask] = 0.0
        rho[~alive[mon], :] = 0.0
        # the worst contingency: the lowest position within the tie band of the largest
        # per-contingency maximum, then its worst monitored branch within that column's band
        cm = rho.max(axis=0)
        jc = first_in_band(cm, tie_eps)
        im = first_in_band(rho[:, jc], tie_eps)
        ovl = float(np.maximum(rho - 1.0, 0.0).sum())
        return n0m, float(cm.max()), ovl, int(vj[jc]), int(im), (cm, rho.argmax(axis=0))

    for ti in range(T):
        if not nvar:
            p = base_flows[:, ti]
            r = metrics(p, Pn[:, ti])
            if want_flows:
                res["n0_flow"][ti] = p[mon]
        else:
            cand = []
            for u in range(nvar):
                p = base_flows[:, ti] + dflow[:, ti, u]
                cand.append((metrics(p, Pn[:, ti] + dP[:, ti, u]), p))
            # Eq. (8): the candidate with the smallest maximum loading (lowest index within the tie band)
            u_best = first_in_band([c[0][1] for c in cand], tie_eps, lowest=True)
            r, p = cand[u_best]
            res["best_var"][ti] = u_best
            if want_flows:
                res["n0_flow"][ti] = p[mon]
        res["n0_max"][ti], res["n1_max"][ti], res["ovl"][ti] = r[0], r[1], r[2]
        res["worst_cont"][ti], res["worst_mon"][ti] = r[3], r[4]
        if want_cmax and r[5] is not None:
            res["cmax"][ti, vj] = r[5][0]
            res["cargmax"][ti, vj] = r[5][1]
    return res


def evaluate(grid, topo, P, mon, cont, limit, var=None, mode="lodf", idx=None,
             want_flows=False, want_cmax=False, ti=None, split_bus=None, outage_cand=None, tie_eps=0.0):
    """Evaluate a batch of topologies (or the subset ``idx``); arrays per topology.
    ti: injection topologies as (ti_ptr [n_topo + 1], ti_mask, inj_bus, inj_p [T, n_inj]).
    split_bus / outage_cand: the study's switchable substations and outage
    candidates (None: every bus / branch); a topology outside them is INVALID.
    tie_eps: the tie band of the reported indices (evaluate_topology)."""
    inc = incident_lists(grid.n_bus, grid.f, grid.t)
    sb = None if split_bus is None else {int(x) for x in split_bus}
    oc = None if outage_cand is None else {int(x) for x in outage_cand}
    P = np.atleast_2d(np.asarray(P, np.float64))
    ids = range(topo.n_topo) if idx is None else [int(i) for i in idx]
    vtuple = None
    if var is not None and var.n_var > 0:
        vtuple = (var.var_ptr, var.var_bus, var.var_delta)
    outs = []
    for i in ids:
        a, c = topo.split_ptr[i], topo.split_ptr[i + 1]
        splits = list(zip(topo.split_sub[a:c], topo.split_mask[a:c]))
        a, c = topo.out_ptr[i], topo.out_ptr[i + 1]
        outages = list(topo.out_branch[a:c])
        tti = None
        if ti is not None:
            tp, tm, ib, ip = ti
            tti = ([int(x) for x in tm[tp[i]:tp[i + 1]]], ib, ip)
        outs.append(evaluate_topology(grid, inc, splits, outages, P, mon, cont, limit,
                                      vtuple, mode, want_flows, want_cmax, tti, sb, oc, tie_eps))
    keys = ["n0_max", "n1_max", "ovl", "worst_cont", "worst_mon", "best_var"]
    r = {k: np.stack([o[k] for o in outs]) if outs else np.zeros((0, P.shape[0])) for k in keys}
    r["status"] = np.array([o["status"] for o in outs], np.int64)
    r["n_island_cont"] = np.array([o["n_island_cont"] for o in outs], np.int64)
    r["n_valid_cont"] = np.array([o["n_valid_cont"] for o in outs], np.int64)
    r["tie_eps"] = float(tie_eps)
    if want_flows:
        r["n0_flow"] = np.stack([o["n0_flow"] for o in outs]) if outs else np.zeros((0, P.shape[0], len(mon)))
    if want_cmax:
        r["cmax"] = np.stack([o["cmax"] for o in outs]) if outs else np.zeros((0, P.shape[0], len(cont)))
        r["cargmax"] = (np.stack([o["cargmax"] for o in outs]) if outs
                        else np.zeros((0, P.shape[0], len(cont)), np.int64))
    return r


def top_cases(cmax, cargmax, k):
    """Sparse worst results (agg_i of Sec. III-A): per (topology, timestep) the k
    N-1 cases with the highest maximum loading, each with its most loaded
    monitored branch -- the top 1 inside every N-1 case, then the top k over
    the cases.  Ties: lower contingency position first.  Returns (cont, mon,
    loading), each [..., k]; slots beyond the valid cases hold -1 / -1 / 0."""
    cm = np.asarray(cmax, np.float64)
    ca = np.asarray(cargmax, np.int64)
    shp = cm.shape[:-1]
    cmf, caf = cm.reshape(-1, cm.shape[-1]), ca.reshape(-1, ca.shape[-1])
    oc = -np.ones((cmf.shape[0], k), np.int64)
    om = -np.ones((cmf.shape[0], k), np.int64)
    ol = np.zeros((cmf.shape[0], k))
    for r in range(cmf.shape[0]):
        valid = [c for c in range(cmf.shape[1]) if cmf[r, c] >= 0]
        order = sorted(valid, key=lambda c: (-cmf[r, c], c))[:k]
        for j, c in enumerate(order):
            oc[r, j], om[r, j], ol[r, j] = c, caf[r, c], cmf[r, c]
    return oc.reshape(shp + (k,)), om.reshape(shp + (k,)), ol.reshape(shp + (k,))


def n1_loading_column(grid, splits, outages, P_t, mon, c_branch, limit, moved=None):
    """|p_n1| / limit over the monitored branches for one contingency branch, by
    refactorisation of the topology without it (None if it islands).  moved:
    optional [(position of an effective split, power)] put on that split's
    busbar B and taken off its bus A (an injection topology, Sec. III-A)."""
    fl, info = topology_flows(grid, splits, list(outages) + [int(c_branch)], P_t, moved)
    if fl is None:
        return None
    return np.abs(fl[np.asarray(mon)]) / np.asarray(limit)[np.asarray(mon)]


def base_flows(grid, P):
    """N-0 flows [T, E] of the unsplit grid: theta = B'^{-1} P, flow = C_w theta (Eq. (1)-(2))."""
    alive = np.ones(grid.n_branch, dtype=bool)
    f = np.asarray(grid.f, np.int64)
    t = np.asarray(grid.t, np.int64)
    fac = _Factor(grid.n_bus, f, t, grid.b, alive, grid.slack)
    th = fac.solve_full(np.atleast_2d(np.asarray(P, np.float64)).T)
    return _flows_from_angles(th, f, t, grid.b, alive).T


def thermal_limits(grid, P, factor=1.2, offset=0.1):
    """Synthetic limits: factor * max_t |base flow| + offset, from the unsplit grid."""
    return factor * np.abs(base_flows(grid, P)).max(axis=0) + offset


def loadflow_count(res, n_timesteps, n_var=0):
    """The throughput metric's numerator (the loadflow arithmetic under the
    benchmark table of Sec. IV: topologies x |T_i| x N-1 cases): the N-1 cases
    actually solved, i.e. the solved contingencies (classify_contingencies) of
    the topologies that neither island nor are invalid, times the timesteps,
    times the injection candidates when there are any."""
    ok = res["status"] == OK
    return int(res["n_valid_cont"][ok].sum()) * n_timesteps * max(1, n_var)


def topology_flows(grid, splits, outages, P, moved=None):
    """N-0 flows [E] (or [E, T]) of one rebuilt topology; also returns (status, n, f2, t2, alive).
    moved: optional [(position of an effective split, power)] moved from its bus A onto its busbar B."""
    inc = incident_lists(grid.n_bus, grid.f, grid.t)
    st, n, f2, t2, alive, _ = build_topology(grid.n_bus, grid.f, grid.t, inc, splits, outages)
    if st != OK or components(n, f2, t2, alive) > 1:
        return None, (st if st != OK else ISLANDED, n, f2, t2, alive)
    fac = _Factor(n, f2, t2, grid.b, alive, grid.slack)
    P = np.asarray(P, np.float64)
    Pn = np.zeros((n,) + P.shape[1:])
    Pn[:grid.n_bus] = P
    if moved:
        _, sbus = eligible_injections(inc, splits, [])
        for i, pw in moved:
            Pn[grid.n_bus + i] += pw
            Pn[sbus[i]] -= pw
    return _flows_from_angles(fac.solve_full(Pn), f2, t2, grid.b, alive), (OK, n, f2, t2, alive)


def generator_n1(grid, topo, P, gen_bus, gen_p, mon, limit, idx=None):
    """Generator-failure N-1 (the "N-1 generator" case of the injection module,
    Sec. III-A): generator g at bus gen_bus[g] with output gen_p[t, g] fails and
    the slack takes up its output.  Per topology the split/outaged graph is
    rebuilt and factored, and the flows of P[t] - gen_p[t, g] e_{gen_bus[g]}
    are solved for every (t, g).  Returns per topology and timestep the maximum
    loading over generators and monitored branches, the failing generator that
    reaches it (lowest index on ties; -1 if none), the overload sum and every
    generator's own maximum (gen_each [T, G]), plus the topology status."""
    P = np.atleast_2d(np.asarray(P, np.float64))
    gp = np.atleast_2d(np.asarray(gen_p, np.float64))
    gb = np.asarray(gen_bus, np.int64)
    mon = np.asarray(mon, np.int64)
    lim = np.asarray(limit, np.float64)[mon]
    T, G = P.shape[0], gb.size
    ids = range(topo.n_topo) if idx is None else [int(i) for i in idx]
    out = {k: [] for k in ("gen_max", "worst_gen", "gen_ovl", "gen_each", "status")}
    for i in ids:
        a, c = topo.split_ptr[i], topo.split_ptr[i + 1]
        splits = list(zip(topo.split_sub[a:c], topo.split_mask[a:c]))
        a, c = topo.out_ptr[i], topo.out_ptr[i + 1]
        outages = list(topo.out_branch[a:c])
        gm, wg, go, ge = np.zeros(T), -np.ones(T, np.int64), np.zeros(T), np.zeros((T, G))
        fl0, info = topology_flows(grid, splits, outages, P.T)
        st = info[0]
        if fl0 is not None and G:
            # injections minus each generator's output, column (t, g) = P[t] - gp[t, g] e_b
            rhs = np.repeat(P.T[:, :, None], G, axis=2)  # [V, T, G]
            for g in range(G):
                rhs[gb[g], :, g] -= gp[:, g]
            fl, _ = topology_flows(grid, splits, outages, rhs.reshape(grid.n_bus, T * G))
            rho = np.abs(fl[mon].reshape(mon.size, T, G)) / lim[:, None, None]  # [M, T, G]
            for t in range(T):
                per_g = rho[:, t, :].max(axis=0)
                ge[t] = per_g
                g = int(np.argmax(per_g))
                gm[t], wg[t] = per_g[g], g
                go[t] = float(np.maximum(rho[:, t, :] - 1.0, 0.0).sum())
        out["gen_max"].append(gm)
        out["worst_gen"].append(wg)
        out["gen_ovl"].append(go)
        out["gen_each"].append(ge)
        out["status"].append(st)
    return {k: np.asarray(v) for k, v in out.items()}


def multi_outage_n1(grid, topo, P, multi, mon, limit, idx=None):
    """N-1 cases that take out several branches at once (Def. 4, MODF; e.g. the
    windings of a three-winding transformer).  multi: list of branch lists.
    Per topology the graph is rebuilt without each set (on top of the
    topology's own outages) and refactored.  A set that islands the topology
    is skipped and counted; a set with a branch the topology already lost is
    skipped and not counted.  Returns per topology and timestep the maximum
    loading over sets and monitored branches, the set reaching it (lowest index
    on ties; -1 if none), the overload sum, every set's own maximum
    (multi_each [T, S], -1 if skipped), and per topology the islanding count
    and the status."""
    P = np.atleast_2d(np.asarray(P, np.float64))
    mon = np.asarray(mon, np.int64)
    lim = np.asarray(limit, np.float64)[mon]
    T, S = P.shape[0], len(multi)
    ids = range(topo.n_topo) if idx is None else [int(i) for i in idx]
    out = {k: [] for k in ("multi_max", "worst_multi", "multi_ovl", "multi_each", "n_island_multi", "status")}
    for i in ids:
        a, c = topo.split_ptr[i], topo.split_ptr[i + 1]
        splits = list(zip(topo.split_sub[a:c], topo.split_mask[a:c]))
        a, c = topo.out_ptr[i], topo.out_ptr[i + 1]
        outages = [int(x) for x in topo.out_branch[a:c]]
        mm, wm, mo = np.zeros(T), -np.ones(T, np.int64), np.zeros(T)
        me = -np.ones((T, S))
        nisl = 0
        fl0, info = topology_flows(grid, splits, outages, P.T)
        st = info[0]
        if fl0 is not None:
            for m, br in enumerate(multi):
                if any(int(b) in outages for b in br):
                    continue
                fl, inf2 = topology_flows(grid, splits, outages + [int(b) for b in br], P.T)
                if fl is None:
                    nisl += 1
                    continue
                rho = np.abs(fl[mon]) / lim[:, None]  # [M, T]; the outaged set carries nothing
                me[:, m] = rho.max(axis=0)
                mo += np.maximum(rho - 1.0, 0.0).sum(axis=0)
            for t in range(T):
                if (me[t] >= 0).any():
                    m = int(np.argmax(me[t]))
                    mm[t], wm[t] = me[t, m], m
        out["multi_max"].append(mm)
        out["worst_multi"].append(wm)
        out["multi_ovl"].append(mo)
        out["multi_each"].append(me)
        out["n_island_multi"].append(nisl)
        out["status"].append(st)
    return {k: np.asarray(v) for k, v in out.items()}
