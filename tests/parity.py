"""Comparison of CUDA-path outputs with the oracle (shared by the GPU tests).

Error metric: flows |x - x_ref| / max(|x_ref|, limit_l); loadings
|rho - rho_ref| / max(rho_ref, 1); overload sums |s - s_ref| / max(s_ref, 1).
Integer outputs: island flags and islanding-contingency counts bit-exact.
The reported worst contingency and worst monitored branch are compared
exactly when the oracle ran with the form's tie band (oracle.first_in_band:
the lowest position within tolerance * max(best, 1) of the best, the rule
the CUDA path applies); against an oracle run without the band they must be
exact wherever the best value beats the runner-up by more than twice the
tolerance, otherwise reach the maximum within the tolerance (near-tie rule).
"""
import numpy as np

import oracle

TOL = {"fp64": 1e-10, "fp32": 1e-4, "bf16x3": 1e-4}
BAND = TOL  # the CUDA path's default tie band of each form equals its tolerance


def _topo_lists(topo, i):
    a, c = topo.split_ptr[i], topo.split_ptr[i + 1]
    splits = list(zip(topo.split_sub[a:c], topo.split_mask[a:c]))
    a, c = topo.out_ptr[i], topo.out_ptr[i + 1]
    return splits, list(topo.out_branch[a:c])


def compare(gpu, ref, w, topo, lim, tol, report=None, column=None):
    """gpu/ref: dicts of per-topology arrays for the same topologies (ref from
    oracle.evaluate(..., want_flows=True, want_cmax=True)).  Raises AssertionError.
    column(i, t, c): the oracle's loading column of contingency position c for
    the near-tie check of the worst monitored branch (default: refactorisation
    with the batch injections w.inj)."""
    rep = {"max_err_flow": 0.0, "max_err_n1": 0.0, "max_err_n0": 0.0, "max_err_ovl": 0.0,
           "near_ties": 0, "exact_argmax": 0}
    np.testing.assert_array_equal(gpu["status"], ref["status"], err_msg="island flags")
    ok = ref["status"] == 0
    np.testing.assert_array_equal(gpu["n_island_cont"][ok], ref["n_island_cont"][ok], err_msg="islanding contingencies")
    mon = np.asarray(w.mon)
    lim_mon = np.asarray(lim)[mon]
    if not ok.any():
        return rep
    if "n0_flow" in gpu and "n0_flow" in ref:
        d = np.abs(gpu["n0_flow"][ok] - ref["n0_flow"][ok]) / np.maximum(np.abs(ref["n0_flow"][ok]), lim_mon)
        rep["max_err_flow"] = float(d.max())
        assert d.max() <= tol, f"N-0 flow error {d.max():.3e}"
    for key, rk in (("n0_max", "max_err_n0"), ("n1_max", "max_err_n1")):
        d = np.abs(gpu[key][ok] - ref[key][ok]) / np.maximum(ref[key][ok], 1.0)
        rep[rk] = float(d.max())
        assert d.max() <= tol, f"{key} error {d.max():.3e}"
    d = np.abs(gpu["ovl"][ok] - ref["ovl"][ok]) / np.maximum(ref["ovl"][ok], 1.0)
    rep["max_err_ovl"] = float(d.max())
    assert d.max() <= tol, f"overload-sum error {d.max():.3e}"
    cmax = ref["cmax"]
    if "cont_max" in gpu:  # per-contingency maxima (screener labels): -1 exactly where skipped
        g = gpu["cont_max"][ok].astype(np.float64)
        r = cmax[ok]
        np.testing.assert_array_equal(g < 0, r < 0, err_msg="skipped contingencies")
        v = r >= 0
        d = np.abs(g[v] - r[v]) / np.maximum(r[v], 1.0)
        rep["max_err_cont_max"] = float(d.max()) if d.size else 0.0
        assert d.size == 0 or d.max() <= max(tol, 2e-7), f"per-contingency max error {d.max():.3e}"
    banded = float(ref.get("tie_eps", 0.0)) == float(tol) and tol > 0
    if banded:  # the same tie band on both sides: the reported indices agree exactly
        np.testing.assert_array_equal(gpu["worst_cont"][ok], ref["worst_cont"][ok], err_msg="worst contingency")
        np.testing.assert_array_equal(gpu["worst_mon"][ok], ref["worst_mon"][ok], err_msg="worst monitored branch")
        rep["exact_argmax"] = int(ok.sum()) * ref["n1_max"].shape[1]
        if report is not None:
            report.update(rep)
        return rep
    for i in np.nonzero(ok)[0]:
        for t in range(ref["n1_max"].shape[1]):
            go, ro = int(gpu["worst_cont"][i, t]), int(ref["worst_cont"][i, t])
            vals = cmax[i, t]
            if ro < 0:
                assert go == -1
                continue
            srt = np.sort(vals[vals >= 0])[::-1]
            gap = srt[0] - srt[1] if srt.size > 1 else np.inf
            if gap > 2 * tol * max(1.0, srt[0]):
                assert go == ro, f"topology {i} t {t}: worst contingency {go} != {ro}"
                rep["exact_argmax"] += 1
            else:
                assert go >= 0 and vals[go] >= srt[0] - 2 * tol * max(1.0, srt[0]), \
                    f"topology {i} t {t}: near-tie pick {go} value {vals[go]} vs {srt[0]}"
                rep["near_ties"] += 1
            gm, rm = int(gpu["worst_mon"][i, t]), int(ref["worst_mon"][i, t])
            if go == ro and gm != rm:
                if column is not None:
                    col = column(i, t, go)
                else:
                    splits, outs = _topo_lists(topo, i)
                    col = oracle.n1_loading_column(w.grid, splits, outs, w.inj[t], mon, w.cont[go], lim)
                best = col.max()
                assert col[gm] >= best - 2 * tol * max(1.0, best), \
                    f"topology {i} t {t}: worst monitored {gm} != {rm} beyond tolerance"
                rep["near_ties"] += 1
    if report is not None:
        report.update(rep)
    return rep
