"""Each plausible mistake planted in the oracle must fail at least one pin.

The mutations are applied with monkeypatch to the oracle module on the CPU
only; they show the pins in test_oracle_pins.py are not vacuous.
"""
import numpy as np
import pytest

import oracle
from oracle import dcflow_ref as ref
import tests.test_oracle_pins as pins


def _fails(fn, *args):
    try:
        fn(*args)
    except AssertionError:
        return True
    except (ValueError, IndexError, np.linalg.LinAlgError, ZeroDivisionError):
        return True
    return False


def _cw_wrong_sign(n_bus, f, t, b):
    Cw = np.zeros((len(f), n_bus))
    for l in range(len(f)):
        Cw[l, f[l]] += b[l]
        Cw[l, t[l]] += b[l]  # planted: + instead of -
    return Cw


def _lodf_no_override(ptdf_m, f, t, k):
    num = ptdf_m[:, f[k]] - ptdf_m[:, t[k]]
    return num / (1.0 - num[k])  # planted: LODF[k,k] = -1 dropped


def _lodf_transposed(ptdf_m, f, t, k):
    num = ptdf_m[k, f] - ptdf_m[k, t]  # planted: row instead of column
    col = num / (1.0 - num[k])
    col[k] = -1.0
    return col


def _modf_no_override(ptdf_m, f, t, outages):
    O = list(outages)
    rhs = ptdf_m[:, [f[k] for k in O]] - ptdf_m[:, [t[k] for k in O]]
    A = np.eye(len(O)) - rhs[O, :]
    return np.linalg.solve(A.T, rhs.T).T  # planted: rows O not set to -I


def _bsdf_corr_on_all(ptdf_m, f, t, b, A, moved, new_bus):
    _, bbc, ext = _orig_bsdf(ptdf_m, f, t, b, A, moved, new_bus)
    E, V = ptdf_m.shape
    inc = [l for l in range(E) if f[l] == A or t[l] == A]
    S = [l for l in inc if l not in set(moved)]
    bS = sum(b[l] for l in S)
    shift = np.zeros(V + 1)
    shift[new_bus] = -1.0
    corr = np.zeros(E)
    for l in S:
        far = t[l] if f[l] == A else f[l]
        shift[far] += b[l] / bS
    for l in inc:  # planted: correction over every incident branch, moved ones too
        corr[l] = b[l] / bS if f[l] == A else -b[l] / bS
    return (ext @ shift + corr) / (1.0 - bbc @ shift), bbc, ext


_orig_bsdf = ref.bsdf


def _incident_descending(n_bus, f, t):
    return [x[::-1] for x in _orig_inc(n_bus, f, t)]  # planted: mask bit order reversed


_orig_inc = ref.incident_lists


def _components_ignores_isolated(n, f, t, alive):
    used = set(np.asarray(f)[alive].tolist()) | set(np.asarray(t)[alive].tolist())
    c = _orig_comp(n, f, t, alive)
    return c - (n - len(used))  # planted: isolated buses are not islands


_orig_comp = ref.components


MUTATIONS = [
    ("weighted_connectivity", _cw_wrong_sign, [(pins.test_three_bus_golden, "golden")]),
    ("lodf_column", _lodf_no_override, [(pins.test_lodf_diagonal_and_outaged_flow, 4)]),
    ("lodf_column", _lodf_transposed, [(pins.test_lodf_equals_refactorisation, 12)]),
    ("modf", _modf_no_override, [(pins.test_modf_equals_refactorisation, 15)]),
    ("bsdf", _bsdf_corr_on_all, [(pins.test_bsdf_sequential_equals_refactorisation, 17)]),
    ("incident_lists", _incident_descending, [(pins.test_split_examples_golden, "golden")]),
    ("components", _components_ignores_isolated, [(pins.test_split_examples_golden, "golden")]),
]


@pytest.mark.parametrize("name,mut,checks", MUTATIONS, ids=[m[1].__name__ for m in MUTATIONS])
def test_planted_mistake_is_caught(monkeypatch, golden_dir, name, mut, checks):
    monkeypatch.setattr(ref, name, mut)
    monkeypatch.setattr(oracle, name, mut, raising=False)
    caught = False
    for fn, arg in checks:
        if arg == "golden":
            caught |= _fails(fn, golden_dir)
        elif arg is None:
            caught |= _fails(fn)
        else:
            caught |= _fails(fn, arg)
    assert caught, f"planted mistake in {name} not detected"


# ---------------------------------------------------------------------------
# screener reference
# ---------------------------------------------------------------------------
from oracle import screener_ref as sref  # noqa: E402
import tests.test_oracle_screener as spins  # noqa: E402


def _bwd_no_relu_mask(params, cache, z, Y, rounding=None):
    Y = np.asarray(Y, np.float64)
    B, C = z.shape
    dz = (sref.sigmoid(z) - Y) / (B * C)
    g = {"W3": dz.T @ cache["h2"], "b3": dz.sum(axis=0)}
    dh2 = dz @ cache["W3"]  # planted: relu' dropped
    g["W2"], g["b2"] = dh2.T @ cache["h1"], dh2.sum(axis=0)
    dh1 = (dh2 @ cache["W2"]) * (cache["h1"] > 0)
    g["W1"], g["b1"] = dh1.T @ cache["x"], dh1.sum(axis=0)
    return g


def _bwd_w2_transposed(params, cache, z, Y, rounding=None):
    Y = np.asarray(Y, np.float64)
    B, C = z.shape
    dz = (sref.sigmoid(z) - Y) / (B * C)
    g = {"W3": dz.T @ cache["h2"], "b3": dz.sum(axis=0)}
    dh2 = (dz @ cache["W3"]) * (cache["h2"] > 0)
    g["W2"], g["b2"] = dh2.T @ cache["h1"], dh2.sum(axis=0)
    dh1 = (dh2 @ cache["W2"].T) * (cache["h1"] > 0)  # planted: W2^T instead of W2
    g["W1"], g["b1"] = dh1.T @ cache["x"], dh1.sum(axis=0)
    return g


def _bwd_no_mean(params, cache, z, Y, rounding=None):
    Y = np.asarray(Y, np.float64)
    dz = sref.sigmoid(z) - Y  # planted: the 1 / (B C) of the mean dropped
    g = {"W3": dz.T @ cache["h2"], "b3": dz.sum(axis=0)}
    dh2 = (dz @ cache["W3"]) * (cache["h2"] > 0)
    g["W2"], g["b2"] = dh2.T @ cache["h1"], dh2.sum(axis=0)
    dh1 = (dh2 @ cache["W2"]) * (cache["h1"] > 0)
    g["W1"], g["b1"] = dh1.T @ cache["x"], dh1.sum(axis=0)
    return g


def _adam_no_bias_correction(params, grads, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    for k in sref.PARAM_NAMES:
        m[k] = beta1 * m[k] + (1 - beta1) * grads[k]
        v[k] = beta2 * v[k] + (1 - beta2) * grads[k] ** 2
        params[k] = params[k] - lr * m[k] / (np.sqrt(v[k]) + eps)  # planted
    return params


def _labels_no_threshold(cmax, k):
    cm = np.asarray(cmax, np.float64)
    flat = cm.reshape(-1, cm.shape[-1])
    Y = np.zeros(flat.shape, np.uint8)
    for r in range(flat.shape[0]):
        for c in sorted(range(flat.shape[1]), key=lambda c: (-flat[r, c], c))[:k]:
            Y[r, c] = 1  # planted: max rho > 1 not required
    return Y.reshape(cm.shape)


def _bf16_truncate(x):
    a = np.asarray(x, np.float64).astype(np.float32)
    u = a.view(np.uint32) & np.uint32(0xFFFF0000)  # planted: truncation, not round-to-nearest-even
    return u.view(np.float32).astype(np.float64)


@pytest.mark.parametrize("name,attr,fake,pin", [
    ("relu mask dropped", "backward", _bwd_no_relu_mask, "fd"),
    ("W2 transposed in backward", "backward", _bwd_w2_transposed, "hand"),
    ("mean dropped", "backward", _bwd_no_mean, "fd"),
    ("adam bias correction dropped", "adam_step", _adam_no_bias_correction, "adam"),
    ("labels without overload test", "labels", _labels_no_threshold, "labels"),
    ("bf16 truncation", "bf16_round", _bf16_truncate, "bf16"),
])
def test_screener_mutation_is_caught(monkeypatch, golden_dir, name, attr, fake, pin):
    monkeypatch.setattr(sref, attr, fake)
    fn = {"fd": lambda: spins.test_gradients_match_central_differences(None),
          "hand": lambda: spins.test_hand_worked_network(golden_dir),
          "adam": spins.test_adam_first_steps_closed_form,
          "labels": spins.test_labels_characterisation,
          "bf16": spins.test_bf16_round_known_values_and_torch}[pin]
    assert _fails(fn), name


def _top_cases_ascending(cmax, cargmax, k):
    cm = np.asarray(cmax, np.float64)
    ca = np.asarray(cargmax, np.int64)
    shp = cm.shape[:-1]
    cmf, caf = cm.reshape(-1, cm.shape[-1]), ca.reshape(-1, ca.shape[-1])
    oc = -np.ones((cmf.shape[0], k), np.int64)
    om = -np.ones((cmf.shape[0], k), np.int64)
    ol = np.zeros((cmf.shape[0], k))
    for r in range(cmf.shape[0]):
        valid = [c for c in range(cmf.shape[1]) if cmf[r, c] >= 0]
        order = sorted(valid, key=lambda c: (cmf[r, c], c))[:k]  # planted: lowest loadings first
        for j, c in enumerate(order):
            oc[r, j], om[r, j], ol[r, j] = c, caf[r, c], cmf[r, c]
    return oc.reshape(shp + (k,)), om.reshape(shp + (k,)), ol.reshape(shp + (k,))


def test_top_cases_mutation_is_caught(monkeypatch):
    monkeypatch.setattr(ref, "top_cases", _top_cases_ascending)
    monkeypatch.setattr(oracle, "top_cases", _top_cases_ascending)
    assert _fails(pins.test_top_cases_k1_is_the_worst_case_and_k3_matches_refactorisation)


def test_generator_n1_mutation_is_caught(monkeypatch):
    """A generator failure that adds its output instead of removing it."""
    orig = ref.generator_n1

    def wrong_sign(grid, topo, P, gen_bus, gen_p, mon, limit, idx=None):
        return orig(grid, topo, P, gen_bus, -np.asarray(gen_p, np.float64), mon, limit, idx)  # planted

    monkeypatch.setattr(ref, "generator_n1", wrong_sign)
    monkeypatch.setattr(oracle, "generator_n1", wrong_sign)
    assert _fails(pins.test_generator_n1_closed_forms)


def test_multi_outage_mutation_is_caught(monkeypatch):
    """A multi-outage case that takes out only the first branch of each set."""
    orig = ref.multi_outage_n1

    def first_only(grid, topo, P, multi, mon, limit, idx=None):
        return orig(grid, topo, P, [list(m)[:1] for m in multi], mon, limit, idx)  # planted

    monkeypatch.setattr(ref, "multi_outage_n1", first_only)
    monkeypatch.setattr(oracle, "multi_outage_n1", first_only)
    assert _fails(pins.test_multi_outage_reduces_to_lodf_and_modf)


_orig_eligible = ref.eligible_injections


def _eligible_descending(inc, splits, inj_bus, cap=64):
    el, buses = _orig_eligible(inc, splits, inj_bus, cap)
    return el[::-1], buses  # planted: mask bits counted from the highest injection index


def _eligible_first_split(inc, splits, inj_bus, cap=64):
    el, buses = _orig_eligible(inc, splits, inj_bus, cap)
    return [(e, 0) for e, _ in el], buses  # planted: every injection onto the first split's busbar B


def _eligible_off_slack(inc, splits, inj_bus, cap=64):
    el, buses = _orig_eligible(inc, splits, inj_bus, cap)
    return el, [0 for _ in buses]  # planted: the moved power is taken off bus 0 (the slack), not bus A


@pytest.mark.parametrize("mut", [_eligible_descending, _eligible_first_split, _eligible_off_slack])
def test_injection_topology_mutation_is_caught(monkeypatch, mut):
    monkeypatch.setattr(ref, "eligible_injections", mut)
    assert _fails(pins.test_injection_topology_flows_match_the_split_grid_by_hand)


_orig_classify = ref.classify_contingencies
_orig_count = ref.loadflow_count


def _classify_bridges_solved(cont, alive, br):
    valid = np.array([bool(alive[c]) for c in cont], dtype=bool)  # planted: bridges counted as solved
    return valid, 0


def _classify_outaged_as_island(cont, alive, br):
    valid, _ = _orig_classify(cont, alive, br)
    return valid, int(sum(1 for c in cont if (not alive[c]) or br[c]))  # planted: outaged counted as islanding


def _count_without_candidate_guard(res, n_timesteps, n_var=0):
    ok = res["status"] == ref.OK
    return int(res["n_valid_cont"][ok].sum()) * n_timesteps * n_var  # planted: max(1, U) dropped


def _count_nominal(res, n_timesteps, n_var=0):
    n = len(res["status"]) * int((res["n_valid_cont"] + res["n_island_cont"]).max())
    return n * n_timesteps * max(1, n_var)  # planted: nominal cases, skipped ones included


@pytest.mark.parametrize("attr,fake", [
    ("classify_contingencies", _classify_bridges_solved),
    ("classify_contingencies", _classify_outaged_as_island),
    ("loadflow_count", _count_without_candidate_guard),
    ("loadflow_count", _count_nominal),
], ids=["bridges_solved", "outaged_as_island", "no_candidate_guard", "nominal_count"])
def test_loadflow_count_mutation_is_caught(monkeypatch, golden_dir, attr, fake):
    monkeypatch.setattr(ref, attr, fake)
    monkeypatch.setattr(oracle, attr, fake, raising=False)
    assert _fails(pins.test_loadflow_count_hand_counted, golden_dir)


_orig_band = ref.first_in_band


def _band_highest_index(values, eps, lowest=False):
    v = np.asarray(values, np.float64)
    best = v.min() if lowest else v.max()
    ok = (v <= best + eps * max(abs(best), 1.0)) if lowest else (v >= best - eps * max(abs(best), 1.0))
    return int(np.nonzero(ok)[0][-1])  # planted: the highest index inside the band


def _band_without_scale(values, eps, lowest=False):
    v = np.asarray(values, np.float64)
    best = v.min() if lowest else v.max()
    ok = (v <= best + eps) if lowest else (v >= best - eps)  # planted: band not scaled by max(|best|, 1)
    return int(np.nonzero(ok)[0][0])


@pytest.mark.parametrize("fake", [_band_highest_index, _band_without_scale])
def test_tie_band_mutation_is_caught(monkeypatch, golden_dir, fake):
    monkeypatch.setattr(ref, "first_in_band", fake)
    monkeypatch.setattr(oracle, "first_in_band", fake)
    caught = _fails(pins.test_first_in_band_hand_values) or \
        _fails(pins.test_series_branches_tie_goes_to_the_lowest_position, golden_dir)
    assert caught
