"""Pins of the screener reference (oracle/screener_ref.py) against hand work,
finite differences, closed forms and an independent library."""
import json
import math
import os

import numpy as np
import pytest

from oracle import screener_ref as sr


def _params(d):
    return {k: np.asarray(v, np.float64) for k, v in d.items()}


def test_hand_worked_network(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "mlp_tiny.json")))
    p = _params(g["params"])
    z, cache = sr.forward(p, np.asarray(g["x"]))
    np.testing.assert_allclose(cache["h1"], g["h1"], atol=0)
    np.testing.assert_allclose(cache["h2"], g["h2"], atol=0)
    np.testing.assert_allclose(z, g["z"], atol=0)
    y = np.asarray(g["y"], np.float64)
    assert sr.bce_loss(z, y) == pytest.approx(math.log1p(math.exp(g["loss_softplus_arg"])), rel=1e-14)
    d = 1.0 / (1.0 + math.exp(1.75)) - 1.0
    gr = sr.backward(p, cache, z, y)
    for k, v in g["grad_over_d"].items():
        np.testing.assert_allclose(gr[k], d * np.asarray(v), rtol=1e-13, atol=1e-15, err_msg=k)


@pytest.mark.parametrize("rounding", [None])
def test_gradients_match_central_differences(rounding):
    rng = np.random.default_rng(7)
    F, H, C, B = 7, 5, 4, 6
    p = sr.init_params(F, H, C, 3)
    for k in ("b1", "b2", "b3"):
        p[k] = rng.normal(0, 0.3, p[k].shape)
    X = rng.normal(0, 1, (B, F))
    Y = (rng.random((B, C)) < 0.3).astype(np.uint8)
    z, cache = sr.forward(p, X)
    g = sr.backward(p, cache, z, Y)
    h = 1e-6
    for k in sr.PARAM_NAMES:
        flat = p[k].reshape(-1)
        for i in range(flat.size):
            old = flat[i]
            flat[i] = old + h
            lp = sr.bce_loss(sr.forward(p, X)[0], Y)
            flat[i] = old - h
            lm = sr.bce_loss(sr.forward(p, X)[0], Y)
            flat[i] = old
            fd = (lp - lm) / (2 * h)
            an = g[k].reshape(-1)[i]
            assert abs(fd - an) <= 1e-7 + 1e-5 * abs(fd), (k, i, fd, an)


def test_bce_special_values():
    z = np.array([[0.0, 0.0]])
    assert sr.bce_loss(z, np.array([[0, 1]])) == pytest.approx(math.log(2.0), rel=1e-15)
    assert sr.bce_loss(np.array([[40.0]]), np.array([[1]])) < 1e-16
    assert sr.bce_loss(np.array([[-40.0]]), np.array([[1]])) == pytest.approx(40.0, rel=1e-15)
    for zz in (-3.0, -0.4, 0.7, 2.5):
        for y in (0, 1):
            s = 1.0 / (1.0 + math.exp(-zz))
            want = -(y * math.log(s) + (1 - y) * math.log(1 - s))
            assert sr.bce_loss(np.array([[zz]]), np.array([[y]])) == pytest.approx(want, rel=1e-12)


def test_adam_first_steps_closed_form():
    rng = np.random.default_rng(1)
    p = {k: rng.normal(size=(3, 2)) for k in sr.PARAM_NAMES}
    g = {k: rng.normal(size=(3, 2)) for k in sr.PARAM_NAMES}
    m = {k: np.zeros((3, 2)) for k in sr.PARAM_NAMES}
    v = {k: np.zeros((3, 2)) for k in sr.PARAM_NAMES}
    p0 = {k: x.copy() for k, x in p.items()}
    lr, eps = 1e-2, 1e-8
    sr.adam_step(p, g, m, v, 1, lr, eps=eps)
    for k in sr.PARAM_NAMES:  # bias-corrected moments are g and g^2 after one step
        np.testing.assert_allclose(p[k], p0[k] - lr * g[k] / (np.abs(g[k]) + eps), rtol=1e-12)
    sr.adam_step(p, g, m, v, 2, lr, eps=eps)  # a constant gradient keeps the step
    for k in sr.PARAM_NAMES:
        np.testing.assert_allclose(p[k], p0[k] - 2 * lr * g[k] / (np.abs(g[k]) + eps), rtol=1e-12)


def test_bf16_round_known_values_and_torch():
    one = 1.0
    assert sr.bf16_round(one) == 1.0
    assert sr.bf16_round(1.0 + 2.0 ** -8) == 1.0                    # halfway, even neighbour below
    assert sr.bf16_round(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6    # halfway, even neighbour above
    assert sr.bf16_round(1.0 + 2.0 ** -8 + 2.0 ** -20) == 1.0 + 2.0 ** -7
    assert sr.bf16_round(-2.5) == -2.5
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(2).normal(0, 10, 20000)
    want = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(sr.bf16_round(x), want)


def test_labels_characterisation():
    rng = np.random.default_rng(4)
    for trial in range(40):
        C = int(rng.integers(1, 30))
        k = int(rng.integers(1, 12))
        row = np.round(rng.uniform(0.0, 2.0, C), 1)  # coarse values: many ties
        row[rng.random(C) < 0.1] = -1.0
        Y = sr.labels(row[None, :], k)[0]
        pos = set(np.nonzero(Y)[0])
        over = [c for c in range(C) if row[c] > 1.0]
        assert len(pos) == min(k, len(over))
        assert all(row[c] > 1.0 for c in pos)
        for c in pos:  # nothing outside the set outranks a member
            for c2 in over:
                if c2 not in pos:
                    assert (row[c2], -c2) < (row[c], -c)


def test_top_k_and_recall():
    s = np.array([[0.1, 0.9, 0.9, 0.3, 0.8]])
    np.testing.assert_array_equal(sr.top_k(s, 2), [[1, 2]])
    np.testing.assert_array_equal(sr.top_k(s, 3), [[1, 2, 4]])
    Y = np.array([[0, 1, 0, 1, 1]])
    assert sr.recall(np.array([[1, 2, 4]]), Y) == pytest.approx(2 / 3)
    assert sr.recall(np.array([[0, 2]]), np.zeros((1, 5))) == 1.0


def test_feature_layout_and_bits():
    from paper_2501_17529_b300 import synth
    from oracle import dcflow_ref as ref
    w = synth.workload(1, n_topo=8)
    lim = ref.thermal_limits(w.grid, w.inj)
    lay, nbits = sr.feature_layout(w.grid, w.subs)
    inc = ref.incident_lists(w.grid.n_bus, w.grid.f, w.grid.t)
    assert nbits == sum(len(inc[s]) for s in w.subs)
    X = sr.features(w.grid, w.topo, w.inj, w.mon, lim, w.subs)
    M = len(w.mon)
    for i in range(w.topo.n_topo):
        bits = np.zeros(nbits)
        for k in range(w.topo.split_ptr[i], w.topo.split_ptr[i + 1]):
            o, d = lay[int(w.topo.split_sub[k])]
            for j in range(d):
                bits[o + j] = (int(w.topo.split_mask[k]) >> j) & 1
        if np.any(X[i, :, :M]):
            np.testing.assert_array_equal(X[i, 0, M:], bits)
    # an empty topology gives the base loadings
    empty = synth.Topologies(np.zeros(2, np.int32), np.zeros(0, np.int32), np.zeros(0, np.uint64),
                             np.zeros(2, np.int32), np.zeros(0, np.int32))
    X0 = sr.features(w.grid, empty, w.inj, w.mon, lim, w.subs)
    np.testing.assert_allclose(X0[0, :, :M], ref.base_flows(w.grid, w.inj)[:, w.mon] / lim[w.mon], rtol=1e-12)
    assert not X0[0, :, M:].any()
