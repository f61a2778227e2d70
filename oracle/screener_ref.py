"""Plain FP64 reference of the learned contingency screener (test infrastructure).

The paper has no learned component; the screener sits beside its method as a
filter in front of the exact N-1 of Def. 3 / Eq. (5): a 3-layer perceptron
predicts, per (topology, timestep), which contingencies are among the most
severe, so that only those are solved exactly.  What this module defines:

* features (per topology and timestep): the signed N-0 loadings
  p_n0[l] / limit_l of the monitored branches (Eq. (2) on the split/outaged
  topology), then one bit per incident branch of every split-capable
  substation (substations in ascending bus id, their branches in ascending
  branch id, the bit order of the busbar masks t_b of Sec. III-A): 1 if the
  branch is on busbar B;
* labels: contingency c is positive for (topology, timestep) if its maximum
  N-1 loading max_l rho[l, c] exceeds 1 AND c is among the k largest of those
  maxima (ties to the lower contingency position); rows of islanded or invalid
  topologies are all-negative;
* network: h1 = relu(x W1^T + b1), h2 = relu(h1 W2^T + b2), z = h2 W3^T + b3;
* loss: binary cross-entropy on the logits, averaged over rows and
  contingencies: mean(softplus(z) - y z);
* gradients by the chain rule (no autograd), Adam (Kingma & Ba, 2015,
  Algorithm 1) with bias correction;
* an optional rounding model: ``rounding="bf16"`` rounds the stored values of
  the mixed-precision form (inputs, weights, h1, h2 and the back-propagated
  dz, dh2, dh1) to bfloat16 (round to nearest even), so that a tensor-core
  implementation that stores those tensors in bf16 and accumulates in FP32 can
  be compared with this reference at a tolerance set by FP32 accumulation
  order rather than by bf16 rounding;
* recall of a predicted set against the labels.

Pins (tests/test_oracle_screener.py): a hand-worked 2-2-2-1 network
(forward, loss and every gradient, tests/golden/mlp_tiny.json), central
finite differences of the loss, the closed form of Adam's first step, BCE
special values, bf16 rounding against known values and against PyTorch's
bf16 conversion, and labels against a brute-force sort.
"""
from __future__ import annotations

import numpy as np

from .dcflow_ref import OK, incident_lists, topology_flows

PARAM_NAMES = ("W1", "b1", "W2", "b2", "W3", "b3")


# ---------------------------------------------------------------------------
# bfloat16 rounding model
# ---------------------------------------------------------------------------
def bf16_round(x):
    """Round to the nearest bfloat16 (ties to even) via IEEE float32; returns float64.

    bfloat16 keeps the sign, the 8 exponent bits and the top 7 mantissa bits of
    a float32.  The value is first rounded to float32 (round to nearest), then
    the low 16 bits are rounded away: add 0x7FFF plus the lowest kept bit and
    truncate, which is round-half-to-even on the dropped half-word."""
    a = np.asarray(x, np.float64).astype(np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    out = (r & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(a)
    if np.any(nan):
        out = np.where(nan, np.nan, out)
    return out


def _r(x, rounding):
    return bf16_round(x) if rounding == "bf16" else x


# ---------------------------------------------------------------------------
# network
# ---------------------------------------------------------------------------
def init_params(F, H, C, seed):
    """He-normal weights, zero biases (a reference initialisation for tests)."""
    rng = np.random.default_rng(seed)
    return {
        "W1": rng.normal(0.0, np.sqrt(2.0 / F), (H, F)), "b1": np.zeros(H),
        "W2": rng.normal(0.0, np.sqrt(2.0 / H), (H, H)), "b2": np.zeros(H),
        "W3": rng.normal(0.0, np.sqrt(2.0 / H), (C, H)), "b3": np.zeros(C),
    }


def forward(params, X, rounding=None):
    """Logits [B, C] and the intermediate values needed by ``backward``."""
    W1 = _r(params["W1"], rounding)
    W2 = _r(params["W2"], rounding)
    W3 = _r(params["W3"], rounding)
    x = _r(np.asarray(X, np.float64), rounding)
    a1 = x @ W1.T + params["b1"]
    h1 = _r(np.maximum(a1, 0.0), rounding)
    a2 = h1 @ W2.T + params["b2"]
    h2 = _r(np.maximum(a2, 0.0), rounding)
    z = h2 @ W3.T + params["b3"]
    return z, dict(x=x, h1=h1, h2=h2, W1=W1, W2=W2, W3=W3)


def softplus(z):
    z = np.asarray(z, np.float64)
    return np.maximum(z, 0.0) + np.log1p(np.exp(-np.abs(z)))


def sigmoid(z):
    z = np.asarray(z, np.float64)
    e = np.exp(-np.abs(z))
    return np.where(z >= 0, 1.0 / (1.0 + e), e / (1.0 + e))


def bce_loss(z, Y):
    """Mean binary cross-entropy with logits over every row and contingency."""
    Y = np.asarray(Y, np.float64)
    return float(np.mean(softplus(z) - Y * z))


def backward(params, cache, z, Y, rounding=None):
    """Gradients of ``bce_loss`` with respect to every parameter (chain rule)."""
    Y = np.asarray(Y, np.float64)
    B, C = z.shape
    dz = _r((sigmoid(z) - Y) / (B * C), rounding)  # d loss / d z
    g = {}
    g["W3"] = dz.T @ cache["h2"]
    g["b3"] = dz.sum(axis=0)
    dh2 = _r((dz @ cache["W3"]) * (cache["h2"] > 0), rounding)  # relu' of a2 (h2 > 0 iff a2 > 0)
    g["W2"] = dh2.T @ cache["h1"]
    g["b2"] = dh2.sum(axis=0)
    dh1 = _r((dh2 @ cache["W2"]) * (cache["h1"] > 0), rounding)
    g["W1"] = dh1.T @ cache["x"]
    g["b1"] = dh1.sum(axis=0)
    return g


def adam_step(params, grads, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (t = 1 for the first step), in place; returns the params."""
    for k in PARAM_NAMES:
        m[k] = beta1 * m[k] + (1.0 - beta1) * grads[k]
        v[k] = beta2 * v[k] + (1.0 - beta2) * grads[k] ** 2
        mh = m[k] / (1.0 - beta1 ** t)
        vh = v[k] / (1.0 - beta2 ** t)
        params[k] = params[k] - lr * mh / (np.sqrt(vh) + eps)
    return params


# ---------------------------------------------------------------------------
# features and labels
# ---------------------------------------------------------------------------
def feature_layout(grid, split_bus):
    """Offsets of the split bits: {substation: (offset, degree)} after the M loadings."""
    inc = incident_lists(grid.n_bus, grid.f, grid.t)
    off, lay = 0, {}
    for s in sorted(int(x) for x in split_bus):
        lay[s] = (off, len(inc[s]))
        off += len(inc[s])
    return lay, off


def features(grid, topo, P, mon, limit, split_bus, idx=None):
    """Feature rows [n_topo, T, M + n_bits] (zero rows for islanded/invalid topologies)."""
    lay, nbits = feature_layout(grid, split_bus)
    mon = np.asarray(mon, np.int64)
    lim = np.asarray(limit, np.float64)[mon]
    P = np.atleast_2d(np.asarray(P, np.float64))
    T = P.shape[0]
    ids = range(topo.n_topo) if idx is None else [int(i) for i in idx]
    out = np.zeros((len(ids), T, mon.size + nbits))
    for r, i in enumerate(ids):
        a, c = topo.split_ptr[i], topo.split_ptr[i + 1]
        splits = list(zip(topo.split_sub[a:c], topo.split_mask[a:c]))
        a, c = topo.out_ptr[i], topo.out_ptr[i + 1]
        outages = list(topo.out_branch[a:c])
        fl, info = topology_flows(grid, splits, outages, P.T)
        if fl is None:
            continue
        out[r, :, :mon.size] = (fl[mon] / lim[:, None]).T
        for s, mask in splits:
            o, d = lay[int(s)]
            for j in range(d):
                out[r, :, mon.size + o + j] = float((int(mask) >> j) & 1)
    return out


def labels(cmax, k):
    """Positive iff max_l rho[l, c] > 1 and c is among the k largest maxima of its row.

    cmax: [..., C] per-contingency maximum loading (negative = not evaluated:
    islanding contingency or invalid topology).  Ties in the ranking go to the
    lower contingency position."""
    cm = np.asarray(cmax, np.float64)
    shp = cm.shape
    flat = cm.reshape(-1, shp[-1])
    Y = np.zeros(flat.shape, np.uint8)
    for r in range(flat.shape[0]):
        order = sorted(range(flat.shape[1]), key=lambda c: (-flat[r, c], c))
        for c in order[:k]:
            if flat[r, c] > 1.0:
                Y[r, c] = 1
    return Y.reshape(shp)


def top_k(scores, k):
    """Indices of the k largest scores of every row (ties to the lower index), ascending."""
    s = np.asarray(scores, np.float64)
    flat = s.reshape(-1, s.shape[-1])
    out = np.zeros((flat.shape[0], min(k, flat.shape[1])), np.int64)
    for r in range(flat.shape[0]):
        order = sorted(range(flat.shape[1]), key=lambda c: (-flat[r, c], c))
        out[r] = np.sort(order[:k])
    return out.reshape(s.shape[:-1] + (out.shape[1],))


def recall(pred, Y):
    """sum |pred ∩ true| / sum |true| over rows; pred: [..., k] index sets, Y: [..., C] labels."""
    Yf = np.asarray(Y).reshape(-1, np.asarray(Y).shape[-1])
    Pf = np.asarray(pred).reshape(Yf.shape[0], -1)
    hit = sum(int(Yf[r, Pf[r]].sum()) for r in range(Yf.shape[0]))
    tot = int(Yf.sum())
    return hit / tot if tot else 1.0


def ok_rows(status):
    return np.asarray(status) == OK
