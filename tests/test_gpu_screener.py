"""Learned screener on the GPU against the FP64 screener reference: forward,
gradients and Adam with identical BF16-rounded weights, labels, features, the
screened solve against the oracle restricted to the evaluated contingencies,
and what a trained network gains over the full N-1."""
import numpy as np
import pytest

from oracle import dcflow_ref as ref
from oracle import screener_ref as sr
from paper_2501_17529_b300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2501_17529_b300.csrc import build
    build.build()


@pytest.fixture(scope="module")
def study():
    w = synth.workload(2, n_topo=24, T=3)
    lim = ref.thermal_limits(w.grid, w.inj)
    from paper_2501_17529_b300.dcflow import Screener, Solver
    s = Solver(w.grid, precision="fp32")
    s.set_study(w.mon, w.cont, lim, split_bus=w.subs)
    scr = Screener(s, max_rows=384, seed=3)
    yield w, lim, s, scr
    scr.close()
    s.close()


def _base_bridges(grid):
    """Branches whose outage islands the unsplit grid (they island every topology)."""
    alive = np.ones(grid.n_branch, dtype=bool)
    return np.asarray(ref.bridges(grid.n_bus, np.asarray(grid.f), np.asarray(grid.t), alive), dtype=bool)


def _random_params(scr, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    p = sr.init_params(scr.F, scr.H, scr.C, seed)
    for k in ("b1", "b2", "b3"):
        p[k] = rng.normal(0, 0.1, p[k].shape)
    for k in p:
        p[k] = (p[k] * scale).astype(np.float32).astype(np.float64)
        scr.set(k, p[k])
    return p


def _bf16_rows(rng, n, F, Fp):
    X = np.zeros((n, Fp))
    X[:, :F] = sr.bf16_round(rng.normal(0, 1, (n, F)))
    return X, torch.tensor(X, dtype=torch.float32).to(torch.bfloat16).cuda()


def test_forward_matches_reference(study):
    w, lim, s, scr = study
    p = _random_params(scr, 11)
    rng = np.random.default_rng(12)
    X, Xd = _bf16_rows(rng, 300, scr.F, scr.F_pad)  # 300 rows: several 128-row tiles and a ragged tail
    Z = scr.logits(Xd).cpu().numpy()
    z, _ = sr.forward(p, X[:, :scr.F], rounding="bf16")
    err = np.abs(Z - z).max()
    assert err <= 5e-3 * np.abs(z).max() + 1e-4, err


def test_gradients_match_reference(study):
    w, lim, s, scr = study
    p = _random_params(scr, 21)
    rng = np.random.default_rng(22)
    X, Xd = _bf16_rows(rng, 320, scr.F, scr.F_pad)
    Y = np.zeros((320, scr.C_pad), np.uint8)
    Y[:, :scr.C] = rng.random((320, scr.C)) < 0.08
    rows = np.sort(rng.choice(320, 200, replace=False)).astype(np.int32)[::-1].copy()  # gathered, reordered
    loss = scr.backward(Xd, torch.tensor(Y).cuda(), rows=torch.tensor(rows).cuda())
    z, cache = sr.forward(p, X[rows, :scr.F], rounding="bf16")
    g = sr.backward(p, cache, z, Y[rows, :scr.C], rounding="bf16")
    assert float(loss.item()) == pytest.approx(sr.bce_loss(z, Y[rows, :scr.C]), rel=1e-4)
    for k in sr.PARAM_NAMES:
        gg = scr.get(k, "grad").astype(np.float64)
        rel = np.linalg.norm(gg - g[k]) / max(np.linalg.norm(g[k]), 1e-30)
        assert rel <= 1e-2, (k, rel)


def test_adam_matches_reference(study):
    w, lim, s, scr = study
    rng = np.random.default_rng(31)
    st = {}
    for k in sr.PARAM_NAMES:
        shp = scr.shape(k)
        st[k] = [rng.normal(0, 1, shp).astype(np.float32) for _ in range(3)]
        st[k].append(np.abs(rng.normal(0, 1, shp)).astype(np.float32))
        for kind, v in zip(("param", "grad", "m", "v"), st[k]):
            scr.set(k, v, kind)
    from paper_2501_17529_b300.dcflow import dcflow_screen_adam_step
    dcflow_screen_adam_step(scr.scr, 6)
    scr.adam(3e-3)
    torch.cuda.synchronize()
    params = {k: st[k][0].astype(np.float64) for k in sr.PARAM_NAMES}
    grads = {k: st[k][1].astype(np.float64) for k in sr.PARAM_NAMES}
    m = {k: st[k][2].astype(np.float64) for k in sr.PARAM_NAMES}
    v = {k: st[k][3].astype(np.float64) for k in sr.PARAM_NAMES}
    sr.adam_step(params, grads, m, v, 7, 3e-3)
    assert dcflow_screen_adam_step(scr.scr) == 7
    for k in sr.PARAM_NAMES:
        np.testing.assert_allclose(scr.get(k), params[k], rtol=1e-5, atol=1e-6, err_msg=k)
        np.testing.assert_allclose(scr.get(k, "m"), m[k], rtol=1e-5, atol=1e-7, err_msg=k)
        np.testing.assert_allclose(scr.get(k, "v"), v[k], rtol=1e-5, atol=1e-7, err_msg=k)


def test_labels_bit_exact(study):
    w, lim, s, scr = study
    rng = np.random.default_rng(41)
    rows = 257
    cm = np.round(rng.uniform(0.0, 1.6, (rows, scr.C)), 2).astype(np.float32)  # coarse: many ties
    cm[rng.random((rows, scr.C)) < 0.05] = -1.0
    cm[7] = -1.0  # a row of an islanded topology
    for k in (1, 64, 700):
        Y = scr.labels(torch.tensor(cm.reshape(-1)).cuda(), k).cpu().numpy()
        np.testing.assert_array_equal(Y[:, :scr.C], sr.labels(cm.astype(np.float64), k))
        assert not Y[:, scr.C:].any()


def test_features_match_reference(study):
    w, lim, s, scr = study
    from paper_2501_17529_b300.dcflow import DeviceBatch
    topo = synth.make_topologies(w.grid, w.subs, 30, 77, (1, 4), (0, 3))
    X, status = scr.features(DeviceBatch(topo, w.inj))
    X = X.float().cpu().numpy().reshape(30, 3, scr.F_pad)
    want = sr.features(w.grid, topo, w.inj, w.mon, lim, w.subs)
    ev = ref.evaluate(w.grid, topo, w.inj, w.mon, w.cont, lim)
    np.testing.assert_array_equal(status.cpu().numpy(), ev["status"])
    M = len(w.mon)
    assert np.all(np.abs(X[..., :M] - want[..., :M]) <= 2.0 ** -8 * np.abs(want[..., :M]) + 1e-5)
    np.testing.assert_array_equal(X[..., M:scr.F], want[..., M:])
    assert not X[..., scr.F:].any()
    assert not X[ev["status"] != 0].any()


def test_screened_solve_matches_oracle_on_evaluated_set(study):
    w, lim, s, scr = study
    from paper_2501_17529_b300.dcflow import DeviceBatch
    p = _random_params(scr, 51, scale=0.5)
    topo = synth.make_topologies(w.grid, w.subs, 12, 78, (1, 4), (0, 3))
    k = 24
    res, rep = s.solve_screened(DeviceBatch(topo, w.inj), scr, top_k=k, want_pred=True)
    out = res.to_host()
    pred = rep["pred"].cpu().numpy().reshape(12, 3, k)
    neval = rep["n_eval"].cpu().numpy()[:12]
    assert not rep["fallback"].cpu().numpy()[:12].any()
    # the predictions are the top k of the reference scores (near-ties either way)
    Xo = sr.features(w.grid, topo, w.inj, w.mon, lim, w.subs)
    z, _ = sr.forward(p, sr.bf16_round(Xo.reshape(36, -1)), rounding="bf16")
    z = z.reshape(12, 3, -1)
    for i in range(12):
        if out["status"][i] != 0:
            assert (pred[i] == -1).all() and neval[i] == 0
            continue
        for t in range(3):
            zz = z[i, t]
            kth = np.sort(zz)[::-1][k - 1]
            tol = 5e-3 * np.abs(zz).max() + 1e-4
            sel = set(pred[i, t].tolist())
            assert len(sel) == k and -1 not in sel
            assert all(zz[c] >= kth - 2 * tol for c in sel)
            assert all(c in sel for c in np.nonzero(zz > kth + 2 * tol)[0])
        union = np.unique(pred[i])
        assert neval[i] == int((~_base_bridges(w.grid)[w.cont[union]]).sum())  # bridges are never evaluated
        # the oracle over exactly the evaluated contingencies
        o = ref.evaluate(w.grid, topo.subset([i]), w.inj, w.mon, w.cont[union], lim)
        np.testing.assert_allclose(out["n1_max"][i], o["n1_max"][0], rtol=1e-4, atol=1e-6)
        np.testing.assert_allclose(out["ovl"][i], o["ovl"][0], rtol=1e-4, atol=1e-4)
        for t in range(3):
            wc = o["worst_cont"][0, t]
            assert out["worst_cont"][i, t] == (union[wc] if wc >= 0 else -1) or \
                abs(out["n1_max"][i, t] - o["n1_max"][0, t]) <= 1e-4 * o["n1_max"][0, t]


def test_screened_fallback_is_the_full_n1(study):
    w, lim, s, scr = study
    from paper_2501_17529_b300.dcflow import DeviceBatch
    _random_params(scr, 61)
    topo = synth.make_topologies(w.grid, w.subs, 16, 79, (1, 4), (0, 3))
    db = DeviceBatch(topo, w.inj)
    full = s.solve(db).to_host()
    res, rep = s.solve_screened(db, scr, top_k=8, fallback_logit=-float("inf"))
    out = res.to_host()
    ok = full["status"] == 0
    assert rep["fallback"].cpu().numpy()[:16][ok].all()
    assert (rep["n_eval"].cpu().numpy()[:16][ok] == int((~_base_bridges(w.grid)[w.cont]).sum())).all()
    np.testing.assert_allclose(out["n1_max"], full["n1_max"], rtol=1e-5)
    np.testing.assert_allclose(out["ovl"], full["ovl"], rtol=1e-4, atol=1e-4)
    np.testing.assert_array_equal(out["status"], full["status"])


def test_checkpoint_round_trip(study, tmp_path):
    w, lim, s, scr = study
    _random_params(scr, 71)
    rng = np.random.default_rng(72)
    X, Xd = _bf16_rows(rng, 128, scr.F, scr.F_pad)
    Z0 = scr.logits(Xd).cpu().numpy()
    scr.save(tmp_path / "ck.npz")
    _random_params(scr, 72)
    assert np.abs(scr.logits(Xd).cpu().numpy() - Z0).max() > 1e-3
    scr.load(tmp_path / "ck.npz")
    np.testing.assert_array_equal(scr.logits(Xd).cpu().numpy(), Z0)


def test_trained_screener_gains_over_full_n1():
    """On the 2000-bus screener study (1,000 contingencies, 8 timesteps): trained on
    solver labels of 40,000 topologies, the screened solve keeps the exact top-64
    overloads of held-out topologies (the threshold of the additions calibrated on
    a third set) and is measured faster than the full N-1 it replaces."""
    from paper_2501_17529_b300 import screener as drv
    from paper_2501_17529_b300.dcflow import Screener, Solver
    w = synth.workload(5, n_topo=40000)
    lim = drv._limits(w)
    s = Solver(w.grid, precision="fp32")
    s.set_study(w.mon, w.cont, lim, split_bus=w.subs)
    scr = Screener(s, max_rows=4096, seed=5)
    ev_topo = synth.make_topologies(w.grid, w.subs, 10000, 605, (1, 8), (0, 0))
    cal_topo = synth.make_topologies(w.grid, w.subs, 5000, 606, (1, 8), (0, 0))
    Xtr, Ytr, _, _, st_tr = drv.dataset(s, scr, w.topo, w.inj)
    Xev, Yev, cm_ev, n1_ev, st_ev = drv.dataset(s, scr, ev_topo, w.inj)
    Xc, Yc, cm_c, n1_c, st_c = drv.dataset(s, scr, cal_topo, w.inj)
    del Xev, Xc
    before = drv.evaluate(s, scr, ev_topo, w.inj, Yev, cm_ev, n1_ev, st_ev, repeats=1)
    hist = drv.train(scr, Xtr, Ytr, st_tr, 8, epochs=30, batch=4096, lr=1e-3, cosine=True)
    plain = drv.evaluate(s, scr, ev_topo, w.inj, Yev, cm_ev, n1_ev, st_ev, repeats=3)
    p_min, curve = drv.calibrate_min_prob(s, scr, cal_topo, w.inj, Yc, cm_c, n1_c, st_c, target=0.98)
    after = drv.evaluate(s, scr, ev_topo, w.inj, Yev, cm_ev, n1_ev, st_ev, repeats=3, min_prob=p_min)
    print("screener before", before)
    print("screener top 64", plain)
    print("screener calibrated", p_min, curve, after)
    assert hist[-1] < hist[0]
    assert plain["recall_at_k"] > before["recall_at_k"] + 0.2
    assert plain["recall_evaluated"] >= 0.9 and plain["speedup"] > 1.5
    assert after["recall_evaluated"] >= 0.97 and after["speedup"] > 1.2
    assert after["evaluated_fraction"] <= 0.35
    assert after["worst_cont_hit_rate"] >= 0.99
    scr.close()
    s.close()


def test_screened_solve_probability_additions(study):
    """min_prob: besides each row's top k, every contingency the network scores above
    the probability is evaluated; the reported evaluated set covers both, and the
    results equal the oracle over exactly that set."""
    w, lim, s, scr = study
    from paper_2501_17529_b300.dcflow import DeviceBatch
    p = _random_params(scr, 53, scale=0.5)
    topo = synth.make_topologies(w.grid, w.subs, 10, 81, (1, 4), (0, 3))
    k, pm = 8, 0.1
    res, rep = s.solve_screened(DeviceBatch(topo, w.inj), scr, top_k=k, want_pred=True, min_prob=pm,
                                want_evaluated=True)
    out = res.to_host()
    C = len(w.cont)
    Wd = (C + 31) // 32
    evw = rep["evaluated"].cpu().numpy()[:10 * Wd].view(np.uint32).reshape(10, Wd)
    ev = ((evw[:, :, None] >> np.arange(32, dtype=np.uint32)) & 1).reshape(10, -1)[:, :C].astype(bool)
    pred = rep["pred"].cpu().numpy().reshape(10, 3, k)
    neval = rep["n_eval"].cpu().numpy()[:10]
    Xo = sr.features(w.grid, topo, w.inj, w.mon, lim, w.subs)
    z, _ = sr.forward(p, sr.bf16_round(Xo.reshape(30, -1)), rounding="bf16")
    z = z.reshape(10, 3, -1)
    br = _base_bridges(w.grid)[w.cont]
    extra = 0
    for i in range(10):
        if out["status"][i] != 0:
            assert not ev[i].any() and neval[i] == 0
            continue
        top = set(np.unique(pred[i]).tolist())
        assert all(ev[i, c] or br[c] for c in top)
        thr = np.log(pm / (1 - pm))
        tol = 5e-3 * np.abs(z[i]).max() + 1e-4
        sure = np.nonzero((z[i] > thr + 2 * tol).any(axis=0))[0]
        assert all(ev[i, c] or br[c] for c in sure)
        extra += int(ev[i].sum()) - len([c for c in top if not br[c]])
        assert neval[i] == int(ev[i].sum())
        o = ref.evaluate(w.grid, topo.subset([i]), w.inj, w.mon, w.cont[ev[i]], lim)
        np.testing.assert_allclose(out["n1_max"][i], o["n1_max"][0], rtol=1e-4, atol=1e-6)
        np.testing.assert_allclose(out["ovl"][i], o["ovl"][0], rtol=1e-4, atol=1e-4)
    assert extra > 0  # the threshold added contingencies beyond the top k


def test_screened_solve_fp64_matches_oracle():
    """The FP64 form of the screened N-1 (selected-contingency kernel in FP64)."""
    from paper_2501_17529_b300.dcflow import DeviceBatch, Screener, Solver
    w = synth.workload(2, n_topo=8, T=2)
    lim = ref.thermal_limits(w.grid, w.inj)
    s = Solver(w.grid, precision="fp64")
    s.set_study(w.mon, w.cont, lim, split_bus=w.subs)
    scr = Screener(s, max_rows=128, seed=9)
    res, rep = s.solve_screened(DeviceBatch(w.topo, w.inj), scr, top_k=16, want_pred=True)
    out = res.to_host()
    pred = rep["pred"].cpu().numpy().reshape(8, 2, 16)
    for i in range(8):
        if out["status"][i] != 0:
            continue
        union = np.unique(pred[i])
        o = ref.evaluate(w.grid, w.topo.subset([i]), w.inj, w.mon, w.cont[union], lim)
        np.testing.assert_allclose(out["n1_max"][i], o["n1_max"][0], rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(out["ovl"][i], o["ovl"][0], rtol=1e-10, atol=1e-10)
    scr.close()
    s.close()
