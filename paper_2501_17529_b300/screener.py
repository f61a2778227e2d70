"""Training and evaluation driver of the learned contingency screener.

Orchestration only: features, labels, the forward/backward passes, Adam and
the screened N-1 all run in libdcflow's kernels; PyTorch supplies device
memory, index permutations and reductions of reported statistics.

The exact full N-1 (``Solver.solve(want_cont_max=True)``) is both the source
of the training labels and the reference the screener is scored against:
recall is measured against it, and the screened solve falls back to it per
topology.

    python -m paper_2501_17529_b300.screener --train 200000 --eval 100000
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from .dcflow import DeviceBatch, DeviceResults, Screener, Solver


def exact(solver: Solver, topo, inj, chunk=20000):
    """Full N-1 with per-contingency maxima, in batches: (cont_max [N*T*C] f32, n1_max [N, T], status [N])."""
    import torch
    N, T, C = topo.n_topo, inj.shape[0], solver.n_cont
    cm = torch.empty(N * T * C, dtype=torch.float32, device="cuda")
    n1 = torch.empty((N, T), dtype=torch.float64, device="cuda")
    st = torch.empty(N, dtype=torch.uint8, device="cuda")
    for a in range(0, N, chunk):
        b = min(N, a + chunk)
        db = DeviceBatch(topo.subset(np.arange(a, b)), inj)
        r = solver.solve(db, want_cont_max=True)
        cm[a * T * C:b * T * C] = r.n1_cont_max[:(b - a) * T * C]
        n1[a:b] = r.n1_max_loading[:(b - a) * T].view(b - a, T)
        st[a:b] = r.island_flag[:b - a]
    return cm, n1, st


def dataset(solver: Solver, screener: Screener, topo, inj, k=64, chunk=20000):
    """Features X [N*T, F_pad] bf16, labels Y [N*T, C_pad] u8, cont_max, n1_max, status."""
    import torch
    N, T = topo.n_topo, inj.shape[0]
    X = torch.empty((N * T, screener.F_pad), dtype=torch.bfloat16, device="cuda")
    for a in range(0, N, chunk):
        b = min(N, a + chunk)
        db = DeviceBatch(topo.subset(np.arange(a, b)), inj)
        Xa, _ = screener.features(db)
        X[a * T:b * T] = Xa
    cm, n1, st = exact(solver, topo, inj, chunk)
    Y = screener.labels(cm, k)
    return X, Y, cm, n1, st


def train(screener: Screener, X, Y, status, T, epochs=4, batch=4096, lr=1e-3, seed=0, log=None, cosine=False):
    """Minibatch Adam over the rows of non-islanded topologies (optionally with a
    cosine-decayed step size); returns the mean loss per epoch."""
    import math

    import torch
    ok = torch.nonzero(status.repeat_interleave(T) == 0).flatten().to(torch.int32)
    g = torch.Generator(device="cuda").manual_seed(seed)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    hist = []
    per_epoch = max(1, ok.numel() // batch)
    total, step = epochs * per_epoch, 0
    for ep in range(epochs):
        perm = ok[torch.randperm(ok.numel(), device="cuda", generator=g)]
        loss.zero_()
        nb = 0
        for a in range(0, perm.numel() - batch + 1, batch):
            lr_t = lr * 0.5 * (1.0 + math.cos(math.pi * step / total)) if cosine else lr
            screener.train_step(X, Y, perm[a:a + batch], lr_t, loss)
            nb += 1
            step += 1
        screener.check()
        hist.append(float(loss.item()) / max(nb, 1))
        if log:
            log(f"epoch {ep}: mean loss {hist[-1]:.5f} over {nb} steps")
    return hist


def recall_at_k(pred, Y, C):
    """sum |pred ∩ true| / sum |true| with pred [rows, k] (−1 padding) and labels Y [rows, C_pad]."""
    import torch
    p = pred.long()
    valid = (p >= 0) & (p < C)
    hit = torch.gather(Y[:, :C].to(torch.int64), 1, torch.where(valid, p, 0)) * valid
    tot = Y[:, :C].sum()
    return float(hit.sum().item()) / max(1, float(tot.item()))


def evaluate(solver: Solver, screener: Screener, topo, inj, Y, cont_max, n1_exact, status, top_k=64,
             fallback_logit=float("inf"), chunk=20000, repeats=3, min_prob=0.0):
    """Screened vs full N-1 on a held-out batch: recall, worst-contingency hits, error, timings
    (repeats = 0: no timings).  min_prob: contingencies predicted above it are evaluated too."""
    import torch
    N, T, C = topo.n_topo, inj.shape[0], solver.n_cont
    W = (C + 31) // 32
    pred = torch.empty((N * T, top_k), dtype=torch.int32, device="cuda")
    evw = torch.empty((N, W), dtype=torch.int32, device="cuda")
    neval = torch.empty(N, dtype=torch.int32, device="cuda")
    fb = torch.empty(N, dtype=torch.uint8, device="cuda")
    n1s = torch.empty((N, T), dtype=torch.float64, device="cuda")
    batches = [(a, min(N, a + chunk)) for a in range(0, N, chunk)]
    dbs = [DeviceBatch(topo.subset(np.arange(a, b)), inj) for a, b in batches]
    ress = [DeviceResults(b - a, T, solver.n_mon, n_cont=C) for a, b in batches]

    def run_screened():
        for (a, b), db, r in zip(batches, dbs, ress):
            _, rep = solver.solve_screened(db, screener, top_k, fallback_logit, results=r, want_pred=True,
                                           min_prob=min_prob, want_evaluated=True)
            pred[a * T:b * T] = rep["pred"][:(b - a) * T * top_k].view(-1, top_k)
            evw[a:b] = rep["evaluated"][:(b - a) * W].view(b - a, W)
            neval[a:b] = rep["n_eval"][:b - a]
            fb[a:b] = rep["fallback"][:b - a]
            n1s[a:b] = r.n1_max_loading[:(b - a) * T].view(b - a, T)

    def run_full():
        for db, r in zip(dbs, ress):
            solver.solve(db, results=r)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(repeats):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3)
        return best

    if repeats > 0:
        t_full = timed(run_full)
        t_scr = timed(run_screened)
    else:
        run_screened()
        t_full = t_scr = float("nan")
    ok = (status == 0).repeat_interleave(T)
    cm = cont_max.view(N * T, C)
    worst = torch.where(cm.max(dim=1).values > 0, cm.argmax(dim=1), torch.full_like(cm[:, 0], -1, dtype=torch.int64))
    # evaluated set per topology, as the solver reports it (the union of its rows' selections)
    bits = (evw.unsqueeze(2) >> torch.arange(32, device="cuda", dtype=torch.int32)) & 1
    ev = bits.view(N, W * 32)[:, :C].bool()
    ev_rows = ev.repeat_interleave(T, dim=0)
    Yc = Y[:, :C].bool()
    okr = ok.view(-1, 1)
    rec64 = recall_at_k(pred[ok], Y[ok], C)
    rec_ev = float((Yc & ev_rows & okr).sum().item()) / max(1, float((Yc & okr).sum().item()))
    wv = worst[ok]
    hit = ev_rows[ok].gather(1, wv.clamp(min=0).view(-1, 1)).flatten() | (wv < 0)
    err = (n1s.flatten()[ok] - n1_exact.flatten()[ok]).abs()
    rel = err / n1_exact.flatten()[ok].abs().clamp(min=1e-12)
    lf_full = int(ok.sum().item()) * C
    return {
        "topologies": N, "timesteps": T, "contingencies": C, "top_k": top_k,
        "recall_at_k": rec64, "recall_evaluated": rec_ev,
        "worst_cont_hit_rate": float(hit.float().mean().item()),
        "n1_max_rel_err_max": float(rel.max().item()) if rel.numel() else 0.0,
        "n1_max_rel_err_mean": float(rel.mean().item()) if rel.numel() else 0.0,
        "evaluated_fraction": float(neval[status == 0].float().mean().item()) / C,
        "fallback_fraction": float(fb[status == 0].float().mean().item()),
        "min_prob": min_prob,
        "full_s": t_full, "screened_s": t_scr, "speedup": t_full / t_scr,
        "full_loadflows_per_s": lf_full / t_full, "screened_equiv_loadflows_per_s": lf_full / t_scr,
    }


def calibrate_min_prob(solver: Solver, screener: Screener, topo, inj, Y, cont_max, n1_exact, status, top_k=64,
                       target=0.99, probs=(0.5, 0.3, 0.2, 0.12, 0.08, 0.05, 0.03, 0.02, 0.01)):
    """The largest probability threshold whose screened solve reaches `target` recall of the
    evaluated set on a calibration batch (held apart from both the training and the held-out
    topologies); returns (threshold, [(threshold, recall, evaluated fraction)])."""
    curve = []
    for p in probs:
        r = evaluate(solver, screener, topo, inj, Y, cont_max, n1_exact, status, top_k, repeats=0, min_prob=p)
        curve.append((p, r["recall_evaluated"], r["evaluated_fraction"]))
        if r["recall_evaluated"] >= target:
            return p, curve
    return probs[-1], curve


def _study():
    from . import synth
    return synth.workload(5, n_topo=16)


def _limits(w):
    base = Solver(w.grid, precision="fp64")
    pt = base.base_ptdf(w.mon).cpu().numpy()
    base.close()
    lim = np.ones(w.grid.n_branch)
    lim[w.mon] = 1.2 * np.abs(w.inj @ pt.T).max(axis=0) + 0.1
    return lim


def profile(a):
    """Timing of a trained screener (loaded from a checkpoint) on held-out topologies."""
    import torch

    from . import synth
    from .csrc import build
    build.build()
    torch.cuda.set_device(0)
    w = _study()
    ev = synth.make_topologies(w.grid, w.subs, a.eval, 605, (1, 8), (0, 0))
    solver = Solver(w.grid, precision="fp32")
    solver.set_study(w.mon, w.cont, _limits(w), split_bus=w.subs)
    scr = Screener(solver, max_rows=a.batch, seed=1)
    scr.load(a.profile)
    db = DeviceBatch(ev, w.inj)
    r = DeviceResults(ev.n_topo, w.inj.shape[0], solver.n_mon, n_cont=solver.n_cont)

    def tm(fn, n=3):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(n):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    t_full = tm(lambda: solver.solve(db, results=r))
    t_scr = tm(lambda: solver.solve_screened(db, scr, a.top_k, a.fallback_logit, results=r))
    rows = 8 * a.batch
    X = torch.zeros(rows, scr.F_pad, dtype=torch.bfloat16, device="cuda")
    X[:, :scr.F] = torch.randn(rows, scr.F, device="cuda").to(torch.bfloat16)
    Y = (torch.rand(rows, scr.C_pad, device="cuda") < 0.06).to(torch.uint8)
    loss = torch.zeros(1, device="cuda")
    perm = torch.randperm(rows, device="cuda").to(torch.int32)

    def steps():
        for i in range(0, rows, a.batch):
            scr.train_step(X, Y, perm[i:i + a.batch], 1e-4, loss)

    t_step = tm(steps, 2) / 8
    print(json.dumps({"topologies": a.eval, "top_k": a.top_k, "full_ms": t_full, "screened_ms": t_scr,
                      "speedup": t_full / t_scr, "train_step_ms": t_step, "train_rows": a.batch}))


def main():
    import torch
    from . import synth
    from .csrc import build

    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--train", type=int, default=200000, help="training topologies")
    ap.add_argument("--eval", type=int, default=100000, help="held-out topologies")
    ap.add_argument("--epochs", type=int, default=6)
    ap.add_argument("--batch", type=int, default=8192)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--top-k", type=int, default=64)
    ap.add_argument("--eval-top-k", default="", help="further k values to evaluate, comma separated")
    ap.add_argument("--cosine", action="store_true", help="cosine-decayed step size")
    ap.add_argument("--fallback-logit", type=float, default=float("inf"))
    ap.add_argument("--save", default=None, help="checkpoint path (.npz)")
    ap.add_argument("--profile", default=None, metavar="CKPT",
                    help="no training: load CKPT and time a full and a screened solve of --eval "
                         "held-out topologies, and 8 training steps of --batch rows")
    a = ap.parse_args()
    if a.profile:
        return profile(a)
    build.build()
    torch.cuda.set_device(0)
    w = synth.workload(5, n_topo=a.train)
    ev_topo = synth.make_topologies(w.grid, w.subs, a.eval, 605, (1, 8), (0, 0))
    lim = _limits(w)
    solver = Solver(w.grid, precision="fp32")
    solver.set_study(w.mon, w.cont, lim, split_bus=w.subs)
    scr = Screener(solver, max_rows=a.batch, seed=1)
    t0 = time.perf_counter()
    Xtr, Ytr, _, _, st_tr = dataset(solver, scr, w.topo, w.inj, a.top_k)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    t0 = time.perf_counter()
    hist = train(scr, Xtr, Ytr, st_tr, w.inj.shape[0], a.epochs, a.batch, a.lr, log=print, cosine=a.cosine)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del Xtr
    Xev, Yev, cm_ev, n1_ev, st_ev = dataset(solver, scr, ev_topo, w.inj, a.top_k)
    del Xev
    rep = evaluate(solver, scr, ev_topo, w.inj, Yev, cm_ev, n1_ev, st_ev, a.top_k, a.fallback_logit)
    for k in [int(x) for x in a.eval_top_k.split(",") if x]:
        r = evaluate(solver, scr, ev_topo, w.inj, Yev, cm_ev, n1_ev, st_ev, k, a.fallback_logit)
        rep[f"top_k_{k}"] = {x: r[x] for x in ("recall_at_k", "recall_evaluated", "worst_cont_hit_rate",
                                               "evaluated_fraction", "speedup", "n1_max_rel_err_mean")}
    rep.update({"train_topologies": a.train, "train_rows": a.train * w.inj.shape[0], "epochs": a.epochs,
                "loss_per_epoch": hist, "data_s": t_data, "train_s": t_train,
                "features": scr.F, "hidden": scr.H})
    if a.save:
        scr.save(a.save)
    print(json.dumps(rep))


if __name__ == "__main__":
    main()
