"""Benchmark: N-1 DC loadflows per second on the 500-bus / 700-branch study.

Workload (synthetic, seeded): 500-bus, 700-branch grid, 50 split-capable
substations, 10,000 topologies with 1-4 bus splits and 0-3 branch outages,
24 timesteps of injections, full N-1 over all 700 branches with every branch
monitored.  One step = one dcflow_solve_batch over the whole batch (N-0 flows,
r x r updates, fused N-1 with max / arg-max / overload reduction), inputs
resident in HBM.  A loadflow is one solved (topology, timestep, contingency)
N-1 case (islanded topologies and islanding or outaged contingencies are not
counted).

The headline form is FP32 (mixed precision: FP64 factor, r x r systems and
N-1 denominators); the plain FP64 form is measured beside it.  Under torchrun
every rank solves its own 10,000-topology batch (weak scaling, no collective
on the data path).  ``--impl reference`` times the CPU oracle on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "N-1 DC loadflows/sec on 1 B300, FP64 plain vs mixed-prec form at stated max err"
WORKLOADS = {
    # name: (shape id, default topologies, description)
    "grid500": (2, 10000, "grid500_splits1-4_outages0-3_T24_fullN1"),
    "grid2000": (3, 1000, "grid2000_splits1-8_outages0-4_T8_cand256_mon3000_cont1000"),
    "grid10000": (4, 50000, "grid10000_splits1-6_T16_mon5000_cont2000"),
}
# dram bytes per launch of the dominant kernel from an ncu capture of the
# 500-bus study (its summary sits under profiles/), keyed by the sha1 of the
# kernel's source and of its argument block at the time of the capture
N1_TRAFFIC = {
    ("c1efdb0101c7", "fp32"): {"bytes": 1.1018e9, "per": "bench step of the 500-bus study",
                               "how": "1,000-topology capture (626 + 374 topologies: 78.67 MB + 31.62 MB of DRAM "
                                      "read + write) scaled by topologies per rank class to 6,233 + 3,767"},
    ("c1efdb0101c7", "bf16x3"): {"bytes": 1.1584e9, "per": "bench step of the 500-bus study",
                                 "how": "1,000-topology capture (626 + 374 topologies: 84.42 MB + 31.55 MB) scaled "
                                        "by topologies per rank class to 6,233 + 3,767"},
}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


def _src_hash():
    h = hashlib.sha1()
    for f in ("n1_reg.cuh", "n1_tma.cuh", "args.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2501_17529_b300", "csrc", f), "rb").read())
    return h.hexdigest()[:12]


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 7:
                self.rows.append(parts)

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[3 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_topologies(w, shape, n_topo, rank):
    """Weak scaling: rank 0 keeps the workload's batch, every other rank draws
    its own batch of the same shape (independent topologies, no exchange)."""
    from paper_2501_17529_b300 import synth
    if rank == 0:
        return w.topo
    spec = {2: ((1, 4), (0, 3)), 3: (synth.geometric_count(0.5, 1, 8), synth.geometric_count(0.5, 0, 4)),
            4: ((1, 6), (0, 0))}[shape]
    return synth.make_topologies(w.grid, w.subs, n_topo, 1000 * rank + 200 + shape, *spec)


def reduce_over_ranks(t_dev, lf, device):
    """Whole-job timing: the slowest rank's device time and the loadflows of all ranks."""
    import torch
    import torch.distributed as dist
    tt = torch.tensor([t_dev], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    lft = torch.tensor([lf], device=device, dtype=torch.float64)
    dist.all_reduce(lft)
    return float(tt.item()), float(lft.item())


def _loadflows(topo, status, n_island_cont, cont, T):
    """N-1 cases solved: valid contingencies of non-islanded topologies x T."""
    cset = set(int(c) for c in cont)
    n = 0
    for i in range(topo.n_topo):
        if status[i] != 0:
            continue
        a, b = topo.out_ptr[i], topo.out_ptr[i + 1]
        n_out_cont = sum(1 for c in topo.out_branch[a:b] if int(c) in cset)
        n += len(cont) - n_out_cont - int(n_island_cont[i])
    return n * T


def _cpu_worker(args):
    shape, idx = args
    import oracle
    from paper_2501_17529_b300 import synth
    w = synth.workload(shape, n_topo=max(idx) + 1)
    lim = oracle.thermal_limits(w.grid, w.inj)
    t0 = time.perf_counter()
    r = oracle.evaluate(w.grid, w.topo, w.inj, w.mon, w.cont, lim, var=w.var, idx=idx, want_cmax=w.var is None)
    dt = time.perf_counter() - t0
    nv = 0 if w.var is None else w.var.n_var
    keep = {k: r[k] for k in ("n0_max", "n1_max", "ovl", "worst_cont", "status", "n_island_cont")}
    keep["idx"] = np.asarray(idx, np.int64)
    if w.var is None:
        # the worst contingency under each form's tie band (the lowest position within
        # band * max(best, 1) of the largest per-contingency maximum), as the CUDA path reports it
        for name, eps in (("band_1e-4", 1e-4), ("band_1e-10", 1e-10)):
            wc = -np.ones_like(r["worst_cont"])
            for i in range(wc.shape[0]):
                for t in range(wc.shape[1]):
                    if r["status"][i] == 0 and (r["cmax"][i, t] >= 0).any():
                        wc[i, t] = oracle.first_in_band(r["cmax"][i, t], eps)
            keep["worst_cont_" + name] = wc
    return oracle.loadflow_count(r, w.inj.shape[0], nv), dt, keep


def cpu_baseline(workload: str, budget_s: float = 20.0):
    """The oracle as it stands on the host cores, on a bounded topology sample."""
    shape, n_all, _ = WORKLOADS[workload]
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    # probe the per-topology cost, then size the sample to the budget
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        probe = pool.map(_cpu_worker, [(shape, [i]) for i in range(cores)])
        per_topo = max(1e-3, statistics.median(dt for _, dt, _ in probe))
        n_each = max(1, int(budget_s / per_topo))
        n_each = min(n_each, max(1, (n_all - cores) // cores))
        chunks = [(shape, list(range(cores + k * n_each, cores + (k + 1) * n_each))) for k in range(cores)]
        t0 = time.perf_counter()
        res = pool.map(_cpu_worker, chunks)
        wall = time.perf_counter() - t0
    lf = sum(r[0] for r in res)
    ntop = n_each * cores
    ref = {k: np.concatenate([r[2][k] for r in probe + res]) for k in probe[0][2]}
    return {"value": lf / wall, "unit": "loadflows/s", "cores": cores, "kind": "oracle",
            "sample": f"{ntop} of the {n_all} topologies of {workload} (all timesteps, candidates and contingencies), "
                      f"{cores} spawn workers, 1 BLAS thread each, {wall:.1f} s wall"}, ref


def _errors(host, ref, form=None):
    """Errors of one form against the oracle on the oracle's topology sample
    (loadings |x - x_ref| / max(x_ref, 1), overload sums likewise; integer
    outputs as the fraction that agrees exactly; the worst contingency against
    the oracle's under the form's tie band when the sample has it)."""
    idx = ref["idx"]
    st = host["status"][idx]
    ok = ref["status"] == 0
    out = {"topologies": int(idx.size), "status_agree": float(np.mean(st == ref["status"])),
           "n_island_cont_agree": float(np.mean(host["n_island_cont"][idx][ok] == ref["n_island_cont"][ok]))
           if ok.any() else 1.0}
    for key, name in (("n0_max", "n0_max_loading"), ("n1_max", "n1_max_loading"), ("ovl", "overload_sum")):
        g, r = host[key][idx][ok], ref[key][ok]
        out[f"max_err_{name}"] = float((np.abs(g - r) / np.maximum(np.abs(r), 1.0)).max()) if ok.any() else 0.0
    key = {"fp64": "worst_cont_band_1e-10", "fp32": "worst_cont_band_1e-4", "bf16x3": "worst_cont_band_1e-4"}.get(form)
    wref = ref[key] if key in ref else ref["worst_cont"]
    out["worst_cont_agree"] = float(np.mean(host["worst_cont"][idx][ok] == wref[ok])) if ok.any() else 1.0
    if key in ref:
        out["worst_cont_rule"] = "lowest position within " + key.split("_")[-1] + " x max(best, 1) of the best"
    return out


def _config(w, desc, n_topo, T, l2):
    """The workload keys of both arms' JSON lines."""
    return {"workload": desc, "topologies": n_topo, "timesteps": T, "monitored": len(w.mon),
            "contingencies": len(w.cont), "candidates": 0 if w.var is None else w.var.n_var,
            "branches": int(w.grid.n_branch), "l2": l2, "max_err_stated": {"fp32": 1e-4, "fp64": 1e-10}}


def _ref_worker(args):
    shape, n_topo, idx = args
    import oracle
    from paper_2501_17529_b300 import synth
    w = synth.workload(shape, n_topo=n_topo)
    lim = oracle.thermal_limits(w.grid, w.inj)
    t0 = time.perf_counter()
    r = oracle.evaluate(w.grid, w.topo, w.inj, w.mon, w.cont, lim, var=w.var, idx=idx)
    nv = 0 if w.var is None else w.var.n_var
    return oracle.loadflow_count(r, w.inj.shape[0], nv), time.perf_counter() - t0


def run_reference(args):
    """The oracle as it stands, on the host cores (one spawn worker per core, one BLAS thread
    each): every step evaluates a bounded sample of the workload's topologies (disjoint
    between steps), sized so that a step takes a few seconds."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import multiprocessing as mp
    from paper_2501_17529_b300 import synth
    shape, n_all, desc = WORKLOADS[args.workload]
    n_topo = args.topologies or n_all
    cores = os.cpu_count() or 1
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    w = synth.workload(shape, n_topo=1)
    ctx = mp.get_context("spawn")
    times, lfs = [], []
    with ctx.Pool(cores) as pool:
        probe = pool.map(_ref_worker, [(shape, n_topo, [i]) for i in range(cores)])
        per_topo = max(1e-3, statistics.median(dt for _, dt in probe))
        per_core = max(1, int(float(os.environ.get("DCFLOW_REF_STEP_S", "4")) / per_topo))
        per_core = min(per_core, max(1, (n_topo - cores) // (cores * (args.warmup + args.steps))))
        nxt = cores
        for s2 in range(args.warmup + args.steps):
            chunks = []
            for _ in range(cores):
                chunks.append((shape, n_topo, [i % n_topo for i in range(nxt, nxt + per_core)]))
                nxt += per_core
            t0 = time.perf_counter()
            res = pool.map(_ref_worker, chunks)
            dt = time.perf_counter() - t0
            if s2 >= args.warmup:
                times.append(dt)
                lfs.append(sum(r[0] for r in res))
    value = sum(lfs) / sum(times)
    sample = (f"{per_core * cores} of the {n_topo} topologies per step ({per_core} per core; all timesteps, "
              f"candidates and contingencies), {cores} spawn workers, 1 BLAS thread each")
    cfg = _config(w, desc, n_topo, w.inj.shape[0], "n/a (host)")
    cfg["topologies_per_step"] = per_core * cores
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "loadflows/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": cfg,
            "cpu_baseline": {"value": value, "unit": "loadflows/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "loadflows/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import torch.distributed as dist

    ws, rank, local = _dist()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    from paper_2501_17529_b300 import synth
    from paper_2501_17529_b300.csrc import build as cbuild
    from paper_2501_17529_b300.dcflow import DeviceBatch, DeviceResults, Solver

    if rank == 0 or ws == 1:
        cbuild.build()
    if ws > 1:
        dist.barrier()
    shape, n_default, desc = WORKLOADS[args.workload]
    n_topo = args.topologies or n_default
    w = synth.workload(shape, n_topo=n_topo)
    w.topo = rank_topologies(w, shape, n_topo, rank)
    # limits from the unsplit grid's N-0 flows on the monitored branches, computed on the device
    base = Solver(w.grid, precision="fp64")
    pt = base.base_ptdf(w.mon).cpu().numpy()
    base.close()
    lim = np.ones(w.grid.n_branch)
    lim[w.mon] = 1.2 * np.abs(w.inj @ pt.T).max(axis=0) + 0.1
    n_mon = len(w.mon)
    T_STEPS = w.inj.shape[0]
    # PTDF row restriction (Sec. II): the study needs the rows of the monitored, contingency, split-bus
    # and outaged branches only; "full" keeps every branch row
    ocand = np.unique(np.asarray(w.topo.out_branch, np.int32)) if args.rows == "restricted" else None
    need = np.zeros(w.grid.n_branch, bool)
    need[w.mon] = need[w.cont] = True
    for v in w.subs:
        need[(w.grid.f == v) | (w.grid.t == v)] = True
    if ocand is None:
        need[:] = True
    else:
        need[ocand] = True

    results, hosts = {}, {}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > 126 MB L2
    peaks, peak_kind = _peaks()
    alu_peak = 148 * 128 * peaks.get("sm_max_mhz", 2032.0) * 1e6 / 1e12  # T issue slots/s, as the N-1 roofline
    fp64_peak = 148 * 2 * peaks.get("sm_max_mhz", 2032.0) * 1e6 / 1e12  # T DFMA lanes/s
    lib = __import__("paper_2501_17529_b300.dcflow", fromlist=["x"])

    def timed(solver, dbx, resx, steps, stream):
        """Warm-up, then `steps` timed solves (L2 flushed before each) with the kernel profile on:
        (seconds over the steps, max over ranks; per-kind kernel milliseconds per step)."""
        for _ in range(args.warmup):
            solver.solve(dbx, results=resx)
        torch.cuda.synchronize()
        evx = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        lib.dcflow_profile(solver.ctx, True)
        for k2 in range(steps):
            flush.fill_(k2 & 0xFF)
            evx[k2][0].record(stream)
            solver.solve(dbx, results=resx)
            evx[k2][1].record(stream)
        torch.cuda.synchronize()
        kp = lib.dcflow_profile_read(solver.ctx)
        lib.dcflow_profile(solver.ctx, False)
        tx = sum(a.elapsed_time(b) for a, b in evx) / 1e3
        if ws > 1:
            tx, _ = reduce_over_ranks(tx, 0, "cuda")
        return tx, {k: v / steps for k, v in kp.items() if k.endswith("_ms")}

    for form in (args.forms.split(",")):
        torch.cuda.synchronize()
        ts = time.perf_counter()
        solver = Solver(w.grid, precision=form, compact_n1=args.compact, chunk_topo=args.chunk)
        solver.set_study(w.mon, w.cont, lim, split_bus=w.subs, outage_cand=ocand)
        torch.cuda.synchronize()
        setup_s = time.perf_counter() - ts
        db = DeviceBatch(w.topo, w.inj, w.var)
        res = DeviceResults(db.n_topo, db.n_time, len(w.mon), want_var=db.n_var > 0)
        stream = torch.cuda.current_stream()
        steps = args.steps if form != "fp64" or args.fp64_steps <= 0 else max(1, min(args.steps, args.fp64_steps))
        for _ in range(args.warmup):
            solver.solve(db, results=res)
        torch.cuda.synchronize()
        host = res.to_host()
        hosts[form] = host
        lf = _loadflows(w.topo, host["status"], host["n_island_cont"], w.cont, T_STEPS) * max(1, db.n_var)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        launches = 0
        lib.dcflow_profile(solver.ctx, True)
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        with ClockSampler(dev) as clk:
            wall0 = time.perf_counter()
            for k in range(steps):
                flush.fill_(k & 0xFF)
                ev[k][0].record(stream)
                solver.solve(db, results=res)
                ev[k][1].record(stream)
                launches += solver.last_launch_count()
            torch.cuda.synchronize()
            wall = time.perf_counter() - wall0
        ms = [a.elapsed_time(b) for a, b in ev]
        t_dev = sum(ms) / 1e3
        kern = lib.dcflow_profile_read(solver.ctx)
        kern = {"n1_ms": kern["n1_ms"], "n1_launches": kern["n1_launches"]}
        lib.dcflow_profile(solver.ctx, False)
        if ws > 1:
            t_dev, lf_all = reduce_over_ranks(t_dev, lf, "cuda")
        else:
            lf_all = lf
        results[form] = {"value": lf_all * steps / t_dev, "ms_per_step": 1e3 * t_dev / steps,
                         "loadflows_per_step": lf_all, "steps": steps, "launches": launches,
                         "clocks": clk.summary(), "wall_s": wall, "kernel": kern, "lf_rank": lf,
                         "n1_ms_per_step": kern["n1_ms"] / steps if kern["n1_ms"] else None}
        # end to end through host buffers: H2D of the batch, solve, D2H of the results
        if form == "fp32" and not args.no_e2e:
            results[form]["e2e"] = _e2e(solver, w, lim, steps, args.warmup, lf)
        # the same solve with the sparse worst results (agg_i, top k per topology and timestep)
        if form == "fp32" and args.top_k > 0:
            rk = DeviceResults(db.n_topo, db.n_time, len(w.mon), want_var=db.n_var > 0, top_k=args.top_k)
            tk, kk = timed(solver, db, rk, steps, stream)
            nok = int((rk.island_flag[:db.n_topo] == 0).sum().item())
            rec = nok * T_STEPS * args.top_k * n_mon  # entries of the cases' recomputed columns
            results[f"fp32_top{args.top_k}"] = {"value": lf_all * steps / tk, "ms_per_step": 1e3 * tk / steps,
                                                "loadflows_per_step": lf_all, "steps": steps,
                                                "kernels": {"name": "k_topcases_tile", "ms_per_step": kk["topcases_ms"],
                                                           "column_entries_per_s_T": rec / (kk["topcases_ms"] / 1e3) / 1e12
                                                           if kk["topcases_ms"] else None},
                                                "note": f"fp32 solve plus the {args.top_k} worst N-1 cases "
                                                        "(contingency, monitored branch, loading) per topology "
                                                        "and timestep"}
        # the same solve with generator-failure N-1 cases (16 generators at seeded buses)
        if form == "fp32" and args.gens > 0:
            rng = np.random.default_rng(700)
            gb = np.sort(rng.choice(np.arange(1, w.grid.n_bus), args.gens, replace=False)).astype(np.int32)
            gp = np.abs(rng.normal(1.0, 0.5, (T_STEPS, args.gens)))
            dbg = DeviceBatch(w.topo, w.inj, w.var, gen_bus=gb, gen_p=gp)
            rg = DeviceResults(db.n_topo, db.n_time, len(w.mon), want_var=db.n_var > 0, want_gen=True)
            tg, kg = timed(solver, dbg, rg, steps, stream)
            ngen_cases = int((rg.island_flag[:db.n_topo] == 0).sum().item()) * T_STEPS * args.gens * ws
            gen_rate = ngen_cases / ws * n_mon / (kg["gen_ms"] / 1e3) / 1e12 if kg["gen_ms"] else None
            results[f"fp32_gen{args.gens}"] = {"value": lf_all * steps / tg, "ms_per_step": 1e3 * tg / steps,
                                               "loadflows_per_step": lf_all,
                                               "generator_cases_per_step": ngen_cases, "steps": steps,
                                               "kernels": {"name": "k_gen_tma", "ms_per_step": kg["gen_ms"],
                                                          "entries_per_s_T": gen_rate, "alu_peak_T": alu_peak,
                                                          "frac": gen_rate / alu_peak if gen_rate else None},
                                               "note": f"fp32 solve plus {args.gens} generator-failure N-1 cases "
                                                       "per topology and timestep (value counts the branch "
                                                       "N-1 cases only)"}
        # injection topologies t_i (Sec. III-A): |T_i| busbar assignments of the injections at the split
        # substations per topology, brute-forced for the lowest agg_m (on a subset of the topologies)
        if form == "fp32" and args.ti > 0 and db.n_var == 0:
            nsub = min(args.ti_topologies, w.topo.n_topo)
            tsub = w.topo.subset(np.arange(nsub))
            tis = synth.make_injection_topologies(w.grid, w.subs, tsub, w.inj, args.ti, 900)
            dbt = DeviceBatch(tsub, w.inj, ti=tis)
            rt = DeviceResults(nsub, db.n_time, len(w.mon), want_var=True)
            tt, kt = timed(solver, dbt, rt, steps, stream)
            st_h = rt.island_flag[:nsub].cpu().numpy()
            ni_h = rt.n_island_cont[:nsub].cpu().numpy()
            lft = _loadflows(tsub, st_h, ni_h, w.cont, T_STEPS) * args.ti
            # the expansion writes every (timestep, assignment)'s N-0 row and N-1 weights
            exp_bytes = int((st_h == 0).sum()) * T_STEPS * args.ti * (((n_mon + 15) // 16 * 16) + len(w.cont)) * 4
            exp_gbs = exp_bytes / (kt["expand_ms"] / 1e3) / 1e9 if kt["expand_ms"] else None
            if ws > 1:
                _, lft = reduce_over_ranks(0.0, lft, "cuda")
            results[f"fp32_ti{args.ti}"] = {
                "value": lft * steps / tt, "ms_per_step": 1e3 * tt / steps, "loadflows_per_step": lft,
                "topologies": nsub, "steps": steps,
                "kernels": {"name": "k_ti_expand", "ms_per_step": kt["expand_ms"], "written_gbs": exp_gbs,
                           "hbm_peak_gbs": peaks.get("hbm_gbs"), "frac": exp_gbs / peaks["hbm_gbs"] if exp_gbs else None,
                           "screening_n1_ms_per_step": kt["n1_ms"]},
                "note": f"injection topologies: {args.ti} busbar assignments of the injections at the split "
                        f"substations per topology ({nsub} topologies x {T_STEPS} timesteps), metric-first "
                        "brute force; loadflows count every (topology, timestep, assignment, contingency)"}
            # the same with the top-k cases (agg_i): metric-first (the chosen assignment's cases only)
            # against output-first (every assignment's cases inside the loop, the chosen one's kept)
            if args.top_k > 0:
                modes = {}
                for of in (False, True):
                    so = solver if not of else Solver(w.grid, precision=form, output_first=True)
                    if of:
                        so.set_study(w.mon, w.cont, lim, split_bus=w.subs, outage_cand=ocand)
                    rk2 = DeviceResults(nsub, db.n_time, len(w.mon), want_var=True, top_k=args.top_k)
                    tk2, kk2 = timed(so, dbt, rk2, steps, stream)
                    modes["output_first" if of else "metric_first"] = {
                        "value": lft * steps / tk2, "ms_per_step": 1e3 * tk2 / steps,
                        "topcases_ms_per_step": kk2["topcases_ms"]}
                    if of:
                        so.close()
                results[f"fp32_ti{args.ti}_top{args.top_k}"] = dict(
                    modes, output_first_over_metric_first=modes["output_first"]["ms_per_step"]
                    / modes["metric_first"]["ms_per_step"],
                    note=f"the injection-topology form with the {args.top_k} worst N-1 cases per (topology, "
                         "timestep): metric-first computes them for the chosen assignment only, output-first "
                         "for every assignment inside the brute-force loop (the modes of Sec. III-A); both "
                         "report the same outputs")
            # |T_i| sweep (the paper's injection-ratio figure): loadflows/s against the number of
            # injection topologies per branch topology, both modes, with the top-k cases
            if args.ti_sweep and args.top_k > 0:
                sweep = {}
                so_of = Solver(w.grid, precision=form, output_first=True)
                so_of.set_study(w.mon, w.cont, lim, split_bus=w.subs, outage_cand=ocand)
                for U_ in (int(x) for x in args.ti_sweep.split(",")):
                    tis_ = synth.make_injection_topologies(w.grid, w.subs, tsub, w.inj, U_, 900)
                    dbs = DeviceBatch(tsub, w.inj, ti=tis_)
                    row = {}
                    for of, so in ((False, solver), (True, so_of)):
                        rks = DeviceResults(nsub, db.n_time, len(w.mon), want_var=True, top_k=args.top_k)
                        tks, _ = timed(so, dbs, rks, steps, stream)
                        st_s = rks.island_flag[:nsub].cpu().numpy()
                        ni_s = rks.n_island_cont[:nsub].cpu().numpy()
                        lfs = _loadflows(tsub, st_s, ni_s, w.cont, T_STEPS) * U_
                        row["output_first" if of else "metric_first"] = {
                            "loadflows_per_s": lfs * steps / tks, "ms_per_step": 1e3 * tks / steps}
                    sweep[str(U_)] = row
                so_of.close()
                results[f"fp32_ti_sweep_top{args.top_k}"] = {
                    "by_ti": sweep, "topologies": nsub,
                    "note": "loadflows/s (every topology, timestep, assignment and contingency) against |T_i|, "
                            "the busbar assignments per branch topology, in both injection-module modes"}
        # the same solve with multi-outage N-1 cases (sets of 2-4 branches that fail together)
        if form == "fp32" and args.multi > 0 and db.n_var == 0:
            rng = np.random.default_rng(800)
            E = w.grid.n_branch
            sets = [[int(b) for b in rng.choice(E, 2 + k % 3, replace=False)] for k in range(args.multi)]
            solver.set_study(w.mon, w.cont, lim, split_bus=w.subs, outage_cand=ocand, multi=sets)
            rm = DeviceResults(db.n_topo, db.n_time, len(w.mon), want_multi=True)
            tm, km = timed(solver, db, rm, steps, stream)
            okm = rm.island_flag[:db.n_topo] == 0
            nm_cases = (int(okm.sum().item()) * args.multi - int(rm.n_island_multi[:db.n_topo][okm].sum().item())) \
                * T_STEPS * ws
            results[f"fp32_multi{args.multi}"] = {
                "value": lf_all * steps / tm, "ms_per_step": 1e3 * tm / steps, "loadflows_per_step": lf_all,
                "multi_cases_per_step": nm_cases, "steps": steps,
                "kernels": {"name": "k_multi_tma", "ms_per_step": km["multi_ms"],
                           "entries_per_s_T": nm_cases / ws * n_mon / (km["multi_ms"] / 1e3) / 1e12 if km["multi_ms"] else None,
                           "alu_peak_T": alu_peak,
                           "frac": (nm_cases / ws * n_mon / (km["multi_ms"] / 1e3) / 1e12 / alu_peak) if km["multi_ms"] else None,
                           "prep_ms_per_step": km["multi_prep_ms"]},
                "note": f"fp32 solve plus {args.multi} multi-outage N-1 sets of 2-4 branches per topology and "
                        "timestep (value counts the single-branch N-1 cases only; multi_cases_per_step counts "
                        "the sets evaluated, sets a topology already lost counted too)"}
        results[form]["setup_s"] = setup_s
        if form == "fp64" and kern["n1_ms"]:
            # the FP64 N-1's floor: one DFMA per entry on the FP64 pipe, 2 lanes per clock per SM
            # (ncu: sm__sass_thread_inst_executed_op_dfma_pred_on peak_sustained = 2 per SM)
            e64 = lf * n_mon * steps / (kern["n1_ms"] / 1e3) / 1e12  # this rank's entries over its kernel time
            results[form]["kernels"] = {"name": "k_n1<double>", "ms_per_step": kern["n1_ms"] / steps,
                                        "entries_per_s_T": e64, "fp64_peak_T": fp64_peak, "frac": e64 / fp64_peak}
        solver.close()
    configs = {}
    run_cfgs = [c for c in args.configs.split(",") if c and c != "none"] if ws == 1 and args.workload == "grid500" \
        else []
    if run_cfgs:
        import multiprocessing as mp
        pool = None
        if not args.no_cpu:
            for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
                os.environ[k] = "1"
            pool = mp.get_context("spawn").Pool(os.cpu_count() or 1)
        if "grid10000" in run_cfgs:  # its oracle jobs start first (the longest; no GPU result needed)
            configs["grid10000"] = run_cfg_grid10000(args, flush, peaks, pool)
        if "cand" in run_cfgs:
            configs["grid2000_cand256"] = run_cfg_candidates(args, flush, peaks, pool)
        if "screen" in run_cfgs:
            configs["grid2000_screen"] = run_cfg_screener(args, peaks)
        if "grid10000" in configs and "_oracle" in configs["grid10000"]:
            configs["grid10000"]["error_vs_oracle"] = _grid10000_errors(configs["grid10000"])
        if "grid2000_cand256" in configs and "_oracle" in configs["grid2000_cand256"]:
            configs["grid2000_cand256"]["error_vs_oracle"] = _cand_errors(configs["grid2000_cand256"])
        if pool is not None:
            pool.close()
            pool.join()
    if rank != 0:
        if ws > 1:
            dist.barrier()
            dist.destroy_process_group()
        return
    head = results.get("fp32") or next(iter(results.values()))
    roof = None
    if "fp32" not in results and "fp64" in results and results["fp64"].get("kernels"):
        k = results["fp64"]["kernels"]
        roof = {"bound": "alu", "achieved": k["entries_per_s_T"], "peak": fp64_peak, "unit": "T N-1 entries/s",
                "frac": k["frac"], "traffic": None, "traffic_note": "no capture for this kernel source and workload",
                "kernel": "k_n1<double> (FP64 fused N-1)",
                "peak_note": f"1 DFMA per entry at the {peak_kind} max SM clock "
                             f"({peaks.get('sm_max_mhz', 2032.0):.0f} MHz), 148 SMs x 2 FP64 lanes",
                "n1_ms_per_step": k["ms_per_step"],
                "n1_share_of_step": k["ms_per_step"] / head["ms_per_step"]}
    elif head.get("kernel"):
        k = head["kernel"]
        # Algorithmic work of the dominant kernel: one N-1 entry per solved
        # (topology, timestep, contingency) case and monitored branch.  Its
        # floor on the CUDA cores is one FP32 issue slot per entry (half a
        # packed FFMA2 for the flow, half a 3-input |max| for the reduction), so
        # the peak is 148 SMs x 128 lanes x the maximum SM clock.
        entries = head["lf_rank"] * n_mon * head["steps"]  # rank 0's entries over rank 0's kernel time
        peak = 148 * 128 * peaks.get("sm_max_mhz", 2032.0) * 1e6 / 1e12
        ach = entries / (k["n1_ms"] / 1e3) / 1e12
        key = (_src_hash(), "fp32" if not args.compact else "fp32_compact")
        roof = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "T N-1 entries/s", "frac": ach / peak,
                "traffic": (N1_TRAFFIC[key]["bytes"] if key in N1_TRAFFIC and args.workload == "grid500"
                            and n_topo == 10000 else None),
                "traffic_note": (N1_TRAFFIC[key] if key in N1_TRAFFIC and args.workload == "grid500"
                                 and n_topo == 10000 else "no capture for this kernel source and workload"),
                "kernel": "k_n1_reg (FP32 fused N-1, " + ("each topology's valid contingencies)" if args.compact
                                                           else "every contingency column)"),
                "peak_note": f"1 FP32 issue slot per entry at the {peak_kind} max SM clock "
                             f"({peaks.get('sm_max_mhz', 2032.0):.0f} MHz), 148 SMs x 128 lanes",
                "n1_ms_per_step": k["n1_ms"] / head["steps"],
                "n1_share_of_step": k["n1_ms"] / (head["ms_per_step"] * head["steps"]),
                # the same rate against the 5 FP32-pipe operations per entry of the method's
                # per-entry accounting (flow FFMA, |.|, max, and the overload max + add)
                "frac_at_5_ops_per_entry": ach * 5 / peak}
    line = {"metric": METRIC,
            "value": head["value"], "unit": "loadflows/s", "n_gpus": ws, "steps": head["steps"],
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(_config(w, desc, n_topo, T_STEPS, "flushed between steps (256 MB write)"),
                           ptdf_rows=int(need.sum())),
            "gpu_launches": head["launches"], "clocks": head["clocks"],
            "forms": {f: {k: v for k, v in r.items() if k not in ("clocks", "kernel", "lf_rank")} for f, r in results.items()}}
    if "fp64" in results and "fp32" in results:
        line["forms"]["fp32_over_fp64_speedup"] = results["fp32"]["value"] / results["fp64"]["value"]
    if "e2e" in head:
        line["e2e"] = head["e2e"]
    if roof:
        line["roofline"] = roof
    if configs:
        line["configs"] = configs
    if ws == 1 and not args.no_cpu:
        line["cpu_baseline"], ref = cpu_baseline(args.workload, args.cpu_budget)
        if n_topo == WORKLOADS[args.workload][1]:  # the oracle's sample is of this very batch
            line["error_vs_oracle"] = {f: _errors(h, ref, f) for f, h in hosts.items()}
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# the other study shapes, one entry each under "configs" of the JSON line:
# 2000-bus with 256 injection candidates (uneven k, autotuned schedule),
# 10000-bus in the FP32 and BF16x3 forms, and the learned screener
# ---------------------------------------------------------------------------

def _device_limits(w):
    """Limits 1.2 max_t |base flow| + 0.1 on the monitored branches, base PTDF rows on the device."""
    from paper_2501_17529_b300.dcflow import Solver
    base = Solver(w.grid, precision="fp64")
    pt = base.base_ptdf(w.mon).cpu().numpy()
    base.close()
    lim = np.ones(w.grid.n_branch)
    lim[w.mon] = 1.2 * np.abs(w.inj @ pt.T).max(axis=0) + 0.1
    return lim


def _cand_rows(w):
    """[U, V] injection change of every candidate."""
    var, U = w.var, w.var.n_var
    D = np.zeros((U, w.grid.n_bus))
    for u in range(U):
        for k in range(var.var_ptr[u], var.var_ptr[u + 1]):
            D[u, var.var_bus[k]] += var.var_delta[k]
    return D


def _cand_oracle_worker(job):
    """Oracle rows of the 2000-bus candidate study for topologies idx: per timestep the
    GPU's chosen candidate first, then `others` (a sample of the rest), each as its own
    timestep of a plain refactorising evaluation."""
    idx, picks, others = job
    import oracle
    from paper_2501_17529_b300 import synth
    w = synth.workload(3, n_topo=max(idx) + 1)
    lim = oracle.thermal_limits(w.grid, w.inj)
    D = _cand_rows(w)
    T = w.inj.shape[0]
    out = []
    for j, i in enumerate(idx):
        rows = []
        for t in range(T):
            rows.append(w.inj[t] + (D[picks[j][t]] if picks[j][t] >= 0 else 0.0))
            rows.extend(w.inj[t] + D[u] for u in others[j][t])
        r = oracle.evaluate(w.grid, w.topo.subset([i]), np.array(rows), w.mon, w.cont, lim, tie_eps=1e-4)
        out.append({k: r[k][0] for k in ("status", "n_island_cont", "n0_max", "n1_max", "ovl", "worst_cont")})
    return out


def _timed_solve(solver, db, res, steps, flush, stream):
    """`steps` solves (L2 flushed before each) by CUDA events with the kernel timers on:
    (seconds, N-1 kernel ms per step, launches per step, clocks)."""
    import torch
    lib = __import__("paper_2501_17529_b300.dcflow", fromlist=["x"])
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    lib.dcflow_profile(solver.ctx, True)
    launches = 0
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clk:
        for k in range(steps):
            flush.fill_(k & 0xFF)
            ev[k][0].record(stream)
            solver.solve(db, results=res)
            ev[k][1].record(stream)
            launches += solver.last_launch_count()
        torch.cuda.synchronize()
    kp = lib.dcflow_profile_read(solver.ctx)
    lib.dcflow_profile(solver.ctx, False)
    t = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    return t, kp["n1_ms"] / steps, launches // steps, clk.summary()


def run_cfg_candidates(args, flush, peaks, pool):
    """2000 buses / 3000 branches, 100,000 topologies of uneven k (1-8 splits + 0-4 outages,
    geometric), 8 timesteps x 256 injection candidates, N-1 over 1000 contingencies, every
    branch monitored; schedule picked by the autotuner on a 512-topology prefix."""
    import torch
    from paper_2501_17529_b300 import synth
    from paper_2501_17529_b300.dcflow import DeviceBatch, DeviceResults, Solver
    n = args.cand_topologies
    w = synth.workload(3, n_topo=n)
    lim = _device_limits(w)
    T, U, M = w.inj.shape[0], w.var.n_var, len(w.mon)
    ocand = np.unique(np.asarray(w.topo.out_branch, np.int32))
    ts = time.perf_counter()
    s = Solver(w.grid, precision=args.cand_form)
    s.set_study(w.mon, w.cont, lim, split_bus=w.subs, outage_cand=ocand)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - ts
    ns = min(512, n)
    sdb = DeviceBatch(w.topo.subset(np.arange(ns)), w.inj, w.var)
    sres = DeviceResults(ns, T, M, want_var=True)
    t0 = time.perf_counter()
    pick, tried = s.autotune(sdb, sres)
    tune_s = time.perf_counter() - t0
    db = DeviceBatch(w.topo, w.inj, w.var)
    res = DeviceResults(n, T, M, want_var=True)
    s.solve(sdb, results=sres)  # warm-up on the prefix (the full batch allocates in its first chunk)
    torch.cuda.synchronize()
    t, n1_ms, launches, clk = _timed_solve(s, db, res, args.cand_steps, flush, torch.cuda.current_stream())
    host = res.to_host()
    lf = _loadflows(w.topo, host["status"], host["n_island_cont"], w.cont, T) * U
    alu_peak = 148 * 128 * peaks.get("sm_max_mhz", 2032.0) * 1e6 / 1e12
    # N-1 entries: the screening pass evaluates every (timestep, candidate, contingency, monitored
    # branch) once; the full pass of the chosen candidate adds 1/U of that
    ach = lf * M * (1.0 + 1.0 / U) / (n1_ms / 1e3) / 1e12
    entry = {"workload": "grid2000_splits1-8geo_outages0-4geo_T8_cand256_mon3000_cont1000", "form": args.cand_form,
             "topologies": n, "timesteps": T, "candidates": U, "monitored": M, "contingencies": len(w.cont),
             "value": lf * args.cand_steps / t, "unit": "loadflows/s", "ms_per_step": 1e3 * t / args.cand_steps,
             "steps": args.cand_steps, "loadflows_per_step": lf, "launches_per_step": launches, "clocks": clk,
             "setup_s": setup_s, "schedule": pick, "schedules_tried": tried, "tune_s": tune_s,
             "roofline": {"bound": "alu", "kernel": "k_n1_reg (screening pass over every (timestep, candidate), "
                                                  "then the full pass of the chosen one)",
                          "achieved": ach, "peak": alu_peak, "unit": "T N-1 entries/s", "frac": ach / alu_peak,
                          "n1_ms_per_step": n1_ms, "n1_share_of_step": n1_ms / (1e3 * t / args.cand_steps)},
             "l2": "flushed before each step (256 MB write); the step's operands exceed L2"}
    job = None
    if pool is not None and args.cand_oracle > 0:
        # oracle sample: the first topologies; per timestep the GPU's pick plus 8 random other candidates
        k = min(args.cand_oracle, n)
        rng = np.random.default_rng(12)
        picks = host["best_var"][:k].astype(np.int64)
        others = [[rng.choice(np.setdiff1d(np.arange(U), [picks[i][t]]), 8, replace=False).tolist()
                   for t in range(T)] for i in range(k)]
        chunks = [list(range(i, k, 16)) for i in range(min(16, k))]
        job = pool.map_async(_cand_oracle_worker, [(c, [picks[i] for i in c], [others[i] for i in c])
                                                   for c in chunks if c])
        entry["_oracle"] = (job, chunks, {kk: host[kk][:k] for kk in ("status", "n_island_cont", "n0_max", "n1_max",
                                                                       "ovl", "worst_cont", "best_var")})
    s.close()
    return entry


def _cand_errors(entry, tol=1e-4):
    job, chunks, g = entry.pop("_oracle")
    rows = {}
    for c, out in zip([c for c in chunks if c], job.get()):
        for i, o in zip(c, out):
            rows[i] = o
    idx = sorted(rows)
    T = g["n1_max"].shape[1]
    K = 1 + 8
    st = np.array([rows[i]["status"] for i in idx])
    ok = st == 0
    e = {"topologies": len(idx), "status_agree": float(np.mean(st == g["status"][idx]))}
    errs_n1, errs_ovl, errs_n0, pick_ok, wc = [], [], [], [], []
    for j, i in enumerate(idx):
        if not ok[j]:
            continue
        r = rows[i]
        for t in range(T):
            ref_n1 = r["n1_max"][t * K]
            errs_n1.append(abs(g["n1_max"][i, t] - ref_n1) / max(ref_n1, 1.0))
            errs_ovl.append(abs(g["ovl"][i, t] - r["ovl"][t * K]) / max(r["ovl"][t * K], 1.0))
            errs_n0.append(abs(g["n0_max"][i, t] - r["n0_max"][t * K]) / max(r["n0_max"][t * K], 1.0))
            others = r["n1_max"][t * K + 1:(t + 1) * K]
            pick_ok.append(bool(ref_n1 <= others.min() + 2 * tol * max(1.0, others.min())))
            wc.append(int(g["worst_cont"][i, t]) == int(r["worst_cont"][t * K]))
    e.update({"max_err_n1_max_loading": float(max(errs_n1, default=0.0)),
              "max_err_overload_sum": float(max(errs_ovl, default=0.0)),
              "max_err_n0_max_loading": float(max(errs_n0, default=0.0)),
              "pick_not_beaten_by_8_random_candidates": float(np.mean(pick_ok)) if pick_ok else 1.0,
              "worst_cont_agree": float(np.mean(wc)) if wc else 1.0,
              "sample": f"first {len(idx)} topologies, every timestep: the oracle evaluated at the chosen "
                        "candidate and at 8 random others (all 256 per topology take the oracle ~4 min)"})
    return e


def run_cfg_grid10000(args, flush, peaks, pool):
    """10,000 buses / 15,000 branches, 5000 monitored x 2000 contingencies, 50,000 topologies
    with 1-6 splits, 16 timesteps; the FP32 and the BF16x3 forms (FP64 denominators)."""
    import torch
    from paper_2501_17529_b300 import synth
    from paper_2501_17529_b300.dcflow import DeviceBatch, DeviceResults, Solver
    n = args.g10k_topologies
    w = synth.workload(4, n_topo=n)
    lim = _device_limits(w)
    T, M = w.inj.shape[0], len(w.mon)
    job = None
    if pool is not None and args.g10k_oracle > 0:
        k = min(args.g10k_oracle, n)
        job = pool.map_async(_cpu_worker, [(4, list(range(i, k, 16))) for i in range(min(16, k))])
    alu_peak = 148 * 128 * peaks.get("sm_max_mhz", 2032.0) * 1e6 / 1e12
    out = {"workload": "grid10000_splits1-6_T16_mon5000_cont2000", "topologies": n, "timesteps": T, "monitored": M,
           "contingencies": len(w.cont), "l2": "flushed before each step (256 MB write)", "forms": {}}
    hosts = {}
    for form in args.g10k_forms.split(","):
        ts = time.perf_counter()
        s = Solver(w.grid, precision=form)
        s.set_study(w.mon, w.cont, lim, split_bus=w.subs, outage_cand=np.zeros(0, np.int32))
        torch.cuda.synchronize()
        setup_s = time.perf_counter() - ts
        db = DeviceBatch(w.topo, w.inj)
        res = DeviceResults(n, T, M)
        s.solve(db, results=res)
        torch.cuda.synchronize()
        t, n1_ms, launches, clk = _timed_solve(s, db, res, args.g10k_steps, flush, torch.cuda.current_stream())
        host = res.to_host()
        hosts[form] = host
        lf = _loadflows(w.topo, host["status"], host["n_island_cont"], w.cont, T)
        ach = lf * M / (n1_ms / 1e3) / 1e12
        out["forms"][form] = {"value": lf * args.g10k_steps / t, "unit": "loadflows/s",
                              "ms_per_step": 1e3 * t / args.g10k_steps, "steps": args.g10k_steps,
                              "loadflows_per_step": lf, "launches_per_step": launches, "setup_s": setup_s,
                              "clocks": clk, "schedule": s.last_schedule(),
                              "roofline": {"bound": "alu", "kernel": "k_n1_reg", "achieved": ach, "peak": alu_peak,
                                           "unit": "T N-1 entries/s", "frac": ach / alu_peak, "n1_ms_per_step": n1_ms}}
        s.close()
    if "fp32" in out["forms"] and "bf16x3" in out["forms"]:
        out["bf16x3_over_fp32_speedup"] = out["forms"]["bf16x3"]["value"] / out["forms"]["fp32"]["value"]
    if job is not None:
        out["_oracle"] = (job, hosts)
    return out


def _grid10000_errors(out):
    job, hosts = out.pop("_oracle")
    res = job.get()
    ref = {k: np.concatenate([r[2][k] for r in res]) for k in res[0][2]}
    e = {f: _errors(h, ref, f) for f, h in hosts.items()}
    e["sample"] = f"first {ref['idx'].size} topologies (the oracle refactorises each: ~26 s per topology per core)"
    return e


def run_cfg_screener(args, peaks):
    """The learned screener on the 2000-bus study: trained on solver-generated N-1 labels of
    200,000 topologies (1-8 splits, 8 timesteps), evaluated on 100,000 held-out ones."""
    import torch
    from paper_2501_17529_b300 import screener as scr_mod
    from paper_2501_17529_b300 import synth
    from paper_2501_17529_b300.dcflow import Screener, Solver
    w = synth.workload(5, n_topo=args.scr_train)
    ev_topo = synth.make_topologies(w.grid, w.subs, args.scr_eval, 605, (1, 8), (0, 0))
    lim = _device_limits(w)
    s = Solver(w.grid, precision="fp32")
    s.set_study(w.mon, w.cont, lim, split_bus=w.subs)
    B = args.scr_batch
    sc = Screener(s, max_rows=B, seed=1)
    t0 = time.perf_counter()
    Xtr, Ytr, _, _, st_tr = scr_mod.dataset(s, sc, w.topo, w.inj, args.scr_top_k)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    t0 = time.perf_counter()
    hist = scr_mod.train(sc, Xtr, Ytr, st_tr, w.inj.shape[0], args.scr_epochs, B, args.scr_lr, cosine=True)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    steps = args.scr_epochs * max(1, int((st_tr.repeat_interleave(w.inj.shape[0]) == 0).sum().item()) // B)
    del Xtr, Ytr
    # the probability threshold of the additions beyond the top k, calibrated on topologies held
    # apart from both the training and the evaluation sets (seed 606) for 0.99 recall
    cal_topo = synth.make_topologies(w.grid, w.subs, args.scr_cal, 606, (1, 8), (0, 0))
    Xc, Yc, cm_c, n1_c, st_c = scr_mod.dataset(s, sc, cal_topo, w.inj, args.scr_top_k)
    del Xc
    p_min, cal_curve = scr_mod.calibrate_min_prob(s, sc, cal_topo, w.inj, Yc, cm_c, n1_c, st_c, args.scr_top_k)
    del Yc, cm_c
    Xev, Yev, cm_ev, n1_ev, st_ev = scr_mod.dataset(s, sc, ev_topo, w.inj, args.scr_top_k)
    del Xev
    rep = scr_mod.evaluate(s, sc, ev_topo, w.inj, Yev, cm_ev, n1_ev, st_ev, args.scr_top_k, min_prob=p_min)
    rep["calibration"] = {"topologies": args.scr_cal, "target_recall": 0.99, "min_prob": p_min,
                          "curve": [{"min_prob": p, "recall_evaluated": r, "evaluated_fraction": f}
                                    for p, r, f in cal_curve]}
    # the plain top k, and the recall / speed curve over larger selections
    rep["curve"] = {}
    for k, pm in ((args.scr_top_k, 0.0), (96, 0.0), (128, 0.0)):
        r = scr_mod.evaluate(s, sc, ev_topo, w.inj, Yev, cm_ev, n1_ev, st_ev, k, repeats=2, min_prob=pm)
        rep["curve"][f"top_{k}"] = {x: r[x] for x in ("recall_at_k", "recall_evaluated", "worst_cont_hit_rate",
                                                       "evaluated_fraction", "speedup")}
    # training GEMM work per step: forward 2BH(F + H + C), backward twice that (B rows)
    F, H, C = sc.F, sc.H, s.n_cont
    flop = 3 * 2 * B * H * (F + H + C) * steps
    tfs = flop / t_train / 1e12
    rep.update({"workload": "grid2000_screen_train200k_eval100k_T8_cont1000_mlp256", "train_topologies": args.scr_train,
                "eval_topologies": args.scr_eval, "epochs": args.scr_epochs, "batch": B, "lr": args.scr_lr,
                "train_steps": steps,
                "loss_first_last": [hist[0], hist[-1]] if hist else None, "data_s": t_data, "train_s": t_train,
                "features": F, "hidden": H,
                "roofline": {"bound": "tensor", "kernel": "training (k_gemm_bf16 forward / backward + Adam)",
                             "achieved": tfs, "peak": peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops")),
                             "unit": "TFLOP/s", "frac": tfs / peaks.get("bf16_tflops_sustained",
                                                                         peaks.get("bf16_tflops", 1800.0))}})
    sc.close()
    s.close()
    return rep



def _e2e(solver, w, lim, steps, warmup, lf):
    import torch
    from paper_2501_17529_b300.dcflow import DeviceBatch, DeviceResults

    db = DeviceBatch(w.topo, w.inj, w.var)
    res = DeviceResults(db.n_topo, db.n_time, len(w.mon), want_var=db.n_var > 0)
    names = ["split_ptr", "split_sub", "split_mask", "out_ptr", "out_branch", "inj"]
    if db.n_var:
        names += ["var_ptr", "var_bus", "var_delta"]
    host_in = {n: getattr(db, n).cpu().pin_memory() for n in names}
    outs = ["n1_max_loading", "overload_sum", "worst_cont", "worst_mon", "island_flag", "n_island_cont"]
    host_out = {n: torch.empty_like(getattr(res, n), device="cpu").pin_memory() for n in outs}
    h2d = sum(t.numel() * t.element_size() for t in host_in.values())
    d2h = sum(t.numel() * t.element_size() for t in host_out.values())
    stream = torch.cuda.current_stream()

    def step():
        for n in names:
            getattr(db, n).copy_(host_in[n], non_blocking=True)
        solver.solve(db, results=res)
        for n in outs:
            host_out[n].copy_(getattr(res, n), non_blocking=True)
        stream.synchronize()

    # untimed warm-up: the per-step time of this loop settles over about ten steps
    # after the device-timed loop (11.6 -> 11.2 ms on the 500-bus study)
    for _ in range(max(warmup, 10)):
        step()
    t0 = time.perf_counter()
    for _ in range(steps):
        step()
    dt = time.perf_counter() - t0
    return {"value": lf * steps / dt, "unit": "loadflows/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}


def run_gemm(shapes):
    """Time the screener's tensor-core GEMM (dcflow_gemm_bf16) on M x N x K shapes:
    bf16 A [M, K] and B [N, K], D = A B^T in FP32, 3 warm-up calls, then 10
    timed with CUDA events; one JSON line with ms and TF/s per shape."""
    import torch
    from paper_2501_17529_b300.csrc import build as cbuild
    from paper_2501_17529_b300.dcflow import dcflow_gemm_bf16
    cbuild.build()
    out = {}
    for sh in shapes:
        M, N, K = (int(x) for x in sh.lower().split("x"))
        A = torch.randn(M, K, device="cuda").to(torch.bfloat16)
        B = torch.randn(N, K, device="cuda").to(torch.bfloat16)
        D = torch.empty(M, N, device="cuda")
        for _ in range(3):
            dcflow_gemm_bf16(A, B, out=D)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(10):
            dcflow_gemm_bf16(A, B, out=D)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 10
        out[sh] = {"ms": ms, "tflops": 2.0 * M * N * K / ms / 1e9}
    print(json.dumps({"gemm_bf16": out}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--forms", default="fp32,bf16x3,fp64")
    ap.add_argument("--fp64-steps", type=int, default=0, help="timed steps of the FP64 form (0 = --steps)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--topologies", type=int, default=0, help="batch size (0 = the workload's own)")
    ap.add_argument("--workload", default="grid500", choices=sorted(WORKLOADS))
    ap.add_argument("--gens", type=int, default=16,
                    help="also time the FP32 solve with this many generator-failure cases; 0 = skip")
    ap.add_argument("--ti", type=int, default=16,
                    help="also time the FP32 solve with this many injection topologies per topology; 0 = skip")
    ap.add_argument("--ti-sweep", default="1,4,16,64",
                    help="assignments per topology of the |T_i| sweep (both injection-module modes); '' = none")
    ap.add_argument("--ti-topologies", type=int, default=1000,
                    help="topologies of the injection-topology form")
    ap.add_argument("--rows", default="restricted", choices=["restricted", "full"],
                    help="PTDF rows of the study: the needed branches only, or every branch")
    ap.add_argument("--chunk", type=int, default=0,
                    help="topologies per internal chunk of the solver (0 = automatic)")
    ap.add_argument("--compact", action="store_true",
                    help="FP32 N-1 over each topology's valid contingencies instead of every contingency column")
    ap.add_argument("--multi", type=int, default=32,
                    help="also time the FP32 solve with this many multi-outage sets; 0 = skip")
    ap.add_argument("--top-k", type=int, default=8,
                    help="also time the FP32 solve with the k worst N-1 cases per (topology, timestep); 0 = skip")
    ap.add_argument("--configs", default="grid10000,cand,screen",
                    help="further study shapes timed after the 500-bus line (comma separated from grid10000, cand, "
                         "screen; 'none' skips them)")
    ap.add_argument("--cand-topologies", type=int, default=100000)
    ap.add_argument("--cand-steps", type=int, default=1)
    ap.add_argument("--cand-form", default="fp32")
    ap.add_argument("--cand-oracle", type=int, default=32, help="oracle sample of the candidate study (topologies)")
    ap.add_argument("--g10k-topologies", type=int, default=50000)
    ap.add_argument("--g10k-steps", type=int, default=3)
    ap.add_argument("--g10k-forms", default="fp32,bf16x3")
    ap.add_argument("--g10k-oracle", type=int, default=64, help="oracle sample of the 10,000-bus study (topologies)")
    ap.add_argument("--scr-train", type=int, default=200000)
    ap.add_argument("--scr-eval", type=int, default=100000)
    ap.add_argument("--scr-epochs", type=int, default=80)
    ap.add_argument("--scr-batch", type=int, default=4096)
    ap.add_argument("--scr-lr", type=float, default=1e-3)
    ap.add_argument("--scr-top-k", type=int, default=64)
    ap.add_argument("--scr-cal", type=int, default=20000, help="calibration topologies of the screener")
    ap.add_argument("--gemm", default="",
                    help="only time the screener's tensor-core GEMM on comma-separated MxNxK shapes")
    args = ap.parse_args()
    if args.gemm:
        run_gemm(args.gemm.split(","))
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
