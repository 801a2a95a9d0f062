"""Benchmark: periodized Stokes SLP+DLP layer-potential sum at N = 128,768 on one GB300.

One step = one stokes_sum_eval (density pack, tiled pair kernel over 3 images, FP64
cross-split reduction with the wall curvature diagonal and the FP64 Kress self term) on the
paper-scale channel: walls y = +-(1 + 0.4 sin x + 0.15 sin 3x) with 16,384 nodes each and
750 vesicles x 128 nodes.  Inputs are resident in HBM when the timed region starts; L2 is
flushed (256 MB write) before every timed step.  The metric is pair-image evaluations per
second, 3 N_t N_s per step (Gpair-evals/s).

Under torchrun each rank runs an independent replica (the sum has no exchange step on one
node); value = pairs processed by all ranks / max-over-ranks time.

``--impl reference`` times the FP64 CPU oracle (the test oracle, a plain double loop) on the
host cores, on bounded target samples of the same workload.

Other measurements (one JSON line each): ``--batch`` (64-channel ensemble in one launch),
``--scaling`` (the sum from N = 1,280 to 524,288), ``--step`` (semi-implicit vesicle step with
the learned warm start), ``--poiseuille`` (the accuracy study of Sec. 5.1), ``--walls`` (the
fast direct wall solver against the dense one), ``--fmm`` (fast multipole node evaluation
against the direct sums).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "paper_n128k"
WORKLOAD_DESCS = {
    "paper_n128k": ("channel walls y=+-(1+0.4 sin x+0.15 sin 3x), 2 x 16384 nodes; 750 vesicles x 128 "
                    "nodes (volume fraction 0.15, gap >= 5h); period 2pi, images m=-1,0,1; N=128768"),
    "mid_n16k": ("channel walls y=+-(1+0.3 sin x), 2 x 4096 nodes; 128 vesicles x 64 nodes "
                 "(volume fraction 0.15); period 2pi, images m=-1,0,1; N=16384 (profiling case)"),
    "small_n1280": ("channel walls y=+-(1+0.3 sin x), 2 x 512 nodes; 4 vesicles x 64 nodes; "
                    "period 2pi, images m=-1,0,1; N=1280"),
}
METRIC = "Stokes SLP+DLP Gpair-evals/s at N≈128k: FP32-comp vs FP64, rel err ≤1e-6"
# Nominal FP32 work of one pair-image evaluation (r, r^2, 1/r^2, log or (r.n), r.q, the
# tensor-vector product and the accumulation), counting every add, multiply, reciprocal and
# log as one flop; used for the roofline's achieved rate.
FLOPS_PER_PAIR = 20
LANES = 128  # FP32 FMA lanes per SM (Blackwell)


def device_sms(device=0) -> int:
    """Streaming multiprocessors of the CUDA device (read from the device, not assumed)."""
    import torch
    return int(torch.cuda.get_device_properties(device).multi_processor_count)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                smax = float(r[2])
            except (ValueError, IndexError):
                continue
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(seconds, device=None):
    """The slowest rank's time (all ranks must call); the single-rank value when not distributed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(seconds)
    t = torch.tensor([float(seconds)], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank, world_size, seconds_max):
    """Whole-job throughput of independent replicas: all ranks' units over the slowest time."""
    return world_size * units_per_rank / seconds_max


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("k_pair.cu", "stokes_internal.cuh", "bulk_pipe.cuh"):
        with open(os.path.join(ROOT, "paper_1510_05616_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per pair-kernel launch from the committed ncu summary, if it still
    describes the current kernel source."""
    p = os.path.join(ROOT, "profiles", "pair_f32k_paper_n128k.traffic.txt")
    if not os.path.exists(p):
        return None
    txt = open(p).read()
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    hm = re.search(r"kernel_source_hash:\s*([0-9a-f]+)", txt)
    if not m or not hm or hm.group(1) != kernel_source_hash():
        return None
    return float(m.group(1))


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"sm_max_mhz": 2070.0}, "fallback"


def cpu_sample_oracle(geom, slp, dlp, budget_s, seed=0):
    """Time the FP64 oracle on a random target sample sized to ~budget_s seconds."""
    from oracle import oracle as O
    threads = os.cpu_count() or 1
    rng = np.random.default_rng(seed)
    n = 64
    sel = np.sort(rng.choice(geom.n_nodes, n, replace=False)).astype(np.int32)
    t0 = time.perf_counter()
    O.sum_nodes(geom, slp, dlp, select=sel, threads=threads)
    t1 = time.perf_counter() - t0
    n2 = int(min(geom.n_nodes, max(n, n * budget_s / max(t1, 1e-3))))
    sel = np.sort(rng.choice(geom.n_nodes, n2, replace=False)).astype(np.int32)
    t0 = time.perf_counter()
    ref = O.sum_nodes(geom, slp, dlp, select=sel, threads=threads)
    dt = time.perf_counter() - t0
    pairs = (3.0 if geom.period else 1.0) * n2 * geom.n_nodes
    return sel, ref, pairs, dt, threads


def rel_err_by_kind(out, ref, geom, sel):
    wall = geom.kind_mask(0)[sel]
    res = {}
    for name, m in (("wall", wall), ("vesicle", ~wall)):
        if m.any():
            scale = np.abs(ref[m]).max(0)
            res[name] = [float(v) for v in np.abs(out[sel][m] - ref[m]).max(0) / scale]
    return res


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_1510_05616_gb300 import inputs as I
    from oracle import oracle as O
    O.build()
    g, slp, dlp = I.workload(WORKLOAD)
    budget = max(1.0, 60.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        cpu_sample_oracle(g, slp, dlp, min(budget, 2.0), seed=1)
    total_pairs, total_t, threads, samples = 0.0, 0.0, 1, []
    for k in range(args.steps):
        sel, _, pairs, dt, threads = cpu_sample_oracle(g, slp, dlp, budget, seed=100 + k)
        total_pairs += pairs
        total_t += dt
        samples.append(len(sel))
    val = total_pairs / total_t / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "Gpair-evals/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total_t / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESCS[WORKLOAD], "N": g.n_nodes, "sample": "random target nodes per step"},
        "cpu_baseline": {"value": val, "unit": "Gpair-evals/s", "cores": threads, "kind": "oracle",
                         "sample": "%s target nodes x all %d sources x 3 images per step"
                                   % (samples, g.n_nodes)},
        "e2e": {"value": val, "unit": "Gpair-evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_batch(args):
    """64 independent channels: one persistent graph-replayed launch vs the plain form
    (one stokes_sum_eval per instance, back to back on one stream)."""
    import torch
    import paper_1510_05616_gb300 as P
    from paper_1510_05616_gb300 import build as B
    from paper_1510_05616_gb300 import inputs as I
    B.build()
    ens = I.ensemble(workers=min(16, os.cpu_count() or 1))
    geoms = [g for g, _, _ in ens]
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    b = P.StokesBatch(geoms)
    ts = torch.as_tensor(P.StokesBatch.stack([s for _, s, _ in ens]), device=dev)
    td = torch.as_tensor(P.StokesBatch.stack([d for _, _, d in ens]), device=dev)
    out = torch.empty((b.N, 2), dtype=torch.float64, device=dev)
    pairs = P.stokes_pair_count(b.h)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def timed(fn, steps):
        ms = []
        for k in range(steps):
            flush.fill_(float(k))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return ms

    res = {}
    for prec_name in ("fp32k", "fp64"):
        prec = P.PRECISIONS[prec_name]
        # the FP64 leg keeps its default shape: timing its candidates would take minutes
        tuned = None if args.no_tune or prec_name != "fp32k" else P.stokes_autotune(b.h, prec, repeats=3)
        steps = args.steps if prec_name == "fp32k" else max(1, args.fp64_steps)
        for _ in range(max(1, args.warmup if prec_name == "fp32k" else 1)):
            P.stokes_batch_eval(b.h, prec, ts, td, 0.0, out, True)
        P.stokes_sync(b.h)
        g_ms = timed(lambda: P.stokes_batch_eval(b.h, prec, ts, td, 0.0, out, True), steps)
        d_ms = timed(lambda: P.stokes_batch_eval(b.h, prec, ts, td, 0.0, out, False), steps)
        res[prec_name] = {"graph_ms": statistics.median(g_ms), "direct_ms": statistics.median(d_ms),
                          "graph_gpairs": pairs / statistics.median(g_ms) / 1e6,
                          "items": P.stokes_batch_info(b.h, prec)[0],
                          "blocks": P.stokes_batch_info(b.h, prec)[1],
                          "shape": dict(zip(("targets_per_thread", "items_per_slot"),
                                            P.stokes_batch_info(b.h, prec)[2:])),
                          "autotune": tuned}
    b.close()
    # plain form: one single-instance context per channel, evaluated back to back
    singles = [P.StokesSum(g) for g in geoms]
    dens = [(torch.as_tensor(s, device=dev), torch.as_tensor(d, device=dev)) for _, s, d in ens]
    outs = [torch.empty((g.n_nodes, 2), dtype=torch.float64, device=dev) for g in geoms]
    for prec_name in ("fp32k",):
        prec = P.PRECISIONS[prec_name]
        # per size class: a context whose class the tuner has not seen yet is tuned; the
        # others took the recorded shape of their class when their geometry was set
        n_tuned = 0
        if not args.no_tune:
            sms = torch.cuda.get_device_properties(0).multi_processor_count
            for h, g in zip(singles, geoms):
                nw = int(g.kind_mask(I.KIND_DLP).sum())
                if P.stokes_tune_lookup(sms, prec, 1, g.n_nodes, nw, g.n_nodes - nw) is None:
                    P.stokes_autotune(h.h, prec, repeats=3)
                    n_tuned += 1
                else:
                    sh = P.stokes_tune_lookup(sms, prec, 1, g.n_nodes, nw, g.n_nodes - nw)
                    P.stokes_set_launch(h.h, prec, sh["source_splits"], sh["targets_per_thread"],
                                        sh["kahan_group"])
        res[prec_name]["plain_size_classes_tuned"] = n_tuned
        for h, (s_, d_), o in zip(singles, dens, outs):
            P.stokes_sum_eval(h.h, prec, s_, d_, 0.0, o)
        torch.cuda.synchronize()

        def plain():
            for h, (s_, d_), o in zip(singles, dens, outs):
                P.stokes_sum_eval(h.h, prec, s_, d_, 0.0, o)
        p_ms = timed(plain, args.steps)
        per = []
        for h, (s_, d_), o, g in zip(singles, dens, outs, geoms):
            ms = timed(lambda: P.stokes_sum_eval(h.h, prec, s_, d_, 0.0, o), 3)
            per.append(P.stokes_pair_count(h.h) / min(ms) / 1e6)
        res[prec_name]["plain_ms"] = statistics.median(p_ms)
        res[prec_name]["plain_gpairs"] = pairs / statistics.median(p_ms) / 1e6
        res[prec_name]["per_instance_gpairs"] = {"min": min(per), "median": statistics.median(per),
                                                 "max": max(per)}
    for h in singles:
        h.close()
    line = {"metric": "batched ensemble Gpair-evals/s (64 channels, one persistent graph launch)",
            "value": res["fp32k"]["graph_gpairs"], "unit": "Gpair-evals/s", "n_gpus": 1,
            "steps": args.steps, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "64 channels: wall nodes {1024..8192}/wall, vesicles U[10,400] x "
                                   "{32..256} nodes, fill U[0.05,0.15]", "instances": len(geoms),
                       "N_total": int(sum(g.n_nodes for g in geoms)), "pairs_per_step": pairs},
            "results": res}
    print(json.dumps(line))
    return 0


def _mode_slice(nm_from, nm_to, history=False):
    """Columns of the nm_from-mode features and targets that hold the nm_to-mode ones (the
    modes k = -nm_to/2..nm_to/2-1 of shape, velocity change and solution change, and the
    tension modes k = 0..nm_to/2-1, are a subset of the larger representation; with history
    features the previous solution and its last change follow in the target layout)."""
    lo = nm_from // 2 - nm_to // 2
    shape = np.arange(2 * lo, 2 * lo + 2 * nm_to)
    targ = np.concatenate([shape, 2 * nm_from + np.arange(nm_to)])
    feat = [shape, 2 * nm_from + shape]
    if history:
        feat += [4 * nm_from + targ, 4 * nm_from + 3 * nm_from + targ]
    return np.concatenate(feat), targ


def run_step_one(args):
    """One mixed-precision zero-guess step of the held-out channel of --step (seed 2000), after
    --warmup warm steps, between cudaProfilerStart/Stop -- for a launch list of one step with
    `ncu --profile-from-start off`.  Settings as --step: --residual-fmm, --sweep-fmm,
    --precond-refresh."""
    import torch
    import paper_1510_05616_gb300 as P
    from paper_1510_05616_gb300 import build as B
    from paper_1510_05616_gb300 import inputs as I
    from paper_1510_05616_gb300 import warmstart as WS
    B.build()
    n_w, modes, nv, n_v, area = I.WORKLOADS[args.step_workload]
    kb = 0.01 * area / I.WORKLOADS["mid_n16k"][4]  # as run_step
    pd = 2 * 1.0 * 2 * math.pi * 0.2
    g = I.channel(n_w, modes, nv, n_v, area, 2000, mu=1.0)
    sim = WS.Simulation(g, kappa_b=kb, restart=200, residual_fmm=args.residual_fmm,
                        sweep_fmm=args.sweep_fmm, precond_refresh=args.precond_refresh,
                        precond_tensor=args.precond_tensor)
    for _ in range(args.warmup):
        sim.step(1e-3, pd, "zero", precision=P.STOKES_FP32_KAHAN)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    st = sim.step(1e-3, pd, "zero", precision=P.STOKES_FP32_KAHAN)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    sim.close()
    print(json.dumps({"metric": "one semi-implicit step (zero guess), profiled", "unit": "ms",
                      "value": st["total_ms"], "warm_steps": args.warmup,
                      "config": {"workload": WORKLOAD_DESCS[args.step_workload],
                                 "residual_fmm_order": args.residual_fmm,
                                 "sweep_fmm_order": args.sweep_fmm,
                                 "precond_refresh": bool(args.precond_refresh),
                                 "precond_tensor": bool(args.precond_tensor)},
                      "stats": st}))
    return 0


def run_step(args):
    """Algorithm 1 on a channel (walls, channel response, GMRES to 1e-10): plain runs give the
    training states, a network per feature size (warm-start modes) is trained with the
    library's kernels, and a held-out channel is stepped from the same state with the zero,
    previous-step and network guesses, for each precision of the Krylov matvecs (FP64;
    FP32-Kahan sweeps inside FP64-accurate refinement -- whose FP64-accurate vesicle sums are
    double-float direct sums, or the FMM with --residual-fmm; double-float).  The FP64 pair sum
    is left out at N = 128,768, where one of its matvecs costs ~1.2 s."""
    import torch
    import paper_1510_05616_gb300 as P
    from paper_1510_05616_gb300 import build as B
    from paper_1510_05616_gb300 import inputs as I
    from paper_1510_05616_gb300 import warmstart as WS
    B.build()
    n_w, modes, nv, n_v, area = I.WORKLOADS[args.step_workload]
    big = args.step_workload == "paper_n128k"
    # bending modulus scaled with the vesicle area (0.01 at the 16k channel's vesicle size): the
    # bending velocity kappa_B / (mu R^2) then stays ~2 and the explicit channel response does
    # not move a vesicle across its wall gap within one step of dt = 1e-3
    dt, mu = 1e-3, 1.0
    kb = 0.01 * area / I.WORKLOADS["mid_n16k"][4]
    pd = 2 * mu * 2 * math.pi * 0.2
    names = {"fp64": P.STOKES_FP64, "fp32k": P.STOKES_FP32_KAHAN, "df": P.STOKES_DOUBLE_FLOAT}
    precs = [p for p in args.step_precisions.split(",") if p] or (
        ["fp32k", "df"] if big else ["fp64", "fp32k", "df"])
    collect_prec = names[args.collect_precision or ("fp32k" if big else "fp64")]
    nets_modes = sorted({int(m) for m in args.step_modes.split(",") if m})
    nm_max = max(nets_modes)
    fmm = args.residual_fmm
    sweep = args.sweep_fmm
    refresh = args.precond_refresh
    base = args.warm_base
    hist = not args.no_warm_history
    res = {"workload": args.step_workload, "dt": dt, "p_drive": pd, "kappa_b": kb, "tol": 1e-10,
           "precisions": precs, "collect_precision": args.collect_precision or
           ("fp32k" if big else "fp64"), "warm_modes": nets_modes,
           "residual_fmm_order": fmm, "sweep_fmm_order": sweep, "precond_refresh": refresh,
           "precond_tensor": bool(args.precond_tensor), "warm_base": base, "history_features": hist}
    t0 = time.perf_counter()
    Xs, Ts, plain_its = [], [], []
    for r in range(args.train_runs):
        g = I.channel(n_w, modes, nv, n_v, area, 1000 + r, mu=mu)
        torch.cuda.synchronize()
        ts = time.perf_counter()
        sim = WS.Simulation(g, kappa_b=kb, restart=200, modes=nm_max, residual_fmm=fmm,
                            history=hist, sweep_fmm=sweep, precond_refresh=refresh, base=base,
                            precond_tensor=args.precond_tensor)
        torch.cuda.synchronize()
        res.setdefault("setup_s", time.perf_counter() - ts)
        res.setdefault("wall_solve", dict(zip(("refinements", "residual"),
                                              P.stokes_sim_wall_stats(sim.h))))
        X, T, st = WS.collect(sim, args.train_steps, dt, pd, precision=collect_prec)
        plain_its += [x["iterations"] for x in st]
        Xs.append(X)
        Ts.append(T)
        sim.close()
    X, T = torch.cat(Xs), torch.cat(Ts)
    res["collect_s"] = time.perf_counter() - t0
    nets, res["train"] = {}, {}
    for nm in nets_modes:
        fc, tc = (torch.as_tensor(c, device="cuda") for c in _mode_slice(nm_max, nm, hist))
        Xm, Tm = X[:, fc].contiguous(), T[:, tc].contiguous()
        net = WS.WarmStartNet(hidden=256, seed=0, modes=nm, history=hist)
        t1 = time.perf_counter()
        losses = net.fit(Xm, Tm, epochs=args.train_epochs, batch=256, lr=2e-3)
        torch.cuda.synchronize()
        res["train"][nm] = {"samples": int(Xm.shape[0]), "features": int(Xm.shape[1]),
                            "targets": int(Tm.shape[1]), "epochs": args.train_epochs, "batch": 256,
                            "adam_steps": args.train_epochs * (int(Xm.shape[0]) // 256),
                            "seconds": time.perf_counter() - t1, "loss_first": losses[0],
                            "loss_last": losses[-1]}
        nets[nm] = net
    del X, T, Xs, Ts
    g = I.channel(n_w, modes, nv, n_v, area, 2000, mu=mu)
    sim = WS.Simulation(g, kappa_b=kb, restart=200, modes=nm_max, residual_fmm=fmm, history=hist,
                        sweep_fmm=sweep, precond_refresh=refresh, base=base,
                        precond_tensor=args.precond_tensor)
    x0, s0, _ = sim.state()
    evs = {}
    for p in precs:
        ev = {}
        for k, nm in enumerate(nets_modes):
            P.stokes_sim_set_warm_modes(sim.h, nm)
            gs = ("zero", "previous", "extrapolate", "mlp") if k == 0 else ("mlp",)
            one = WS.evaluate(sim, x0, s0, args.steps, dt, pd, model=nets[nm], guesses=gs,
                              precision=names[p])
            one["mlp%d" % nm] = one.pop("mlp")
            ev.update(one)
        evs[p] = ev
    sim.close()
    for net in nets.values():
        net.close()
    for p, ev in evs.items():
        res["eval_" + p] = ev
    head = evs[precs[0]]
    z = head["zero"]

    def summary(ev):
        return {k: {kk: v[kk] for kk in ("mean_iterations", "step_ms", "gmres_ms",
                                          "mean_refinements", "mean_accurate_residuals")}
                for k, v in ev.items()}

    line = {"metric": "semi-implicit vesicle step, GMRES to 1e-10: mean iterations and ms per step",
            "value": z["step_ms"], "unit": "ms/step (zero guess, %s matvecs)" % precs[0],
            "higher_is_better": False, "n_gpus": 1, "steps": args.steps, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_DESCS[args.step_workload], "vesicles": nv,
                       "nodes_per_vesicle": n_v, "wall_nodes": 2 * n_w,
                       "training_states": int(res["train"][nets_modes[0]]["samples"]),
                       "warm_modes": nets_modes, "residual_fmm_order": fmm,
                       "sweep_fmm_order": sweep, "precond_refresh": refresh,
                       "precond_tensor": bool(args.precond_tensor), "warm_base": base},
            "iterations_saved_vs_zero": {p: {k: ev["zero"]["mean_iterations"] - v["mean_iterations"]
                                             for k, v in ev.items()} for p, ev in evs.items()},
            "by_precision": {p: summary(ev) for p, ev in evs.items()},
            "details": res}
    print(json.dumps(line))
    return 0


def run_poiseuille(args):
    """Accuracy study of Sec. 5.1 on the GPU: the pressure-driven channel with wall data of the
    exact Poiseuille flow u_e = (-p_drive/(2 mu d) y^2, 0), p_e = -p_drive x / d (+ const),
    mu = 0.7, alpha = 0.2, d = 2 pi; errors at the probes (0.8, 0), (3.2, 0), (4.8, 0) as the
    wall nodes N (K = 32, M = 128) and the side points K (M = 4K, N = 512) vary, for both sine
    channels.  Velocity error: max over probes of |u - u_e| / max |u_e| on the walls; pressure
    error: max over probes of |p - p_e - c| / p_drive with c the mean offset (the
    representation fixes its own additive constant).  Also times the FP64 pressure and
    traction sums at free points."""
    import torch
    import paper_1510_05616_gb300 as P
    from paper_1510_05616_gb300 import build as B
    from paper_1510_05616_gb300 import inputs as I
    B.build()
    mu, d = 0.7, 2 * math.pi
    pd = 2 * mu * d * 0.2
    probes = np.array([[0.8, 0.0], [3.2, 0.0], [4.8, 0.0]])
    ue = lambda q: np.stack([-(pd / (2 * mu * d)) * q[:, 1] ** 2, 0 * q[:, 1]], 1)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")

    def errors(shape, n_w, K, M):
        lo, up = I.wall_curves(n_w, shape)
        xw = np.vstack([lo.nodes, up.nodes])
        h = P.stokes_sim_create(0)
        P.stokes_sim_set_walls(h, n_w, xw, np.concatenate([lo.weights, up.weights]),
                               np.vstack([lo.normals, up.normals]),
                               np.concatenate([lo.curvature, up.curvature]), d, mu, K, M)
        u = torch.zeros((len(probes), 2), dtype=torch.float64, device="cuda")
        p = torch.zeros(len(probes), dtype=torch.float64, device="cuda")
        P.stokes_sim_empty_channel(h, pd, dev(ue(xw)), dev(probes), u)
        P.stokes_sim_empty_channel_pressure(h, pd, dev(ue(xw)), dev(probes), p)
        P.stokes_sim_destroy(h)
        u, p = u.cpu().numpy(), p.cpu().numpy()
        eu = float(np.abs(u - ue(probes)).max() / np.abs(ue(xw)).max())
        off = p + pd * probes[:, 0] / d
        ep = float(np.abs(off - off.mean()).max() / pd)
        return eu, ep

    shapes = {"1+0.3 sin x": I.WALL_SHAPE_SMALL, "1+0.4 sin x+0.15 sin 3x": I.WALL_SHAPE_LARGE}
    res = {"by_N": {}, "by_K": {}}
    for name, shape in shapes.items():
        res["by_N"][name] = {n: errors(shape, n, 32, 128) for n in (32, 48, 64, 96, 128, 192, 256, 512)}
        res["by_K"][name] = {k: errors(shape, 512, k, 4 * k) for k in (4, 6, 8, 12, 16, 24, 32)}
    # throughput of the FP64 field sums at the paper-scale geometry
    g, slp, dlp = I.workload("paper_n128k")
    s = P.StokesSum(g)
    rng = np.random.default_rng(0)
    T = 16384
    pts = dev(np.stack([rng.uniform(0, d, T), rng.uniform(-0.5, 0.5, T)], 1))
    nrm = dev(np.tile([[0.0, 1.0]], (T, 1)))
    ts, td = dev(slp), dev(dlp)
    pr = torch.zeros(T, dtype=torch.float64, device="cuda")
    tr = torch.zeros((T, 2), dtype=torch.float64, device="cuda")
    timing = {}
    for name, fn in (("pressure", lambda: P.stokes_sum_eval_pressure(s.h, ts, td, pts, pr)),
                     ("traction", lambda: P.stokes_sum_eval_traction(s.h, ts, td, pts, nrm, tr))):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            fn()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 3
        timing[name] = {"ms": ms, "gpair_per_s": 3.0 * T * g.n_nodes / ms / 1e6}
    s.close()
    line = {"metric": "Poiseuille accuracy study (Sec. 5.1): relative errors at 3 probes",
            "unit": "relative error", "n_gpus": 1, "data": "synthetic", "dtype": "f64",
            "config": {"mu": mu, "alpha": 0.2, "period": d, "probes": probes.tolist(),
                       "field_timing_targets": T, "field_timing_sources": g.n_nodes},
            "velocity_pressure_errors": res, "field_sums": timing}
    print(json.dumps(line))
    return 0


def run_walls(args):
    """Wall solvers at a channel's walls (default: the paper's, 2 x 16,384 nodes): the fast
    direct solver of Sec. 4 (HBS inverse of A_0, low-rank neighbour factors, SMW) against the
    dense FP32-LU inverse with FP64 refinement.  Set-up wall clock and device memory, median
    time of one solve (one right-hand side) and of 256 right-hand sides, and the relative
    residual max|A x - b| / max|b| with A applied by the FP64 double-layer pair sum.  The
    one-right-hand-side solves of the fast solver run between cudaProfilerStart/Stop, so a
    profiler started with --profile-from-start off sees only them."""
    import torch
    import paper_1510_05616_gb300 as P
    from paper_1510_05616_gb300 import build as B
    from paper_1510_05616_gb300 import inputs as I
    B.build()
    mu, d = 0.7, 2 * math.pi
    n_w = args.walls_nodes
    lo, up = I.wall_curves(n_w, I.WALL_SHAPE_LARGE)
    xw = np.vstack([lo.nodes, up.nodes])
    rng = np.random.default_rng(0)
    b = torch.as_tensor(rng.normal(size=(4, 4 * n_w)), device="cuda")
    peaks, peak_kind = measured_peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    # fds_plain: the fast direct solver without the column recompression of its neighbour
    # factors (R = A_m(J, :) stored dense)
    modes = {"fds": P.STOKES_WALLS_FDS, "fds_plain": P.STOKES_WALLS_FDS,
             "lu32_refine": P.STOKES_WALLS_LU32_REFINE}
    res = {}
    sols = {}
    # warm-up: a small channel with each solver (library loading, first cuBLAS/cuSOLVER calls)
    wl, wu = I.wall_curves(256, I.WALL_SHAPE_LARGE)
    for name in args.walls_solvers.split(","):
        h = P.stokes_sim_create(0)
        P.stokes_sim_set_wall_solver(h, modes[name])
        P.stokes_sim_set_fds_recompress(h, name != "fds_plain")
        P.stokes_sim_set_walls(h, 256, np.vstack([wl.nodes, wu.nodes]),
                               np.concatenate([wl.weights, wu.weights]),
                               np.vstack([wl.normals, wu.normals]),
                               np.concatenate([wl.curvature, wu.curvature]), d, mu, 32, 128)
        P.stokes_sim_destroy(h)
    for name in args.walls_solvers.split(","):
        h = P.stokes_sim_create(0)
        P.stokes_sim_set_wall_solver(h, modes[name])
        P.stokes_sim_set_fds_recompress(h, name != "fds_plain")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        t0 = time.perf_counter()
        P.stokes_sim_set_walls(h, n_w, xw, np.concatenate([lo.weights, up.weights]),
                               np.vstack([lo.normals, up.normals]),
                               np.concatenate([lo.curvature, up.curvature]), d, mu, 32, 128)
        setup = time.perf_counter() - t0
        mem = (free0 - torch.cuda.mem_get_info()[0]) / 1e9
        info = P.stokes_sim_fds_info(h)
        X = b[0].clone()
        for _ in range(max(args.warmup, 3)):
            X.copy_(b[0])
            P.stokes_sim_wall_solve(h, X)
        ts = []
        if name == "fds":
            torch.cuda.profiler.start()
        for _ in range(max(args.steps, 5)):
            X.copy_(b[0])
            torch.cuda.synchronize()
            t = time.perf_counter()
            P.stokes_sim_wall_solve(h, X)  # synchronous
            ts.append(time.perf_counter() - t)
        if name == "fds":
            torch.cuda.profiler.stop()
        one_ms = 1e3 * statistics.median(ts)
        Xs = b.clone()
        P.stokes_sim_wall_solve(h, Xs)
        Xm = torch.as_tensor(rng.normal(size=(256, 4 * n_w)), device="cuda")
        torch.cuda.synchronize()
        t = time.perf_counter()
        P.stokes_sim_wall_solve(h, Xm)
        many_ms = 1e3 * (time.perf_counter() - t)
        del Xm
        P.stokes_sim_destroy(h)
        torch.cuda.empty_cache()
        sols[name] = Xs
        r = {"setup_s": setup, "device_gb": mem, "solve_ms": one_ms, "solve_256_ms": many_ms}
        if name in ("fds", "fds_plain"):
            r["fds"] = {k: info[k] for k in ("levels", "max_rank", "root_size", "neighbour_rank",
                                             "neighbour_col_rank", "sections", "host_ms",
                                             "device_ms", "device_bytes", "solve_bytes")}
            gbs = info["solve_bytes"] / (one_ms * 1e-3) / 1e9
            r["roofline"] = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                             "frac": gbs / hbm, "basis": "matrices read once per solve / "
                             "wall-clock of the synchronous call, of %s copy peak" % peak_kind}
        res[name] = r
    # residuals through the FP64 double-layer pair sum (an independent application of A)
    geom = I.Geometry([lo, up], d, mu, {})
    s = P.StokesSum(geom)
    for name, Xs in sols.items():
        rr = []
        for k in range(Xs.shape[0]):
            Ax = s.eval(None, Xs[k].view(-1, 2).contiguous(), precision="fp64", jump=-0.5)
            rr.append((Ax.reshape(-1) - b[k]).abs().max().item() / b[k].abs().max().item())
        res[name]["residual_max"] = max(rr)
    s.close()
    for other in ("lu32_refine", "fds_plain"):
        if "fds" in sols and other in sols:
            a, c = sols["fds"], sols[other]
            res["fds_vs_%s_max_rel" % other] = ((a - c).abs().max() / c.abs().max()).item()
    line = {"metric": "channel wall solve: fast direct solver (Sec. 4) vs dense LU32 + FP64 refinement",
            "unit": "ms / s / GB", "n_gpus": 1, "data": "synthetic", "dtype": "f64",
            "config": {"workload": "walls y=+-(1+0.4 sin x+0.15 sin 3x), 2 x %d nodes, period 2pi, "
                                   "mu 0.7, K=32, M=128" % n_w, "unknowns": 4 * n_w},
            "solvers": res}
    print(json.dumps(line))
    return 0


def run_close(args):
    """Close evaluation (the near-pair correction of the vesicles' single layer, F2) on channels
    packed with a gap of only `--close-gap` node spacings, so that close pairs exist: plan time
    (host pair search), time per correction call (CUDA events, median after warm-up) against
    the plain node sums it corrects, the close pairs found, and how much the correction moves
    the FP64 node sum (max over nodes, relative to max |u|)."""
    import torch
    import paper_1510_05616_gb300 as P
    from paper_1510_05616_gb300 import build as B
    from paper_1510_05616_gb300 import inputs as I
    B.build()
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")

    def timed(fn, reps=7):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    rows = {}
    for name in args.close_workloads.split(","):
        n_w, modes, nv, n_v, area = I.WORKLOADS[name]
        t0 = time.perf_counter()
        g = I.channel(n_w, modes, nv, n_v, area, I.WORKLOAD_SEED[name] + 500,
                      gap_factor=args.close_gap)
        slp, dlp = I.densities(g, I.WORKLOAD_SEED[name] + 500)
        gen_s = time.perf_counter() - t0
        s = P.StokesSum(g)
        ts, td = dev(slp), dev(dlp)
        N = g.n_nodes
        out = torch.zeros((N, 2), dtype=torch.float64, device="cuda")
        r = {"N": N, "vesicles": nv, "nodes_per_vesicle": n_v, "gap_spacings": args.close_gap,
             "generation_s": gen_s}
        for prec in ("fp32k", "df"):
            r["plain_" + prec + "_ms"] = timed(lambda: s.eval(ts, td, precision=prec, out=out))
        base = s.eval(ts, td, precision="df").clone()
        for K in (8, 16):
            t0 = time.perf_counter()
            cl = P.stokes_close_create(s.h, args.close_factor, K)
            plan_ms = 1e3 * (time.perf_counter() - t0)
            info = P.stokes_close_get_info(cl)

            def call():
                P.stokes_close_eval(cl, ts, out)
                P.stokes_sync(s.h)
            out.copy_(base)
            ms = timed(call)
            out.copy_(base)
            call()
            moved = float((out - base).abs().max() / base.abs().max())
            r["close_K%d" % K] = {"ms": ms, "plan_ms": plan_ms, "pairs": info["pairs"],
                                  "targets": info["targets"], "vesicles": info["vesicles"],
                                  "share_of_fp32k_sum": ms / r["plain_fp32k_ms"],
                                  "share_of_df_sum": ms / r["plain_df_ms"],
                                  "max_change_rel": moved}
            P.stokes_close_destroy(cl)
        s.close()
        rows[name] = r
    print(json.dumps({"metric": "close evaluation of the vesicles' single layer: time per call",
                      "unit": "ms", "higher_is_better": False, "n_gpus": 1, "dtype": "f64",
                      "data": "synthetic", "factor": args.close_factor, "results": rows}))
    return 0


def run_fmm(args):
    """The pair sum at the nodes by the fast multipole method (FP64 expansions, orders 20 and
    28) against the direct GPU sums, from N = 1,280 to 524,288: evaluation time (median of
    CUDA-event-timed calls after warm-up), the equivalent pair rate 3 N_t N_s / t, plan time,
    and the FMM's error against the FP64-accurate double-float direct sum."""
    import torch
    import paper_1510_05616_gb300 as P
    from paper_1510_05616_gb300 import build as B
    from paper_1510_05616_gb300 import inputs as I
    B.build()
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    rows = {}
    orders = [("fp64", int(o)) for o in args.fmm_orders.split(",") if o] + \
             [("fp32", int(o)) for o in args.fmm_fp32_orders.split(",") if o]
    for name in args.fmm_workloads.split(","):
        g, slp, dlp = I.workload(name)
        if args.fmm_vesicles_only:  # the step's vesicle sums: vesicle curves only
            ves = [c for c in g.curves if c.kind == I.KIND_SLP]  # slp rows are the vesicle nodes
            g, dlp = I.Geometry(ves, g.period, g.mu, dict(g.meta)), None
        s = P.StokesSum(g)
        ts, td = dev(slp), (dev(dlp) if dlp is not None else None)
        N = g.n_nodes
        pairs = 3.0 * N * N
        out = torch.zeros((N, 2), dtype=torch.float64, device="cuda")
        # the library's calls run on its own stream and end with a sync, so events on the
        # current stream bracket them completely
        r = {"N": N, "pairs": pairs}
        ref = None
        for prec in ("fp32k", "df") + (("fp64",) if N <= 20000 else ()):
            ms = timed(lambda: s.eval(ts, td, precision=prec, out=out), 3 if N > 200000 else 5)
            r["direct_" + prec] = {"ms": ms, "gpair_per_s": pairs / ms / 1e6}
            if prec == "df":
                ref = out.cpu().numpy().copy()
        for arith, order in orders:
            t0 = time.perf_counter()
            f = P.stokes_fmm_create(s.h, order, args.fmm_leaf)
            plan_ms = 1e3 * (time.perf_counter() - t0)
            P.stokes_fmm_set_precision(f, P.STOKES_FP32_KAHAN if arith == "fp32" else P.STOKES_FP64)

            def call():
                P.stokes_fmm_eval(f, ts, td, 0.0, out)
                P.stokes_sync(s.h)
            first = (arith, order) == orders[0]
            if first:  # a profiler started with --profile-from-start off sees these calls
                torch.cuda.profiler.start()
            ms = timed(call, 5)
            if first:
                torch.cuda.profiler.stop()
            u = out.cpu().numpy()
            err = float((np.abs(u - ref).max(0) / np.abs(ref).max(0)).max())
            info = P.stokes_fmm_get_info(f)
            P.stokes_fmm_destroy(f)
            r["fmm_p%d" % order + ("_fp32" if arith == "fp32" else "")] = {
                                    "ms": ms, "equiv_gpair_per_s": pairs / ms / 1e6, "plan_ms": plan_ms,
                                    "rel_err_vs_df": err, "levels": info["levels"],
                                    "m2l_pairs": info["m2l_pairs"], "near_pairs": info["near_pairs"]}
        s.close()
        rows[name] = r
    line = {"metric": "node evaluation of the layer-potential sum: FMM (FP64 expansions) vs direct",
            "unit": "ms per evaluation", "n_gpus": 1, "data": "synthetic", "dtype": "f64",
            "config": {"workloads": {k: WORKLOAD_DESCS.get(k, k) for k in rows},
                       "vesicles_only": bool(args.fmm_vesicles_only),
                       "leaf_size": args.fmm_leaf, "direct_shapes": "default (not autotuned)"},
            "results": rows}
    print(json.dumps(line))
    return 0


def run_scaling(args):
    """The FP32-Kahan node sum (autotuned shape) at N = 1,280 / 16,384 / 128,768 / 524,288:
    throughput, pair-kernel fraction of the FP32 FMA peak and the error against the FP64
    oracle on sampled nodes.  (The largest channel takes a couple of minutes to generate.)"""
    import torch
    import paper_1510_05616_gb300 as P
    from paper_1510_05616_gb300 import build as B
    from paper_1510_05616_gb300 import inputs as I
    from oracle import oracle as O
    B.build()
    O.build()
    peaks, _ = measured_peaks()
    peak = device_sms() * LANES * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
    rows = {}
    for name in ("small_n1280", "mid_n16k", "paper_n128k", "large_n512k"):
        t0 = time.perf_counter()
        g, slp, dlp = I.workload(name)
        gen_s = time.perf_counter() - t0
        s = P.StokesSum(g)
        tuned = P.stokes_autotune(s.h, P.STOKES_FP32_KAHAN, repeats=3)
        ts, td = torch.as_tensor(slp, device="cuda"), torch.as_tensor(dlp, device="cuda")
        out = torch.empty((g.n_nodes, 2), dtype=torch.float64, device="cuda")
        for _ in range(3):
            P.stokes_sum_eval(s.h, P.STOKES_FP32_KAHAN, ts, td, 0.0, out)
        P.stokes_sync(s.h)
        # the sum's device time: sums issued back to back by the library (small geometries
        # replay a captured graph) ...
        ms = [P.stokes_time_sums(s.h, P.STOKES_FP32_KAHAN, ts, td, 0.0, out,
                                 reps=50 if g.n_nodes < 100000 else 5) for _ in range(5)]
        # ... the same one call at a time through the Python binding (host overhead included) ...
        call_ms = []
        for _ in range(7):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            P.stokes_sum_eval(s.h, P.STOKES_FP32_KAHAN, ts, td, 0.0, out)
            e1.record()
            torch.cuda.synchronize()
            call_ms.append(e0.elapsed_time(e1))
        graphs = P.stokes_graph_stats(s.h)
        # ... and the pair kernel alone (phase events; profiled calls launch directly)
        P.stokes_set_profiling(s.h, True)
        pair_ms = []
        for _ in range(5):
            P.stokes_sum_eval(s.h, P.STOKES_FP32_KAHAN, ts, td, 0.0, out)
            P.stokes_sync(s.h)
            pair_ms.append(P.stokes_last_timing(s.h)[1])
        P.stokes_set_profiling(s.h, False)
        pairs = P.stokes_pair_count(s.h)
        rng = np.random.default_rng(0)
        k = min(g.n_nodes, 400)
        sel = np.sort(rng.choice(g.n_nodes, k, replace=False)).astype(np.int32)
        ref = O.sum_nodes(g, slp, dlp, select=sel)
        err = rel_err_by_kind(out.cpu().numpy(), ref, g, sel)
        s.close()
        m, pm = statistics.median(ms), statistics.median(pair_ms)
        rows[name] = {"N": g.n_nodes, "pairs": pairs, "ms": m, "gpair_per_s": pairs / m / 1e6,
                      "python_call_ms": statistics.median(call_ms),
                      "graph_captures_launches": graphs,
                      "pair_ms": pm, "frac_fp32_fma_peak": FLOPS_PER_PAIR * pairs / (pm / 1e3) / 1e12 / peak,
                      "shape": {k2: tuned[k2] for k2 in ("source_splits", "targets_per_thread", "kahan_group")},
                      "rel_err_vs_oracle": err, "oracle_sample": int(k), "generation_s": gen_s}
    print(json.dumps({"metric": "FP32-Kahan node sum vs problem size", "unit": "Gpair-evals/s",
                      "n_gpus": 1, "dtype": "f32", "data": "synthetic", "results": rows}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--precision", default="fp32k", choices=["fp32k", "fp64"])
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--df-steps", type=int, default=3,
                    help="timed double-float evaluations beside the FP32-Kahan leg")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(WORKLOAD_DESCS))
    ap.add_argument("--batch", action="store_true",
                    help="time the 64-channel batched ensemble instead (separate JSON line)")
    ap.add_argument("--scaling", action="store_true",
                    help="FP32-Kahan sum from N = 1,280 to N = 524,288 (throughput, roofline, error)")
    ap.add_argument("--fmm", action="store_true",
                    help="fast multipole node evaluation vs the direct sums, N = 1,280 .. 524,288")
    ap.add_argument("--fmm-workloads", default="small_n1280,mid_n16k,paper_n128k,large_n512k")
    ap.add_argument("--fmm-leaf", type=int, default=32)
    ap.add_argument("--fmm-orders", default="20,28", help="--fmm: FP64 evaluation orders")
    ap.add_argument("--fmm-fp32-orders", default="", help="--fmm: FP32 evaluation orders")
    ap.add_argument("--fmm-vesicles-only", action="store_true",
                    help="--fmm: the vesicle curves of each workload only (the step's vesicle sums)")
    ap.add_argument("--walls", action="store_true",
                    help="wall solvers: fast direct solver vs dense LU32 at a channel's walls")
    ap.add_argument("--walls-nodes", type=int, default=16384)
    ap.add_argument("--walls-solvers", default="fds,lu32_refine")
    ap.add_argument("--poiseuille", action="store_true",
                    help="accuracy study of the pressure-driven channel (velocity and pressure)")
    ap.add_argument("--step", action="store_true",
                    help="time the semi-implicit vesicle step with the learned warm start instead")
    ap.add_argument("--step-workload", default="mid_n16k",
                    choices=["paper_n128k", "mid_n16k", "small_n1280"])
    ap.add_argument("--step-precisions", default="",
                    help="comma list of fp64, fp32k, df (default: all three; fp32k,df at N=128,768)")
    ap.add_argument("--collect-precision", default="", choices=["", "fp64", "fp32k", "df"])
    ap.add_argument("--train-runs", type=int, default=2)
    ap.add_argument("--train-steps", type=int, default=40)
    ap.add_argument("--train-epochs", type=int, default=40)
    ap.add_argument("--step-modes", default="16",
                    help="warm-start Fourier modes, one network each (e.g. 16,32)")
    ap.add_argument("--close", action="store_true",
                    help="time the close-evaluation correction on densely packed channels")
    ap.add_argument("--close-workloads", default="mid_n16k,paper_n128k")
    ap.add_argument("--close-gap", type=float, default=1.5,
                    help="vesicle gap in node spacings for --close (the other workloads use 5)")
    ap.add_argument("--close-factor", type=float, default=5.0)
    ap.add_argument("--no-warm-history", action="store_true",
                    help="warm-start features without the previous solution and its last change")
    ap.add_argument("--warm-base", default="previous", choices=["previous", "extrapolate"],
                    help="--step: what the network's predicted change is added to (and trained on)")
    ap.add_argument("--step-one", action="store_true",
                    help="one zero-guess step of the --step held-out channel after --warmup steps, "
                         "between cudaProfilerStart/Stop")
    ap.add_argument("--precond-refresh", action="store_true",
                    help="--step: refresh the preconditioner inverse by Newton-Schulz from the "
                         "previous step's instead of factorising every step")
    ap.add_argument("--precond-tensor", action="store_true",
                    help="--step: the FP32 preconditioner's GEMMs by cuBLAS's BF16x9 FP32 emulation "
                         "on the tensor cores")
    ap.add_argument("--sweep-fmm", type=int, default=0,
                    help="--step, fp32k: the Krylov sweeps' vesicle sums by the step's FMM plan at "
                         "this order (0: FP32-Kahan direct sums)")
    ap.add_argument("--residual-fmm", type=int, default=0,
                    help="FMM order of the FP64-accurate vesicle sums of FP32-Kahan steps "
                         "(0: double-float direct sums)")
    ap.add_argument("--tune-file", default=None,
                    help="shapes file of the autotuner: loaded when it exists (no tuning), "
                         "else written after tuning")
    ap.add_argument("--no-tune", action="store_true",
                    help="skip the launch-shape autotuner (wave-model default shapes)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.batch:
        return run_batch(args)
    if args.step_one:
        return run_step_one(args)
    if args.step:
        return run_step(args)
    if args.poiseuille:
        return run_poiseuille(args)
    if args.walls:
        return run_walls(args)
    if args.close:
        return run_close(args)
    if args.fmm:
        return run_fmm(args)
    if args.scaling:
        return run_scaling(args)

    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    import paper_1510_05616_gb300 as P
    from paper_1510_05616_gb300 import build as B
    from paper_1510_05616_gb300 import inputs as I
    if rank == 0:
        B.build()
    if ws > 1:
        torch.distributed.barrier()
    B.build()

    g, slp, dlp = I.workload(args.workload)
    dev = torch.device("cuda", local)
    from_file = bool(args.tune_file) and os.path.exists(args.tune_file) and not args.no_tune
    if from_file:
        P.stokes_tune_load(args.tune_file)  # the context takes its class's shape at geometry set
    s = P.StokesSum(g, device=local)
    ts = torch.as_tensor(slp, device=dev)
    td = torch.as_tensor(dlp, device=dev)
    out = torch.empty((g.n_nodes, 2), dtype=torch.float64, device=dev)
    prec = P.PRECISIONS[args.precision]
    pairs = P.stokes_pair_count(s.h)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    # launch shape: the library's autotuner times its candidates on this geometry (untimed)
    tuned = None if (args.no_tune or from_file) else P.stokes_autotune(s.h, prec, repeats=3)
    if tuned is not None and args.tune_file and rank == 0:
        P.stokes_tune_save(args.tune_file)
    launch = dict(zip(("source_splits", "targets_per_thread", "kahan_group"),
                      P.stokes_get_launch(s.h, prec)))
    launch["autotuned"] = tuned is not None or from_file
    if from_file:
        launch["shapes_file"] = os.path.basename(args.tune_file)
    if tuned is not None:
        launch["candidates"] = tuned["candidates"]
        launch["default_shape_ms"] = tuned["initial_ms"]

    # warm-up
    for _ in range(max(args.warmup, 0)):
        P.stokes_sum_eval(s.h, prec, ts, td, 0.0, out)
    P.stokes_sync(s.h)

    # timed region: K steps, each preceded by an L2 flush outside its events
    P.stokes_set_profiling(s.h, True)
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    pair_ms = []
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    for k in range(args.steps):
        flush.fill_(float(k))
        ev0[k].record(stream)
        P.stokes_sum_eval(s.h, prec, ts, td, 0.0, out)
        ev1[k].record(stream)
        pair_ms.append(P.stokes_last_timing(s.h)[1])
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    P.stokes_set_profiling(s.h, False)
    P.stokes_sync(s.h)
    step_ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    t_total = max_over_ranks(sum(step_ms) / 1e3, dev)
    value = aggregate_rate(pairs * args.steps, ws, t_total) / 1e9
    pair_avg = statistics.mean(pair_ms)
    gpu_out = out.cpu().numpy()

    # FP64 GPU path on the same inputs (the "beats FP64" comparison)
    fp64 = None
    if args.precision == "fp32k" and args.fp64_steps > 0:
        out64 = torch.empty_like(out)
        P.stokes_sum_eval(s.h, P.STOKES_FP64, ts, td, 0.0, out64)
        P.stokes_sync(s.h)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t64 = 0.0
        for _ in range(args.fp64_steps):
            flush.fill_(1.0)
            e0.record(stream)
            P.stokes_sum_eval(s.h, P.STOKES_FP64, ts, td, 0.0, out64)
            e1.record(stream)
            torch.cuda.synchronize()
            t64 += e0.elapsed_time(e1) / 1e3
        P.stokes_sync(s.h)
        fp64 = {"value": pairs * args.fp64_steps / t64 / 1e9, "unit": "Gpair-evals/s",
                "ms_per_step": 1e3 * t64 / args.fp64_steps}
        d = np.abs(gpu_out - out64.cpu().numpy()).max(0) / np.abs(out64.cpu().numpy()).max(0)
        fp64["fp32k_rel_diff_vs_fp64"] = [float(v) for v in d]

    # double-float path (FP64 accuracy on the FP32 pipes) on the same inputs
    dfl = None
    if args.precision == "fp32k" and args.df_steps > 0:
        outdf = torch.empty_like(out)
        P.stokes_sum_eval(s.h, P.STOKES_DOUBLE_FLOAT, ts, td, 0.0, outdf)
        P.stokes_sync(s.h)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tdf = 0.0
        for _ in range(args.df_steps):
            flush.fill_(1.0)
            e0.record(stream)
            P.stokes_sum_eval(s.h, P.STOKES_DOUBLE_FLOAT, ts, td, 0.0, outdf)
            e1.record(stream)
            torch.cuda.synchronize()
            tdf += e0.elapsed_time(e1) / 1e3
        P.stokes_sync(s.h)
        dfl = {"value": pairs * args.df_steps / tdf / 1e9, "unit": "Gpair-evals/s",
               "ms_per_step": 1e3 * tdf / args.df_steps}
        df_out = outdf.cpu().numpy()
        if fp64 is not None:
            o64 = out64.cpu().numpy()
            d = np.abs(df_out - o64).max(0) / np.abs(o64).max(0)
            dfl["rel_diff_vs_fp64"] = [float(v) for v in d]

    # end to end through the host-buffer C entry point (pinned host memory)
    hs = torch.as_tensor(slp).pin_memory()
    hd = torch.as_tensor(dlp).pin_memory()
    ho = torch.empty((g.n_nodes, 2), dtype=torch.float64).pin_memory()
    P.stokes_sum_eval_host(s.h, prec, hs, hd, 0.0, ho)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        P.stokes_sum_eval_host(s.h, prec, hs, hd, 0.0, ho)
    te = max_over_ranks(time.perf_counter() - t0, dev)
    e2e = {"value": aggregate_rate(pairs * args.steps, ws, te) / 1e9, "unit": "Gpair-evals/s",
           "h2d_bytes_per_step": int(hs.numel() * 8 + hd.numel() * 8),
           "d2h_bytes_per_step": int(ho.numel() * 8)}

    if rank != 0:
        s.close()
        if ws > 1:
            torch.distributed.destroy_process_group()
        return 0

    peaks, peak_kind = measured_peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    sms = device_sms(torch.cuda.current_device())
    peak_tflops = sms * LANES * 2 * sm_mhz * 1e6 / 1e12
    achieved = FLOPS_PER_PAIR * pairs / (pair_avg / 1e3) / 1e12
    traffic = profiled_traffic()
    line = {
        "metric": METRIC, "value": value, "unit": "Gpair-evals/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "fp32k" else "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESCS[args.workload], "N": g.n_nodes, "pairs_per_step": pairs,
                   "precision": args.precision, "l2": "flushed before each timed step (256 MB write)",
                   "parallelism": "replicas" if ws > 1 else "single", "launch": launch},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                     "frac": achieved / peak_tflops, "traffic": traffic,
                     "kernel": "pair_f32k_kernel" if args.precision == "fp32k" else "pair_f64_kernel",
                     "kernel_ms": pair_avg,
                     "peak_basis": "FP32 FMA peak %d SM x 128 lanes x 2 flop x sm_max_mhz (%s clocks)" % (sms, peak_kind),
                     "flops_per_pair": FLOPS_PER_PAIR},
        "e2e": e2e,
        "gpu_launches": 5 * args.steps,  # per step: self (side stream), pack, pair, 2 finish
        "clocks": clk,
        "fp64_path": fp64,
        "double_float_path": dfl,
    }
    if not args.no_cpu_baseline and ws == 1:
        sel, ref, cpairs, dt, threads = cpu_sample_oracle(g, slp, dlp, args.cpu_budget)
        line["cpu_baseline"] = {"value": cpairs / dt / 1e9, "unit": "Gpair-evals/s", "cores": threads,
                                "kind": "oracle",
                                "sample": "%d random target nodes x all %d sources x 3 images"
                                          % (len(sel), g.n_nodes)}
        line["rel_err_vs_oracle"] = rel_err_by_kind(gpu_out, ref, g, sel)
        if dfl is not None:
            dfl["rel_err_vs_oracle"] = rel_err_by_kind(df_out, ref, g, sel)
    print(json.dumps(line))
    s.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
