"""Benchmark of the coupled LB + rigid-RBC time step on GB300.

Default workload: the largest single-GPU configuration, a straight tube of
radius 120 in a 256^3 box (11,582,464 fluid nodes, periodic along z) with
51,846 cells (hematocrit 0.45 of the lumen), driven by the axial force
density that gives a wall shear rate of 1e-4 in plain plasma, FP32
populations in the compact layout.  One step is one full coupled step: cell
list + Gay-Berne forces, per-cell sampling + rigid update + spreading, and
the fused lattice pass.

Prints one JSON line (rank 0): value = fluid-node updates per second over all
ranks (MLUPS) from CUDA events around K graph-launched steps, with live
per-kernel event timing of the lattice pass for the roofline, nvidia-smi clock
samples taken during the timed region, the end-to-end figure through the
public API with host buffers (init from host arrays, K steps, fields read
back; the init time beside it), the FP64 oracle timed on a bounded sample on
the host, and (``serving``) the batched request server on the serving mix at
full step counts against the plain FP32 single-instance path.

``--impl reference`` times the oracle (plain FP64 CPU implementation) on the
same workload and prints the same line with ``"impl": "reference"``.
Multi-GPU (torchrun): every rank runs an independent replica of the
workload (the step has no exchange between replicas); value = sum of
node updates / max time over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1107_4889_gb300 import workloads as wl  # noqa: E402

METRIC = "coupled-step MLUPS"
UNIT = "MLUPS"
L2_BYTES = 129e6


PREC_NAME = {"f32": "FP32", "f16": "binary16", "bf16": "bfloat16"}


def _prec_name(precision, rounding="stochastic"):
    return PREC_NAME[precision] + ("" if precision == "f32" else f" ({rounding} rounding)")


def _workload(name, precision="f32", planes=20, rounding="stochastic"):
    if name == "channel":
        g, c, p = wl.channel_workload()
        desc = "walled channel 64x64x256, 3650 RBC (H=0.35), G=5.376e-7"
    elif name == "box32":
        g, c, p = wl.box_workload()
        desc = "periodic box 32^3, 32 RBC (H=0.098), G=1e-6"
    elif name == "ybif":
        g, c, p = wl.ybif_workload()
        desc = (f"Y-bifurcation in 512^3 (parent r=60, daughters r=45 at +-35 deg), {wl.fluid_count(g)} fluid nodes "
                f"(node list), {len(c['pos'])} RBC (H={len(c['pos']) * wl.CELL_VOLUME / wl.fluid_count(g):.2f} of the "
                f"lumen, slot-limited), inlet Poiseuille u_max={g['inlet_umax']}, pressure outlets")
    elif name in ("box256", "box128"):
        L = int(name[3:])
        g = wl.periodic_box(L, body_force=(1e-6, 0.0, 0.0))
        c, p = None, wl.params()
        desc = f"periodic box {L}^3, fluid only, G=1e-6"
    elif name == "tube":
        g, c, p = wl.tube_workload()
        desc = (f"tube r=120 in 256^3, {len(c['pos'])} RBC (H={wl.tube_hematocrit(g, len(c['pos'])):.2f} "
                f"of the lumen), G_z={g['body_force'][2]:.3e}")
    elif name == "tube_slab":
        g, c, p = wl.tube_slab(nz=planes)
        desc = (f"slab of the tube: r=120 in 256x256x{g['nz']} (periodic z), {len(c['pos'])} RBC, "
                f"G_z={g['body_force'][2]:.3e}")
    else:
        raise SystemExit(f"unknown workload {name}")
    p = dict(p, precision=precision)
    if precision != "f32":
        p["rounding"] = rounding
    return g, c, p, f"{desc}, {_prec_name(precision, rounding)} populations"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _barrier_and_max(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64,
                     device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if f[5 + k].lower() in ("active", "0x1", "1"):
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def _lb_source_hash():
    h = hashlib.sha256()
    for f in ("lb.cu", "rbc_device.cuh"):
        with open(os.path.join(ROOT, "paper_1107_4889_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _profiled_lb(workload, precision="f32"):
    """From the committed ncu summary of the lattice pass, if it was taken on
    the current kernel source: DRAM bytes per launch and the launch's time
    alone (serialised under ncu, default launch shape, in us; None when the
    summary gives none).  None when there is no current summary."""
    path = os.path.join(ROOT, "profiles", f"lb_pass_{workload}.md")
    if precision != "f32":
        path = os.path.join(ROOT, "profiles", f"lb_pass_{workload}_{precision}.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m_hash = re.search(r"source_sha256_16:\s*([0-9a-f]{16})", txt)
    m_bytes = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    m_us = re.search(r"alone_us_per_launch:\s*([0-9.eE+]+)", txt)
    if not m_hash or not m_bytes or m_hash.group(1) != _lb_source_hash():
        return None
    return {"traffic": float(m_bytes.group(1)), "alone_us": float(m_us.group(1)) if m_us else None,
            "summary": os.path.relpath(path, ROOT)}


def _profiled_traffic(workload, precision="f32"):
    """DRAM bytes per lattice-pass launch from the committed ncu summary, if
    it was taken on the current kernel source; else None."""
    prof = _profiled_lb(workload, precision)
    return prof["traffic"] if prof else None


def _algorithmic_bytes_per_node(geom, params, has_cells=True):
    # populations 19 x e B read + written (e = 4 FP32, 2 for the 16-bit
    # stores); u (3) written; with cells, G (3) and theta (1) read and sigma
    # (6) written when the elongational torque is on; the node's solid flag
    # (1 B) on walled lattices
    e = 4 if params.get("precision", "f32") == "f32" else 2
    b = 2 * 19 * e + 3 * 4
    if has_cells:
        b += 4 * 4
        if params.get("alpha_tt", 0.04) != 0.0:
            b += 6 * 4
    if geom["solid"] is not None:
        b += 1
    return b


def _cpu_sample(name, precision):
    """The bounded sample of a workload the oracle is timed on: the whole
    workload, except for the tube, whose oracle step takes about a minute
    (and whose cell-wall search is brute force over 193,000 wall particles
    per cell): there a 20-plane slab of it, the same cross-section, drive
    and cell density."""
    return _workload("tube_slab" if name == "tube" else name, precision)


def _oracle_rate(geom, cells, params, budget_s):
    """Run the FP64 oracle for about budget_s seconds; returns (MLUPS, steps, seconds)."""
    from oracle import oracle as orc
    nf = wl.fluid_count(geom)
    o = orc.Oracle(geom, cells, params)
    t0 = time.perf_counter()
    o.step(1)
    t1 = time.perf_counter()
    steps = 1
    per = t1 - t0
    more = int(max(0, budget_s - per) / per)
    if more:
        o.step(more)
        steps += more
    dt = time.perf_counter() - t0
    o.close()
    return nf * steps / dt / 1e6, steps, dt


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    geom, cells, params, desc = _workload(args.workload, args.precision, args.planes, args.rounding)
    nf = wl.fluid_count(geom)
    sg, sc, sp, sdesc = _cpu_sample(args.workload, args.precision)
    rate, steps, dt = _oracle_rate(sg, sc, sp, args.reference_budget)
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / steps * nf / wl.fluid_count(sg),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": desc, "fluid_nodes": nf, "cells": 0 if cells is None else len(cells["pos"])},
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{steps} coupled steps of {sdesc} ({dt:.1f} s), "
                                   f"capped by a {args.reference_budget:.0f} s budget"},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch

    from paper_1107_4889_gb300 import build as B
    from paper_1107_4889_gb300.rbc import Solver

    ws, rank, local = _dist()
    # the device first, so that NCCL binds each rank's communicator to its own GPU
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    if rank == 0:
        B.build()
    _barrier(ws)
    geom, cells, params, desc = _workload(args.workload, args.precision, args.planes, args.rounding)
    if args.layout != "auto":
        params = dict(params, layout=args.layout)
        desc += f", {args.layout} layout"
    if args.node_list:
        params = dict(params, node_list=args.node_list)
        desc += ", node-list pass" if args.node_list > 0 else ", row-staged pass"
    if args.no_cells and cells is not None:
        cells, desc = None, desc + ", cells removed"
    nf = wl.fluid_count(geom)
    N = geom["nx"] * geom["ny"] * geom["nz"]

    s = Solver(geom, cells, params)
    s.step(args.warmup)
    # the launch shape of the lattice pass (ring depth, CTAs per SM) picked
    # by timing real steps of this solve
    tune = s.autotune(args.tune_steps) if args.tune_steps > 0 else None
    # capture the timed step graphs now, outside the timed region
    s.set_timing(1)
    s.set_timing(0)
    torch.cuda.synchronize()
    st = s.stats()

    # timed region: K graph-launched steps in 8 chunks; the first eighth of
    # each chunk runs the step graphs with event nodes around the kernels
    # (live timing of the lattice pass and the per-cell kernel, sampled over
    # the whole region), the rest the plain graphs
    clocks = Clocks(local)
    stream = s.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    nchunk = min(8, args.steps)
    sizes = [args.steps // nchunk + (1 if c < args.steps % nchunk else 0) for c in range(nchunk)]
    kms, kcount = np.zeros(2), np.zeros(2, dtype=np.int64)
    _barrier(ws)
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    e0.record(stream)
    for n_c in sizes:
        s.set_timing(max(1, n_c // 8))
        s.step(n_c)
        k_ms, k_cnt = s.kernel_times()
        kms += k_ms
        kcount += k_cnt
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    _barrier(ws)
    ms = e0.elapsed_time(e1)
    st2 = s.stats()
    launches = s.launches_per_step() * args.steps
    ws_bytes = s.workspace_bytes
    s.close()
    ms_max = _barrier_and_max(ms, ws)
    value = nf * args.steps * ws / (ms_max * 1e-3) / 1e6

    # end to end through the public API with host buffers; the set-up
    # (rbc_init: host tables, uploads, graph capture, the first cell list)
    # is timed on its own as well
    _barrier(ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s2 = Solver(geom, cells, params)
    torch.cuda.synchronize()
    init_s = time.perf_counter() - t0
    s2.step(args.steps)
    f = s2.fields()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    layout = s2.layout()
    s2.close()
    e2e_s = _barrier_and_max(e2e_s, ws)
    init_s = _barrier_and_max(init_s, ws)
    n = 0 if cells is None else len(cells["pos"])
    h2d = (0 if geom["solid"] is None else N) + n * (3 + 4 + 3 + 3) * 8
    d2h = N * 8 + N * 3 * 8 + n * 13 * 8
    e2e = {"value": nf * args.steps * ws / e2e_s / 1e6, "unit": UNIT,
           "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
           "init_s": init_s, "steps_s": e2e_s - init_s,
           "note": "job = init from host arrays (init_s) + K steps + fields read back"}
    assert np.isfinite(f["u"]).all()

    if rank != 0:
        return
    lb_ms = kms[0] / max(kcount[0], 1)
    bpn = _algorithmic_bytes_per_node(geom, params, n > 0)
    peak, peak_kind = _peaks()
    achieved = bpn * nf / (lb_ms * 1e-3) / 1e9
    # the committed summaries profile the pass with cells
    prof = _profiled_lb(args.workload, args.precision) if n > 0 else None
    traffic = prof["traffic"] if prof else None
    roof = {"kernel": "lattice pass (k_lb)", "bound": "hbm", "achieved": achieved, "peak": peak,
            "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
            "peak_source": f"{peak_kind} hbm_gbs", "bytes_per_fluid_node": bpn,
            "lb_ms_per_launch": lb_ms, "cell_work_ms_per_step": kms[1] / max(kcount[1], 1)}
    if prof and prof["alone_us"]:
        # the same pass with nothing beside it (the step's live launch shares
        # the SMs with the cell kernels that the graph runs next to it)
        a_gbs = bpn * nf / (prof["alone_us"] * 1e-6) / 1e9
        roof["alone"] = {"us_per_launch": prof["alone_us"], "achieved": a_gbs, "frac": a_gbs / peak,
                         "how": f"serialised under ncu, default launch shape ({prof['summary']})"}

    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        sg, sc, sp, sdesc = _cpu_sample(args.workload, args.precision)
        rate, csteps, cdt = _oracle_rate(sg, sc, sp, args.cpu_budget)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{csteps} coupled steps of {sdesc} ({cdt:.1f} s, one core)"}
    serving = None
    if ws == 1 and not args.no_serve:
        serving = serve_measure(args)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "f32" else f"f32 ({args.precision} storage)", "data": "synthetic",
        "config": {"workload": desc, "nodes": N, "fluid_nodes": nf, "cells": n,
                   "layout": "compact" if layout["compact"] else "dense", "stored_entries": layout["entries"],
                   "parallelism": "replicas" if ws > 1 else "single GPU",
                   "l2": f"inputs larger than L2: per-step working set "
                         f"{ws_bytes / 1e6:.0f} MB > {L2_BYTES / 1e6:.0f} MB",
                   "steps_per_s": args.steps / (ms_max * 1e-3),
                   "lattice_launch": None if tune is None else
                   {"stages": tune["stages"], "ctas_per_sm": tune["ctas_per_sm"],
                    "lattice_first": tune["lattice_first"],
                    "shape_list_blocks_per_sm": tune["wt_blocks_per_sm"],
                    "gay_berne_blocks_per_sm": tune["gb_blocks_per_sm"], "particle_bin_scale": tune["bin_scale"],
                    "spread_split": tune["split_spread"], "autotuned": True}},
        "clocks": clk, "e2e": e2e, "gpu_launches": launches, "roofline": roof, "cpu_baseline": cpu,
        "budget": {"mass_drift_rel": (st2["mass"] - st["mass"]) / st["mass"], "max_u": st2["max_u"],
                   "gb_clamps": st2["gb_clamps"]},
        "serving": serving,
    }
    print(json.dumps(line), flush=True)


def run_serve(args):
    """The serving measurement alone, as its own JSON line."""
    import torch

    from paper_1107_4889_gb300 import build as B

    B.build()
    torch.cuda.set_device(0)
    line = serve_measure(args)
    line = {"metric": "batched serving solves/s (binary16, continuous batching)", "value": line["solves_per_s"],
            "unit": "solves/s", "n_gpus": 1, "higher_is_better": True, "data": "synthetic", **line}
    print(json.dumps(line), flush=True)


def serve_measure(args):
    """Batched serving of the request stream: solves/s and p50/p99
    time-to-result of the binary16 request server (continuous batching,
    Poisson arrivals at 0.8 of its measured capacity) against the plain FP32
    single-instance path (the same requests one after another through
    Solver), and the per-request work-rate (effective viscosity) error of
    binary16 against FP32."""
    import torch

    from paper_1107_4889_gb300.rbc import Server, Solver

    reqs16 = wl.serving_stream(args.serve_requests, precision="f16", step_scale=args.serve_step_scale)
    n = len(reqs16)

    def serve(reqs, arrivals=None):
        srv = Server(int(args.serve_arena_gb * 2 ** 30), max_active=args.serve_slots, tick_steps=args.serve_tick)
        torch.cuda.synchronize()
        t0 = srv.clock()
        order = list(range(len(reqs))) if arrivals is None else list(np.argsort(arrivals))
        k, res = 0, []
        while True:
            now = srv.clock() - t0
            while k < len(order) and (arrivals is None or arrivals[order[k]] <= now):
                g, c, p, steps, info = reqs[order[k]]
                srv.submit(g, c, p, steps, steps // 2, tag=int(order[k]))
                k += 1
            a, q = srv.poll()
            res += srv.results()
            if a == 0 and q == 0 and k == len(order):
                break
            if a == 0 and q == 0:
                time.sleep(1e-4)
        res += srv.results()
        makespan = max(r["t_done"] for r in res) - t0
        srv.close()
        res.sort(key=lambda r: r["tag"])
        return res, makespan

    # plain FP32 single instance: the same requests, one after another
    nseq = min(n, args.serve_baseline_requests)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    p32 = []
    for g, c, p, steps, info in reqs16[:nseq]:
        s = Solver(g, c, dict(p, precision="f32"))
        acc = []
        for done in range(0, steps, args.serve_tick):
            s.step(min(args.serve_tick, steps - done))
            st = s.stats()
            if done + args.serve_tick >= steps // 2:
                acc.append(st["power"])
        p32.append(float(np.mean(acc)))
        s.close()
    torch.cuda.synchronize()
    seq_rate = nseq / (time.perf_counter() - t0)

    # closed loop (all submitted at once): capacity of the batched server
    res_cl, span_cl = serve(reqs16)
    capacity = n / span_cl
    # open loop: Poisson arrivals at 0.8 of capacity
    rng = np.random.default_rng(wl.SEED_BASE + 40)
    arrivals = np.cumsum(rng.exponential(1.0 / (0.8 * capacity), n))
    res_ol, span_ol = serve(reqs16, arrivals)
    ttr = np.array([r["t_done"] - r["t_submit"] for r in res_ol])
    errs = [abs(res_cl[k]["mean_power"] / p32[k] - 1.0) for k in range(nseq)]
    fluid = [wl.fluid_count(g) * steps for g, c, p, steps, i in reqs16]
    return {
        "solves_per_s": capacity,
        "config": {"workload": f"{n} requests: boxes {list(wl.SERVING_BOXES)}, periodic (Kolmogorov drive) or walled "
                               f"(uniform drive), hematocrit U[0.1,0.5] (slot-limited), shear rate logU[1e-5,1e-3], "
                               f"steps U[2000,10000] x {args.serve_step_scale}, binary16 populations",
                   "requests": n, "steps_total": int(sum(st for _, _, _, st, _ in reqs16)),
                   "slots": args.serve_slots, "tick_steps": args.serve_tick},
        "fp32_single_instance": {"value": seq_rate, "unit": "solves/s", "requests": nseq},
        "speedup_vs_fp32_single": capacity / seq_rate,
        "mlups_batched": float(np.sum(fluid)) / span_cl / 1e6,
        "open_loop": {"arrival_rate": 0.8 * capacity, "p50_s": float(np.percentile(ttr, 50)),
                      "p99_s": float(np.percentile(ttr, 99)), "makespan_s": span_ol},
        "viscosity_error_vs_fp32": {"max": float(np.max(errs)), "median": float(np.median(errs)),
                                    "within_1pct": int(np.sum(np.array(errs) < 0.01)), "of": nseq},
        "failed": int(sum(r["status"] != 0 for r in res_cl + res_ol)),
    }


def run_stats(args):
    """Long-run statistics of the channel workload (64 x 64 x 256, 3,650
    cells, hematocrit 0.35): eta_rel = P_0 / P_H (time-averaged work rate of
    the uniform drive without and with cells, i.e. the flow rate ratio
    Q_0 / Q_H) and the near-wall hematocrit profile (cell centres in 1-lu
    bins of y, time-averaged, as the local volume fraction V_cell count /
    (n_x n_z)), each with FP32 and with binary16 populations; samples every
    100 steps over the second half of --steps."""
    import torch

    from paper_1107_4889_gb300 import build as B
    from paper_1107_4889_gb300.rbc import Solver

    B.build()
    torch.cuda.set_device(0)
    every = 100
    res = {}
    for prec in ("f32", "f16"):
        out = {}
        for with_cells in (False, True):
            geom, cells, params, desc = _workload("channel", prec, rounding=args.rounding)
            s = Solver(geom, cells if with_cells else None, params)
            powers, done = [], 0
            t0 = time.perf_counter()
            while done < args.steps:
                s.step(every)
                done += every
                if done > args.steps // 2:
                    powers.append(s.stats()["power"])
                    if with_cells:
                        s.profile_accumulate(1)
            out["P_H" if with_cells else "P_0"] = float(np.mean(powers))
            if with_cells:
                prof = s.profile()[0]
                out["profile"] = prof * wl.CELL_VOLUME / (geom["nx"] * geom["nz"])
                out["samples"] = len(powers)
            out["s_" + ("H" if with_cells else "0")] = time.perf_counter() - t0
            s.close()
        out["eta_rel"] = out["P_0"] / out["P_H"]
        res[prec] = out
    a, b = res["f32"], res["f16"]
    ny = len(a["profile"])
    core = a["profile"][ny // 4: 3 * ny // 4].mean()

    def cfl(prof):
        # distance from the wall plane y = 0.5 to the first bin whose local
        # hematocrit reaches half the core value, averaged over both walls
        d = []
        for side in (prof, prof[::-1]):
            k = int(np.argmax(side >= 0.5 * core))
            d.append(k - 0.5)
        return float(np.mean(d))

    line = {"metric": f"channel long-run statistics, {_prec_name('f16', args.rounding)} vs FP32", "workload": desc,
            "steps": args.steps, "samples": a["samples"], "sample_every": every,
            "eta_rel": {"f32": a["eta_rel"], "f16": b["eta_rel"], "rel_diff": b["eta_rel"] / a["eta_rel"] - 1.0},
            "near_wall_hematocrit": {"f32": [round(float(v), 4) for v in a["profile"][:12]],
                                     "f16": [round(float(v), 4) for v in b["profile"][:12]],
                                     "core_mean_f32": float(core),
                                     "profile_l1_rel": float(np.abs(b["profile"] - a["profile"]).sum() /
                                                             a["profile"].sum())},
            "cell_free_layer_lu": {"f32": cfl(a["profile"]), "f16": cfl(b["profile"])},
            "seconds": {k: res[k]["s_0"] + res[k]["s_H"] for k in res}}
    print(json.dumps(line), flush=True)


def run_tank_treading(args):
    """The tank-treading test of Sec. 3 (E2), in a Kolmogorov flow: one cell
    at a plane where the plasma velocity u_x = U sin(2 pi y / n) vanishes
    and its shear rate is largest (the paper shears with Lees-Edwards
    boundaries, which it only cites; near that plane the flow is simple shear
    to within the curvature of the profile over the cell, cos(2 pi a / n) =
    0.92 for a = 4 in n = 64).  The cell starts with its short (symmetry)
    axis in the shear plane, 10 degrees off the gradient direction.  For each
    coefficient alpha of the elongational torque (Eq. pheno_torque_diss) the
    short axis' angle phi in the shear plane is sampled; the cell tumbles if
    phi advances by more than a quarter turn over the second half of the
    run, else it holds a fixed inclination, reported as the angle of its
    long axis in the shear plane to the flow direction (mean over the last
    quarter).  The paper finds the transition at alpha = 0.063 with an
    inclination of about 40 degrees (20-35 degrees in a bounded slab)."""
    import torch

    from paper_1107_4889_gb300 import build as B
    from paper_1107_4889_gb300.rbc import RbcError, Solver

    B.build()
    torch.cuda.set_device(0)
    n, rate, steps, every = 64, 1e-3, args.steps, 200
    # the paper's range, then up to where the elongational torque can match
    # the vorticity-driven one (gamma_R I omega~ under the App. A integrator)
    alphas = [0.0, 0.04, 0.063, 0.1, 1.0, 10.0, 30.0, 100.0, 300.0, 1000.0]
    nu = (wl.PAPER_PARAMS["tau0"] - 0.5) / 3.0
    geom = wl.periodic_box(n, body_force_wave=(wl.kolmogorov_amplitude(n, rate, nu), 0.0, 0.0))
    # short axis in the shear plane at 80 degrees from the flow: body z to lab
    # x (a quarter turn about y), then 80 degrees about z
    a, b = math.radians(80.0) / 2, math.pi / 4
    q0 = np.array([[math.cos(a) * math.cos(b), -math.sin(a) * math.sin(b), math.cos(a) * math.sin(b),
                    math.sin(a) * math.cos(b)]])
    rows = []
    for alpha in alphas:
        cells = wl.cells_dict(np.array([[n / 2 + 0.2, n / 2, n / 2 + 0.3]]), q0)
        p = wl.params(alpha_tt=alpha)
        s = Solver(geom, cells, p)
        phis, ratios, done = [], [], 0
        try:
            while done < steps:
                s.step(every)
                done += every
                w, x, y, z = s.fields(rho=False, u=False)["quat"][0]
                e = np.array([2 * (x * z + w * y), 2 * (y * z - w * x), 1 - 2 * (x * x + y * y)])  # lab short axis
                phis.append(math.atan2(e[1], e[0]))
                if done > steps // 2:
                    dg = s.cell_diag()
                    # elongational torque against the vorticity-driven one,
                    # gamma_R I omega~ (z: the vorticity axis)
                    ratios.append(abs(dg["T_S"][0, 2]) /
                                  max(p["gamma_R"] * p["inertia"][2] * abs(dg["omega_s"][0, 2]), 1e-30))
        except RbcError as err:
            # a strong elongational torque, spread back as force density,
            # drives the lattice past the Mach guard
            rows.append({"alpha": alpha, "unstable_at_step": done, "error": str(err)[:60]})
            s.close()
            continue
        s.close()
        phi = np.unwrap(np.array(phis))
        half = len(phi) // 2
        turn = float(phi[-1] - phi[half])
        tumbling = abs(turn) > math.pi / 2
        # long axis in the shear plane: perpendicular to the short axis
        incl = np.degrees(np.angle(np.exp(2j * (phi[3 * len(phi) // 4:] - math.pi / 2))) / 2.0)
        rows.append({"alpha": alpha, "tumbling": bool(tumbling),
                     "turns_second_half": turn / (2 * math.pi),
                     "inclination_deg": None if tumbling else float(np.mean(np.abs(incl))),
                     "torque_ratio_TS_over_vorticity": float(np.mean(ratios))})
    steady = [r["alpha"] for r in rows if r.get("tumbling") is False]
    line = {"metric": "tank-treading test (Sec. 3): tumbling or fixed inclination vs alpha",
            "workload": f"one cell, {n}^3 periodic box, Kolmogorov flow with peak shear rate {rate}, cell at its "
                        f"zero-velocity plane, {steps} steps per alpha",
            "paper": {"transition_alpha": 0.063, "inclination_deg": 40, "bounded_slab_deg": [20, 35]},
            "transition_alpha": min(steady) if steady else None, "runs": rows}
    print(json.dumps(line), flush=True)


def run_mobility(args):
    """The mobility test of Sec. 3: one cell (M = 10, I = 1000, no viscosity
    contrast) in a 60^3 periodic box of quiescent fluid, pushed by a constant
    external force (the counter-force spread uniformly over the fluid keeps
    the total momentum at zero) or turned by a constant external torque.
    The terminal velocity (angular velocity), averaged over the last third
    of the run, over the push is the mobility mu; against the bare mobility
    1 / (M gamma_T) (1 / (I gamma_R)) it is a line whose intercept at
    infinite friction is the mesh-induced mobility the paper reports
    (1 / (M gamma_T^mesh) = 6.6 frontal, 10.3 side-wise; gamma_R^mesh =
    1/44 about the smallest radius, 1/38 about the largest).  Frontal: push
    along the short axis; side-wise: along a long axis."""
    import torch

    from paper_1107_4889_gb300 import build as B
    from paper_1107_4889_gb300.rbc import Solver

    B.build()
    torch.cuda.set_device(0)
    L, steps = 60, args.steps
    N = L ** 3
    gammas = [0.05, 0.1, 0.2, 0.4, 0.8]
    base = dict(delta=0.0, alpha_tt=0.0)
    if args.mobility_xi_half:
        # the alternative reading of the shape-function radii: xi = a / 2
        base["xi"] = tuple(0.5 * a for a in wl.PAPER_PARAMS["semi_axes"])
    out = {}
    cases = {"frontal": ("force", 2), "side": ("force", 0), "spin_smallest_radius": ("torque", 2),
             "spin_largest_radius": ("torque", 0)}
    for name, (kind, axis) in cases.items():
        rows = []
        for g in gammas:
            push = np.zeros(3)
            push[axis] = 1e-5 if kind == "force" else 1e-3
            cells = wl.cells_dict(np.array([[30.2, 29.7, 30.4]]), np.array([[1.0, 0.0, 0.0, 0.0]]))
            cells["force_ext" if kind == "force" else "torque_ext"] = push[None, :]
            geom = wl.periodic_box(L, body_force=tuple(-push / N) if kind == "force" else (0.0, 0.0, 0.0))
            p = wl.params(**base, gamma_T=g, gamma_R=g)
            s = Solver(geom, cells, p)
            vals = []
            done, chunk = 0, 100
            while done < steps:
                s.step(chunk)
                done += chunk
                if done > 2 * steps // 3:
                    f = s.fields(rho=False, u=False)
                    vals.append(f["vel"][0, axis] if kind == "force" else f["omega"][0, axis])
            s.close()
            mu = float(np.mean(vals)) / push[axis]
            bare = 1.0 / ((p["mass"] if kind == "force" else p["inertia"][axis]) * g)
            rows.append((g, bare, mu))
        bare = np.array([r[1] for r in rows])
        mu = np.array([r[2] for r in rows])
        slope, icpt = np.polyfit(bare, mu, 1)
        out[name] = {"gamma": gammas, "mu": [float(m) for m in mu], "bare_mobility": [float(b) for b in bare],
                     "slope": float(slope), "intercept_mesh_mobility": float(icpt)}
        if kind == "force":
            out[name]["gamma_mesh"] = float(1.0 / (p["mass"] * icpt))
            out[name]["a_T_mesh"] = float(1.0 / icpt / (6 * np.pi / 6.0))
        else:
            gm = 1.0 / (p["inertia"][axis] * icpt)
            out[name]["gamma_R_mesh"] = float(gm)
            out[name]["a_R_mesh"] = float((p["inertia"][axis] * gm / (8 * np.pi / 6.0)) ** (1.0 / 3.0))
    line = {"metric": "mobility of one cell vs friction (Sec. 3 mobility test)",
            "workload": f"one cell, 60^3 periodic box, M=10, I=1000, delta=0, xi={tuple(base.get('xi', wl.PAPER_PARAMS['xi']))}, "
                        f"{steps} steps per point",
            "paper": {"frontal": 6.6, "side": 10.3, "gamma_R_mesh_smallest": 1 / 44, "gamma_R_mesh_largest": 1 / 38},
            **out}
    print(json.dumps(line), flush=True)


def run_wss_map(args):
    """Time-averaged wall-shear-stress map of the workload (ybif by default)
    with binary16 storage against the FP32 run of the same seed: --steps
    coupled steps each, the stress sampled every 20 steps over the second
    half; prints relative L2 and percentiles of the magnitude difference and
    the MLUPS of both runs."""
    import torch

    from paper_1107_4889_gb300 import build as B
    from paper_1107_4889_gb300.rbc import Solver

    B.build()
    torch.cuda.set_device(0)
    name = args.workload if args.workload != "channel" else "ybif"
    res = {}
    for prec in ("f32", "f16"):
        geom, cells, params, desc = _workload(name, prec)
        nf = wl.fluid_count(geom)
        s = Solver(geom, cells, params)
        s.step(args.warmup)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        done = 0
        while done < args.steps:
            k = min(20, args.steps - done)
            s.step(k)
            done += k
            if done >= args.steps // 2:
                s.wss_accumulate()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        nodes, tau, samples = s.wss()
        st = s.stats()
        s.close()
        res[prec] = dict(mag=np.linalg.norm(tau[np.argsort(nodes)], axis=1), mlups=nf * args.steps / dt / 1e6,
                         samples=samples, max_u=st["max_u"], desc=desc)
    a, b = res["f16"]["mag"], res["f32"]["mag"]
    rel = np.abs(a - b) / np.maximum(b, 1e-3 * b.max())
    line = {"metric": "wall-shear-stress map, binary16 vs FP32", "workload": res["f32"]["desc"],
            "steps": args.steps, "samples": res["f32"]["samples"], "wall_nodes": int(len(b)),
            "rel_l2": float(np.linalg.norm(a - b) / np.linalg.norm(b)),
            "rel_median": float(np.median(rel)), "rel_p99": float(np.percentile(rel, 99)),
            "mean_wss_f32": float(b.mean()), "mean_wss_f16": float(a.mean()),
            "mlups_f32": res["f32"]["mlups"], "mlups_f16": res["f16"]["mlups"],
            "max_u": [res["f32"]["max_u"], res["f16"]["max_u"]]}
    print(json.dumps(line), flush=True)


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["channel", "box32", "tube", "tube_slab", "box256", "box128", "ybif"],
                    default="tube")
    ap.add_argument("--wss-map", action="store_true",
                    help="wall-shear-stress map of the workload, binary16 against FP32")
    ap.add_argument("--mobility", action="store_true", help="mobility of one cell against the friction rates")
    ap.add_argument("--mobility-xi-half", action="store_true", help="mobility test with xi = semi-axes / 2")
    ap.add_argument("--tank-treading", action="store_true",
                    help="tank-treading test: tumbling or fixed inclination of one cell in shear vs alpha")
    ap.add_argument("--stats", action="store_true",
                    help="relative viscosity and near-wall hematocrit of the channel, binary16 against FP32")
    ap.add_argument("--planes", type=int, default=20, help="planes of the tube_slab workload")
    ap.add_argument("--no-cells", action="store_true", help="drop the workload's cells (lattice pass alone)")
    ap.add_argument("--layout", choices=["auto", "dense", "compact"], default="auto",
                    help="storage layout of the lattice fields (auto: compact for sparse walled lattices)")
    ap.add_argument("--node-list", type=int, default=0, choices=[-1, 0, 1],
                    help="lattice pass over a fluid-node list (1), whole rows (-1), or the library's choice (0)")
    ap.add_argument("--precision", choices=["f32", "f16", "bf16"], default="f32")
    ap.add_argument("--rounding", choices=["stochastic", "nearest"], default="stochastic",
                    help="rounding of the 16-bit population stores")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tune-steps", type=int, default=50,
                    help="steps per launch shape the autotuner times during warm-up (0: no tuning)")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--reference-budget", type=float, default=60.0)
    ap.add_argument("--serve", action="store_true", help="batched-serving benchmark instead of the step benchmark")
    ap.add_argument("--no-serve", action="store_true", help="leave the serving measurement out of the step line")
    ap.add_argument("--serve-requests", type=int, default=48)
    ap.add_argument("--serve-step-scale", type=float, default=1.0)
    ap.add_argument("--serve-baseline-requests", type=int, default=8)
    ap.add_argument("--serve-slots", type=int, default=48)
    ap.add_argument("--serve-tick", type=int, default=100)
    ap.add_argument("--serve-arena-gb", type=float, default=64.0)
    return ap.parse_args(argv)


def main():
    args = parse_args()
    if args.serve:
        run_serve(args)
        return
    if args.wss_map:
        run_wss_map(args)
        return
    if args.stats:
        run_stats(args)
        return
    if args.tank_treading:
        run_tank_treading(args)
        return
    if args.mobility:
        run_mobility(args)
        return
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
