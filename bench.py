#!/usr/bin/env python
"""Benchmark of the radiative-transfer step: cell crossings per second.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl crash|reference]
                [--workload NAME]

One step = one whole pass of the hot path (source budget, emission, traversal
with attenuation and int64 deposition, per-cell chemistry) over the
workload's packets for one time step.  The metric is cell crossings per
second: (packet, cell) segments with positive length, counted on the device.

Timing: W untimed warm-up steps, then K steps bracketed by a barrier and
torch.cuda.synchronize(), timed with CUDA events on the library's stream;
every step moves a state far larger than L2 (or L2 is flushed between
steps, see config.l2).  With N > 1 (torchrun) every rank runs an
independent replica with its own seed (weak scaling; the step needs no
exchange between replicas) and rank 0 prints the max-over-ranks time.

--impl reference times the CPU oracle on a bounded sample of the same
workload on the host cores (the baseline arm).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell crossings/s"


# ---------------------------------------------------------------- workloads
def workload(name):
    from paper_1101_4127_gb300 import inputs, native
    if name == "hhe_bb_128":
        w = inputs.hhe_blackbody_128()
        return w, native.CRASH_FP64_PLAIN
    if name == "hhe_bb_128_mixed":       # the same workload in the mixed form
        return inputs.hhe_blackbody_128(), native.CRASH_MIXED
    if name == "stromgren_32":
        return inputs.stromgren_32(), native.CRASH_FP64_PLAIN
    if name == "lognormal_128":
        return inputs.lognormal_128(), native.CRASH_MIXED
    if name == "lognormal_128_thin":
        return inputs.lognormal_128(thin=True), native.CRASH_MIXED
    if name == "batch_64":
        return inputs.batch_64(), native.CRASH_MIXED
    if name == "lognormal_256_thin":      # profiling case: a few GB on the device
        return inputs.lognormal_512(n=256, n_src=2000, packets=4_000_000, thin=True), native.CRASH_MIXED
    if name == "lognormal_512_thin":
        return inputs.lognormal_512(thin=True), native.CRASH_MIXED
    if name == "stromgren_rec_128":      # diffuse recombination field (Test 1 set-up)
        return inputs.stromgren_rec(n=128, packets=10_000_000), native.CRASH_MIXED
    if name == "stromgren_rec_128_fp64":
        return inputs.stromgren_rec(n=128, packets=10_000_000), native.CRASH_FP64_PLAIN
    if name == "cloudy_hhe_64":          # Test-3 H+He set-up
        return inputs.cloudy_hhe(n=64), native.CRASH_MIXED
    if name == "lognormal_512_neutral":
        return inputs.lognormal_512(thin=False), native.CRASH_MIXED
    raise SystemExit(f"unknown workload {name}")


def bytes_per_crossing(box, precision):
    """Algorithmic bytes one crossing must move: the crossed cell's frozen
    absorbers (1 value for pure H, 3 with He; 8 B in FP64, 4 B in FP32) and its
    deposit payload (one int64 per species present, plus the heating counter
    when T evolves)."""
    from paper_1101_4127_gb300 import native
    he = box.he_over_h > 0
    n_abs = 3 if he else 1
    w = 8 if precision == native.CRASH_FP64_PLAIN else 4
    n_dep = (3 if he else 1) + (0 if box.isothermal else 1)
    return n_abs * w + 8 * n_dep


# ---------------------------------------------------------------- helpers
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def traffic_for(workload_name, kernel_src):
    """DRAM bytes per crossing of the transport from the committed ncu summary
    (profiles/traffic.md), if taken on the current kernel source; the row of
    the workload itself, else the row of the smaller case it names."""
    p = os.path.join(ROOT, "profiles", "traffic.md")
    if not os.path.exists(p):
        return None
    sha = hashlib.sha256(open(kernel_src, "rb").read()).hexdigest()[:12]
    for ln in open(p):
        c = [x.strip() for x in ln.strip().strip("|").split("|")]
        if len(c) >= 3 and workload_name in [x.strip() for x in c[0].split(",")] and c[1] == sha:
            try:
                return float(c[2])                # DRAM bytes per crossing
            except ValueError:
                return None
    return None


# ---------------------------------------------------------------- reference arm
_ORACLE_CACHE = {}


def oracle_sample(w, seconds=15.0):
    """Time the CPU oracle (one core) on a bounded sample of one step of the
    workload and extrapolate to the whole step.

    Transport: packet ids [0, K) of every source, K grown until the step
    takes about seconds/2 beyond a step with no packets (the fixed per-step
    cost of freezing the absorbers is timed alone and counted once, not
    scaled with the packets).  Chemistry: the per-cell update of that step on
    every S-th cell of the whole grid, with the window's deposits scaled by
    Ns/K to those of the full step, less the same step without chemistry,
    scaled by S.  Returns (crossings/s, description, seconds spent)."""
    import oracle
    box = w.boxes[0]
    P = w.packets_per_step[0]
    Ns = P // box.n_src
    ncell = int(np.prod(box.shape_xyz))
    spent = 0.0
    # one oracle grid per workload and process; every timed step starts from
    # the workload's initial state and step index
    if _ORACLE_CACHE.get("name") != w.name:
        _ORACLE_CACHE.clear()
        o = oracle.OracleGrid.from_box(box)
        fields = (oracle.F_XHII, oracle.F_XHEII, oracle.F_XHEIII, oracle.F_T)
        _ORACLE_CACHE.update(name=w.name, grid=o, state=[(f, o.read(f)) for f in fields])
    o = _ORACLE_CACHE["grid"]

    def timed_step(K):
        o.set_options(chemistry=0, pkt_begin=0, pkt_end=K)
        o.set_step_index(0)
        t0 = time.perf_counter()
        o.step(w.dt_s, P)
        t = time.perf_counter() - t0
        return t, int(o.read(oracle.F_BUDGET)[3])

    t_fixed, _ = timed_step(0)
    spent += t_fixed
    K = 1
    while True:
        t, cross = timed_step(K)
        spent += t
        t_tr = max(t - t_fixed, 1e-6)
        if t_tr > seconds / 2 or K >= Ns:
            break
        # grow at most 8x per trial: a short trial's time is mostly noise
        K = min(Ns, K * 8, max(K * 2, int(K * (seconds / 2) / t_tr)))
    # chemistry of that step alone on every stride-th cell, deposits scaled
    # to the full step (the state is put back afterwards)
    stride = max(1, ncell // 200_000)
    o.set_chem_sample(stride, Ns / K)
    t0 = time.perf_counter()
    o.chemistry(w.dt_s)
    t_chem = time.perf_counter() - t0
    spent += t_chem
    o.set_chem_sample(1, 1.0)
    for f, a in _ORACLE_CACHE["state"]:
        o.write(f, a)
    t_step = t_fixed + t_tr * (Ns / K) + t_chem * stride
    cross_step = cross * (Ns / K)
    rate = cross_step / t_step
    desc = (f"one step of {w.name}: transport of packet ids [0,{K}) of each of the {box.n_src} "
            f"sources ({cross} crossings, {t_tr:.2f} s beyond the {t_fixed:.2f} s fixed cost) scaled "
            f"to {Ns} per source, plus the per-cell update of every {stride}-th of the {ncell} cells "
            f"with the full step's deposits ({t_chem:.2f} s) scaled to all cells")
    return rate, desc, spent


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w, _prec = workload(args.workload)
    vals = []
    desc = ""
    for _ in range(args.warmup):
        oracle_sample(w, seconds=min(args.ref_seconds, 2.0))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r, desc, el = oracle_sample(w, seconds=args.ref_seconds / max(1, args.steps))
        vals.append(r)
    total = time.perf_counter() - t0
    v = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "crossings/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / max(1, args.steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "sample": desc},
            "cpu_baseline": {"value": v, "unit": "crossings/s", "cores": 1, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": v, "unit": "crossings/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- main arm
def run_crash(args):
    import torch
    from paper_1101_4127_gb300 import build, native

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
        if rank == 0:
            build.build()
        dist.barrier()
    else:
        torch.cuda.set_device(0)
        build.build()
    dev = torch.device("cuda", local)

    w, prec = workload(args.workload)
    boxes = w.boxes
    box = boxes[0]
    for bx in boxes:
        bx.seed = bx.seed + rank          # independent replica per rank
    if args.packets:
        w.packets_per_step = [max(bx.n_src, args.packets // bx.n_src * bx.n_src) for bx in boxes]
    Plist = list(w.packets_per_step)
    P = Plist[0]
    batch = len(boxes) > 1
    step_arg = Plist if batch else P
    ncell_all = sum(bx.n ** 3 for bx in boxes)
    g = native.Grid(boxes, prec)
    graph = bool(args.graph)
    pers = {"persistent": 1, "per-pass": 0}.get(args.launch, 1)
    g.set_options(timing=0 if graph else 1, use_graph=1 if graph else 0, persistent=pers,
                  reg_cap=args.reg_cap)
    stream = torch.cuda.ExternalStream(g.stream(), device=dev)
    state_bytes = ncell_all * (4 + 4 * 8 + 32 + (32 if prec == native.CRASH_FP64_PLAIN else 16))
    l2_bytes = 129 * 2**20
    flush = None
    if state_bytes < 2 * l2_bytes:
        flush = torch.empty(256 * 2**20, dtype=torch.uint8, device=dev)

    # the optically thin idealisation is held: every step starts from the thin
    # state (restored on the device inside the timed region), otherwise the
    # medium recombines step by step and stops being thin
    hold = args.workload.endswith("_thin")
    if hold:
        g.checkpoint(native.CKPT_SAVE)

    def one_step():
        if flush is not None:
            with torch.cuda.stream(stream):
                flush.fill_(1)
        if hold:
            g.checkpoint(native.CKPT_RESTORE_STATE)
        g.step(w.dt_s, step_arg)

    def totals():
        t = np.zeros(8, np.int64)
        for i in range(len(boxes)):
            t += g.read(native.F_TOTALS, i)
        return t

    tuned = None
    tuned_kw = {}
    for k in range(args.warmup):
        one_step()
        if k == 0 and prec == native.CRASH_MIXED and not args.no_autotune:
            if hold:
                g.checkpoint(native.CKPT_RESTORE_STATE)   # tune on the state that is timed
            g.sync()
            # block, crossings per pass, re-sort, register cap, tiles, key curve
            tuned = g.autotune(w.dt_s, Plist)
            if args.launch == "auto":           # the autotuner also chose the launch style
                pers = int(g.get_options()["persistent"])
            tuned_kw.update(block_size=tuned[0], seg_per_iter=tuned[1], resort_interval=tuned[2],
                            reg_cap=tuned[3], tile=tuned[4], sort_curve=tuned[5], persistent=pers)
            g.set_options(timing=0 if graph else 1, use_graph=1 if graph else 0, **tuned_kw)
    g.sync()
    if prec == native.CRASH_FP64_PLAIN:
        launch_style = "one thread per packet"
    elif g.get_options()["tile"]:
        launch_style = "tile passes"
    else:
        launch_style = "one persistent launch per step" if g.get_options()["persistent"] \
            else "one launch per pass"
    g.reset_kernel_time()
    tot0 = totals()
    launches0 = g.launch_count()
    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        one_step()
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ck = clocks.stop()
    ms = e0.elapsed_time(e1)
    tot1 = totals()
    launches = g.launch_count() - launches0
    kms, klaunches = g.kernel_time()
    if graph:      # no per-launch events inside a replayed graph: time whole steps
        kms, klaunches = ms, args.steps
    crossings = int(tot1[3] - tot0[3])
    if dist:
        t = torch.tensor([ms, float(crossings)], dtype=torch.float64, device=dev)
        tmax = t.clone()
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        tsum = t.clone()
        dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
        ms_max = float(tmax[0])
        cross_all = float(tsum[1])
    else:
        ms_max, cross_all = ms, float(crossings)
    value = cross_all / (ms_max * 1e-3)

    # roofline of the dominant (transport) kernel
    bpc = bytes_per_crossing(box, prec)
    peak, peak_kind = measured_peaks()
    achieved = (crossings * bpc) / (kms * 1e-3) / 1e9 if kms > 0 else None
    ksrc = os.path.join(ROOT, "paper_1101_4127_gb300", "csrc",
                        "k_fp64.cu" if prec == native.CRASH_FP64_PLAIN else "k_mixed.cu")
    dram_per_crossing = traffic_for(args.workload, ksrc)
    traffic = None
    if dram_per_crossing is not None and klaunches:
        # DRAM bytes of this run's average transport launch
        traffic = dram_per_crossing * crossings / klaunches

    # end-to-end through the C ABI with host buffers (pinned): every step
    # uploads its inputs (the sources, and for the held thin state the four
    # state fields), steps, and reads back the four state fields (x_HII,
    # x_HeII, x_HeIII, T) of every box and the budget
    e2e = None
    if rank == 0 and not args.no_e2e:
        g.set_options(timing=0, **tuned_kw)
        ncell = box.n ** 3
        pin = lambda dt_, n_=ncell: torch.empty(n_, dtype=dt_, pin_memory=True).numpy()
        fields = (native.F_XHII, native.F_XHEII, native.F_XHEIII, native.F_T)
        outs = [[pin(torch.float64, bx.n ** 3) for _ in fields] for bx in boxes]
        bud = np.empty(8, np.int64)
        state_in = []
        if hold:
            for val in (box.x_HII0, box.x_HeII0, box.x_HeIII0, box.T0):
                a_ = pin(torch.float64)
                a_[:] = val
                state_in.append(a_)
        nb = len(box.bin_eV)
        h2d = sum(bx.n_src for bx in boxes) * (3 + 1 + nb) * 8 + len(boxes) * nb * 8 + \
            sum(a_.nbytes for a_ in state_in)
        d2h = sum(a_.nbytes for o_ in outs for a_ in o_) + len(boxes) * bud.nbytes
        t_e2e = 0.0
        cr_e2e = 0
        n_e2e = 5
        for _ in range(n_e2e):
            g.sync()
            t0 = time.perf_counter()
            for f_, a_ in zip(fields, state_in):
                g._check(g.L.crash_write_fields(g.ctx, f_, a_.ctypes.data))
            for i_, bx in enumerate(boxes):
                g.add_sources(bx.src_pos, bx.src_ndot, bx.bin_eV, bx.bin_frac, box=i_)
            g.step(w.dt_s, step_arg)
            cr_step = 0
            for i_ in range(len(boxes)):
                for f_, a_ in zip(fields, outs[i_]):
                    g._check(g.L.crash_read_fields_box(g.ctx, i_, f_, a_.ctypes.data))
                g._check(g.L.crash_read_fields_box(g.ctx, i_, native.F_BUDGET, bud.ctypes.data))
                cr_step += int(bud[3])
            t_e2e += time.perf_counter() - t0
            cr_e2e += cr_step
        e2e = {"value": cr_e2e / t_e2e, "unit": "crossings/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "steps": n_e2e,
               "read_back": "x_HII, x_HeII, x_HeIII, T of every box, and the budget"}

    fp64 = None
    if rank == 0 and prec == native.CRASH_MIXED and not args.no_fp64 and not batch:
        # the FP64 form and the mixed form on the same inputs: the transport of
        # the same window of packet ids of every source, the same (second)
        # step from the same initial state, kernel time of each (the FP64
        # pipe of this GPU is narrow, so the window is small)
        g.close()
        g = None
        Ns = P // box.n_src
        K = max(1, min(Ns, (1 << 21) // box.n_src))

        def window_rate(precision, **opts):
            gw = native.Grid(box, precision)
            gw.set_options(chemistry=0, timing=1, pkt_begin=0, pkt_end=K, **opts)
            gw.step(w.dt_s, P)
            gw.sync()
            gw.reset_kernel_time()
            t0 = gw.read(native.F_TOTALS)
            gw.step(w.dt_s, P)
            gw.sync()
            t1 = gw.read(native.F_TOTALS)
            ms_w, _ = gw.kernel_time()
            gw.close()
            return float(t1[3] - t0[3]) / (ms_w * 1e-3), int(t1[3] - t0[3])

        r64, c64 = window_rate(native.CRASH_FP64_PLAIN)
        rmx, cmx = window_rate(native.CRASH_MIXED, **{k: v for k, v in tuned_kw.items()})
        fp64 = {"value": r64, "unit": "crossings/s",
                "sample": f"transport of packet ids [0,{K}) of each of the {box.n_src} sources, "
                          f"second step, kernel time", "crossings": c64,
                "mixed_same_sample": {"value": rmx, "unit": "crossings/s", "crossings": cmx},
                "mixed_over_fp64": rmx / r64}

    # a batch against the same boxes stepped one at a time, each in its own
    # context (the launches of every box's step issued in turn; host clock
    # around K steps of all boxes, the device synchronised on both sides)
    one_by_one = None
    if rank == 0 and batch and args.one_by_one:
        if g is not None:
            g.close()
            g = None
        singles = []
        for bx, pb in zip(boxes, Plist):
            gs = native.Grid(bx, prec)
            gs.set_options(use_graph=1 if graph else 0, **{k: v for k, v in tuned_kw.items()})
            gs.step(w.dt_s, pb)
            singles.append((gs, pb))
        for gs, _ in singles:
            gs.sync()
        c0 = sum(int(gs.read(native.F_TOTALS)[3]) for gs, _ in singles)
        l0 = sum(gs.launch_count() for gs, _ in singles)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            for gs, pb in singles:
                gs.step(w.dt_s, pb)
        for gs, _ in singles:
            gs.sync()
        t_one = time.perf_counter() - t0
        c1 = sum(int(gs.read(native.F_TOTALS)[3]) for gs, _ in singles)
        l1 = sum(gs.launch_count() for gs, _ in singles)
        for gs, _ in singles:
            gs.close()
        one_by_one = {"value": (c1 - c0) / t_one, "unit": "crossings/s",
                      "ms_per_step": 1e3 * t_one / args.steps,
                      "launches_per_step": (l1 - l0) / args.steps,
                      "how": f"{len(boxes)} contexts, one per box, stepped in turn (host clock)"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r, desc, _ = oracle_sample(w, seconds=args.ref_seconds)
        cpu = {"value": r, "unit": "crossings/s", "cores": 1, "kind": "oracle", "sample": desc}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "crossings/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == native.CRASH_FP64_PLAIN else "f32+i64",
            "data": "synthetic",
            "config": {"workload": w.name,
                       "grid": [bx.n for bx in boxes] if batch else box.n,
                       "sources": sum(bx.n_src for bx in boxes),
                       "packets_per_step": sum(Plist), "bins": len(box.bin_eV),
                       "cuda_graph": graph,
                       "transport_launch": launch_style,
                       "precision": "fp64" if prec == native.CRASH_FP64_PLAIN else "mixed",
                       "l2": "flushed between steps (256 MiB write)" if flush is not None
                             else "state larger than L2",
                       "state": "thin state restored on the device before every step (timed)"
                                if hold else "evolving from the initial state",
                       "parallelism": f"replicas{world}"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": (achieved / peak) if achieved else None,
                         "traffic": traffic, "peak_kind": peak_kind,
                         "kernel": "whole step (graph replay)" if graph else "transport",
                         "bytes_per_crossing": bpc,
                         "kernel_ms_per_launch": kms / max(1, klaunches)},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "fp64_plain": fp64,
            "one_by_one": one_by_one,
            "autotuned": {"block": tuned[0], "crossings_per_pass": tuned[1],
                          "resort_interval": tuned[2], "reg_cap": tuned[3],
                          "tile": tuned[4], "sort_curve": ["morton", "hilbert"][tuned[5]]}
                         if tuned else None,
            "gpu_launches": int(launches),
            "clocks": ck,
            "crossings_per_step": crossings / args.steps,
            "transport_ms_per_step": kms / args.steps,
            "chem_substeps_per_cell": float(tot1[7] - tot0[7]) / (args.steps * ncell_all),
        }
        if any(getattr(bx, "f_rec", 0.0) > 0 for bx in boxes):
            # diffuse recombination field: re-emission packets traced per step
            # beyond the sources' packets
            line["config"]["f_rec"] = max(getattr(bx, "f_rec", 0.0) for bx in boxes)
            line["reemitted_packets_per_step"] = (float(tot1[4] - tot0[4]) / args.steps
                                                  - float(sum(Plist)))
        print(json.dumps(line), flush=True)
    if g is not None:
        g.close()
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="crash", choices=["crash", "reference"])
    ap.add_argument("--workload", default="lognormal_512_thin")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--graph", action="store_true", help="replay each step as a CUDA graph")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--ref-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--packets", type=int, default=0, help="override packets per step (small cases)")
    ap.add_argument("--reg-cap", type=int, default=0, choices=[0, 1],
                    help="without autotuning: 1 = transport kernels capped at 64 registers")
    ap.add_argument("--one-by-one", action="store_true",
                    help="batched workloads: also time the same boxes stepped one at a time")
    ap.add_argument("--launch", default="auto", choices=["auto", "persistent", "per-pass"],
                    help="transport launch style: one persistent launch per step, one launch per "
                         "wavefront pass, or (auto) the autotuner's choice (persistent when not tuned)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_crash(args)


if __name__ == "__main__":
    main()
