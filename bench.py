#!/usr/bin/env python3
"""Benchmark of the RPY matvec hot path on GB300.

One step = the whole hot path on one system resident in HBM: bounding cube,
Morton keys, radix sort, adaptive octree, U/V/W/X lists (tree build), then
the matvec (P2P near field, upward pass, plane-wave M2X / X2X / X2L, P2L,
downward pass, L2P + W-list M2P + Eq. (2.8) combine, unpermute).

Default workload: 1,000,000 beads, 90% on a sphere surface of radius 0.5 and
10% uniform in the unit cube, a = 1e-4, forces N(0,1), kT/(6 pi eta a) = 1,
FP64, 6-digit setting (rel-L2 <= 1e-6 against the FP64 oracle).

Multi-GPU: replicas only (every rank runs its own copy of the system; the
method needs no exchange between independent systems), weak scaling.

--impl reference times the CPU oracle (direct O(N^2) FP64 sum) on a bounded
sample of targets of the same workload.

Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RPY matvec Mbeads/s at rel-L2 <=1e-3 (3-digit) / <=1e-6 (6-digit) vs FP64 oracle"
CONFIGS = {
    "sphere1m_6digit_fp64": dict(gen="config2", digits=6, precision=0, leaf_cap=0,
                                 desc="1,000,000 beads: sphere surface r=0.5 + 10% uniform cube, a=1e-4, "
                                      "6-digit, FP64"),
    "sphere1m_9digit_fp64": dict(gen="config2", digits=9, precision=0, leaf_cap=0,
                                 desc="1,000,000 beads: sphere surface r=0.5 + 10% uniform cube, a=1e-4, "
                                      "9-digit, FP64 (the paper's third accuracy setting)"),
    # the paper's other timed workloads (Sec. 4.3, 512 Cray XC30 nodes): 15M cube at 6 and 9
    # digits, 8M sphere surface at 3, 6 and 9 digits (Mbeads/s = N / time)
    "cube15m_6digit_fp64": dict(gen="config3", digits=6, precision=0, leaf_cap=0, paper_mbeads_s=15.787,
                                desc="15,000,000 beads uniform cube, a=2e-5, 6-digit, FP64"),
    "cube15m_9digit_fp64": dict(gen="config3", digits=9, precision=0, leaf_cap=0, paper_mbeads_s=12.185,
                                desc="15,000,000 beads uniform cube, a=2e-5, 9-digit, FP64"),
    "sphere8m_3digit_fp64": dict(gen="sphere8m", digits=3, precision=0, leaf_cap=0, paper_mbeads_s=18.448,
                                 desc="8,000,000 beads uniform on a sphere surface, a=1e-4, 3-digit, FP64"),
    "sphere8m_6digit_fp64": dict(gen="sphere8m", digits=6, precision=0, leaf_cap=0, paper_mbeads_s=5.310,
                                 desc="8,000,000 beads uniform on a sphere surface, a=1e-4, 6-digit, FP64"),
    "sphere8m_9digit_fp64": dict(gen="sphere8m", digits=9, precision=0, leaf_cap=0, paper_mbeads_s=1.912,
                                 desc="8,000,000 beads uniform on a sphere surface, a=1e-4, 9-digit, FP64"),
    "cube4096_3digit_fp64": dict(gen="config1", digits=3, precision=0, leaf_cap=40,
                                 desc="4,096 beads uniform cube, a=0.004, 3-digit, FP64, leaf cap 40"),
    "cube15m_3digit_fp32": dict(gen="config3", digits=3, precision=1, leaf_cap=0,
                                desc="15,000,000 beads uniform cube, a=2e-5, 3-digit, FP32 precision form"),
    # paper_mbeads_s: the paper's own figure for this workload (15M cube, 3 digits, FP64:
    # 0.666 s on 512 Cray XC30 nodes, Sec. 4.3), the denominator of vs_baseline
    "cube15m_3digit_fp64": dict(gen="config3", digits=3, precision=0, leaf_cap=0, paper_mbeads_s=22.5,
                                desc="15,000,000 beads uniform cube, a=2e-5, 3-digit, FP64 (the FP32 precision "
                                     "form of the same workload is measured beside it)"),
    "sphere200k_6digit_fp64": dict(gen="sphere200k", digits=6, precision=0, leaf_cap=0,
                                   desc="200,000 beads: sphere surface + 10% cube (seed 2), a=1e-4, 6-digit, FP64 "
                                        "(small case for ncu captures)"),
    "sphere200k_6digit_fp32": dict(gen="sphere200k", digits=6, precision=1, leaf_cap=0,
                                   desc="200,000 beads: sphere surface + 10% cube (seed 2), a=1e-4, 6-digit, FP32 "
                                        "precision form (small case for ncu captures)"),
    "cube2m_3digit_fp32": dict(gen="cube2m", digits=3, precision=1, leaf_cap=0,
                               desc="2,000,000 beads uniform cube (seed 3), a=2e-5, 3-digit, FP32 precision form "
                                    "(small case of the 15M cube's near field for ncu captures: ~60 beads per leaf)"),
    "batch24_3digit_fp32": dict(gen="config4_24", digits=3, precision=1, leaf_cap=0,
                                desc="24 systems in one forest drawn like the 256-system batch (seed 4), 3-digit, "
                                     "FP32 precision form (small case for ncu captures)"),
    "batch256_3digit_fp32": dict(gen="config4", digits=3, precision=1, leaf_cap=0,
                                 desc="256 systems in one forest, sizes log-uniform 1e3..2e5 (seed 4), uniform "
                                      "cube or Plummer cluster, a=0.5/N^(1/3), 3-digit, FP32 precision form"),
}
DEFAULT = "sphere1m_6digit_fp64"


def replica_value(n_per_rank, ms_local, ws, device=None):
    """Whole-job rate of N independent replicas: every rank times its own
    system; the step time is the maximum over ranks (all_reduce MAX after a
    barrier), the value counts every rank's beads.  Returns (Mbeads/s, ms)."""
    ms = float(ms_local)
    if ws > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.barrier()
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ws * n_per_rank / (ms * 1e-3) / 1e6, ms


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


class Forest:
    """Many systems concatenated (caller order = system order)."""

    def __init__(self, systems):
        self.systems = systems
        self.pos = np.concatenate([sy.pos for sy in systems])
        self.f = np.concatenate([sy.f for sy in systems])
        self.off = np.concatenate([[0], np.cumsum([sy.n for sy in systems])]).astype(np.int64)
        self.a_list = [sy.a for sy in systems]
        self.s_list = [sy.s for sy in systems]
        self.n = int(self.off[-1])


def make_workload(name):
    import synth
    gen = CONFIGS[name]["gen"]
    if gen == "sphere200k":
        return synth.sphere_plus_cube(200000, 2, 1e-4)
    if gen == "config4_24":
        return Forest(synth.config4(nsys=24))
    if gen == "cube2m":
        return synth.uniform_cube(2000000, 3, 2e-5)
    w = getattr(synth, gen)()
    return Forest(w) if isinstance(w, list) else w


def host_cpu():
    """The host the CPU baseline ran on: model name, online cores, cores in this
    process's affinity mask."""
    model = platform.processor() or platform.machine()
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"model": model, "nproc": os.cpu_count(), "affinity": len(os.sched_getaffinity(0))}


def run_ours(args, ws, rank, local, config=None, steps=None, warmup=None, profile=True):
    import torch
    import paper_1711_02976_gb300 as rp

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    config = config or args.config
    steps = steps or args.steps
    warmup = args.warmup if warmup is None else warmup
    cfg = CONFIGS[config]
    sysm = make_workload(config)
    forest = isinstance(sysm, Forest)
    n = sysm.n
    P = torch.from_numpy(sysm.pos).to(dev)
    F = torch.from_numpy(sysm.f).to(dev)
    U = torch.empty_like(F)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (129 MB)
    off = sysm.off if forest else [0, n]
    a_list = sysm.a_list if forest else [sysm.a]
    s_list = sysm.s_list if forest else [sysm.s]
    tune = None
    prec = cfg["precision"]
    bp = {"leaf_cap": cfg["leaf_cap"], "order_p": 0, "direct_w": 0, "direct_x": 0, "quad": 0}
    if getattr(args, "params", None):
        vals = [int(v) for v in args.params.split(",")]
        bp = dict(zip(("leaf_cap", "order_p", "direct_w", "direct_x", "quad"), vals))
    elif args.autotune:
        # parameter search (untimed): order p, leaf capacity and direct-substitution
        # thresholds, by sampled-target error against the GPU direct sum and timed matvecs
        tune = rp.rpy_autotune(P, off, a_list, F, s_list, cfg["digits"], cfg["precision"])
        bp = {k: tune["best"][k] for k in ("leaf_cap", "order_p", "direct_w", "direct_x", "quad")}
        prec = tune["best"]["precision"]   # an FP32 choice that fails verification falls back to FP64
    tree = rp.rpy_forest_build(P, off, a_list, cfg["digits"], precision=prec, **bp)
    matvec = lambda: rp.rpy_forest_matvec(tree, F, s_list, U)

    for _ in range(warmup):
        rp.rpy_tree_update_positions(tree, P)
        matvec()
    torch.cuda.synchronize()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    launches0 = rp.rpy_launch_count()
    times, tb, tm = [], [], []
    for _ in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        rp.rpy_tree_update_positions(tree, P)
        e1.record(stream)
        matvec()
        e2.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e2))
        tb.append(e0.elapsed_time(e1))
        tm.append(e1.elapsed_time(e2))
    launches = (rp.rpy_launch_count() - launches0) // max(1, steps)
    clocks = sampler.stop()
    value, ms = replica_value(n, sum(times) / len(times), ws, dev)
    stats = rp.rpy_tree_stats(tree)

    # repeated matvecs on the resident tree (the Krylov use), replayed as a CUDA graph: median of 20
    reps = []
    for _ in range(20):
        flush.zero_()
        torch.cuda.synchronize()
        e1, e2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e1.record(stream)
        matvec()
        e2.record(stream)
        torch.cuda.synchronize()
        reps.append(e1.elapsed_time(e2))
    stage_ms = {}
    if profile:
        rp.rpy_tree_set_profiling(tree, True)
        prof = []
        for _ in range(3):
            flush.zero_()
            matvec()
            prof.append(rp.rpy_tree_stage_times(tree))
        rp.rpy_tree_set_profiling(tree, False)
        stage_ms = {k: statistics.median(p[k] for p in prof) for k in prof[0]}
    matvec()
    torch.cuda.synchronize()
    u_dev = U.cpu().numpy()

    result = {
        "metric": METRIC, "value": round(value, 4), "unit": "Mbeads/s", "n_gpus": ws, "steps": steps,
        "warmup": warmup, "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": (round(value / cfg["paper_mbeads_s"], 4) if cfg.get("paper_mbeads_s") else None),
        "dtype": "f64" if prec == 0 else "f32+f64",
        "data": "synthetic (seeded numpy; shapes of the paper's sphere/cube workloads)",
        "config": {"workload": config, "description": cfg["desc"], "n_beads": n, "digits": cfg["digits"],
                   "precision": "fp64" if prec == 0 else "fp32", "parallelism": f"replicas x{ws}",
                   "l2": "flushed between timed steps (256 MB write)", "step": "tree build + matvec",
                   "leaf_cap": stats["leaf_cap"], "order_p": stats["order_p"], "exp_terms": stats["exp_terms"],
                   "direct_w": bp["direct_w"], "direct_x": bp["direct_x"], "quad_rule": stats["quad"],
                   "params": "autotuned" if tune is not None else ("fixed" if getattr(args, "params", None)
                                                                    else "defaults")},
        "build_ms": round(statistics.median(tb), 4), "matvec_ms": round(statistics.median(tm), 4),
        "matvec_only_mbeads_s": round(ws * n / (statistics.median(tm) * 1e-3) / 1e6, 4),
        "resident_tree_matvec_ms": round(statistics.median(reps), 4),
        "resident_tree_matvec_mean5_ms": round(sum(reps[:5]) / 5, 4),   # the paper's mean of 5
        "stages_ms": {k: round(v, 4) for k, v in stage_ms.items()},
        "tree": {k: stats[k] for k in ("n_systems", "n_boxes", "n_leaves", "depth", "u_pairs", "d_pairs", "n_wlist",
                                       "n_xlist", "n_dlist", "max_leaf_count", "leaves_over_cap", "device_bytes")},
        "gpu_launches": int(launches), "clocks": clocks,
        "autotune": None if tune is None else {
            "chosen": dict(bp, precision="fp64" if prec == 0 else "fp32"), "est_rel_l2": tune["est_rel_l2"],
            "goal": tune["goal"], "tune_ms": round(tune["tune_ms"], 1), "n_trials": len(tune["trials"]),
            "samples": 256, "verify_rel_l2": tune["verify_rel_l2"], "n_verify": tune["n_verify"],
            "verify_ok": tune["verify_ok"],
            "method": "per plane-wave rule, smallest p with sampled error <= goal; fastest (rule, p); then leaf cap "
                      "and direct thresholds by timed matvecs; verified on 1,024 fresh targets (half in the two "
                      "deepest leaf levels) at 0.5 x bound"},
    }
    work = rp.rpy_tree_work(tree)
    tree.close()
    return result, sysm, u_dev, stats, stage_ms, work


# DRAM bytes per bead of the FP64 near-field launch (the merged pass over U lists and
# direct substitutes, k_p2p), from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum) of the 200,000-bead sphere + cube workload at 6 digits, FP64
# (bench.py --config sphere200k_6digit_fp64): 10,747,648 B per launch.  The traffic is
# the sources' positions and forces, so it grows with the bead count; it is reported
# only for that kernel.
P2P64_DRAM_BYTES_PER_BEAD = 10747648.0 / 200000.0


def hbm_peak_gbs():
    """Measured copy bandwidth of the GB300s (MEASURED_PEAKS.json, written by the
    driver next to this file), else the profiling recipe's fallback figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured (MEASURED_PEAKS.json: STREAM-style copy)"
    except Exception:
        return 6800.0, "fallback (6.8 TB/s, one earlier GB300 measurement)"


def roofline(precision, stage_ms, work, peaks, n_beads=None):
    """Roofline of the dominant stage (largest time) and the fractions of every stage.
    work[stage] = (algorithmic FLOPs, algorithmic DRAM bytes) of one matvec on the tree
    (rpy_tree_work); the achieved rates divide them by the stage's CUDA-event time.  A
    stage's bound is the roof it is closer to: the FP64 or FP32 FMA peak measured on
    this GPU (rpy_alu_peak) or the measured HBM copy bandwidth."""
    hbm, hbm_src = hbm_peak_gbs()
    alu = peaks["fp64"] if precision == "fp64" else peaks["fp32"]
    per = {}
    for k, ms in stage_ms.items():
        fl, by = work.get(k, (0.0, 0.0))
        if ms <= 0:
            continue
        fa = fl / (ms * 1e-3) / alu if fl else 0.0
        fh = by / (ms * 1e-3) / 1e9 / hbm if by else 0.0
        per[k] = {"ms": round(ms, 4), "frac_alu": round(fa, 4), "frac_hbm": round(fh, 4)}
    top = max(stage_ms, key=lambda k: stage_ms[k])
    fl, by = work[top]
    t = stage_ms[top] * 1e-3
    fa, fh = fl / t / alu, by / t / 1e9 / hbm
    if fa >= fh:
        out = {"kernel": top, "bound": "alu", "achieved": round(fl / t / 1e12, 4), "peak": round(alu / 1e12, 4),
               "unit": "TFLOP/s", "frac": round(fa, 4),
               "peak_source": f"measured {precision.upper()} FMA-chain probe on this GPU (rpy_alu_peak)"}
    else:
        out = {"kernel": top, "bound": "hbm", "achieved": round(by / t / 1e9, 1), "peak": hbm, "unit": "GB/s",
               "frac": round(fh, 4), "peak_source": hbm_src}
    out["algorithmic"] = {"flops": fl, "bytes": by, "stage_ms": round(stage_ms[top], 4)}
    out["traffic"] = None
    if top == "p2p" and precision == "fp64" and n_beads:
        out["traffic"] = round(P2P64_DRAM_BYTES_PER_BEAD * n_beads)
        out["traffic_note"] = ("dram__bytes_read.sum + dram__bytes_write.sum of k_p2p per bead from an ncu capture "
                               "of the 200k-bead sphere (6 digits, FP64), scaled by bead count")
    out["stages"] = per
    return out


def e2e_host(args, sysm, cfg, bp=None, precision=None):
    """The same work through the C ABI with host buffers, every step: one call of
    rpy_tree_matvec_host on the resident tree with page-locked host arrays, which copies
    the positions to the device, rebuilds the tree for them, copies the forces, applies
    the matvec and copies the velocities back (the Brownian-dynamics / serving step).
    The tree is built once before the timed steps."""
    import torch
    import paper_1711_02976_gb300 as rp
    n = sysm.n
    pos_h = torch.from_numpy(sysm.pos).pin_memory().numpy()
    f_h = torch.from_numpy(sysm.f).pin_memory().numpy()
    u_h = torch.empty((n, 3), dtype=torch.float64).pin_memory().numpy()
    forest = isinstance(sysm, Forest)
    off = sysm.off if forest else [0, n]
    a_list = sysm.a_list if forest else [sysm.a]
    s_list = sysm.s_list if forest else [sysm.s]
    kw = bp if bp is not None else {"leaf_cap": cfg["leaf_cap"]}
    P = torch.from_numpy(sysm.pos).cuda()
    tree = rp.rpy_forest_build(P, off, a_list, cfg["digits"],
                               precision=cfg["precision"] if precision is None else precision, **kw)
    del P
    call = lambda: rp.rpy_tree_matvec_host(tree, pos_h, f_h, s_list, u_h)
    for _ in range(2):
        call()
    ts = []
    for _ in range(max(2, min(args.steps, 5))):
        t0 = time.perf_counter()
        call()
        ts.append(time.perf_counter() - t0)
    tree.close()
    t = statistics.median(ts)
    return {"value": round(n / t / 1e6, 4), "unit": "Mbeads/s", "h2d_bytes_per_step": 2 * n * 3 * 8,
            "d2h_bytes_per_step": n * 3 * 8, "ms_per_step": round(t * 1e3, 3),
            "api": "per step one rpy_tree_matvec_host call (C ABI, page-locked host arrays): H2D positions, "
                   "tree rebuild, H2D forces, matvec, D2H velocities, on the resident tree"}


def cpu_oracle_sample(sysm, k):
    """Oracle velocities on k sampled targets (for a forest: spread over the
    systems, each against its own system)."""
    import oracle
    import synth
    th = oracle.default_threads()
    if isinstance(sysm, Forest):
        rng = np.random.default_rng(12345)
        pick = rng.choice(len(sysm.systems), min(len(sysm.systems), 32), replace=False)
        per = max(1, k // len(pick))
        tg, refs, dt = [], [], 0.0
        for j in sorted(pick):
            sy = sysm.systems[j]
            loc = synth.sample_targets(sy.n, per)
            t0 = time.perf_counter()
            refs.append(oracle.rpy_direct(sy.pos, sy.f, sy.a, sy.s, targets=loc, threads=th))
            dt += time.perf_counter() - t0
            tg.append(sysm.off[j] + loc)
        return np.concatenate(tg), np.concatenate(refs), dt, th
    # small systems (the 4,096-bead case) are checked and timed in full
    tg = np.arange(sysm.n, dtype=np.int64) if sysm.n <= 5000 else synth.sample_targets(sysm.n, k)
    t0 = time.perf_counter()
    ref = oracle.rpy_direct(sysm.pos, sysm.f, sysm.a, sysm.s, targets=tg, threads=th)
    dt = time.perf_counter() - t0
    return tg, ref, dt, th


def self_term(sysm, tg):
    if isinstance(sysm, Forest):
        sysid = np.searchsorted(sysm.off, tg, side="right") - 1
        c = np.array([sysm.s_list[j] / (6 * math.pi * sysm.a_list[j]) for j in sysid])
        return c[:, None] * sysm.f[tg]
    return sysm.s / (6 * math.pi * sysm.a) * sysm.f[tg]


def precision_form(args, local, sysm_cfg):
    """The FP32 precision form on the same workload and digit setting."""
    cfg = dict(CONFIGS[sysm_cfg])
    name = sysm_cfg + "__fp32"
    CONFIGS[name] = dict(cfg, precision=1, desc=cfg["desc"].replace("FP64", "FP32 precision form"))
    res, sysm, u, stats, stage_ms, work = run_ours(args, 1, 0, local, config=name, steps=3, warmup=2, profile=True)
    return res, sysm, u, stage_ms, work


class ServeClient:
    """Client of the serving loop for the resident systems of the serving workload:
    request data (jittered positions, fresh N(0,1) forces) drawn before any timing, a
    few variants per system, so that the arrival process is not held up by random-number
    generation; velocities land in page-locked buffers; a collector thread waits for the
    requests in submission order and hands their velocity buffers back."""

    def __init__(self, systems, srv, variants=2, seed=55):
        import torch
        rng = np.random.default_rng(seed)
        # the server copies positions and forces into its own page-locked buffers at submit
        self.systems, self.srv = systems, srv
        self.data = [[(np.ascontiguousarray(synth_jitter(rng, sy.pos)), rng.standard_normal(sy.pos.shape))
                      for _ in range(variants)] for sy in systems]
        self.free_u = [[] for _ in systems]
        self.lock = threading.Lock()

    def _u(self, k):
        import torch
        with self.lock:
            if self.free_u[k]:
                return self.free_u[k].pop()
        return torch.empty(self.systems[k].pos.shape, dtype=torch.float64).pin_memory().numpy()

    def run(self, order, rate, rng):
        """Submit one request per entry of `order` (system indices): back to back when
        rate is 0, else at Poisson arrivals of `rate` per second.  Returns the wall time
        from the first submit to the last completion and per-request records."""
        import paper_1711_02976_gb300 as rp
        import queue
        q = queue.Queue()
        recs = []

        def collect():
            while True:
                item = q.get()
                if item is None:
                    return
                rid, k, u = item
                st, lat, tm = rp.rpy_server_wait_times(self.srv, rid)
                recs.append((st, lat, k, tm))
                with self.lock:
                    self.free_u[k].append(u)

        th = threading.Thread(target=collect, daemon=True)
        th.start()
        t0 = time.perf_counter()
        t_next = t0
        for r, k in enumerate(order):
            sy = self.systems[k]
            pos, f = self.data[k][r % len(self.data[k])]
            u = self._u(k)
            if rate:
                t_next += rng.exponential(1.0 / rate)
                while time.perf_counter() < t_next:
                    time.sleep(0.0002)
            q.put((rp.rpy_server_submit(self.srv, k, pos, f, sy.s, u), k, u))
        q.put(None)
        th.join()
        return time.perf_counter() - t0, recs


def synth_jitter(rng, pos):
    import synth
    return synth.jitter(rng, pos)


def serving(args, local, loads=(0.7,), n_req=None):
    """Serving form: requests from the 64 resident systems of the serving workload
    (sizes log-uniform 1e4..2e6 beads, cube or sphere, jittered positions and fresh
    forces per request, 3-digit FP32 / 6-digit FP64 alternating by system), admitted by
    device-memory footprint, four worker slots.  Measures (1) every system's request
    alone (the serial bound: beads / sum of solo latencies, and the kernel-only bound
    from the device time of each solo request's rebuild and matvec), (2) a closed loop
    (all requests submitted at once) and (3) Poisson arrivals at a fraction of the
    closed-loop capacity, with p50 / p99 latency and per-phase times."""
    import torch
    import paper_1711_02976_gb300 as rp
    import synth
    torch.cuda.set_device(local)
    n_req = n_req or args.serve_requests or 1000
    systems = synth.config5(nsys=args.serve_systems)
    srv = rp.rpy_server_create(slots=args.serve_slots)
    for k, sy in enumerate(systems):
        d, prec = (3, 1) if k % 2 == 0 else (6, 0)
        rp.rpy_server_add_system(srv, sy.pos, sy.a, d, precision=prec)
    cl = ServeClient(systems, srv)
    rng = np.random.default_rng(56)
    nsys = len(systems)
    # warm every system (its first admission builds its tree), then each request alone
    cl.run(list(range(nsys)), 0, rng)
    solo = {}
    for k in range(nsys):
        _, recs = cl.run([k], 0, rng)
        st, lat, _, tm = recs[0]
        solo[k] = (lat, tm["build_ms"] + tm["matvec_ms"], tm)
    beads = np.array([sy.n for sy in systems], dtype=np.float64)
    serial_bound = beads.sum() / sum(v[0] for v in solo.values()) / 1e3
    kernel_bound = beads.sum() / sum(v[1] for v in solo.values()) / 1e3

    def summarise(wall, recs):
        ok = [r for r in recs if r[0] == 0]
        lat = np.array([r[1] for r in ok])
        nb = sum(systems[r[2]].n for r in ok)
        ph = {key: round(float(np.mean([r[3][key] for r in ok])), 3) for key in
              ("queue_ms", "run_ms", "h2d_ms", "build_ms", "matvec_ms", "d2h_ms")}
        return {"requests": len(recs), "failed": len(recs) - len(ok), "req_s": round(len(recs) / wall, 3),
                "Mbeads_s": round(nb / wall / 1e6, 3), "p50_ms": round(float(np.percentile(lat, 50)), 2),
                "p99_ms": round(float(np.percentile(lat, 99)), 2), "mean_phase_ms": ph}

    order = [int(x) for x in rng.integers(nsys, size=max(256, n_req // 4))]
    wall, recs = cl.run(order, 0, rng)
    closed = summarise(wall, recs)
    cap = closed["req_s"]
    out = {"workload": f"{nsys} resident systems, log-uniform 1e4..2e6 beads (seed 5), half cube / half sphere, "
                       "a = 0.5 N^(-1/3); per request jittered positions (sigma 1e-3) and fresh N(0,1) forces; "
                       "3-digit FP32 and 6-digit FP64 systems alternating",
           "unit": "Mbeads/s", "systems": nsys, "total_beads": int(beads.sum()), "slots": args.serve_slots,
           "serial_bound_Mbeads_s": round(serial_bound, 3), "kernel_bound_Mbeads_s": round(kernel_bound, 3),
           "closed_loop": closed,
           "closed_loop_vs_serial_bound": round(closed["Mbeads_s"] / serial_bound, 3),
           "closed_loop_vs_kernel_bound": round(closed["Mbeads_s"] / kernel_bound, 3), "loads": []}
    for frac in loads:
        order = [int(x) for x in rng.integers(nsys, size=n_req)]
        wall, recs = cl.run(order, frac * cap, rng)
        out["loads"].append(dict(load=frac, **summarise(wall, recs)))
    out["server"] = {k: v for k, v in rp.rpy_server_stats_get(srv).items() if k in
                     ("completed", "failed", "evictions", "rebuilds", "peak_resident_bytes", "resident_systems")}
    rp.rpy_server_destroy(srv)
    return out


def serve(args, local):
    out = serving(args, local, loads=(0.3, 0.5, 0.7, 0.9), n_req=args.serve_requests or 2000)
    out.update({"mode": "serve", "metric": "served RPY matvec Mbeads/s (mixed 3-digit FP32 / 6-digit FP64)"})
    return out


def bd(args, local):
    """Brownian-dynamics form: Ermak-McCammon steps (drift D F and Lanczos D^{1/2} xi on the
    resident tree, then the rebuild for the new positions) on the default workload, with the
    autotuned parameters; fresh N(0,1) forces and xi every step."""
    import torch
    import paper_1711_02976_gb300 as rp
    torch.cuda.set_device(local)
    cfg = CONFIGS[args.config]
    sysm = make_workload(args.config)
    forest = isinstance(sysm, Forest)
    n = sysm.n
    off = sysm.off if forest else [0, n]
    a_list = sysm.a_list if forest else [sysm.a]
    s_list = sysm.s_list if forest else [sysm.s]
    P = torch.from_numpy(sysm.pos).cuda()
    F = torch.from_numpy(sysm.f).cuda()
    tune = rp.rpy_autotune(P, off, a_list, F, s_list, cfg["digits"], cfg["precision"])
    bp = {k: tune["best"][k] for k in ("leaf_cap", "order_p", "direct_w", "direct_x", "quad")}
    tree = rp.rpy_forest_build(P, off, a_list, cfg["digits"], precision=tune["best"]["precision"], **bp)
    rng = torch.Generator(device="cuda").manual_seed(77)
    a0 = float(np.min(a_list))
    kT, eta = 1.0, 1.0 / (6 * math.pi * a0)   # kT/eta = 6 pi a: D_ii = 1 for the smallest bead
    dt = 1e-3 * a0 * a0                        # rms step sqrt(2 dt) ~ 0.045 a
    tol = 1e-3   # relative change of the Lanczos noise vector between steps
    its, ts = [], []
    for k in range(args.warmup + args.steps):
        F.normal_(generator=rng)
        xi = torch.randn(P.shape, dtype=torch.float64, device="cuda", generator=rng)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        it = rp.rpy_bd_step(tree, P, F, xi, kT, eta, dt, m_max=60, tol=tol)
        torch.cuda.synchronize()
        if k >= args.warmup:
            ts.append(time.perf_counter() - t0)
            its.append(it)
    t = statistics.median(ts)
    return {"mode": "bd", "metric": "Ermak-McCammon steps/s (drift + Lanczos noise + rebuild)",
            "value": round(1.0 / t, 4), "unit": "steps/s", "ms_per_step": round(t * 1e3, 2),
            "Mbead_steps_per_s": round(n / t / 1e6, 4), "lanczos_iters_median": statistics.median(its),
            "lanczos_tol": tol, "dt": dt, "n_beads": n, "workload": args.config, "params": bp,
            "matvecs_per_step": 1 + statistics.median(its)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default=DEFAULT, choices=sorted(CONFIGS))
    ap.add_argument("--targets", type=int, default=2000, help="oracle sample for the CPU baseline / error")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the FP32 precision-form measurement")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="build with the default leaf capacity / order instead of the autotuner's choice")
    ap.add_argument("--params", default=None,
                    help="fixed build parameters leaf_cap,order_p,direct_w,direct_x,quad (no autotuning), "
                         "e.g. to profile the autotuned configuration")
    ap.add_argument("--mode", default="bench", choices=["bench", "serve", "bd"])
    ap.add_argument("--serve-systems", type=int, default=64)
    ap.add_argument("--serve-requests", type=int, default=None,
                    help="requests per arrival rate (default: 1,000 in the default run's serving object, "
                         "2,000 per rate with --mode serve)")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement of the default run")
    ap.add_argument("--serve-slots", type=int, default=4)
    args = ap.parse_args()
    ws, rank, local = _dist()
    if ws > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    if args.impl == "reference":
        if rank != 0:
            return
        sysm = make_workload(args.config)
        k = max(1, min(args.targets, 400))
        for _ in range(max(0, min(args.warmup, 1))):
            cpu_oracle_sample(sysm, 16)
        ts = []
        for _ in range(args.steps):
            tg, ref, dt, th = cpu_oracle_sample(sysm, k)
            ts.append(dt)
        t = sum(ts) / len(ts)
        v = k / t / 1e6
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": round(v, 6), "unit": "Mbeads/s",
                          "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": round(t * 1e3, 3), "higher_is_better": True, "scaling": "weak",
                          "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                          "config": {"workload": args.config, "description": CONFIGS[args.config]["desc"]},
                          "cpu_baseline": {"value": round(v, 6), "unit": "Mbeads/s", "cores": th, "kind": "oracle",
                                           "host": host_cpu(),
                                           "sample": f"{k} targets x all {sysm.n} sources per step; extrapolated "
                                                     f"O(N^2) direct rate"},
                          "e2e": {"value": round(v, 6), "unit": "Mbeads/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}), flush=True)
        return
    if args.mode == "serve":
        if rank == 0:
            print(json.dumps(serve(args, local)), flush=True)
        return
    if args.mode == "bd":
        if rank == 0:
            print(json.dumps(bd(args, local)), flush=True)
        return
    result, sysm, u_dev, stats, stage_ms, work = run_ours(args, ws, rank, local)
    import paper_1711_02976_gb300 as rp
    peaks = {"fp64": rp.rpy_alu_peak(rp.RPY_FP64), "fp32": rp.rpy_alu_peak(rp.RPY_FP32)}
    result["alu_peaks_tflops"] = {k: round(v / 1e12, 3) for k, v in peaks.items()}
    result["roofline"] = roofline(result["config"]["precision"], stage_ms, work, peaks, stats["n_beads"])
    if not args.no_e2e:
        c = result["config"]
        bp = ({k: c[k] for k in ("leaf_cap", "order_p", "direct_w", "direct_x")} | {"quad": c["quad_rule"]}
              if c["params"] in ("autotuned", "fixed") else None)
        result["e2e"] = e2e_host(args, sysm, CONFIGS[args.config], bp, 0 if c["precision"] == "fp64" else 1)
    if rank == 0:
        import oracle
        tg, ref, dt, th = cpu_oracle_sample(sysm, args.targets)
        err = oracle.rel_l2(u_dev[tg], ref)
        selft = self_term(sysm, tg)
        err_far = oracle.rel_l2(u_dev[tg] - selft, ref - selft)
        result["rel_l2"] = err
        result["rel_l2_far"] = err_far
        if not args.no_forms and CONFIGS[args.config]["precision"] == 0 and CONFIGS[args.config]["digits"] != 9:
            pf, psys, pu, pstage, pwork = precision_form(args, local, args.config)
            result["precision_form"] = {
                "value": pf["value"], "unit": "Mbeads/s", "ms_per_step": pf["ms_per_step"],
                "resident_tree_matvec_ms": pf["resident_tree_matvec_ms"], "dtype": "f32+f64",
                "rel_l2": oracle.rel_l2(pu[tg], ref), "rel_l2_far": oracle.rel_l2(pu[tg] - selft, ref - selft),
                "leaf_cap": pf["config"]["leaf_cap"], "order_p": pf["config"]["order_p"],
                "params": pf["config"]["params"], "stages_ms": pf["stages_ms"],
                "roofline": roofline("fp32", pstage, pwork, peaks),
                "note": "same workload and digit setting: P2P in FP32 with compensated (Kahan) sums, translations "
                        "in FP32 with every expansion's fourth charge set about its own box centre; bounding "
                        "cube, Morton keys, r ~ 0 pairs and per-bead sums in FP64"}
        if not args.no_serve and args.config == DEFAULT and ws == 1:
            # the serving form (BASELINE metric: p50 / p99 latency served), after the timed steps
            t0 = time.perf_counter()
            result["serving"] = serving(args, local, loads=(0.7,))
            result["serving"]["wall_s"] = round(time.perf_counter() - t0, 1)
        result["cpu_baseline"] = {"value": round(len(tg) / dt / 1e6, 6), "unit": "Mbeads/s", "cores": th,
                                  "kind": "oracle", "host": host_cpu(),
                                  "sample": (f"all {sysm.n} beads (full direct sum)" if len(tg) == sysm.n else
                                             f"{len(tg)} targets (seed 12345) x all {sysm.n} sources; extrapolated "
                                             f"O(N^2) direct rate = targets/s")}
        print(json.dumps(result), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
