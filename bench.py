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
    "cube4096_3digit_fp64": dict(gen="config1", digits=3, precision=0, leaf_cap=40,
                                 desc="4,096 beads uniform cube, a=0.004, 3-digit, FP64, leaf cap 40"),
    "cube15m_3digit_fp32": dict(gen="config3", digits=3, precision=1, leaf_cap=0,
                                desc="15,000,000 beads uniform cube, a=2e-5, 3-digit, FP32 precision form"),
}
DEFAULT = "sphere1m_6digit_fp64"


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


def make_workload(name):
    import synth
    return getattr(synth, CONFIGS[name]["gen"])()


def flops_model(stats, stage):
    """Algorithmic floating-point operations of one stage (FMA = 2), counted
    from the kernel source: the direct RPY pair costs 46 in the
    FP64 kernel (3 sub, r^2 5, Newton reciprocal sqrt 5, scalars 3, R.F 5,
    t1 3, t2 5, accumulate 12) and 45 in the FP32 kernel (no Newton step;
    Kahan adds 4 per component)."""
    if stage == "p2p":
        per = 46.0 if stats["precision"] == 0 else 45.0
        return (stats["u_pairs"] + stats["d_pairs"]) * per
    return None


def run_ours(args, ws, rank, local):
    import torch
    import paper_1711_02976_gb300 as rp

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfg = CONFIGS[args.config]
    sysm = make_workload(args.config)
    n = sysm.n
    P = torch.from_numpy(sysm.pos).to(dev)
    F = torch.from_numpy(sysm.f).to(dev)
    U = torch.empty_like(F)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (129 MB)

    def build():
        return rp.rpy_tree_build(P, n, sysm.a, cfg["digits"], leaf_cap=cfg["leaf_cap"], precision=cfg["precision"])

    tree = build()

    def step():
        rp.rpy_tree_update_positions(tree, P)
        rp.rpy_matvec(tree, F, sysm.s, U)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    launches0 = rp.rpy_launch_count()
    times, tb, tm = [], [], []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        rp.rpy_tree_update_positions(tree, P)
        e1.record(stream)
        rp.rpy_matvec(tree, F, sysm.s, U)
        e2.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e2))
        tb.append(e0.elapsed_time(e1))
        tm.append(e1.elapsed_time(e2))
    launches = (rp.rpy_launch_count() - launches0) // max(1, args.steps)
    clocks = sampler.stop()
    ms = sum(times) / len(times)
    if ws > 1:
        import torch.distributed as dist
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.barrier()
        ms = float(t.item())
    value = ws * n / (ms * 1e-3) / 1e6
    stats = rp.rpy_tree_stats(tree)

    # stage profile of one matvec (separate, untimed for the headline)
    rp.rpy_tree_set_profiling(tree, True)
    prof = []
    for _ in range(3):
        flush.zero_()
        rp.rpy_matvec(tree, F, sysm.s, U)
        prof.append(rp.rpy_tree_stage_times(tree))
    rp.rpy_tree_set_profiling(tree, False)
    stage_ms = {k: statistics.median(p[k] for p in prof) for k in prof[0]}
    u_dev = U.cpu().numpy()

    result = {
        "metric": METRIC, "value": round(value, 4), "unit": "Mbeads/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if cfg["precision"] == 0 else "f32+f64",
        "data": "synthetic (seeded numpy; shapes of the paper's sphere/cube workloads)",
        "config": {"workload": args.config, "description": cfg["desc"], "n_beads": n, "digits": cfg["digits"],
                   "precision": "fp64" if cfg["precision"] == 0 else "fp32", "parallelism": f"replicas x{ws}",
                   "l2": "flushed between timed steps (256 MB write)", "step": "tree build + matvec",
                   "leaf_cap": stats["leaf_cap"], "order_p": stats["order_p"], "exp_terms": stats["exp_terms"]},
        "build_ms": round(statistics.median(tb), 4), "matvec_ms": round(statistics.median(tm), 4),
        "matvec_only_mbeads_s": round(ws * n / (statistics.median(tm) * 1e-3) / 1e6, 4),
        "stages_ms": {k: round(v, 4) for k, v in stage_ms.items()},
        "tree": {k: stats[k] for k in ("n_boxes", "n_leaves", "depth", "u_pairs", "d_pairs", "n_wlist", "n_xlist",
                                       "n_dlist", "max_leaf_count", "leaves_over_cap", "device_bytes")},
        "gpu_launches": int(launches), "clocks": clocks,
    }
    return result, sysm, u_dev, stats, stage_ms, tree


def roofline(result, stats, stage_ms, peaks):
    top = max(stage_ms, key=lambda k: stage_ms[k])
    fl = flops_model(stats, top)
    prec = result["config"]["precision"]
    if fl is not None and stage_ms[top] > 0:
        peak = peaks["fp64"] if prec == "fp64" else peaks["fp32"]
        ach = fl / (stage_ms[top] * 1e-3) / 1e12
        return {"kernel": top, "bound": "alu", "achieved": round(ach, 4), "peak": round(peak / 1e12, 4),
                "unit": "TFLOP/s", "frac": round(ach / (peak / 1e12), 4), "traffic": None,
                "peak_source": "measured FMA-chain probe on this GPU (rpy_alu_peak)"}
    return {"kernel": top, "bound": "alu", "achieved": None, "peak": None, "unit": "TFLOP/s", "frac": None,
            "traffic": None}


def e2e_host(args, sysm, cfg):
    """The same matvec through the host-array entry point: H2D of positions and
    forces from pinned memory, build, matvec, D2H of velocities, every step."""
    import torch
    import paper_1711_02976_gb300 as rp
    n = sysm.n
    pos_h = torch.from_numpy(sysm.pos).pin_memory()
    f_h = torch.from_numpy(sysm.f).pin_memory()
    u_h = torch.empty((n, 3), dtype=torch.float64).pin_memory()
    lib = rp.load()

    def call():
        st = lib.rpy_matvec_host(pos_h.data_ptr(), n, sysm.a, f_h.data_ptr(), sysm.s, cfg["digits"], cfg["precision"],
                                 u_h.data_ptr(), rp._stream(None))
        if st:
            raise rp.RpyError(st, "rpy_matvec_host")

    for _ in range(2):
        call()
    torch.cuda.synchronize()
    ts = []
    for _ in range(max(2, min(args.steps, 5))):
        t0 = time.perf_counter()
        call()
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
    t = statistics.median(ts)
    return {"value": round(n / t / 1e6, 4), "unit": "Mbeads/s", "h2d_bytes_per_step": 2 * n * 3 * 8,
            "d2h_bytes_per_step": n * 3 * 8, "ms_per_step": round(t * 1e3, 3),
            "api": "rpy_matvec_host (pinned host arrays in, velocities out)"}


def cpu_oracle_sample(sysm, k):
    import oracle
    import synth
    tg = synth.sample_targets(sysm.n, k)
    th = oracle.default_threads()
    t0 = time.perf_counter()
    ref = oracle.rpy_direct(sysm.pos, sysm.f, sysm.a, sysm.s, targets=tg, threads=th)
    dt = time.perf_counter() - t0
    return tg, ref, dt, th


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default=DEFAULT, choices=sorted(CONFIGS))
    ap.add_argument("--targets", type=int, default=2000, help="oracle sample for the CPU baseline / error")
    ap.add_argument("--no-e2e", action="store_true")
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
                                           "sample": f"{k} targets x all {sysm.n} sources per step; extrapolated "
                                                     f"O(N^2) direct rate"},
                          "e2e": {"value": round(v, 6), "unit": "Mbeads/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}), flush=True)
        return
    result, sysm, u_dev, stats, stage_ms, tree = run_ours(args, ws, rank, local)
    import paper_1711_02976_gb300 as rp
    peaks = {"fp64": rp.rpy_alu_peak(rp.RPY_FP64), "fp32": rp.rpy_alu_peak(rp.RPY_FP32)}
    result["alu_peaks_tflops"] = {k: round(v / 1e12, 3) for k, v in peaks.items()}
    result["roofline"] = roofline(result, stats, stage_ms, peaks)
    if not args.no_e2e:
        result["e2e"] = e2e_host(args, sysm, CONFIGS[args.config])
    if rank == 0:
        import oracle
        tg, ref, dt, th = cpu_oracle_sample(sysm, args.targets)
        err = oracle.rel_l2(u_dev[tg], ref)
        selft = sysm.s / (6 * math.pi * sysm.a) * sysm.f[tg]
        err_far = oracle.rel_l2(u_dev[tg] - selft, ref - selft)
        result["rel_l2"] = err
        result["rel_l2_far"] = err_far
        result["cpu_baseline"] = {"value": round(len(tg) / dt / 1e6, 6), "unit": "Mbeads/s", "cores": th,
                                  "kind": "oracle",
                                  "sample": f"{len(tg)} targets (seed 12345) x all {sysm.n} sources; extrapolated "
                                            f"O(N^2) direct rate = targets/s"}
        print(json.dumps(result), flush=True)
    tree.close()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
