#!/usr/bin/env python
"""Throughput of the coupled shallow-water + Lagrangian-mean step on GB300.

One bench step is one averaging interval (lmean_begin, n_steps RK4 steps,
lmean_end) of the 256^2 turbulence-plus-Poincare-wave workload, Strategies 1
and 2 side by side on two CUDA streams, FP32 stepping with FP64 end-of-interval
recovery.  Metric: grid-point-steps/s = runs * N^2 * RK4 steps / device time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun): every rank runs an independent replica (the method
shards into independent runs; there is no collective on the data path);
value = all ranks' grid-point-steps / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import sw_inputs as si  # noqa: E402

METRIC = "grid-point-steps/s incl. Lagrangian means"
UNIT = "grid-point-steps/s"
FIELDS = ("zeta", "h", "u", "v")
OUT_KEYS = list(FIELDS) + ["pos_x", "pos_y"] + ["e_" + f for f in FIELDS]
L2_FLUSH_BYTES = 256 << 20


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
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
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def workload():
    w = si.WORKLOADS["plain-256"]
    return w


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ------------------------------------------------------------------------------
def oracle_sample(w, steps_per_strategy):
    """Time the FP64 oracle on a bounded sample of the workload (both strategies)."""
    from oracle import SWOracle
    u, v, h = w.initial_condition()
    t0 = time.perf_counter()
    for strategy in w.strategies:
        o = SWOracle(w.N, w.dt, u, v, h, f0=w.f0, c2=w.c2, nu8=w.nu8)
        o.lmean_begin(strategy, fields=FIELDS, pos=True, eulerian=True, n_steps=steps_per_strategy)
        o.lmean_step(steps_per_strategy)
    dt = time.perf_counter() - t0
    gp = len(w.strategies) * w.N * w.N * steps_per_strategy
    return gp / dt, dt


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    w = workload()
    sample = 12
    for _ in range(args.warmup):
        oracle_sample(w, 2)
    vals, tot = [], 0.0
    for _ in range(args.steps):
        v, dt = oracle_sample(w, sample)
        vals.append(v)
        tot += dt
    value = len(vals) * len(w.strategies) * w.N * w.N * sample / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": config_dict(w, "oracle f64"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{sample} RK4 steps per strategy of the {w.N}^2 workload per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def config_dict(w, form):
    return {"workload": f"{w.name}: {w.N}x{w.N} turbulence (Ro {w.ro}) + Poincare waves |k| "
                        f"{w.k_lo:g}-{w.k_hi:g} (energy ratio {w.ratio:g}), Strategies 1 and 2 side "
                        f"by side, {w.n_steps} RK4 steps per averaging interval (3.6 wave periods)",
            "N": w.N, "strategies": list(w.strategies), "n_steps_per_interval": w.n_steps,
            "dt": w.dt, "fields": list(FIELDS) + ["pos", "eulerian"], "form": form,
            "step": "one averaging interval", "l2": "flushed between timed steps (256 MiB write)"}


# ------------------------------------------------------------------------------
def run_ours(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import paper_2208_02682_gb300 as lm
    lm.build()
    w = workload()
    N, n = w.N, w.n_steps
    prec = args.precision
    ic = np.ascontiguousarray(np.stack(w.initial_condition()))
    streams = [torch.cuda.Stream() for _ in w.strategies]
    params = lm.make_params(N, w.dt, precision=prec, f0=w.f0, c2=w.c2, nu8=w.nu8)
    hs = [lm.sw_create(params, ic, s.cuda_stream) for s in streams]
    outs = [{k: torch.empty((N, N), dtype=torch.float64, device="cuda") for k in OUT_KEYS}
            for _ in hs]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    main = torch.cuda.current_stream()
    chunk = 64

    def interval():
        for h, strat in zip(hs, w.strategies):
            lm.lmean_begin(h, lm.make_lm_params(strat, FIELDS, pos=True, eulerian=True, n_steps=n))
        done = 0
        while done < n:
            c = min(chunk, n - done)
            for h in hs:
                lm.lmean_step(h, c)
            done += c
        for h, o in zip(hs, outs):
            lm.lmean_end(h, o)

    def timed_interval():
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(main)
        for s in streams:
            s.wait_event(ev0)
        interval()
        for s in streams:
            e = torch.cuda.Event()
            e.record(s)
            main.wait_event(e)
        ev1.record(main)
        return ev0, ev1

    for _ in range(args.warmup):
        interval()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = sum(lm.sw_launch_count(h) for h in hs)
    clk = ClockSampler(local)
    clk.start()
    evs = []
    t_wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()
        evs.append(timed_interval())
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    clocks = clk.stop()
    launches = sum(lm.sw_launch_count(h) for h in hs) - launches0
    ms = sum(a.elapsed_time(b) for a, b in evs)
    if dist:
        t = torch.tensor([ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    gp_per_step = len(hs) * N * N * n
    value = world * gp_per_step * args.steps / (ms * 1e-3)

    # per-kernel device times (kernels launched one by one, same stream)
    ktimes = {}
    nk = 16
    for h, strat in zip(hs, w.strategies):
        lm.lmean_begin(h, lm.make_lm_params(strat, FIELDS, pos=True, eulerian=True, n_steps=nk))
        for k, (t, c, b) in lm.sw_kernel_times(h, nk).items():
            a = ktimes.setdefault(k, [0.0, 0, 0.0])
            a[0] += t
            a[1] += c
            a[2] += b
        lm.lmean_step(h, 0)
        lm.lmean_end(h, {})
    torch.cuda.synchronize()
    tot = sum(v[0] for v in ktimes.values())
    dom = max(ktimes, key=lambda k: ktimes[k][0])
    t_ms, cnt, byt = ktimes[dom]
    peak, peak_src = peaks()
    achieved = (byt / cnt) / (t_ms / cnt * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": None, "kernel": dom,
                "peak_source": peak_src,
                "note": "256^2 working set is L2-resident; see DESIGN.md for the 1024^2 figures"}
    kernel_share = {k: {"ms_per_launch": v[0] / v[1], "launches": v[1], "share": v[0] / tot,
                        "GBps_algorithmic": (v[2] / v[1]) / (v[0] / v[1] * 1e-3) / 1e9}
                    for k, v in sorted(ktimes.items(), key=lambda kv: -kv[1][0])}

    # end to end through the C ABI with pinned host buffers, copies timed
    e2e = None
    if not args.no_e2e:
        ic_pin = torch.from_numpy(ic).pin_memory()
        ic_host = ic_pin.numpy()
        host_out = [{k: torch.empty((N, N), dtype=torch.float64).pin_memory().numpy() for k in OUT_KEYS}
                    for _ in hs]

        def e2e_interval():
            for h in hs:
                lm.sw_set_fields(h, ic_host)
            for h, strat in zip(hs, w.strategies):
                lm.lmean_begin(h, lm.make_lm_params(strat, FIELDS, pos=True, eulerian=True, n_steps=n))
            done = 0
            while done < n:
                c = min(chunk, n - done)
                for h in hs:
                    lm.lmean_step(h, c)
                done += c
            for h, o in zip(hs, host_out):
                lm.lmean_end(h, o)

        e2e_interval()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            e2e_interval()
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        if dist:
            t = torch.tensor([te], dtype=torch.float64, device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            te = float(t.item())
        e2e = {"value": world * gp_per_step * args.steps / te, "unit": UNIT,
               "h2d_bytes_per_step": len(hs) * ic.nbytes,
               "d2h_bytes_per_step": len(hs) * len(OUT_KEYS) * N * N * 8,
               "note": "sw_set_fields from pinned host memory + interval + lmean_end to pinned host"}

    for h in hs:
        lm.sw_destroy(h)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        sample = 12
        v, dt = oracle_sample(w, sample)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{sample} RK4 steps of each strategy at {N}^2 ({dt:.1f} s, numpy FP64, one thread)"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == "f32" else "f64",
        "data": "synthetic", "config": config_dict(w, prec + " stepping, fp64 end-of-interval recovery"),
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
        "gpu_launches": launches, "kernels": kernel_share, "wall_s": t_wall,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="f32", choices=["f32", "f64"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
