"""Run one configuration for a few RK4 steps and print per-kernel device times.

Used for profiling captures and quick timings of a single grid:

  python -m paper_2208_02682_gb300.runcase --N 2048 --strategy 1 --precision f32 --steps 4

It creates one handle from the seeded turbulence-plus-wave initial condition,
opens an averaging interval, runs one untimed step (graph capture and
upload), replays `--graph-steps` steps from the captured graphs (timed with
CUDA events), then launches `--steps` steps kernel by kernel through
sw_kernel_times and prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--N", type=int, default=1024)
    ap.add_argument("--strategy", type=int, default=1, choices=[0, 1, 2])
    ap.add_argument("--precision", default="f32", choices=["f32", "f64"])
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--graph-steps", type=int, default=16)
    ap.add_argument("--fields", default="zeta,h,u,v")
    ap.add_argument("--seed", type=int, default=1003)
    ap.add_argument("--cufft", action="store_true",
                    help="also time cuFFT (torch.fft) on the same transform counts, for comparison")
    ap.add_argument("--shapes", action="store_true",
                    help="also time the step under every row-pass launch shape the grid admits "
                         "(sw_batch_set_shape on a batch of one)")
    args = ap.parse_args(argv)

    import torch

    import paper_2208_02682_gb300 as lm
    import sw_inputs as si

    lm.build()
    N = args.N
    K = (N - 1) // 3
    dt = 5e-3 if N <= 1024 else 2.5e-3
    ic = np.ascontiguousarray(np.stack(si.turbulence_plus_waves(N, 0.05, 2.0, 8.0, 12.0, args.seed)))
    h = lm.sw_create(lm.make_params(N, dt, precision=args.precision, nu8=10.0 / K ** 8), ic)
    fields = tuple(f for f in args.fields.split(",") if f)
    total = 1 + args.graph_steps + args.steps
    if args.strategy:
        lm.lmean_begin(h, lm.make_lm_params(args.strategy, fields, n_steps=total))
    step = (lambda n: lm.lmean_step(h, n)) if args.strategy else (lambda n: lm.sw_step(h, n))
    step(1)  # untimed: captures and uploads the step graphs
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    step(args.graph_steps)
    e1.record()
    torch.cuda.synchronize()
    graph_ms = e0.elapsed_time(e1) / max(1, args.graph_steps)
    kt = lm.sw_kernel_times(h, args.steps)
    shapes = None
    if args.shapes:
        # graph replays of a batch of one under each shape, each on a fresh
        # interval (the first half untimed: a new graph's first replay uploads it)
        if args.strategy:
            lm.lmean_end(h, {})
        shapes = {}
        b = lm.sw_batch_create([h])
        reps = max(2, args.graph_steps // 2)
        for c in range(16):
            pts = (256, 512, 1024, 2048)[c // 4]
            if pts < N:
                continue
            lm.sw_batch_set_shape(b, c)
            if args.strategy:
                lm.lmean_begin(h, lm.make_lm_params(args.strategy, fields, n_steps=2 * reps))
            lm.sw_batch_step(b, reps)
            torch.cuda.synchronize()
            e0.record()
            lm.sw_batch_step(b, reps)
            e1.record()
            torch.cuda.synchronize()
            shapes[f"{pts}pts_{(1, 2, 3, 'all')[c % 4]}pairs"] = e0.elapsed_time(e1) / reps
            if args.strategy:
                lm.lmean_end(h, {})
        lm.sw_batch_destroy(b)
    lm.sw_destroy(h)
    tot = sum(v[0] for v in kt.values())
    out = {
        "N": N, "strategy": args.strategy, "precision": args.precision, "fields": list(fields),
        "graph_ms_per_step": graph_ms,
        "gp_steps_per_s": N * N / (graph_ms * 1e-3),
        "kernels": {k: {"ms_per_launch": t / c, "launches": c, "share": t / tot,
                        "GBps_algorithmic": (b / c) / (t / c * 1e-3) / 1e9}
                    for k, (t, c, b) in sorted(kt.items(), key=lambda kv: -kv[1][0])},
    }
    if shapes is not None:
        out["step_ms_by_row_pass_shape"] = shapes
    if args.cufft:
        out["cufft_comparison"] = cufft_reference(torch, N, args.precision, kt)
    print(json.dumps(out))


def cufft_reference(torch, N, precision, kt):
    """cuFFT (through torch.fft, a library call timed only for comparison) on
    the transforms one RK stage of Strategy 1 (zeta, h, u, v, positions)
    performs: the row pass's complex N-point FFTs (N rows x 8 paired inverse
    and 6 paired forward transforms) and the column passes' (K+1 columns x 16
    inverse and 11 forward transforms).  Data movement and the physical-space
    products of the stage kernels are not included."""
    K = (N - 1) // 3
    dt = torch.complex64 if precision == "f32" else torch.complex128
    rows = torch.randn(14 * N, N, dtype=dt, device="cuda")
    cols = torch.randn(27 * (K + 1), N, dtype=dt, device="cuda")
    res = {}
    for name, x in (("row_transforms", rows), ("column_transforms", cols)):
        for _ in range(3):
            torch.fft.fft(x, dim=1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 10
        e0.record()
        for _ in range(reps):
            torch.fft.fft(x, dim=1)
        e1.record()
        torch.cuda.synchronize()
        res[name + "_ms"] = e0.elapsed_time(e1) / reps
    res["note"] = "out-of-place batched C2C, data resident; the stage kernels also read, write and form products"
    per = {k: t / c for k, (t, c, b) in kt.items()}
    res["ours_row_prod_ms"] = per.get("row_prod")
    res["ours_col_inv_plus_col_fwd_ms"] = per.get("col_inv", 0.0) + per.get("col_fwd", 0.0)
    return res


if __name__ == "__main__":
    main()
