"""Oracle runs for the large parity cases, computed in worker processes.

The production-size parity tests compare the CUDA path with the FP64 oracle
at 256^2 over a whole interval and at 512^2-2048^2 over a few steps; the
oracle needs seconds to minutes for each of those.  The runs are named here
(`CASES`), started together in a process pool when the first test asks for
one (the pool uses the "spawn" start method, so it is safe after CUDA has
been initialised in the test process), and each test waits only for the
runs it compares with.  Inputs are generated inside the workers from the
seeded generators of ``sw_inputs``; nothing here touches the GPU.
"""
from __future__ import annotations

import concurrent.futures as cf
import multiprocessing as mp
import os

FIELDS = ("zeta", "h", "u", "v")


def _dt(N):
    # RK4's imaginary-axis limit with the fastest gravity wave, |omega| dt <= 2.8:
    # 5e-3 up to 1024^2, 2e-3 at 2048^2
    return 5e-3 if N <= 1024 else 2e-3


def case_inputs(name):
    """(N, dt, nu8, uvh, n_steps) of a named case."""
    import sw_inputs as si

    kind, N, n = CASES[name][:3]
    K = (N - 1) // 3
    if kind == "plain":
        w = si.WORKLOADS["plain-64" if N == 64 else "plain-256"]
        return w.N, w.dt, w.nu8, w.initial_condition(), n
    if kind == "prec":
        # the 1024^2 precision form's generator (Ro 0.05, waves |k| 8-12, ratio 2)
        uvh = si.turbulence_plus_waves(N, 0.05, 2.0, 8.0, 12.0, 1003 + N)
    else:
        uvh = si.turbulence_plus_waves(N, 0.1, 1.0, 4.0, 6.0, 1002 + N)
    return N, _dt(N), 10.0 / K ** 8, uvh, n


# name -> (inputs kind, N, steps, strategy)
CASES = {
    "plain64-s1-full": ("plain", 64, 1219, 1),
    "plain256-s1-full": ("plain", 256, 1097, 1),
    "plain256-s2-full": ("plain", 256, 1097, 2),
    "plain256-s1-12": ("plain", 256, 12, 1),
    "plain256-s2-12": ("plain", 256, 12, 2),
    "turb512-s1-3": ("turb", 512, 3, 1),
    "turb512-s2-3": ("turb", 512, 3, 2),
    "prec1024-s1-3": ("prec", 1024, 3, 1),
    "prec1024-s2-3": ("prec", 1024, 3, 2),
    "prec2048-s1-2": ("prec", 2048, 2, 1),
    "prec2048-s2-2": ("prec", 2048, 2, 2),
}


def run_case(name):
    """Oracle interval of a named case: (C-ABI-named outputs, final u, v, h)."""
    import numpy as np

    from oracle import SWOracle

    N, dt, nu8, uvh, n = case_inputs(name)
    strategy = CASES[name][3]
    o = SWOracle(N, dt, *uvh, nu8=nu8)
    o.lmean_begin(strategy, fields=FIELDS, pos=True, eulerian=True, n_steps=n)
    o.lmean_step(n)
    r = o.lmean_end()
    out = {("e_" + k[2:] if k.startswith("E_") else k): v for k, v in r.items()}
    return out, np.stack(o.fields())


_pool = None
_futures = {}


def start(names=None):
    """Submit the named oracle runs (default: all) to the worker pool."""
    global _pool
    names = list(CASES) if names is None else list(names)
    if _pool is None:
        # the longest runs first; one worker per run up to the host's cores
        workers = max(1, min(len(CASES), os.cpu_count() or 1))
        _pool = cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"))
    order = sorted(names, key=lambda k: -CASES[k][1] ** 2 * CASES[k][2] * CASES[k][3])
    for k in order:
        if k not in _futures:
            _futures[k] = _pool.submit(run_case, k)


def result(name):
    start([name])
    return _futures[name].result()


def shutdown():
    """Stop the pool; runs still in progress (a session that stopped at a
    failure) are ended with their worker processes."""
    global _pool
    if _pool is not None:
        procs = list(getattr(_pool, "_processes", {}).values())
        _pool.shutdown(wait=False, cancel_futures=True)
        for p in procs:
            if p.is_alive():
                p.terminate()
        _pool = None
        _futures.clear()
