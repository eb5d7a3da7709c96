"""Shared helpers for the GPU parity tests (run the CUDA path and the oracle
on the same seeded inputs and compare)."""
import numpy as np

import sw_inputs as si
from oracle import SWOracle, rel_l2

FIELDS = ("zeta", "h", "u", "v")


def gpu():
    import paper_2208_02682_gb300 as lm
    lm.build()
    lm.api.load()
    return lm


def run_gpu_interval(lm, N, dt, uvh, strategy, n_steps, precision="f64", fields=FIELDS,
                     eulerian=True, pos=True, pre_steps=0, chunks=None, **kw):
    p = lm.make_params(N, dt, precision=precision, **kw)
    h = lm.sw_create(p, np.ascontiguousarray(np.stack(uvh)))
    try:
        if pre_steps:
            lm.sw_step(h, pre_steps)
        lm.lmean_begin(h, lm.make_lm_params(strategy, fields, pos=pos, eulerian=eulerian, n_steps=n_steps))
        for c in (chunks or [n_steps]):
            lm.lmean_step(h, c)
        out = {}
        keys = list(fields) + (["pos_x", "pos_y"] if (pos or strategy == 2) else [])
        keys += ["e_" + f for f in fields] if eulerian else []
        for k in keys:
            out[k] = np.zeros((N, N))
        lm.lmean_end(h, out)
        uvh_out = np.zeros((3, N, N))
        lm.sw_get_fields(h, uvh_out)
        return out, uvh_out
    finally:
        lm.sw_destroy(h)


def run_oracle_interval(N, dt, uvh, strategy, n_steps, fields=FIELDS, eulerian=True, pos=True,
                        pre_steps=0, nu8=0.0, lm_nu8=None, f0=1.0, c2=1.0, model="sw", adv=(0.0, 0.0)):
    o = SWOracle(N, dt, *uvh, f0=f0, c2=c2, nu8=nu8, lm_nu8=lm_nu8, model=model, adv=adv)
    if pre_steps:
        o.step(pre_steps)
    o.lmean_begin(strategy, fields=fields, pos=pos, eulerian=eulerian, n_steps=n_steps)
    o.lmean_step(n_steps)
    r = oracle_keys(o.lmean_end())
    return r, np.stack(o.fields())


def oracle_keys(r):
    """Oracle output names -> C-ABI output names (E_f -> e_f)."""
    return {("e_" + k[2:] if k.startswith("E_") else k): v for k, v in r.items()}


# Positions are reported as absolute coordinates (up to about 2 pi), so each
# value, on either side, is rounded to a spacing of 2^-50 (one ulp of 2 pi);
# the grid coordinate subtracted to form the displacement differs by as
# much.  Two ulps per point are the representation floor of a displacement
# comparison; it matters only when the displacement is tiny (intervals of a
# few steps) and is not counted against the tolerance.
POS_FLOOR = 2.0 * 2.0 ** -50


def _pos_err(a, ref, grid):
    d = float(np.linalg.norm(a - ref))
    floor = POS_FLOOR * np.sqrt(a.size)
    den = float(np.linalg.norm(ref - grid))
    return max(0.0, d - floor) / (den if den > 0 else 1.0)


def compare(gpu_out, ref_out, N, strategy):
    """Per-field relative L2 errors; depth as eta = h - 1, positions as the
    displacement from the grid point (so the norms are not set by 1 or x),
    less the representation floor of absolute coordinates (POS_FLOOR)."""
    x = 2 * np.pi * np.arange(N) / N
    X = x[None, :] + 0 * x[:, None]
    Y = x[:, None] + 0 * x[None, :]
    errs = {}
    for k, ref in ref_out.items():
        a = gpu_out[k]
        if k in ("h", "e_h"):
            errs[k] = rel_l2(a - 1.0, ref - 1.0)
        elif k == "pos_x":
            errs[k] = _pos_err(a, ref, X)
        elif k == "pos_y":
            errs[k] = _pos_err(a, ref, Y)
        else:
            errs[k] = rel_l2(a, ref)
    return errs


def compare_uvh(a, b):
    return {"u": rel_l2(a[0], b[0]), "v": rel_l2(a[1], b[1]), "h": rel_l2(a[2] - 1.0, b[2] - 1.0)}


def turbulence(N, seed=1001, ro=0.1, ratio=1.0, k_lo=4.0, k_hi=6.0):
    return si.turbulence_plus_waves(N, ro, ratio, k_lo, k_hi, seed)
