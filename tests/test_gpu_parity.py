"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs.  Tolerances: relative L2 <= 1e-12 per field in FP64 mode,
<= 2e-5 in FP32 mode (h compared as h - 1, positions as displacements)."""
import numpy as np
import pytest

import sw_inputs as si
from oracle import SWOracle, rel_l2

from _helpers import (FIELDS, compare, compare_uvh, gpu, oracle_keys, run_gpu_interval,
                      run_oracle_interval, turbulence)

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-5


@pytest.fixture(scope="module")
def lm():
    return gpu()


def _max(errs):
    return max(errs.values())


# -- transforms -----------------------------------------------------------------
@pytest.mark.parametrize("N", [16, 64, 256])
@pytest.mark.parametrize("prec,tol", [("f64", 1e-14), ("f32", 1e-6)])
def test_initial_transform_round_trip(lm, N, prec, tol):
    uvh = si.smooth_flow(N, (N - 1) // 3, seed=3, uamp=0.1, eamp=0.05)
    p = lm.make_params(N, 1e-3, precision=prec)
    h = lm.sw_create(p, np.ascontiguousarray(np.stack(uvh)))
    try:
        out = np.zeros((3, N, N))
        lm.sw_get_fields(h, out)
    finally:
        lm.sw_destroy(h)
    e = compare_uvh(out, np.stack(uvh))
    assert _max(e) < tol, e


# -- dynamics only ------------------------------------------------------------------
@pytest.mark.parametrize("N,steps", [(16, 30), (64, 30), (128, 10)])
def test_dynamics_fp64(lm, N, steps):
    uvh = turbulence(N, seed=7)
    nu8 = 10.0 / ((N - 1) // 3) ** 8
    p = lm.make_params(N, 5e-3, nu8=nu8)
    h = lm.sw_create(p, np.ascontiguousarray(np.stack(uvh)))
    try:
        lm.sw_step(h, steps)
        out = np.zeros((3, N, N))
        lm.sw_get_fields(h, out)
        d = lm.sw_diag(h)
    finally:
        lm.sw_destroy(h)
    o = SWOracle(N, 5e-3, *uvh, nu8=nu8)
    o.step(steps)
    e = compare_uvh(out, np.stack(o.fields()))
    assert _max(e) < TOL64, e
    md, ed, zd = o.diag()
    assert abs(d[0] - md) < 1e-15
    assert abs(d[1] - ed) / ed < 1e-13 and abs(d[2] - zd) / zd < 1e-13


# -- one averaging interval, both strategies -----------------------------------------
@pytest.mark.parametrize("strategy", [1, 2])
@pytest.mark.parametrize("N,n", [(32, 40), (64, 40), (128, 12)])
def test_interval_fp64(lm, strategy, N, n):
    uvh = turbulence(N, seed=11)
    nu8 = 10.0 / ((N - 1) // 3) ** 8
    g, gs = run_gpu_interval(lm, N, 5e-3, uvh, strategy, n, nu8=nu8, chunks=[n // 2, n - n // 2])
    r, rs = run_oracle_interval(N, 5e-3, uvh, strategy, n, nu8=nu8)
    e = compare(g, r, N, strategy)
    e.update({"sw_" + k: v for k, v in compare_uvh(gs, rs).items()})
    assert _max(e) < TOL64, e


@pytest.mark.parametrize("strategy", [1, 2])
def test_interval_with_pv_fp64(lm, strategy):
    N, n = 64, 30
    uvh = turbulence(N, seed=5)
    fields = ("zeta", "h", "u", "v", "q")
    g, _ = run_gpu_interval(lm, N, 5e-3, uvh, strategy, n, fields=fields, nu8=1e-10)
    r, _ = run_oracle_interval(N, 5e-3, uvh, strategy, n, fields=fields, nu8=1e-10)
    e = compare(g, r, N, strategy)
    assert _max(e) < TOL64, e


@pytest.mark.parametrize("strategy", [1, 2])
def test_interval_fp32(lm, strategy):
    N, n = 64, 40
    uvh = turbulence(N, seed=11)
    nu8 = 10.0 / 21 ** 8
    g, gs = run_gpu_interval(lm, N, 5e-3, uvh, strategy, n, precision="f32", nu8=nu8)
    r, rs = run_oracle_interval(N, 5e-3, uvh, strategy, n, nu8=nu8)
    e = compare(g, r, N, strategy)
    e.update({"sw_" + k: v for k, v in compare_uvh(gs, rs).items()})
    assert _max(e) < TOL32, e


@pytest.mark.parametrize("strategy", [1, 2])
def test_kinematic_model(lm, strategy):
    N, n = 32, 60
    rng = np.random.default_rng(4)
    F = si.random_smooth_field(N, 4, rng, 1.0)
    G = si.random_smooth_field(N, 4, rng, 1.0)
    uvh = (F, G, 1.0 + 0.1 * F)
    kw = dict(model="kinematic", adv=(0.7, -0.4))
    g, _ = run_gpu_interval(lm, N, 5e-3, uvh, strategy, n, fields=("u", "h"), **kw)
    r, _ = run_oracle_interval(N, 5e-3, uvh, strategy, n, fields=("u", "h"), **kw)
    e = compare(g, r, N, strategy)
    assert _max(e) < TOL64, e


def test_interval_after_spin_up_and_partial_mask(lm):
    # interval opened at tau > 0, Strategy 1 without positions, no Eulerian means
    N, n = 64, 25
    uvh = turbulence(N, seed=2)
    g, _ = run_gpu_interval(lm, N, 5e-3, uvh, 1, n, fields=("zeta", "v"), pos=False, eulerian=False,
                            pre_steps=15, nu8=1e-10)
    r, _ = run_oracle_interval(N, 5e-3, uvh, 1, n, fields=("zeta", "v"), pos=False, eulerian=False,
                               pre_steps=15, nu8=1e-10)
    e = compare(g, r, N, 1)
    assert _max(e) < TOL64, e


def test_consecutive_intervals_reset_state(lm):
    # Sec. 2: each interval starts from a zero mean state
    N, n = 32, 20
    uvh = turbulence(N, seed=8)
    p = lm.make_params(N, 5e-3, nu8=1e-8)
    h = lm.sw_create(p, np.ascontiguousarray(np.stack(uvh)))
    o = SWOracle(N, 5e-3, *uvh, nu8=1e-8)
    try:
        for k, strat in enumerate((1, 2, 1)):
            lm.lmean_begin(h, lm.make_lm_params(strat, ("zeta", "h"), n_steps=n))
            lm.lmean_step(h, n)
            out = {f: np.zeros((N, N)) for f in ("zeta", "h", "pos_x", "pos_y", "e_zeta", "e_h")}
            lm.lmean_end(h, out)
            o.lmean_begin(strat, fields=("zeta", "h"), n_steps=n)
            o.lmean_step(n)
            r = oracle_keys(o.lmean_end())
            e = compare(out, r, N, strat)
            assert _max(e) < TOL64, (k, e)
    finally:
        lm.sw_destroy(h)


# -- checkpoint / resume --------------------------------------------------------------
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_checkpoint_resume_bitwise(lm, prec):
    N, n = 64, 30
    uvh = np.ascontiguousarray(np.stack(turbulence(N, seed=12)))
    p = lm.make_params(N, 5e-3, precision=prec, nu8=1e-10)
    lp = lm.make_lm_params(1, FIELDS, n_steps=n)
    keys = list(FIELDS) + ["pos_x", "pos_y"] + ["e_" + f for f in FIELDS]

    h = lm.sw_create(p, uvh)
    lm.lmean_begin(h, lp)
    lm.lmean_step(h, n)
    ref = {k: np.zeros((N, N)) for k in keys}
    lm.lmean_end(h, ref)
    lm.sw_destroy(h)

    h = lm.sw_create(p, uvh)
    lm.lmean_begin(h, lp)
    lm.lmean_step(h, 13)
    blob = lm.sw_get_state(h)
    lm.sw_destroy(h)
    h2 = lm.sw_create(p, np.ascontiguousarray(np.zeros_like(uvh) + 1.0))
    lm.sw_set_state(h2, blob)
    assert lm.lmean_progress(h2) == (13, n - 13)
    lm.lmean_step(h2, n - 13)
    out = {k: np.zeros((N, N)) for k in keys}
    lm.lmean_end(h2, out)
    lm.sw_destroy(h2)
    for k in keys:
        assert np.array_equal(out[k], ref[k]), k


# -- device-resident outputs -------------------------------------------------------------
def test_device_outputs_match_host(lm):
    import torch
    N, n = 32, 10
    uvh = np.stack(turbulence(N, seed=3))
    p = lm.make_params(N, 5e-3, nu8=1e-8)
    res = []
    for dev in (False, True):
        ic = torch.from_numpy(uvh).cuda() if dev else np.ascontiguousarray(uvh)
        h = lm.sw_create(p, ic)
        lm.lmean_begin(h, lm.make_lm_params(2, ("zeta",), n_steps=n))
        lm.lmean_step(h, n)
        if dev:
            out = {k: torch.zeros((N, N), dtype=torch.float64, device="cuda") for k in ("zeta", "pos_x")}
        else:
            out = {k: np.zeros((N, N)) for k in ("zeta", "pos_x")}
        lm.lmean_end(h, out)
        lm.sw_destroy(h)
        res.append({k: (v.cpu().numpy() if dev else v) for k, v in out.items()})
    for k in res[0]:
        assert np.array_equal(res[0][k], res[1][k])


# -- error paths that need a live handle ---------------------------------------------------
def test_state_errors(lm):
    N = 16
    uvh = np.ascontiguousarray(np.stack(si.uniform_flow(N, 0.1, 0.0)))
    h = lm.sw_create(lm.make_params(N, 1e-2), uvh)
    try:
        with pytest.raises(lm.SWError) as ei:
            lm.lmean_step(h, 1)
        assert ei.value.code == lm.api.SW_ESTATE
        lm.lmean_begin(h, lm.make_lm_params(1, ("u",), n_steps=3))
        with pytest.raises(lm.SWError) as ei:
            lm.sw_step(h, 1)
        assert ei.value.code == lm.api.SW_EBUSY
        with pytest.raises(lm.SWError) as ei:
            lm.lmean_step(h, 4)
        assert ei.value.code == lm.api.SW_ERANGE
        lm.lmean_step(h, 0)
        with pytest.raises(lm.SWError) as ei:
            lm.lmean_end(h, {"u": np.zeros((N, N))})
        assert ei.value.code == lm.api.SW_ESTATE
        lm.lmean_step(h, 3)
        with pytest.raises(lm.SWError) as ei:
            lm.lmean_end(h, {"zeta": np.zeros((N, N))})
        assert ei.value.code == lm.api.SW_EINVAL
        out = {"u": np.zeros((N, N))}
        lm.lmean_end(h, out)
        T = 3 * 1e-2
        # uniform inertial oscillation, f0 = 1: u mean = U0 sin(T)/T up to the
        # RK4 error (about (f0 dt)^4 U0 / 120 per step)
        assert abs(out["u"].mean() - 0.1 * np.sin(T) / T) < 1e-10
    finally:
        lm.sw_destroy(h)
