"""GPU checks of the semi-Lagrangian Strategy 1 (sw_sl_*, App. B).

* Against the oracle (oracle.gbla) on the same FP64 run: both schemes, both
  interpolants, ragged grids; the GPU takes its physical fields from its own
  FP64 transforms, so agreement is to rounding (rel-L2 1e-10), not bits.
* One grid cell of motion per step (kinematic model): every departure point
  is a node, so the mean positions take their closed forms.
* At the bench workload (256^2, one interval, FP32 dynamics): the trapezoid
  with cubic interpolation, remapped (Eq. remap-strat1), agrees with the
  GPU Strategy-2 means to the discretisation error.
* Error codes: an open lmean interval, steps beyond the interval, results
  before its end.
"""
import numpy as np
import pytest

import sw_inputs as si
from oracle import SWOracle, rel_l2
from oracle.gbla import SLInterval

from _helpers import gpu

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

FIELDS = ("zeta", "h", "u", "v", "q")


@pytest.fixture(scope="module")
def lm():
    return gpu()


def _grid(N):
    x = 2 * np.pi * np.arange(N) / N
    return np.meshgrid(x, x)


def _gpu_sl(lm, N, dt, uvh, n, scheme, interp, fields=FIELDS, **kw):
    h = lm.sw_create(lm.make_params(N, dt, precision="f64", **kw), np.ascontiguousarray(np.stack(uvh)))
    try:
        s = lm.sw_sl_create(h, lm.make_sl_params(fields, pos=True, scheme=scheme, interp=interp, n_steps=n))
        lm.sw_sl_step(s, 5)
        lm.sw_sl_step(s, n - 5)
        out = {k: np.zeros((N, N)) for k in fields + ("pos_x", "pos_y")}
        lm.sw_sl_end(s, out)
    finally:
        lm.sw_destroy(h)
    return out


@pytest.mark.parametrize("N", [32, 64])
@pytest.mark.parametrize("scheme", ["euler", "trapezoid"])
@pytest.mark.parametrize("interp", ["linear", "cubic"])
def test_matches_oracle(lm, N, scheme, interp):
    n, dt = 60, 5e-3
    u, v, h = si.smooth_flow(N, 2, seed=21, uamp=0.15, eamp=0.05)
    g = _gpu_sl(lm, N, dt, (u, v, h), n, scheme, interp)
    sl = SLInterval(SWOracle(N, dt, u, v, h), fields=FIELDS, scheme=scheme, interp=interp, n_steps=n)
    sl.step(n)
    ref = sl.end()
    X, Y = _grid(N)
    for k in FIELDS:
        e = rel_l2(g[k], ref[k])
        assert e < 1e-10, (k, e)
    d_g = np.concatenate([(g["pos_x"] - X).ravel(), (g["pos_y"] - Y).ravel()])
    d_r = np.concatenate([(ref["pos_x"] - X).ravel(), (ref["pos_y"] - Y).ravel()])
    assert rel_l2(d_g, d_r) < 1e-10


@pytest.mark.parametrize("scheme", ["euler", "trapezoid"])
def test_one_cell_per_step_positions(lm, scheme):
    N, dt, n = 32, 5e-3, 12
    dx = 2 * np.pi / N
    X, Y = _grid(N)
    cx, cy = dx / dt, -dx / dt
    F0 = np.cos(X + 0.3) + 0.5 * np.sin(Y - X)
    g = _gpu_sl(lm, N, dt, (F0, 0 * X, 1 + 0.1 * F0), n, scheme, "cubic", fields=("u",), model="kinematic",
                adv=(cx, cy), nu8=0.0, lm_nu8=0.0)
    T = n * dt
    w = 0.5 if scheme == "trapezoid" else 0.0
    shift = (T - dt + 2 * w * dt) / 2
    np.testing.assert_allclose(g["pos_x"], X - cx * shift, rtol=0, atol=1e-12)
    np.testing.assert_allclose(g["pos_y"], Y - cy * shift, rtol=0, atol=1e-12)


def test_remapped_agrees_with_strategy2_at_bench_size(lm):
    w = si.WORKLOADS["plain-256"]
    N, n = w.N, w.n_steps
    ic = np.ascontiguousarray(np.stack(w.initial_condition()))
    keys = ("zeta", "h", "u", "v")
    # semi-Lagrangian Strategy 1 on FP32 dynamics
    h1 = lm.sw_create(lm.make_params(N, w.dt, precision="f32", nu8=w.nu8), ic)
    s = lm.sw_sl_create(h1, lm.make_sl_params(keys, pos=True, scheme="trapezoid", interp="cubic", n_steps=n))
    lm.sw_sl_step(s, n)
    sl = {k: torch.empty((N, N), dtype=torch.float64, device="cuda") for k in keys + ("pos_x", "pos_y")}
    lm.sw_sl_end(s, sl)
    lm.sw_destroy(h1)
    # Strategy 2 directly
    h2 = lm.sw_create(lm.make_params(N, w.dt, precision="f32", nu8=w.nu8), ic)
    lm.lmean_begin(h2, lm.make_lm_params(2, keys, n_steps=n))
    lm.lmean_step(h2, n)
    s2 = {k: torch.empty((N, N), dtype=torch.float64, device="cuda") for k in keys + ("pos_x", "pos_y")}
    lm.lmean_end(h2, s2)
    lm.sw_destroy(h2)
    r = lm.lmean_remap(sl["pos_x"], sl["pos_y"], {k: sl[k] for k in keys}, iters=30)
    torch.cuda.synchronize()
    for k in keys:
        a, b = r[k].cpu().numpy(), s2[k].cpu().numpy()
        e = rel_l2(a - b.mean(), b - b.mean())
        assert e < 0.05, (k, e)


def test_error_codes(lm):
    N = 32
    u, v, h = si.smooth_flow(N, 2, seed=3)
    hd = lm.sw_create(lm.make_params(N, 5e-3, precision="f64"), np.ascontiguousarray(np.stack([u, v, h])))
    try:
        lm.lmean_begin(hd, lm.make_lm_params(1, ("u",), n_steps=2))
        with pytest.raises(lm.SWError) as ei:
            lm.sw_sl_create(hd, lm.make_sl_params(("u",), n_steps=3))
        assert ei.value.code == lm.api.SW_EBUSY
        lm.lmean_step(hd, 2)
        lm.lmean_end(hd, {})
        s = lm.sw_sl_create(hd, lm.make_sl_params(("u",), n_steps=3))
        with pytest.raises(lm.SWError) as ei:
            lm.sw_sl_step(s, 4)
        assert ei.value.code == lm.api.SW_ERANGE
        lm.sw_sl_step(s, 2)
        with pytest.raises(lm.SWError) as ei:
            lm.sw_sl_end(s, {"u": np.zeros((N, N))})
        assert ei.value.code == lm.api.SW_ESTATE
        lm.sw_sl_step(s, 1)
        lm.sw_sl_end(s, {"u": np.zeros((N, N))})
    finally:
        lm.sw_destroy(hd)
