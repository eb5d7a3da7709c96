"""GPU checks of the two-dimensional Euler model (Sec. 4.1's test flow).

* Against the oracle on the same FP64 runs (Heun and RK4, both strategies,
  zeta, u, v and positions): relative L2 <= 1e-12 per field, state included.
* The paper's vortex-merger check, Eq. (vorticity_itsmean), at its own
  setup (128^2, Heun, dt = 0.005, tau = 0, T = 25): Strategy 1's zeta~^L
  equals zeta(T) up to the time stepping, so the difference falls by about
  4 when dt is halved (the identity is exact in the semi-discrete system).
* Fig. 3's comparison on the same run: the pseudospectral zeta~^L is closer
  to zeta(T) than the semi-Lagrangian one with cubic interpolation, and that
  one closer than with linear interpolation.
* Error codes: depth or PV means, sw_diag, and a semi-Lagrangian depth mean.
"""
import numpy as np
import pytest

import sw_inputs as si
from oracle import SWOracle, rel_l2

from _helpers import gpu, oracle_keys, run_gpu_interval

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

FIELDS = ("zeta", "u", "v")


@pytest.fixture(scope="module")
def lm():
    return gpu()


def _grid(N):
    x = 2 * np.pi * np.arange(N) / N
    return np.meshgrid(x, x)


@pytest.mark.parametrize("stepper", ["heun", "rk4"])
@pytest.mark.parametrize("strategy", [1, 2])
@pytest.mark.parametrize("N", [32, 64])
def test_matches_oracle_fp64(lm, stepper, strategy, N):
    n, dt = 24, 5e-3
    uvz = si.vortex_pair(N)
    g, gs = run_gpu_interval(lm, N, dt, uvz, strategy, n, fields=FIELDS, chunks=[7, n - 7], model="euler2d",
                             stepper=stepper, nu8=0.0)
    o = SWOracle(N, dt, *uvz, model="euler2d", stepper=stepper)
    o.lmean_begin(strategy, fields=FIELDS, pos=True, eulerian=True, n_steps=n)
    o.lmean_step(n)
    r = oracle_keys(o.lmean_end())
    X, Y = _grid(N)
    for k, ref in r.items():
        a = g[k]
        if k == "pos_x":
            a, ref = a - X, ref - X
        elif k == "pos_y":
            a, ref = a - Y, ref - Y
        assert rel_l2(a, ref) < 1e-12, (k, rel_l2(a, ref))
    for a, b in zip(gs, o.fields()):
        assert rel_l2(a, b) < 1e-12


def _merger(lm, dt, T=25.0, N=128, precision="f64"):
    n = int(round(T / dt))
    h = lm.sw_create(lm.make_params(N, dt, precision=precision, model="euler2d", stepper="heun", nu8=0.0),
                     np.ascontiguousarray(np.stack(si.vortex_pair(N))))
    try:
        lm.lmean_begin(h, lm.make_lm_params(1, ("zeta",), pos=True, eulerian=False, n_steps=n))
        lm.lmean_step(h, n)
        out = {k: np.zeros((N, N)) for k in ("zeta", "pos_x", "pos_y")}
        lm.lmean_end(h, out)
        uvz = np.zeros((3, N, N))
        lm.sw_get_fields(h, uvz)
    finally:
        lm.sw_destroy(h)
    return out, uvz[2]


def test_vortex_merger_material_conservation(lm):
    # the paper's setup; then dt halved
    out1, z1 = _merger(lm, 5e-3)
    out2, z2 = _merger(lm, 2.5e-3)
    e1, e2 = rel_l2(out1["zeta"], z1), rel_l2(out2["zeta"], z2)
    assert e1 < 1e-2, e1
    assert 3.2 < e1 / e2 < 4.8, (e1, e2)
    # the two runs agree on zeta(T) to the stepper's error
    assert rel_l2(z1, z2) < 0.2


def test_vortex_merger_pseudospectral_beats_semi_lagrangian(lm):
    N, dt, T = 128, 5e-3, 25.0
    n = int(round(T / dt))
    ps, zT = _merger(lm, dt)
    err = {"pseudospectral": rel_l2(ps["zeta"], zT)}
    for interp in ("linear", "cubic"):
        h = lm.sw_create(lm.make_params(N, dt, precision="f64", model="euler2d", stepper="heun", nu8=0.0),
                         np.ascontiguousarray(np.stack(si.vortex_pair(N))))
        try:
            s = lm.sw_sl_create(h, lm.make_sl_params(("zeta",), pos=True, scheme="trapezoid", interp=interp,
                                                     n_steps=n))
            lm.sw_sl_step(s, n)
            out = {k: np.zeros((N, N)) for k in ("zeta", "pos_x", "pos_y")}
            lm.sw_sl_end(s, out)
            uvz = np.zeros((3, N, N))
            lm.sw_get_fields(h, uvz)
        finally:
            lm.sw_destroy(h)
        err[interp] = rel_l2(out["zeta"], uvz[2])
    assert err["pseudospectral"] < err["cubic"] < err["linear"], err


def test_error_codes(lm):
    N = 32
    h = lm.sw_create(lm.make_params(N, 5e-3, precision="f64", model="euler2d"),
                     np.ascontiguousarray(np.stack(si.vortex_pair(N))))
    try:
        for f in (("zeta", "h"), ("q",)):
            with pytest.raises(lm.SWError) as ei:
                lm.lmean_begin(h, lm.make_lm_params(1, f, n_steps=2))
            assert ei.value.code == lm.api.SW_EINVAL
        with pytest.raises(lm.SWError) as ei:
            lm.sw_diag(h)
        assert ei.value.code == lm.api.SW_EINVAL
        with pytest.raises(lm.SWError) as ei:
            lm.sw_sl_create(h, lm.make_sl_params(("h",), n_steps=2))
        assert ei.value.code == lm.api.SW_EINVAL
    finally:
        lm.sw_destroy(h)
