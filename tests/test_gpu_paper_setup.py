"""GPU run of Sec. 4.2.1's first shallow-water set-up: Ro = 0.1, Fr = 0.5,
the Laplacian at Re = 3840 on the momentum, a mode-1 Poincare wave of
amplitude -1.8 (Eq. initial_wave) on balanced turbulence (a synthetic
stand-in for the paper's Navier-Stokes field), forward Euler with dt =
1.25e-4, Strategy 2 with bilinear interpolation, inviscid mean equations:
against the oracle at 64^2 over 60 steps (FP64; zeta and q, positions,
Eulerian means, state), relative L2 <= 1e-12.  (The PV rearrangement of
Sec. 4.2.1 is checked on a smooth inviscid flow in test_gpu_diagnostics.py:
with this stand-in the wave steepens into fronts at 64^2-128^2.)
"""
import numpy as np
import pytest

import sw_inputs as si
from oracle import SWOracle, rel_l2

from _helpers import gpu, oracle_keys

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

FIELDS = ("zeta", "q")


@pytest.fixture(scope="module")
def lm():
    return gpu()


def _params(lm, N, p, precision):
    return lm.make_params(N, p["dt"], precision=precision, f0=p["f0"], c2=p["c2"], nu8=p["nu"], lm_nu8=0.0,
                          stepper="euler", visc="laplace")


def test_matches_oracle_fp64(lm):
    N, n = 64, 60
    uvh, p = si.paper_sw_setup(N)
    h = lm.sw_create(_params(lm, N, p, "f64"), np.ascontiguousarray(np.stack(uvh)))
    try:
        lm.lmean_begin(h, lm.make_lm_params(2, FIELDS, pos=True, eulerian=True, n_steps=n))
        lm.lmean_step(h, 25)
        lm.lmean_step(h, n - 25)
        keys = list(FIELDS) + ["pos_x", "pos_y"] + ["e_" + f for f in FIELDS]
        g = {k: np.zeros((N, N)) for k in keys}
        lm.lmean_end(h, g)
        gs = lm.sw_get_fields(h, np.zeros((3, N, N)))
    finally:
        lm.sw_destroy(h)
    o = SWOracle(N, p["dt"], *uvh, f0=p["f0"], c2=p["c2"], nu8=p["nu"], lm_nu8=0.0, stepper="euler",
                 visc="laplace")
    o.lmean_begin(2, fields=FIELDS, pos=True, eulerian=True, n_steps=n)
    o.lmean_step(n)
    r = oracle_keys(o.lmean_end())
    x = 2 * np.pi * np.arange(N) / N
    X, Y = np.meshgrid(x, x)
    for k, ref in r.items():
        a = g[k]
        if k == "pos_x":
            a, ref = a - X, ref - X
        elif k == "pos_y":
            a, ref = a - Y, ref - Y
        else:
            a, ref = a - ref.mean(), ref - ref.mean()
        assert rel_l2(a, ref) < 1e-12, (k, rel_l2(a, ref))
    ou, ov, oh = o.fields()
    assert rel_l2(gs[0], ou) < 1e-12 and rel_l2(gs[1], ov) < 1e-12 and rel_l2(gs[2] - 1, oh - 1) < 1e-12
