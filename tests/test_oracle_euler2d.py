"""Pins of the oracle's two-dimensional Euler model (Sec. 4.1's test flow).

No GPU.  The model carries the vorticity and slaves the velocity to it
through the streamfunction.  Pinned against:

* closed forms: zeta = 2 sin x sin y has u = sin x cos y, v = -cos x sin y and
  is a steady state; for a band-limited zeta whose products stay inside the
  2/3 box the right-hand side equals -u.grad zeta computed analytically;
* invariants of the inviscid flow: the mean vorticity (exactly, the k = 0
  coefficient), kinetic energy and enstrophy (to the stepper's error);
* material conservation, Eq. (vorticity_itsmean): for f = zeta the function
  g = (t - tau) zeta solves Eq. (gtilde-evol) exactly in the semi-discrete
  system, so Strategy 1's zeta~^L equals zeta(tau + T) up to the time
  stepping alone: the difference falls at the stepper's order (Heun 2, RK4
  4) under dt halving, on the paper's vortex-pair initial condition.
"""
import numpy as np
import pytest

import sw_inputs as si
from oracle import SWOracle, rel_l2


def _grid(N):
    x = 2 * np.pi * np.arange(N) / N
    return np.meshgrid(x, x)


def test_velocity_from_vorticity_and_steady_cellular_flow():
    N = 16
    X, Y = _grid(N)
    z0 = np.zeros((N, N))
    o = SWOracle(N, 1e-2, z0, z0, 2 * np.sin(X) * np.sin(Y), model="euler2d")
    u, v, zeta = o.fields()
    np.testing.assert_allclose(u, np.sin(X) * np.cos(Y), atol=1e-14)
    np.testing.assert_allclose(v, -np.cos(X) * np.sin(Y), atol=1e-14)
    o.step(50)
    np.testing.assert_allclose(o.fields()[2], 2 * np.sin(X) * np.sin(Y), atol=1e-13)


def test_rhs_is_analytic_advection():
    N, a, b, c = 32, 0.7, -0.4, 0.9
    X, Y = _grid(N)
    zeta = a * np.cos(X) + b * np.cos(2 * Y) + c * np.sin(X + Y)
    z0 = np.zeros((N, N))
    o = SWOracle(N, 1e-2, z0, z0, zeta, model="euler2d")
    # psi_k = -zeta_k/|k|^2 per mode; u = -d_y psi, v = d_x psi
    u = -(b / 2) * np.sin(2 * Y) + (c / 2) * np.cos(X + Y)
    v = a * np.sin(X) - (c / 2) * np.cos(X + Y)
    zx = -a * np.sin(X) + c * np.cos(X + Y)
    zy = -2 * b * np.sin(2 * Y) + c * np.cos(X + Y)
    uu, vv, _ = o.fields()
    np.testing.assert_allclose(uu, u, atol=1e-14)
    np.testing.assert_allclose(vv, v, atol=1e-14)
    rhs = o._rhs(o._state(), 0.0)["sw"]
    np.testing.assert_allclose(o.phys(rhs[2]), -(u * zx + v * zy), atol=1e-13)
    assert np.abs(rhs[0]).max() == 0 and np.abs(rhs[1]).max() == 0


def test_invariants_of_the_vortex_pair():
    N, n = 32, 200
    o = SWOracle(N, 5e-3, *si.vortex_pair(N), model="euler2d", stepper="rk4")
    m0 = o.hh[0, 0]
    _, e0, z0 = o.diag()
    o.step(n)
    _, e1, z1 = o.diag()
    assert o.hh[0, 0] == m0  # the mean vorticity takes no tendency
    assert abs(e1 - e0) / e0 < 1e-9 and abs(z1 - z0) / z0 < 1e-9


def _material_error(stepper, dt, N=32, T=1.0):
    o = SWOracle(N, dt, *si.vortex_pair(N), model="euler2d", stepper=stepper)
    n = int(round(T / dt))
    o.lmean_begin(1, fields=("zeta",), pos=True, eulerian=False, n_steps=n)
    o.lmean_step(n)
    r = o.lmean_end()
    return rel_l2(r["zeta"], o.fields()[2])


@pytest.mark.parametrize("stepper,order", [("heun", 2), ("rk4", 4)])
def test_material_conservation_at_the_steppers_order(stepper, order):
    e1, e2 = _material_error(stepper, 1e-2), _material_error(stepper, 5e-3)
    assert e1 < (3e-6 if stepper == "heun" else 2e-11)
    ratio = e1 / e2
    assert 2 ** order * 0.9 < ratio < 2 ** order * 1.1, (e1, e2, ratio)


def test_rejects_depth_and_pv_means():
    o = SWOracle(16, 1e-2, *si.vortex_pair(16), model="euler2d")
    with pytest.raises(ValueError):
        o.lmean_begin(1, fields=("zeta", "h"), n_steps=2)
    with pytest.raises(ValueError):
        o.lmean_begin(2, fields=("q",), n_steps=2)


def test_fig3_ordering_of_the_three_discretisations():
    # Fig. 3 (Sec. 4.1, App. B): for the materially conserved vorticity the
    # pseudospectral zeta~^L is closest to zeta(T), the semi-Lagrangian one
    # with cubic interpolation next, with linear interpolation last
    from oracle.gbla import SLInterval
    N, dt, n = 32, 1e-2, 300
    o = SWOracle(N, dt, *si.vortex_pair(N), model="euler2d", stepper="heun")
    o.lmean_begin(1, fields=("zeta",), pos=True, eulerian=False, n_steps=n)
    o.lmean_step(n)
    err = {"pseudospectral": rel_l2(o.lmean_end()["zeta"], o.fields()[2])}
    for interp in ("linear", "cubic"):
        sl = SLInterval(SWOracle(N, dt, *si.vortex_pair(N), model="euler2d", stepper="heun"), fields=("zeta",),
                        scheme="trapezoid", interp=interp, n_steps=n)
        sl.step(n)
        err[interp] = rel_l2(sl.end()["zeta"], sl.o.fields()[2])
    assert err["pseudospectral"] < 1e-4 < err["cubic"] < err["linear"], err
