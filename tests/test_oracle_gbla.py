"""Pins of the semi-Lagrangian Strategy-1 oracle (App. B).

No GPU.  With a uniform velocity that moves one grid cell per step, every
departure point is a grid point, so the recursions of Eqs.
(sdiscrete_gtilde) and (sdiscrete_gtilde_trapez) become sums along exact
characteristics that a test can form from the run's own state history by
rolling the arrays; the mean positions have closed forms.  On a shallow-
water flow the trapezoidal rule with cubic interpolation approaches the
spectral Strategy 1 (Eq. gtilde-evol) as the grid is refined, and is much
closer to it than backward Euler with linear interpolation.
"""
import numpy as np
import pytest

import sw_inputs as si
from oracle import SWOracle, rel_l2
from oracle.gbla import SLInterval, interp_cubic, interp_linear, lagrange4


def _grid(N):
    x = 2 * np.pi * np.arange(N) / N
    return np.meshgrid(x, x)


def test_interpolants_reproduce_polynomials_and_nodes():
    N = 16
    X, Y = _grid(N)
    f = np.random.default_rng(4).standard_normal((N, N))
    z = np.zeros((N, N))
    assert np.array_equal(interp_linear(f, z, z), f)
    np.testing.assert_allclose(interp_cubic(f, z, z), f, rtol=0, atol=1e-15)
    # Lagrange weights: partition of unity, exact on cubics
    a = np.linspace(0, 1, 7)
    w = lagrange4(a)
    np.testing.assert_allclose(sum(w), 1.0, atol=1e-15)
    for p in range(4):
        np.testing.assert_allclose(sum(wk * (k ** p) for wk, k in zip(w, (-1, 0, 1, 2))), a ** p, atol=1e-14)
    # bilinear exact on a field linear in x within one cell
    dx = 2 * np.pi / N
    np.testing.assert_allclose(interp_linear(X, 0.3 * dx + z, z)[:, :-1], (X + 0.3 * dx)[:, :-1], atol=1e-14)


@pytest.mark.parametrize("scheme", ["euler", "trapezoid"])
@pytest.mark.parametrize("interp", ["linear", "cubic"])
def test_one_cell_per_step_matches_characteristic_sums(scheme, interp):
    N, dt, n = 32, 5e-3, 12
    dx = 2 * np.pi / N
    X, Y = _grid(N)
    cx, cy = dx / dt, -dx / dt  # one cell in +x and one in -y per step
    F0 = np.cos(X + 0.3) + 0.5 * np.sin(Y - X)
    args = dict(model="kinematic", adv=(cx, cy), nu8=0.0, lm_nu8=0.0)
    # the run's state history
    o = SWOracle(N, dt, F0, 0 * X, 1 + 0.1 * F0, **args)
    hist = [o.fields()[0].copy()]
    for _ in range(n):
        o.step(1)
        hist.append(o.fields()[0].copy())
    # the semi-Lagrangian interval on an identical run
    o2 = SWOracle(N, dt, F0, 0 * X, 1 + 0.1 * F0, **args)
    sl = SLInterval(o2, fields=("u",), scheme=scheme, interp=interp, n_steps=n)
    sl.step(n)
    out = sl.end()
    T = n * dt

    def at_end(k):  # f(X - c (T - t_k), t_k): k steps of history moved n - k cells
        return np.roll(np.roll(hist[k], n - k, axis=1), -(n - k), axis=0)

    if scheme == "euler":
        g = sum(dt * at_end(k) for k in range(1, n + 1))
        w = 0.0
    else:
        g = sum(dt * (at_end(k - 1) + at_end(k)) / 2 for k in range(1, n + 1))
        w = 0.5
    np.testing.assert_allclose(out["u"], g / T, rtol=0, atol=1e-12)
    # mean positions: D = sum_k (s_k + w dt) dt c, uniform in space
    shift = (T - dt + 2 * w * dt) / 2
    np.testing.assert_allclose(out["pos_x"], X - cx * shift, rtol=0, atol=1e-12)
    np.testing.assert_allclose(out["pos_y"], Y - cy * shift, rtol=0, atol=1e-12)


def test_approaches_the_spectral_strategy1():
    errs = {}
    for N in (32, 64):
        u, v, h = si.smooth_flow(N, 2, seed=21, uamp=0.15, eamp=0.05)
        o = SWOracle(N, 5e-3, u, v, h)
        o.lmean_begin(1, fields=("zeta", "u"), pos=True, eulerian=False, n_steps=200)
        o.lmean_step(200)
        ref = o.lmean_end()
        for scheme, interp in (("euler", "linear"), ("trapezoid", "cubic")):
            sl = SLInterval(SWOracle(N, 5e-3, u, v, h), fields=("zeta", "u"), scheme=scheme, interp=interp,
                            n_steps=200)
            sl.step(200)
            out = sl.end()
            errs[(N, scheme)] = max(rel_l2(out["zeta"], ref["zeta"]), rel_l2(out["u"], ref["u"]))
    assert errs[(64, "trapezoid")] < 2e-3
    assert errs[(32, "trapezoid")] > 1.5 * errs[(64, "trapezoid")]
    for N in (32, 64):
        assert errs[(N, "euler")] > 5 * errs[(N, "trapezoid")]
