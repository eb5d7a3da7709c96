"""Pins of the oracle's alternative steppers and viscosity (the paper's own
setup: Heun, Sec. 4.1; forward Euler and the Laplacian viscosity, Sec. 4.2.1).

No GPU.  For a uniform flow only the Coriolis term acts, so u + i v is
multiplied each step by the stepper's stability polynomial R(-i f0 dt); with
a Laplacian on a single small mode the integrating factor makes the damping
exact, z_n = (exp(-nu |k|^2 dt) R(-i f0 dt))^n z_0; on a nonlinear flow with
an open Strategy-1 interval (whose right-hand sides depend on the stage time
through s u) the error against a fine RK4 reference falls at the stepper's
order under dt halving.
"""
import math

import numpy as np
import pytest

import sw_inputs as si
from oracle import SWOracle, rel_l2

R = {"euler": lambda z: 1 + z, "heun": lambda z: 1 + z + z * z / 2,
     "rk4": lambda z: 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24}


@pytest.mark.parametrize("stepper", ["euler", "heun"])
def test_uniform_inertial_oscillation(stepper):
    N, dt, f0, U0, n = 16, 5e-3, 1.3, 0.7, 300
    u, v, h = si.uniform_flow(N, U0, 0.0)
    o = SWOracle(N, dt, u, v, h, f0=f0, stepper=stepper)
    o.lmean_begin(1, fields=("u", "v"), pos=True, eulerian=True, n_steps=n)
    o.lmean_step(n)
    z = U0 * R[stepper](-1j * f0 * dt) ** n
    uu, vv, _ = o.fields()
    assert abs(uu.mean() - z.real) < 1e-13 and abs(vv.mean() - z.imag) < 1e-13
    assert np.abs(uu - uu.mean()).max() < 1e-14


@pytest.mark.parametrize("stepper", ["euler", "heun", "rk4"])
@pytest.mark.parametrize("n", [1, 2, 9])
def test_strategy2_uniform_flow_exact(stepper, n):
    # Strategy 2 (Eqs. xi_evol, barf_xi) in a uniform flow U with f0 = 0: the
    # flow stays uniform and every gradient vanishes, so the equations reduce
    # to d xi/ds = U - xi/s and d g/ds = f(x + xi) = U, whose solutions from
    # xi = g = 0 are xi = U s/2 (the partial mean position of Eq. (barphi)
    # moves at half the particle speed) and g = U s.  Forward Euler's first
    # step is xi_1 = dt (U - w(0)), so it reproduces them only with the limit
    # w = u/2 at s = 0; Heun and RK4 are exact for any value of that limit
    # (their later stages cancel it), which this also checks: the stage
    # combinations of every stepper carry the -w term and the stage times.
    N, dt, U0, V0 = 16, 5e-3, 0.7, -0.3
    u, v, h = si.uniform_flow(N, U0, V0)
    o = SWOracle(N, dt, u, v, h, f0=0.0, stepper=stepper)
    o.lmean_begin(2, fields=("zeta", "h", "u", "v"), pos=True, eulerian=True, n_steps=n)
    o.lmean_step(n)
    r = o.lmean_end()
    T = n * dt
    x = 2 * np.pi * np.arange(N) / N
    X, Y = np.meshgrid(x, x)
    np.testing.assert_allclose(r["pos_x"] - X, U0 * T / 2, atol=1e-15)
    np.testing.assert_allclose(r["pos_y"] - Y, V0 * T / 2, atol=1e-15)
    np.testing.assert_allclose(r["u"], U0, atol=1e-14)
    np.testing.assert_allclose(r["v"], V0, atol=1e-14)
    np.testing.assert_allclose(r["h"], 1.0, atol=1e-14)
    np.testing.assert_allclose(r["zeta"], 0.0, atol=1e-14)
    np.testing.assert_allclose(r["E_u"], U0, atol=1e-14)


@pytest.mark.parametrize("stepper", ["euler", "heun", "rk4"])
def test_laplacian_integrating_factor_exact(stepper):
    N, dt, f0, n = 16, 1e-2, 1.3, 120
    kx, ky = 2, 1
    nu = 0.2 / (kx * kx + ky * ky)
    x = 2 * np.pi * np.arange(N) / N
    X, Y = np.meshgrid(x, x)
    eps = 1e-9
    u = eps * np.cos(kx * X + ky * Y)
    v = eps * 0.3 * np.sin(kx * X + ky * Y)
    o = SWOracle(N, dt, u, v, 1.0 + 0 * u, f0=f0, c2=0.0, nu8=nu, stepper=stepper, visc="laplace")
    z0 = o.uh[ky, kx] + 1j * o.vh[ky, kx]
    o.step(n)
    z1 = o.uh[ky, kx] + 1j * o.vh[ky, kx]
    amp = math.exp(-nu * (kx * kx + ky * ky) * dt) * R[stepper](-1j * f0 * dt)
    assert abs(z1 - z0 * amp ** n) < 1e-6 * abs(z0)


def _run(stepper, dt, T=0.4, N=32):
    u, v, h = si.smooth_flow(N, 2, seed=8, uamp=0.15, eamp=0.05)
    n = int(round(T / dt))
    o = SWOracle(N, dt, u, v, h, nu8=0.0, stepper=stepper)
    o.lmean_begin(1, fields=("zeta",), pos=True, eulerian=False, n_steps=n)
    o.lmean_step(n)
    return o.lmean_end()


@pytest.mark.parametrize("stepper,order", [("euler", 1), ("heun", 2)])
def test_order_of_accuracy_with_an_open_interval(stepper, order):
    ref = _run("rk4", 1e-3 / 4)
    errs = []
    for dt in (4e-3, 2e-3):
        out = _run(stepper, dt)
        errs.append(max(rel_l2(out["zeta"], ref["zeta"]), np.abs(out["pos_x"] - ref["pos_x"]).max()))
    ratio = errs[0] / errs[1]
    assert 2 ** order * 0.8 < ratio < 2 ** order * 1.25, (errs, ratio)


@pytest.mark.parametrize("visc", ["laplace", "hyper8"])
def test_viscosity_placement_on_depth(visc):
    # at rest with c2 = 0 the depth perturbation has no dynamics: the
    # Laplacian of Eq. (sw_momentum_dimless) leaves it unchanged (the mass
    # equation has no viscous term); the hyperviscosity damps each mode by
    # exp(-nu |k|^8 t)
    N, dt, n, nu = 16, 1e-2, 50, 3e-4
    x = 2 * np.pi * np.arange(N) / N
    X, Y = np.meshgrid(x, x)
    kx, ky = 3, 2
    h = 1.0 + 0.1 * np.cos(kx * X + ky * Y)
    o = SWOracle(N, dt, 0 * X, 0 * X, h, f0=0.7, c2=0.0, nu8=nu, stepper="heun", visc=visc)
    e0 = o.hh[ky, kx]
    o.step(n)
    k2 = kx * kx + ky * ky
    damp = 1.0 if visc == "laplace" else math.exp(-nu * k2 ** 4 * dt * n)
    assert abs(o.hh[ky, kx] - e0 * damp) < 1e-14
    assert np.abs(o.uh).max() < 1e-300 and np.abs(o.vh).max() < 1e-300


def test_paper_setup_initial_condition():
    # Sec. 4.2.1: f0 = 1/Ro = 10, c2 = 1/Fr^2 = 4, omega = 10.2; the stand-in
    # turbulence (the initial condition minus the Eq. (initial_wave) wave) has
    # the requested rms velocity and is in geostrophic balance,
    # f0 z x u = -c2 grad eta
    N = 64
    (u, v, h), p = si.paper_sw_setup(N)
    assert p["f0"] == 10.0 and p["c2"] == 4.0 and p["n_steps"] == 17600
    assert abs(si.wave_frequency(1.0, p["f0"], p["c2"]) - 10.2) < 5e-3
    uw, vw, hw = si.mode1_wave(N, -1.8, p["f0"], p["c2"])
    ub, vb, eb = u - uw, v - vw, h - hw
    assert abs(np.sqrt(np.mean(ub * ub + vb * vb)) - 0.3) < 1e-12
    k = np.fft.fftfreq(N, 1.0 / N)
    KX, KY = np.meshgrid(k, k)
    ex = np.real(np.fft.ifft2(1j * KX * np.fft.fft2(eb)))
    ey = np.real(np.fft.ifft2(1j * KY * np.fft.fft2(eb)))
    np.testing.assert_allclose(-p["f0"] * vb, -p["c2"] * ex, atol=1e-12)
    np.testing.assert_allclose(p["f0"] * ub, -p["c2"] * ey, atol=1e-12)
    assert h.min() > 0.2


def test_xi_first_uniform_flow_exact():
    # Sec. 4.2's xi-first discretisation with the mean equations stepping by
    # 2 dt: in a uniform flow (f0 = 0) the partial mean displacement is
    # xi = U s/2 and the mean of u is U exactly, at every completed mean step
    N, dt, U0, V0, n = 16, 5e-3, 0.7, -0.3, 40
    u, v, h = si.uniform_flow(N, U0, V0)
    o = SWOracle(N, dt, u, v, h, f0=0.0, stepper="euler")
    o.lmean_begin(2, fields=("u", "v"), pos=True, eulerian=False, n_steps=n, scheme="xi_first")
    o.lmean_step(n)
    r = o.lmean_end()
    T = n * dt
    x = 2 * np.pi * np.arange(N) / N
    X, Y = np.meshgrid(x, x)
    np.testing.assert_allclose(r["pos_x"] - X, U0 * T / 2, atol=1e-14)
    np.testing.assert_allclose(r["pos_y"] - Y, V0 * T / 2, atol=1e-14)
    np.testing.assert_allclose(r["u"], U0, atol=1e-14)
    np.testing.assert_allclose(r["v"], V0, atol=1e-14)


def _run_xi_first(dt, T=0.4, N=32):
    u, v, h = si.smooth_flow(N, 2, seed=8, uamp=0.15, eamp=0.05)
    n = int(round(T / dt))
    o = SWOracle(N, dt, u, v, h, nu8=0.0, stepper="euler")
    o.lmean_begin(2, fields=("zeta", "u"), pos=True, eulerian=False, n_steps=n, scheme="xi_first")
    o.lmean_step(n)
    return o.lmean_end()


def test_xi_first_first_order_against_a_fine_reference():
    u, v, h = si.smooth_flow(32, 2, seed=8, uamp=0.15, eamp=0.05)
    o = SWOracle(32, 1e-3 / 4, u, v, h, nu8=0.0)
    n = int(round(0.4 / (1e-3 / 4)))
    o.lmean_begin(2, fields=("zeta", "u"), pos=True, eulerian=False, n_steps=n)
    o.lmean_step(n)
    ref = o.lmean_end()
    errs = []
    for dt in (4e-3, 2e-3):
        out = _run_xi_first(dt)
        errs.append(max(rel_l2(out["zeta"], ref["zeta"]), rel_l2(out["u"], ref["u"]),
                        np.abs(out["pos_x"] - ref["pos_x"]).max()))
    ratio = errs[0] / errs[1]
    assert 2 * 0.8 < ratio < 2 * 1.25, (errs, ratio)


def test_xi_first_needs_strategy2_euler_and_even_steps():
    u, v, h = si.smooth_flow(16, 2, seed=1)
    with pytest.raises(ValueError):
        SWOracle(16, 1e-3, u, v, h, stepper="euler").lmean_begin(1, n_steps=4, scheme="xi_first")
    with pytest.raises(ValueError):
        SWOracle(16, 1e-3, u, v, h, stepper="heun").lmean_begin(2, n_steps=4, scheme="xi_first")
    with pytest.raises(ValueError):
        SWOracle(16, 1e-3, u, v, h, stepper="euler").lmean_begin(2, n_steps=5, scheme="xi_first")
