"""Pins of the diagnostic oracles: fields at lifted positions and shell spectra.

No GPU.  `lift` evaluates fields at the lift map Xi (Sec. 3.2) by the
bilinear rule; it is checked against exact cases, against analytic fields at
second order, and against the paper's statement that the Lagrangian mean PV
is a rearrangement of the PV, qbar^L(x) = q(Xi(x), tau+T) (Sec. 4.2.1), on
an inviscid oracle run.  `spectrum` (Sec. 4.2.2's enstrophy spectra) is
checked against closed forms for single modes, Parseval's identity and a
direct DFT sum on a small grid.
"""
import numpy as np

import sw_inputs as si
from oracle import SWOracle, rel_l2
from oracle.remap import grid, lift, shells, spectrum


def _F(X, Y):
    return np.cos(2 * X + Y) + 0.5 * np.sin(X - 3 * Y)


def test_lift_exact_cases():
    N = 32
    X, Y = grid(N)
    f = np.random.default_rng(3).standard_normal((N, N))
    assert np.array_equal(lift({"f": f}, X.copy(), Y.copy())["f"], f)
    dx = 2 * np.pi / N
    g = lift({"f": f}, X + 2 * dx, Y - 5 * dx)["f"]
    np.testing.assert_allclose(g, np.roll(np.roll(f, -2, axis=1), 5, axis=0), rtol=0, atol=1e-13)
    # a field constant along x is exact under any x-displacement
    h = np.sin(Y)
    np.testing.assert_allclose(lift({"h": h}, X + 0.37, Y.copy())["h"], h, rtol=0, atol=1e-15)


def test_lift_second_order_on_analytic_fields():
    errs = []
    for N in (32, 64, 128):
        X, Y = grid(N)
        px, py = X + 0.3 * np.sin(Y), Y + 0.2 * np.cos(X)
        errs.append(np.abs(lift({"f": _F(X, Y)}, px, py)["f"] - _F(px, py)).max())
    for a, b in zip(errs, errs[1:]):
        assert 3.4 < a / b < 4.6


def _pv(o):
    u, v, h = o.fields()
    zeta = o.phys(o.dx(o.vh) - o.dy(o.uh))
    return (o.f0 + zeta) / h


def test_lagrangian_mean_pv_is_a_rearrangement_of_pv():
    # Sec. 4.2.1: without dissipation q is materially conserved, so
    # qbar^L(x) = q(Xi(x), tau+T); its extrema match those of q, and the
    # Eulerian mean has smaller extrema.  Strategy 2 gives qbar^L and Xi.
    errs = []
    for N in (32, 64):
        u, v, h = si.smooth_flow(N, 2, seed=5, uamp=0.2, eamp=0.05)
        o = SWOracle(N, 5e-3, u, v, h, nu8=0.0, lm_nu8=0.0)
        o.lmean_begin(2, fields=("q",), pos=True, eulerian=True, n_steps=300)
        o.lmean_step(300)
        out = o.lmean_end()
        q_end = _pv(o)
        qx = lift({"q": q_end}, out["pos_x"], out["pos_y"])["q"]
        qbar = out["q"]
        errs.append(rel_l2(qx - qbar.mean(), qbar - qbar.mean()))
        # the Eulerian mean is no rearrangement: further from q(Xi)
        assert rel_l2(qx - qbar.mean(), out["E_q"] - qbar.mean()) > errs[-1]
        span = q_end.max() - q_end.min()
        assert abs(qbar.max() - q_end.max()) < 0.05 * span
        assert abs(qbar.min() - q_end.min()) < 0.05 * span
    assert errs[-1] < 2e-2
    assert errs[0] > 2.0 * errs[1]


def test_spectrum_single_modes_and_box():
    N = 64
    K = (N - 1) // 3
    X, Y = grid(N)
    s = spectrum(0.8 * np.cos(3 * X + 4 * Y + 0.4))
    assert len(s) == shells(N) == int(np.floor(np.sqrt(2) * K + 0.5)) + 1
    np.testing.assert_allclose(s[5], 0.8 ** 2 / 4, rtol=1e-13)
    assert np.abs(np.delete(s, 5)).max() < 1e-28
    # constant mode: shell 0 holds c^2 / 2
    np.testing.assert_allclose(spectrum(np.full((N, N), 1.5))[0], 1.5 ** 2 / 2, rtol=1e-14)
    # a mode outside the 2/3 box is dropped
    assert spectrum(np.cos((K + 1) * X)).max() < 1e-28


def test_spectrum_parseval_and_direct_dft():
    rng = np.random.default_rng(9)
    N = 16
    K = (N - 1) // 3
    f = rng.standard_normal((N, N))
    s = spectrum(f)
    # direct DFT on the box, shell by shell
    X, Y = grid(N)
    ref = np.zeros(shells(N))
    for ky in range(-K, K + 1):
        for kx in range(-K, K + 1):
            F = np.sum(f * np.exp(-1j * (kx * X + ky * Y))) / (N * N)
            ref[int(np.floor(np.hypot(kx, ky) + 0.5))] += 0.5 * abs(F) ** 2
    np.testing.assert_allclose(s, ref, rtol=1e-12, atol=1e-15)
    # Parseval for the box-limited field
    Fb = np.fft.fft2(f) / (N * N)
    k = np.fft.fftfreq(N, 1.0 / N)
    KX, KY = np.meshgrid(k, k)
    Fb[(np.abs(KX) > K) | (np.abs(KY) > K)] = 0
    fb = np.real(np.fft.ifft2(Fb) * N * N)
    np.testing.assert_allclose(s.sum(), 0.5 * np.mean(fb ** 2), rtol=1e-12)
