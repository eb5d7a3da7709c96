"""Pins of the Strategy-1 remap oracle (Eq. remap-strat1) to closed forms.

No GPU.  The remap evaluates fbar^L(y) = f~^L(Xi(y)) with Xi the inverse of
the Strategy-1 mean-position map Xi^{-1}; these tests check it against maps
whose inverse is known exactly, against the exact inverse of a 2D map found
by Newton's method on the analytic functions (no interpolation), and
against the Strategy-2 solver, which computes the same fbar^L directly.
"""
import numpy as np
import pytest

import sw_inputs as si
from oracle import SWOracle, rel_l2
from oracle.remap import grid, remap_strategy1


def _F(X, Y):
    return np.cos(2 * X + Y) + 0.5 * np.sin(X - 3 * Y)


def test_identity_map_returns_the_input():
    N = 16
    X, Y = grid(N)
    f = np.random.default_rng(1).standard_normal((N, N))
    out, xx, yy, res = remap_strategy1({"f": f}, X.copy(), Y.copy(), iters=5)
    assert np.array_equal(out["f"], f)
    assert np.array_equal(xx, X) and np.array_equal(yy, Y)
    assert res.max() == 0.0


def test_whole_cell_shift_is_an_exact_roll():
    # Xi^{-1}(x) = x - c with c = (3, -2) cells: Xi(y) = y + c, so
    # fbar^L(y) = f~^L(y + c), a periodic roll of the grid field (to the
    # rounding of x - Xi^{-1}(x), which puts the point a few ulps off the node).
    N = 32
    dx = 2 * np.pi / N
    X, Y = grid(N)
    f = np.random.default_rng(2).standard_normal((N, N))
    out, xx, yy, _ = remap_strategy1({"f": f}, X - 3 * dx, Y + 2 * dx, iters=4)
    np.testing.assert_allclose(out["f"], np.roll(np.roll(f, -3, axis=1), 2, axis=0), rtol=0, atol=1e-13)
    np.testing.assert_allclose(xx - X, 3 * dx, rtol=0, atol=1e-14)
    np.testing.assert_allclose(yy - Y, -2 * dx, rtol=0, atol=1e-14)


def test_shear_map_exact_inverse_and_second_order():
    # Xi^{-1}(x, y) = (x - eps sin y, y): Xi(y) = (y1 + eps sin y2, y2) exactly
    # (the displacement is constant along x, so its interpolant is exact), and
    # fbar^L = F(Xi(y)) for f~^L = F up to the bilinear error in x.
    eps = 0.3
    errs = []
    for N in (32, 64, 128):
        X, Y = grid(N)
        out, xx, yy, _ = remap_strategy1({"f": _F(X, Y)}, X - eps * np.sin(Y), Y.copy(), iters=3)
        np.testing.assert_allclose(xx, X + eps * np.sin(Y), rtol=0, atol=1e-13)
        np.testing.assert_allclose(yy, Y, rtol=0, atol=0)
        errs.append(np.abs(out["f"] - _F(xx, yy)).max())
    assert errs[-1] < 2e-3
    for a, b in zip(errs, errs[1:]):
        assert 3.4 < a / b < 4.6


def _exact_lift(Xg, Yg, eps, n=60):
    # Newton's method on Xi^{-1}(p) = p - eps (sin p_y, sin p_x) = y (analytic)
    px, py = Xg.copy(), Yg.copy()
    for _ in range(n):
        rx = px - eps * np.sin(py) - Xg
        ry = py - eps * np.sin(px) - Yg
        a, b = 1.0, -eps * np.cos(py)
        c, d = -eps * np.cos(px), 1.0
        det = a * d - b * c
        px, py = px - (d * rx - b * ry) / det, py - (-c * rx + a * ry) / det
    return px, py


def test_two_dimensional_map_against_newton_inverse():
    eps = 0.25
    errs_pos, errs_f = [], []
    for N in (32, 64, 128):
        X, Y = grid(N)
        pos_x = X - eps * np.sin(Y)
        pos_y = Y - eps * np.sin(X)
        out, xx, yy, res = remap_strategy1({"f": _F(X, Y)}, pos_x, pos_y, iters=40)
        ex, ey = _exact_lift(X, Y, eps)
        assert res.max() < 1e-12  # contraction: |grad d| <= eps
        errs_pos.append(max(np.abs(xx - ex).max(), np.abs(yy - ey).max()))
        errs_f.append(np.abs(out["f"] - _F(ex, ey)).max())
    assert errs_pos[-1] < 1e-3 and errs_f[-1] < 5e-3
    for e in (errs_pos, errs_f):
        for a, b in zip(e, e[1:]):
            assert 3.2 < a / b < 4.8


def test_fixed_point_converges_geometrically():
    N = 64
    eps = 0.25
    X, Y = grid(N)
    pos_x, pos_y = X - eps * np.sin(Y), Y - eps * np.sin(X)
    r = [remap_strategy1({}, pos_x, pos_y, iters=k)[3].max() for k in (4, 8, 12)]
    assert r[0] > r[1] > r[2] > 0
    assert r[1] / r[0] < eps ** 3 and r[2] / r[1] < eps ** 3


@pytest.mark.parametrize("field", ["zeta", "u"])
def test_remapped_strategy1_matches_strategy2(field):
    # Both give fbar^L on the mean-position grid: Strategy 2 directly, Strategy
    # 1 through Eq. (remap-strat1).  They agree to the order of the bilinear
    # interpolation both use, and Xi agrees with the Strategy-2 positions.
    errs = []
    for N in (32, 64):
        u, v, h = si.smooth_flow(N, 2, seed=21, uamp=0.15, eamp=0.05)
        out = {}
        for s in (1, 2):
            o = SWOracle(N, 5e-3, u, v, h)
            o.lmean_begin(s, fields=(field,), pos=True, eulerian=False, n_steps=200)
            o.lmean_step(200)
            out[s] = o.lmean_end()
        fb, xx, yy, res = remap_strategy1({field: out[1][field]}, out[1]["pos_x"], out[1]["pos_y"], iters=30)
        assert res.max() < 1e-12
        X, Y = grid(N)
        ref = out[2][field]
        errs.append((rel_l2(fb[field] - ref.mean(), ref - ref.mean()),
                     rel_l2(np.concatenate([(xx - X).ravel(), (yy - Y).ravel()]),
                            np.concatenate([(out[2]["pos_x"] - X).ravel(), (out[2]["pos_y"] - Y).ravel()]))))
    assert errs[-1][0] < 2e-2 and errs[-1][1] < 2e-2
    assert errs[0][0] > 2.5 * errs[1][0]
