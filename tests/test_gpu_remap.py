"""GPU checks of lmean_remap (Strategy-1 remap, Eq. remap-strat1).

* Against the oracle on the same inputs, bit for bit: the kernel rounds
  every FP64 operation separately in the oracle's order, so fbar^L, Xi and
  the residual must be identical (grids 16^2 to 1024^2, smooth random maps
  and fields; and the outputs of an oracle Strategy-1 interval).
* Edge cases: one iteration (Xi = y + d(y) exactly), no fields, the
  identity map, a whole-cell shift.
* At the bench workload (256^2, one full interval, FP64): the GPU Strategy-1
  run remapped agrees with the GPU Strategy-2 run (same fbar^L computed
  directly) to the order of the bilinear interpolation both use.
"""
import numpy as np
import pytest

import sw_inputs as si
from oracle import SWOracle, rel_l2
from oracle.remap import grid, remap_strategy1

from _helpers import gpu

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lm():
    return gpu()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _smooth_map(N, seed, eps=0.2):
    rng = np.random.default_rng(seed)
    X, Y = grid(N)
    dx = eps * np.sin(Y + 0.3) + 0.05 * si.random_smooth_field(N, 3, rng)
    dy = eps * np.sin(X - 0.7) + 0.05 * si.random_smooth_field(N, 3, rng)
    fields = {"a": si.random_smooth_field(N, 6, rng), "b": si.random_smooth_field(N, 10, rng),
              "c": np.cos(2 * X + Y)}
    return X - dx, Y - dy, fields


def _gpu_remap(lm, pos_x, pos_y, fields, iters):
    out = lm.lmean_remap(_dev(pos_x), _dev(pos_y), {k: _dev(v) for k, v in fields.items()}, iters=iters)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("N,iters", [(16, 7), (64, 20), (256, 20), (1024, 12)])
def test_bit_exact_against_oracle(lm, N, iters):
    pos_x, pos_y, fields = _smooth_map(N, 100 + N)
    g = _gpu_remap(lm, pos_x, pos_y, fields, iters)
    fb, xx, yy, res = remap_strategy1(fields, pos_x, pos_y, iters=iters)
    for k in fields:
        assert np.array_equal(g[k], fb[k]), k
    assert np.array_equal(g["xi_x"], xx) and np.array_equal(g["xi_y"], yy)
    assert np.array_equal(g["resid"], res)
    if iters >= 20:
        assert res.max() < 1e-6  # contraction factor about 0.4 for these maps


def test_bit_exact_on_oracle_strategy1_outputs(lm):
    N = 64
    u, v, h = si.smooth_flow(N, 2, seed=21, uamp=0.15, eamp=0.05)
    o = SWOracle(N, 5e-3, u, v, h)
    o.lmean_begin(1, fields=("zeta", "h", "u", "v"), pos=True, eulerian=False, n_steps=200)
    o.lmean_step(200)
    out = o.lmean_end()
    ft = {k: out[k] for k in ("zeta", "h", "u", "v")}
    g = _gpu_remap(lm, out["pos_x"], out["pos_y"], ft, 25)
    fb, xx, yy, res = remap_strategy1(ft, out["pos_x"], out["pos_y"], iters=25)
    for k in ft:
        assert np.array_equal(g[k], fb[k]), k
    assert np.array_equal(g["xi_x"], xx) and np.array_equal(g["xi_y"], yy)


def test_edge_cases(lm):
    N = 32
    X, Y = grid(N)
    pos_x, pos_y, fields = _smooth_map(N, 7)
    # one iteration: xi = d at the grid point itself
    g = _gpu_remap(lm, pos_x, pos_y, fields, 1)
    assert np.array_equal(g["xi_x"], X + (X - pos_x)) and np.array_equal(g["xi_y"], Y + (Y - pos_y))
    # no fields: positions only
    g0 = _gpu_remap(lm, pos_x, pos_y, {}, 20)
    _, xx, yy, _ = remap_strategy1({}, pos_x, pos_y, iters=20)
    assert np.array_equal(g0["xi_x"], xx) and np.array_equal(g0["xi_y"], yy)
    # identity map
    gi = _gpu_remap(lm, X, Y, fields, 5)
    for k in fields:
        assert np.array_equal(gi[k], fields[k])
    assert gi["resid"].max() == 0.0
    # whole-cell shift: a periodic roll
    dx = 2 * np.pi / N
    gs = _gpu_remap(lm, X - 3 * dx, Y + 2 * dx, fields, 4)
    for k in fields:
        np.testing.assert_allclose(gs[k], np.roll(np.roll(fields[k], -3, axis=1), 2, axis=0), rtol=0, atol=1e-13)


def test_aliasing_rejected(lm):
    N = 32
    pos_x, pos_y, fields = _smooth_map(N, 8)
    px, py = _dev(pos_x), _dev(pos_y)
    a = _dev(fields["a"])
    lib = lm.api.load()
    DP = lm.api._DP
    fin = (DP * 1)(lm.api._ptr(a)[0])
    rc = lib.lmean_remap(N, lm.api._ptr(px)[0], lm.api._ptr(py)[0], 1, fin, fin, 10, None, None, None, None)
    assert rc == lm.api.SW_EINVAL


def test_strategy1_remapped_matches_strategy2_at_bench_size(lm):
    w = si.WORKLOADS["plain-256"]
    N = w.N
    ic = np.ascontiguousarray(np.stack(w.initial_condition()))
    keys = ("zeta", "h", "u", "v")
    res = {}
    for s in (1, 2):
        h = lm.sw_create(lm.make_params(N, w.dt, precision="f64", nu8=w.nu8), ic)
        lm.lmean_begin(h, lm.make_lm_params(s, keys, n_steps=w.n_steps))
        lm.lmean_step(h, w.n_steps)
        out = {k: torch.empty((N, N), dtype=torch.float64, device="cuda") for k in keys + ("pos_x", "pos_y")}
        lm.lmean_end(h, out)
        lm.sw_destroy(h)
        res[s] = out
    r = lm.lmean_remap(res[1]["pos_x"], res[1]["pos_y"], {k: res[1][k] for k in keys}, iters=30)
    torch.cuda.synchronize()
    assert r["resid"].max().item() < 1e-10
    X, Y = grid(N)
    for k in keys:
        a, b = r[k].cpu().numpy(), res[2][k].cpu().numpy()
        e = rel_l2(a - b.mean(), b - b.mean())
        assert e < 0.05, (k, e)
    xi1 = np.concatenate([(r["xi_x"].cpu().numpy() - X).ravel(), (r["xi_y"].cpu().numpy() - Y).ravel()])
    xi2 = np.concatenate([(res[2]["pos_x"].cpu().numpy() - X).ravel(), (res[2]["pos_y"].cpu().numpy() - Y).ravel()])
    assert rel_l2(xi1, xi2) < 0.05
