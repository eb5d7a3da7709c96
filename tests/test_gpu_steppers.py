"""GPU checks of the paper's alternative steppers and viscosity: Heun (Sec.
4.1), forward Euler and the Laplacian viscosity (Sec. 4.2.1).

* Against the oracle on the same FP64 run, both strategies: relative L2
  <= 1e-12 per field (the tolerance of the RK4 parity tests).
* A uniform flow turns at the Coriolis frequency, multiplied each step by
  the stepper's stability polynomial R(-i f0 dt): a closed form.
* A batch runs one stepper (mixed batches are refused); a batch of Heun
  runs matches its members run alone bit for bit; a server that mixes
  steppers batches them apart and each job matches its run alone.
* Repeated runs agree bit for bit (forward Euler's single stage reads the
  state it updates, so its update is committed in a separate pass).
"""
import time

import numpy as np
import pytest

import sw_inputs as si
from oracle import SWOracle

from _helpers import FIELDS, compare, gpu, oracle_keys, run_gpu_interval, turbulence

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
R = {"euler": lambda z: 1 + z, "heun": lambda z: 1 + z + z * z / 2}


@pytest.fixture(scope="module")
def lm():
    return gpu()


def _nu(visc, N):
    K = (N - 1) // 3
    return 1e-3 if visc == "laplace" else 10.0 / K ** 8


def _oracle(N, dt, uvh, strategy, n, stepper, visc, nu):
    o = SWOracle(N, dt, *uvh, nu8=nu, stepper=stepper, visc=visc)
    o.lmean_begin(strategy, fields=FIELDS, pos=True, eulerian=True, n_steps=n)
    o.lmean_step(n)
    return oracle_keys(o.lmean_end()), np.stack(o.fields())


@pytest.mark.parametrize("stepper,visc", [("heun", "hyper8"), ("heun", "laplace"), ("euler", "hyper8"),
                                          ("euler", "laplace"), ("rk4", "laplace")])
@pytest.mark.parametrize("strategy", [1, 2])
@pytest.mark.parametrize("N", [32, 64])
def test_interval_matches_oracle_fp64(lm, stepper, visc, strategy, N):
    n, dt = 24, 5e-3
    uvh = si.smooth_flow(N, 2, seed=5, uamp=0.15, eamp=0.05)
    nu = _nu(visc, N)
    g, guvh = run_gpu_interval(lm, N, dt, uvh, strategy, n, chunks=[5, n - 5], nu8=nu, stepper=stepper, visc=visc)
    r, ruvh = _oracle(N, dt, uvh, strategy, n, stepper, visc, nu)
    errs = compare(g, r, N, strategy)
    assert max(errs.values()) < TOL64, errs
    d = np.abs(guvh - ruvh).max()
    assert d < 1e-12 * np.abs(ruvh - [[[0]], [[0]], [[1]]]).max(), d


@pytest.mark.parametrize("stepper", ["euler", "heun"])
def test_uniform_inertial_oscillation_closed_form(lm, stepper):
    N, dt, f0, U0, n = 16, 5e-3, 1.3, 0.7, 300
    u, v, h = si.uniform_flow(N, U0, 0.0)
    p = lm.make_params(N, dt, precision="f64", f0=f0, stepper=stepper)
    hd = lm.sw_create(p, np.ascontiguousarray(np.stack([u, v, h])))
    try:
        lm.sw_step(hd, n)
        out = np.zeros((3, N, N))
        lm.sw_get_fields(hd, out)
    finally:
        lm.sw_destroy(hd)
    z = U0 * R[stepper](-1j * f0 * dt) ** n
    assert abs(out[0].mean() - z.real) < 1e-13 and abs(out[1].mean() - z.imag) < 1e-13
    assert np.abs(out[0] - out[0].mean()).max() < 1e-13


def _heun_handles(lm, prec, n):
    hs = []
    for i, N in enumerate((64, 128)):
        uvh = np.ascontiguousarray(np.stack(turbulence(N, seed=40 + i)))
        h = lm.sw_create(lm.make_params(N, 5e-3, precision=prec, nu8=_nu("hyper8", N), stepper="heun"), uvh)
        lm.lmean_begin(h, lm.make_lm_params(1 + i, ("zeta", "u"), n_steps=n))
        hs.append(h)
    return hs


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_heun_batch_matches_members_alone_bitwise(lm, prec):
    n = 14
    Ns = (64, 128)

    def end(hs):
        res = []
        for h, N in zip(hs, Ns):
            out = {k: np.zeros((N, N)) for k in ("zeta", "u", "pos_x", "pos_y", "e_zeta", "e_u")}
            lm.lmean_end(h, out)
            lm.sw_destroy(h)
            res.append(out)
        return res

    hs = _heun_handles(lm, prec, n)
    for h in hs:
        lm.lmean_step(h, 5)
        lm.lmean_step(h, n - 5)
    ref = end(hs)
    hs = _heun_handles(lm, prec, n)
    b = lm.sw_batch_create(hs)
    try:
        lm.sw_batch_step(b, 5)
        lm.sw_batch_step(b, n - 5)
    finally:
        lm.sw_batch_destroy(b)
    got = end(hs)
    for i, (a, c) in enumerate(zip(ref, got)):
        for k in a:
            assert np.array_equal(a[k], c[k]), (i, k)


def test_batch_rejects_mixed_steppers(lm):
    N = 64
    uvh = np.ascontiguousarray(np.stack(turbulence(N, seed=1)))
    ha = lm.sw_create(lm.make_params(N, 5e-3, precision="f32", stepper="heun"), uvh)
    hb = lm.sw_create(lm.make_params(N, 5e-3, precision="f32"), uvh)
    try:
        with pytest.raises(lm.SWError) as ei:
            lm.sw_batch_create([ha, hb])
        assert ei.value.code == lm.api.SW_EINVAL
    finally:
        lm.sw_destroy(ha)
        lm.sw_destroy(hb)


def test_server_mixes_steppers(lm):
    jobs = [(64, "rk4", 1, 17), (64, "heun", 2, 21), (128, "euler", 1, 9), (128, "rk4", 2, 12)]

    def params(N, st):
        return lm.make_params(N, 5e-3, precision="f32", nu8=_nu("hyper8", N), stepper=st)

    def outputs(N):
        return {k: np.zeros((N, N)) for k in ("zeta", "pos_x", "pos_y", "e_zeta")}

    srv = lm.sw_server_create("f32", max_active=8, chunk_steps=8)
    try:
        for i, (N, st, strat, n) in enumerate(jobs):
            ic = np.stack(turbulence(N, seed=90 + i))
            lm.sw_server_submit(srv, params(N, st), lm.make_lm_params(strat, ("zeta",), n_steps=n), ic,
                                outputs(N), tag=i)
        done = []
        t0 = time.time()
        while len(done) < len(jobs) and time.time() - t0 < 60:
            done += lm.sw_server_poll(srv, wait_ms=200)
    finally:
        lm.sw_server_destroy(srv)
    assert len(done) == len(jobs)
    for d in done:
        assert d["status"] == 0
        N, st, strat, n = jobs[d["tag"]]
        h = lm.sw_create(params(N, st), np.ascontiguousarray(np.stack(turbulence(N, seed=90 + d["tag"]))))
        lm.lmean_begin(h, lm.make_lm_params(strat, ("zeta",), n_steps=n))
        lm.lmean_step(h, n)
        ref = outputs(N)
        lm.lmean_end(h, ref)
        lm.sw_destroy(h)
        for k in ref:
            assert np.array_equal(d["out"][k], ref[k]), (d["tag"], k)


@pytest.mark.parametrize("stepper", ["euler", "heun", "rk4"])
def test_repeated_runs_are_bitwise_equal(lm, stepper):
    # a step must never read a state element that another thread of the same
    # pass overwrites: two identical runs (and a run split into chunks) agree
    # bit for bit
    N, n = 128, 12
    ic = np.ascontiguousarray(np.stack(turbulence(N, seed=77)))
    outs = []
    for chunks in ([n], [n], [5, 7]):
        h = lm.sw_create(lm.make_params(N, 5e-3, precision="f32", nu8=_nu("hyper8", N), stepper=stepper), ic)
        try:
            lm.lmean_begin(h, lm.make_lm_params(1, ("zeta", "h", "u", "v"), n_steps=n))
            for c in chunks:
                lm.lmean_step(h, c)
            out = {k: np.zeros((N, N)) for k in ("zeta", "h", "u", "v", "pos_x", "pos_y")}
            lm.lmean_end(h, out)
        finally:
            lm.sw_destroy(h)
        outs.append(out)
    for o in outs[1:]:
        for k in o:
            assert np.array_equal(o[k], outs[0][k]), k


@pytest.mark.parametrize("N", [32, 64])
@pytest.mark.parametrize("fields", [("zeta", "h", "u", "v"), ("q",)])
def test_xi_first_matches_oracle_fp64(lm, N, fields):
    # the paper's Strategy-2 discretisation (Sec. 4.2, 4.2.1); the interval
    # is stepped in chunks that split a mean step (odd boundary)
    n, dt = 24, 5e-3
    uvh = si.smooth_flow(N, 2, seed=11, uamp=0.15, eamp=0.05)
    nu = _nu("hyper8", N)
    p = lm.make_params(N, dt, precision="f64", nu8=nu, stepper="euler")
    h = lm.sw_create(p, np.ascontiguousarray(np.stack(uvh)))
    try:
        lm.lmean_begin(h, lm.make_lm_params(2, fields, pos=True, eulerian=True, n_steps=n, scheme="xi_first"))
        lm.lmean_step(h, 7)
        lm.lmean_step(h, n - 7)
        keys = list(fields) + ["pos_x", "pos_y"] + ["e_" + f for f in fields]
        g = {k: np.zeros((N, N)) for k in keys}
        lm.lmean_end(h, g)
    finally:
        lm.sw_destroy(h)
    o = SWOracle(N, dt, *uvh, nu8=nu, stepper="euler")
    o.lmean_begin(2, fields=fields, pos=True, eulerian=True, n_steps=n, scheme="xi_first")
    o.lmean_step(n)
    r = oracle_keys(o.lmean_end())
    errs = compare(g, r, N, 2)
    assert max(errs.values()) < TOL64, errs


def test_xi_first_uniform_flow_closed_form(lm):
    N, dt, U0, V0, n = 16, 5e-3, 0.7, -0.3, 40
    u, v, h0 = si.uniform_flow(N, U0, V0)
    h = lm.sw_create(lm.make_params(N, dt, precision="f64", f0=0.0, stepper="euler"),
                     np.ascontiguousarray(np.stack([u, v, h0])))
    try:
        lm.lmean_begin(h, lm.make_lm_params(2, ("u", "v"), pos=True, eulerian=False, n_steps=n, scheme="xi_first"))
        lm.lmean_step(h, n)
        out = {k: np.zeros((N, N)) for k in ("u", "v", "pos_x", "pos_y")}
        lm.lmean_end(h, out)
    finally:
        lm.sw_destroy(h)
    T = n * dt
    x = 2 * np.pi * np.arange(N) / N
    X, Y = np.meshgrid(x, x)
    np.testing.assert_allclose(out["pos_x"] - X, U0 * T / 2, atol=1e-13)
    np.testing.assert_allclose(out["pos_y"] - Y, V0 * T / 2, atol=1e-13)
    np.testing.assert_allclose(out["u"], U0, atol=1e-13)
    np.testing.assert_allclose(out["v"], V0, atol=1e-13)


def test_xi_first_error_codes(lm):
    N = 32
    uvh = np.ascontiguousarray(np.stack(si.smooth_flow(N, 2, seed=3)))
    for stepper, strategy, n in (("euler", 1, 4), ("rk4", 2, 4), ("euler", 2, 5)):
        h = lm.sw_create(lm.make_params(N, 5e-3, precision="f64", stepper=stepper), uvh)
        try:
            with pytest.raises(lm.SWError) as ei:
                lm.lmean_begin(h, lm.make_lm_params(strategy, ("u",), n_steps=n, scheme="xi_first"))
            assert ei.value.code == lm.api.SW_EINVAL
        finally:
            lm.sw_destroy(h)
