"""Batches: uneven members stepped in shared launches give the same bits as
each member stepped alone (the per-run arithmetic does not depend on the
batch or on the tuned launch shapes)."""
import numpy as np
import pytest

from _helpers import gpu, turbulence

pytestmark = pytest.mark.gpu

# (N, strategy or 0 for dynamics only, fields, pos, eulerian, steps before the interval)
MEMBERS = [
    (64, 1, ("zeta", "h", "u", "v"), True, True, 0),
    (128, 2, ("zeta", "q"), True, False, 3),
    (256, 1, ("h",), False, True, 0),
    (128, 0, (), False, False, 0),
    (512, 2, ("u",), True, True, 1),
]


@pytest.fixture(scope="module")
def lm():
    return gpu()


def _make(lm, prec):
    hs = []
    for i, (N, strat, fields, pos, eul, pre) in enumerate(MEMBERS):
        K = (N - 1) // 3
        p = lm.make_params(N, 5e-3, precision=prec, nu8=10.0 / K ** 8)
        h = lm.sw_create(p, np.ascontiguousarray(np.stack(turbulence(N, seed=40 + i))))
        if pre:
            lm.sw_step(h, pre)
        hs.append(h)
    return hs


def _begin(lm, hs, n):
    for h, (N, strat, fields, pos, eul, pre) in zip(hs, MEMBERS):
        if strat:
            lm.lmean_begin(h, lm.make_lm_params(strat, fields, pos=pos, eulerian=eul, n_steps=n))


def _finish(lm, hs):
    res = []
    for h, (N, strat, fields, pos, eul, pre) in zip(hs, MEMBERS):
        out = {}
        if strat:
            keys = list(fields) + (["pos_x", "pos_y"] if (pos or strat == 2) else [])
            keys += ["e_" + f for f in fields] if eul else []
            out = {k: np.zeros((N, N)) for k in keys}
            lm.lmean_end(h, out)
        uvh = np.zeros((3, N, N))
        lm.sw_get_fields(h, uvh)
        out["uvh"] = uvh
        res.append(out)
        lm.sw_destroy(h)
    return res


def _alone(lm, prec, n):
    hs = _make(lm, prec)
    _begin(lm, hs, n)
    for h, m in zip(hs, MEMBERS):
        if m[1]:
            lm.lmean_step(h, n // 2)
            lm.lmean_step(h, n - n // 2)
        else:
            lm.sw_step(h, n)
    return _finish(lm, hs)


def _batched(lm, prec, n, tune=False):
    hs = _make(lm, prec)
    _begin(lm, hs, n)
    b = lm.sw_batch_create(hs)
    try:
        if tune:
            lm.sw_batch_tune(b, 4)
        lm.sw_batch_step(b, 7)
        lm.sw_batch_step(b, n - 7)
        assert lm.sw_batch_launch_count(b) > 0
    finally:
        lm.sw_batch_destroy(b)
    return _finish(lm, hs)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_batch_matches_members_alone_bitwise(lm, prec):
    n = 20
    ref = _alone(lm, prec, n)
    got = _batched(lm, prec, n)
    for i, (a, b) in enumerate(zip(ref, got)):
        for k in a:
            assert np.array_equal(a[k], b[k]), (i, k)


def test_tuned_batch_matches_members_alone_bitwise(lm):
    n = 16
    ref = _alone(lm, "f32", n)
    got = _batched(lm, "f32", n, tune=True)
    for i, (a, b) in enumerate(zip(ref, got)):
        for k in a:
            assert np.array_equal(a[k], b[k]), (i, k)


def test_batch_errors(lm):
    N = 64
    uvh = np.ascontiguousarray(np.stack(turbulence(N, seed=1)))
    h32 = lm.sw_create(lm.make_params(N, 5e-3, precision="f32"), uvh)
    h64 = lm.sw_create(lm.make_params(N, 5e-3, precision="f64"), uvh)
    big = lm.sw_create(lm.make_params(1024, 5e-3, precision="f32"),
                       np.ascontiguousarray(np.stack(turbulence(1024, seed=2))))
    try:
        for hs in ([h32, h64], [h32, h32], [h32, big]):
            with pytest.raises(lm.SWError) as ei:
                lm.sw_batch_create(hs)
            assert ei.value.code == lm.api.SW_EINVAL
        lm.lmean_begin(h32, lm.make_lm_params(1, ("u",), n_steps=3))
        b = lm.sw_batch_create([h32])
        with pytest.raises(lm.SWError) as ei:
            lm.sw_batch_step(b, 4)
        assert ei.value.code == lm.api.SW_ERANGE
        lm.sw_batch_step(b, 3)
        assert lm.lmean_progress(h32) == (3, 0)
        lm.sw_batch_destroy(b)
    finally:
        for h in (h32, h64, big):
            lm.sw_destroy(h)
