"""Parity with the FP64 oracle in the launch configurations that the large
grids and the bench run (relative L2 per field <= 1e-12 in FP64 and <= 2e-5
in FP32; depth as h - 1, positions as displacements).

* 256^2 (the bench's grid), Strategies 1 and 2 stepped as one batch, under
  every row-pass launch shape the autotuner can pick (sw_batch_set_shape):
  one to all product pairs per block, one to several groups of threads per
  row (the multi-group row pass), one to eight rows per block.
* 512^2 and 1024^2, where the row-pass groups synchronise with named
  barriers, under every shape the grid admits; 2048^2 under every shape.
* The automatic shape of a single handle at 512^2-2048^2 (lmean_step).

The oracle runs come from a pool of worker processes (tests/_oracle_pool.py)
started when the session begins.
"""
import numpy as np
import pytest

from _helpers import FIELDS, compare, compare_uvh, gpu
from _oracle_pool import case_inputs

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 2e-5}
KEYS = list(FIELDS) + ["pos_x", "pos_y"] + ["e_" + f for f in FIELDS]
POINTS = (256, 512, 1024, 2048)


@pytest.fixture(scope="module")
def lm():
    return gpu()


def _batched(lm, name1, name2, prec, choice):
    """Strategies 1 and 2 of one case as a batch of two, with row-pass shape
    `choice` (None: the automatic shape), stepped in two chunks."""
    N, dt, nu8, uvh, n = case_inputs(name1)
    ic = np.ascontiguousarray(np.stack(uvh))
    hs = [lm.sw_create(lm.make_params(N, dt, precision=prec, nu8=nu8), ic) for _ in range(2)]
    try:
        for h, s in zip(hs, (1, 2)):
            lm.lmean_begin(h, lm.make_lm_params(s, FIELDS, n_steps=n))
        b = lm.sw_batch_create(hs)
        try:
            if choice is not None:
                lm.sw_batch_set_shape(b, choice)
            lm.sw_batch_step(b, n // 2)
            lm.sw_batch_step(b, n - n // 2)
        finally:
            lm.sw_batch_destroy(b)
        outs, uvhs = [], []
        for h in hs:
            out = {k: np.zeros((N, N)) for k in KEYS}
            lm.lmean_end(h, out)
            u = np.zeros((3, N, N))
            lm.sw_get_fields(h, u)
            outs.append(out)
            uvhs.append(u)
        return outs, uvhs
    finally:
        for h in hs:
            lm.sw_destroy(h)


def _check(outs, uvhs, refs, N, tol):
    for s, (out, u, (ref, ruvh)) in enumerate(zip(outs, uvhs, refs)):
        e = compare(out, ref, N, s + 1)
        e.update({"sw_" + k: v for k, v in compare_uvh(u, ruvh).items()})
        assert max(e.values()) < tol, (s + 1, e)


def _shapes(N):
    return [c for c in range(16) if POINTS[c // 4] >= N]


CASES = [("plain256-s1-12", "plain256-s2-12", 256), ("turb512-s1-3", "turb512-s2-3", 512),
         ("prec1024-s1-3", "prec1024-s2-3", 1024), ("prec2048-s1-2", "prec2048-s2-2", 2048)]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("c1,c2,N", CASES, ids=[str(c[2]) for c in CASES])
def test_every_row_pass_shape_matches_oracle(lm, oracle_pool, c1, c2, N, prec):
    refs = [oracle_pool.result(c1), oracle_pool.result(c2)]
    for choice in _shapes(N):
        outs, uvhs = _batched(lm, c1, c2, prec, choice)
        try:
            _check(outs, uvhs, refs, N, TOL[prec])
        except AssertionError as ex:
            raise AssertionError(f"row-pass shape {choice}: {ex}") from None


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("c1,c2,N", CASES[1:], ids=[str(c[2]) for c in CASES[1:]])
def test_single_handle_automatic_shape_matches_oracle(lm, oracle_pool, c1, c2, N, prec):
    refs = [oracle_pool.result(c1), oracle_pool.result(c2)]
    outs, uvhs = [], []
    for name, s in ((c1, 1), (c2, 2)):
        N_, dt, nu8, uvh, n = case_inputs(name)
        h = lm.sw_create(lm.make_params(N, dt, precision=prec, nu8=nu8), np.ascontiguousarray(np.stack(uvh)))
        try:
            lm.lmean_begin(h, lm.make_lm_params(s, FIELDS, n_steps=n))
            lm.lmean_step(h, 1)
            lm.lmean_step(h, n - 1)
            out = {k: np.zeros((N, N)) for k in KEYS}
            lm.lmean_end(h, out)
            u = np.zeros((3, N, N))
            lm.sw_get_fields(h, u)
        finally:
            lm.sw_destroy(h)
        outs.append(out)
        uvhs.append(u)
    _check(outs, uvhs, refs, N, TOL[prec])


def test_shape_setter_rejects_shapes_below_the_grid(lm):
    N, dt, nu8, uvh, n = case_inputs("turb512-s1-3")
    h = lm.sw_create(lm.make_params(N, dt, precision="f32", nu8=nu8), np.ascontiguousarray(np.stack(uvh)))
    b = lm.sw_batch_create([h])
    try:
        for bad in (-1, 16, 0, 3):  # out of range; 256 points per block < 512
            with pytest.raises(lm.SWError) as ei:
                lm.sw_batch_set_shape(b, bad)
            assert ei.value.code == lm.api.SW_EINVAL
        lm.sw_batch_set_shape(b, 4)
    finally:
        lm.sw_batch_destroy(b)
        lm.sw_destroy(h)
