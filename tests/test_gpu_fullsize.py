"""Checks at the workloads' full sizes and step counts.

* 64^2, one interval of 4 wave periods (1219 RK4 steps), Strategy 1, FP64
  and FP32: element-wise against the oracle.
* 256^2, one full interval (1097 steps) of Strategies 1 and 2 stepped as one
  batch (the launch configuration bench.py times), FP64 and FP32:
  element-wise against the oracle (which takes minutes here and runs in a
  worker process from the start of the session), the FP32 form against the
  FP64 form on the GPU, and properties that hold at any size: bitwise mass
  conservation and the agreement of the two strategies through
  Eq. (tildebar) at the order of the bilinear interpolation.
* 1024^2 precision form, one interval: FP32 against FP64 per field.
"""
import numpy as np
import pytest

import sw_inputs as si
from oracle import rel_l2

from _helpers import FIELDS, compare, gpu

pytestmark = pytest.mark.gpu

KEYS = list(FIELDS) + ["pos_x", "pos_y"] + ["e_" + f for f in FIELDS]


@pytest.fixture(scope="module")
def lm():
    return gpu()


def _interval(lm, w, prec, strategies, batched=True):
    N = w.N
    ic = np.ascontiguousarray(np.stack(w.initial_condition()))
    hs = [lm.sw_create(lm.make_params(N, w.dt, precision=prec, nu8=w.nu8), ic) for _ in strategies]
    for h, s in zip(hs, strategies):
        lm.lmean_begin(h, lm.make_lm_params(s, FIELDS, n_steps=w.n_steps))
    if batched:
        b = lm.sw_batch_create(hs)
        lm.sw_batch_step(b, w.n_steps)
        lm.sw_batch_destroy(b)
    else:
        for h in hs:
            lm.lmean_step(h, w.n_steps)
    outs, diag = [], []
    for h in hs:
        out = {k: np.zeros((N, N)) for k in KEYS}
        lm.lmean_end(h, out)
        outs.append(out)
        diag.append(lm.sw_diag(h))
        lm.sw_destroy(h)
    return outs, diag


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 2e-5)])
def test_plain64_full_interval_matches_oracle(lm, oracle_pool, prec, tol):
    w = si.WORKLOADS["plain-64"]
    assert w.n_steps == 1219
    outs, _ = _interval(lm, w, prec, (1,), batched=False)
    ref, _ = oracle_pool.result("plain64-s1-full")
    e = compare(outs[0], ref, w.N, 1)
    assert max(e.values()) < tol, e


def test_plain256_full_interval_batched(lm, oracle_pool):
    w = si.WORKLOADS["plain-256"]
    assert w.n_steps == 1097
    o32, d32 = _interval(lm, w, "f32", (1, 2))
    o64, d64 = _interval(lm, w, "f64", (1, 2))
    for s in range(2):
        e = compare(o32[s], o64[s], w.N, s + 1)
        assert max(e.values()) < 2e-5, (s + 1, e)
    # element by element against the oracle over the whole interval
    for s in range(2):
        ref, _ = oracle_pool.result(f"plain256-s{s + 1}-full")
        e64 = compare(o64[s], ref, w.N, s + 1)
        assert max(e64.values()) < 1e-12, ("f64", s + 1, e64)
        e32 = compare(o32[s], ref, w.N, s + 1)
        assert max(e32.values()) < 2e-5, ("f32", s + 1, e32)
    # mass: <h> is the k = 0 depth coefficient, unchanged bit for bit in FP64
    h0 = float(np.mean(w.initial_condition()[2]))
    for d in d64:
        assert abs(d[0] - h0) < 1e-15
    # Strategy 1 vs 2 (Eq. tildebar): f~^L(y + xi(y)) = fbar^L(y), evaluated
    # by Fourier interpolation of the Strategy-1 output
    N = w.N
    x = 2 * np.pi * np.arange(N) / N
    X = x[None, :] + 0 * x[:, None]
    Y = x[:, None] + 0 * x[None, :]
    xi_x, xi_y = o64[1]["pos_x"] - X, o64[1]["pos_y"] - Y
    F = np.fft.rfft2(o64[0]["zeta"]) / (N * N)
    kx = np.arange(N // 2 + 1)
    ky = np.fft.fftfreq(N, 1.0 / N)
    px, py = (X + xi_x).ravel(), (Y + xi_y).ravel()
    ex = np.exp(1j * np.outer(px, kx))
    ey = np.exp(1j * np.outer(py, ky))
    wgt = np.where(kx == 0, 1.0, 2.0)
    z1 = np.real(np.sum((ey @ F) * ex * wgt[None, :], axis=1))
    err = rel_l2(z1, o64[1]["zeta"].ravel())
    assert err < 0.05, err


def test_precision1024_fp32_against_fp64(lm):
    w = si.WORKLOADS["precision-1024"]
    o32, _ = _interval(lm, w, "f32", (1,), batched=False)
    o64, _ = _interval(lm, w, "f64", (1,), batched=False)
    e = compare(o32[0], o64[0], w.N, 1)
    assert max(e.values()) < 2e-5, e
