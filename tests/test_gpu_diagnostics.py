"""GPU checks of the diagnostics: lmean_lift (fields at the lift map) and
sw_spectrum (shell spectra on the 2/3 box).

* lmean_lift against the oracle's lift on the same inputs, bit for bit
  (separately rounded FP64 in the oracle's order), 16^2 to 1024^2.
* sw_spectrum against the oracle's spectrum, to 1e-12 relative (the GPU
  sums shells with atomics, in no fixed order), from host and device
  fields; the handle's state is left as it was.
* Sec. 4.2.1's rearrangement on a GPU Strategy-2 run: the lifted final PV
  q(Xi(x), tau+T) matches the Lagrangian mean PV at the bilinear order and
  is closer to it than the Eulerian mean is.
"""
import numpy as np
import pytest

import sw_inputs as si
from oracle import rel_l2
from oracle.remap import grid, lift, spectrum

from _helpers import gpu

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lm():
    return gpu()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("N", [16, 64, 256, 1024])
def test_lift_bit_exact_against_oracle(lm, N):
    rng = np.random.default_rng(N)
    X, Y = grid(N)
    px = X + 0.3 * np.sin(Y + 0.2) + 0.05 * si.random_smooth_field(N, 3, rng)
    py = Y - 0.2 * np.cos(X) + 0.05 * si.random_smooth_field(N, 3, rng)
    fields = {"a": si.random_smooth_field(N, 6, rng), "b": np.cos(2 * X + Y)}
    g = lm.lmean_lift(_dev(px), _dev(py), {k: _dev(v) for k, v in fields.items()})
    torch.cuda.synchronize()
    ref = lift(fields, px, py)
    for k in fields:
        assert np.array_equal(g[k].cpu().numpy(), ref[k]), k


def test_lift_identity_and_aliasing(lm):
    N = 32
    X, Y = grid(N)
    f = np.random.default_rng(1).standard_normal((N, N))
    g = lm.lmean_lift(_dev(X), _dev(Y), {"f": _dev(f)})
    assert np.array_equal(g["f"].cpu().numpy(), f)
    px, fx = _dev(X), _dev(f)
    lib = lm.api.load()
    DP = lm.api._DP
    arr = (DP * 1)(lm.api._ptr(fx)[0])
    assert lib.lmean_lift(N, lm.api._ptr(px)[0], lm.api._ptr(px)[0], 1, arr, arr, None) == lm.api.SW_EINVAL


@pytest.mark.parametrize("N", [32, 256])
def test_spectrum_against_oracle(lm, N):
    rng = np.random.default_rng(7 + N)
    ic = np.ascontiguousarray(np.stack(si.turbulence_plus_waves(N, 0.1, 1.0, 4.0, 6.0, 11)))
    h = lm.sw_create(lm.make_params(N, 5e-3, precision="f32"), ic)
    try:
        before = lm.sw_get_fields(h, np.zeros((3, N, N)))
        f = si.random_smooth_field(N, N // 4, rng) + 0.3
        ref = spectrum(f)
        s_host = lm.sw_spectrum(h, np.ascontiguousarray(f), N)
        s_dev = lm.sw_spectrum(h, _dev(f), N)
        for s in (s_host, s_dev):
            assert len(s) == len(ref)
            np.testing.assert_allclose(s, ref, rtol=1e-12, atol=1e-14 * ref.sum())
        after = lm.sw_get_fields(h, np.zeros((3, N, N)))
        assert np.array_equal(before, after)
        # too few shells, and a missing field, are rejected
        lib = lm.api.load()
        DP = lm.api._DP
        out = np.zeros(len(ref))
        fh = np.ascontiguousarray(f)
        assert lib.sw_spectrum(h, fh.ctypes.data_as(DP), 0, out.ctypes.data_as(DP), 2) == lm.api.SW_EINVAL
        assert lib.sw_spectrum(h, None, 0, out.ctypes.data_as(DP), len(ref)) == lm.api.SW_EINVAL
    finally:
        lm.sw_destroy(h)


def _pv(N, uvh):
    u, v, h = uvh
    k = np.fft.fftfreq(N, 1.0 / N)
    KX, KY = np.meshgrid(k, k)
    zeta = np.real(np.fft.ifft2(1j * KX * np.fft.fft2(v) - 1j * KY * np.fft.fft2(u)))
    return (1.0 + zeta) / h


def test_lifted_pv_matches_lagrangian_mean_pv(lm):
    N, n = 128, 300
    u, v, h = si.smooth_flow(N, 2, seed=5, uamp=0.2, eamp=0.05)
    ic = np.ascontiguousarray(np.stack([u, v, h]))
    hd = lm.sw_create(lm.make_params(N, 5e-3, precision="f64", nu8=0.0, lm_nu8=0.0), ic)
    try:
        lm.lmean_begin(hd, lm.make_lm_params(2, ("q",), pos=True, eulerian=True, n_steps=n))
        lm.lmean_step(hd, n)
        out = {k: torch.empty((N, N), dtype=torch.float64, device="cuda") for k in ("q", "pos_x", "pos_y", "e_q")}
        lm.lmean_end(hd, out)
        q_end = _pv(N, lm.sw_get_fields(hd, np.zeros((3, N, N))))
    finally:
        lm.sw_destroy(hd)
    qx = lm.lmean_lift(out["pos_x"], out["pos_y"], {"q": _dev(q_end)})["q"].cpu().numpy()
    qbar, eq = out["q"].cpu().numpy(), out["e_q"].cpu().numpy()
    m = qbar.mean()
    e_lag = rel_l2(qx - m, qbar - m)
    assert e_lag < 2e-3, e_lag
    assert rel_l2(qx - m, eq - m) > 2 * e_lag
