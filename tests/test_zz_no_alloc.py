"""sw_project_static: the allocation-free entry point, for callers that cannot
allocate device memory (a framework allocator that owns the GPU memory, or a
loop that cannot afford cudaMalloc's synchronisation).

Its output is checked against an independent numpy projection (rfft2, keep
|kx|, |ky| <= floor((N-1)/3), irfft2) and against the allocating path that
computes the same projection (sw_create transforms and truncates the initial
condition, sw_get_fields transforms it back), on two calls in a row, and in
place (the same tensor as input and output).  The file is named so that
pytest collects it last.
"""
import numpy as np
import pytest

from _helpers import gpu

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


def _reference_projection(lm, f):
    """Projection through the allocating path: sw_create + sw_get_fields."""
    N = f.shape[0]
    uvh = np.ascontiguousarray(np.stack([f, np.zeros_like(f), np.ones_like(f)]))
    h = lm.sw_create(lm.make_params(N, 1e-3), uvh)
    try:
        out = np.zeros((3, N, N))
        lm.sw_get_fields(h, out)
    finally:
        lm.sw_destroy(h)
    return out[0]


def _numpy_projection(f):
    """The square 2/3 rule on the real FFT of f, in numpy."""
    N = f.shape[0]
    K = (N - 1) // 3
    kx = np.arange(N // 2 + 1)[None, :]
    ky = np.fft.fftfreq(N, 1.0 / N)[:, None]
    box = (kx <= K) & (np.abs(ky) <= K)
    return np.fft.irfft2(np.where(box, np.fft.rfft2(f), 0.0), s=(N, N))


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("N", [64, 512])
def test_project_static_matches_allocating_path_twice(N):
    import torch

    lm = gpu()
    rng = np.random.default_rng(N)
    stream = torch.cuda.current_stream()
    # full-spectrum inputs, so the 2/3 truncation removes something
    fields = [rng.standard_normal((N, N)), rng.standard_normal((N, N))]
    for f in fields:
        ref = _reference_projection(lm, f)
        ref_np = _numpy_projection(f)
        assert _rel(ref, ref_np) < TOL64
        dev_in = torch.from_numpy(f).cuda()
        dev_out = torch.full((N, N), float("nan"), dtype=torch.float64, device="cuda")
        lm.sw_project_static(dev_in, dev_out, N, stream.cuda_stream)
        stream.synchronize()
        got = dev_out.cpu().numpy()
        assert _rel(got, ref_np) < TOL64
        assert _rel(got, ref) < TOL64
        assert _rel(got, f) > 0.1  # the projection removed the modes outside the box
        # in place: input and output are the same buffer
        inplace = torch.from_numpy(f.copy()).cuda()
        lm.sw_project_static(inplace, inplace, N, stream.cuda_stream)
        stream.synchronize()
        assert _rel(inplace.cpu().numpy(), ref_np) < TOL64


def test_project_static_rejects_sizes_beyond_its_scratch():
    import torch

    lm = gpu()
    N = 1024
    x = torch.zeros((N, N), dtype=torch.float64, device="cuda")
    with pytest.raises(lm.SWError) as ei:
        lm.sw_project_static(x, x, N)
    assert ei.value.code == lm.api.SW_EINVAL
    assert "power of two" in lm.sw_last_error(None)
