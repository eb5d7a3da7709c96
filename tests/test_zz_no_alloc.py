"""sw_project_static: the allocation-free entry point, for callers that cannot
allocate device memory (a framework allocator that owns the GPU memory, or a
loop that cannot afford cudaMalloc's synchronisation).

Its output is checked against the allocating path that computes the same
projection (sw_create transforms and truncates the initial condition,
sw_get_fields transforms it back), on two calls in a row.  The file is named
so that pytest collects it last.
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
        dev_in = torch.from_numpy(f).cuda()
        dev_out = torch.full((N, N), float("nan"), dtype=torch.float64, device="cuda")
        lm.sw_project_static(dev_in, dev_out, N, stream.cuda_stream)
        stream.synchronize()
        got = dev_out.cpu().numpy()
        assert _rel(got, ref) < TOL64
        assert _rel(got, f) > 0.1  # the projection removed the modes outside the box


def test_project_static_rejects_sizes_beyond_its_scratch():
    import torch

    lm = gpu()
    N = 1024
    x = torch.zeros((N, N), dtype=torch.float64, device="cuda")
    with pytest.raises(lm.SWError) as ei:
        lm.sw_project_static(x, x, N)
    assert ei.value.code == lm.api.SW_EINVAL
    assert "power of two" in lm.sw_last_error(None)
