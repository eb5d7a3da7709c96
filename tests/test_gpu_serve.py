"""Serving: continuous batching under an HBM budget.  Jobs that arrive while
others run are admitted as memory frees up, share batched launches (grids
64..512 in one group, each larger size in a group of its own: two 2048^2 and
two 1024^2 jobs here), the groups step on streams of their own, and each
result is the same (bit for bit) as the job run alone."""
import time

import numpy as np
import pytest

from _helpers import gpu, turbulence

pytestmark = pytest.mark.gpu

# (N, strategy, fields, steps)
JOBS = [
    (64, 1, ("zeta", "h"), 37),
    (128, 2, ("zeta", "u"), 25),
    (256, 1, ("u", "v"), 18),
    (64, 2, ("q",), 44),
    (512, 1, ("zeta",), 12),
    (1024, 2, ("h",), 6),
    (128, 1, ("zeta", "h", "u", "v", "q"), 30),
    (2048, 1, ("zeta", "h"), 5),
    (1024, 1, ("v",), 7),
    (2048, 2, ("u",), 4),
]


@pytest.fixture(scope="module")
def lm():
    return gpu()


def _params(lm, N):
    K = (N - 1) // 3
    return lm.make_params(N, 5e-3 if N <= 1024 else 2e-3, precision="f32", nu8=10.0 / K ** 8)


def _outputs(N, strat, fields):
    keys = list(fields) + ["pos_x", "pos_y"] + ["e_" + f for f in fields]
    return {k: np.zeros((N, N)) for k in keys}


def _alone(lm, i, job):
    N, strat, fields, n = job
    ic = np.ascontiguousarray(np.stack(turbulence(N, seed=70 + i)))
    h = lm.sw_create(_params(lm, N), ic)
    lm.lmean_begin(h, lm.make_lm_params(strat, fields, n_steps=n))
    lm.lmean_step(h, n)
    out = _outputs(N, strat, fields)
    lm.lmean_end(h, out)
    lm.sw_destroy(h)
    return out


@pytest.mark.parametrize("budget_jobs", [100, 2])
def test_served_jobs_match_jobs_alone(lm, budget_jobs):
    # a budget of ~2 of the largest jobs forces queueing behind memory
    big = max(lm.sw_state_bytes(_params(lm, j[0])) for j in JOBS)
    srv = lm.sw_server_create("f32", max_active=8, chunk_steps=8, hbm_budget=budget_jobs * big)
    try:
        for i, (N, strat, fields, n) in enumerate(JOBS):
            ic = np.stack(turbulence(N, seed=70 + i))
            lm.sw_server_submit(srv, _params(lm, N), lm.make_lm_params(strat, fields, n_steps=n), ic,
                                _outputs(N, strat, fields), tag=i)
            time.sleep(0.01 * (i % 3))  # arrivals while earlier jobs run
        done = []
        t0 = time.time()
        while len(done) < len(JOBS) and time.time() - t0 < 120:
            done += lm.sw_server_poll(srv, wait_ms=200)
        st = lm.sw_server_stats_get(srv)
    finally:
        lm.sw_server_destroy(srv)
    assert len(done) == len(JOBS)
    assert st["completed"] == len(JOBS) and st["failed"] == 0
    assert st["peak_bytes"] <= budget_jobs * big
    for d in done:
        assert d["status"] == 0
        assert d["t_submit"] <= d["t_admit"] <= d["t_done"]
        ref = _alone(lm, d["tag"], JOBS[d["tag"]])
        for k in ref:
            assert np.array_equal(d["out"][k], ref[k]), (d["tag"], k)
