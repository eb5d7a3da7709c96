"""GB300 library for on-the-fly Lagrangian means of rotating shallow water
(Kafiabad & Vanneste, "Computing Lagrangian means", arXiv 2208.02682).

The compute path is liblagmean.so (CUDA for sm_103a) behind the C ABI of
include/lagmean.h; ``api`` is its thin ctypes binding.
"""
from ._build import build  # noqa: F401
from . import api  # noqa: F401
from .api import (  # noqa: F401
    SWError, make_params, make_lm_params, sw_create, sw_destroy, sw_step, lmean_begin,
    lmean_step, lmean_end, lmean_progress, sw_get_fields, sw_set_fields, sw_diag,
    sw_get_state, sw_set_state, sw_time, sw_sync, sw_last_error, sw_version, sw_kernel_times,
    sw_launch_count, sw_project_static, sw_batch_create, sw_batch_step, sw_batch_tune, sw_batch_set_shape,
    sw_batch_launch_count, sw_batch_last_error, sw_batch_destroy, sw_server_create, sw_server_submit,
    sw_server_poll, sw_server_stats_get, sw_server_clock, sw_server_destroy, sw_state_bytes,
    lmean_remap, lmean_lift, sw_spectrum, spectrum_shells, make_sl_params, sw_sl_create, sw_sl_step,
    sw_sl_end, sw_sl_destroy, sw_fma_peak,
)
