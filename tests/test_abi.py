"""C-ABI checks that need no GPU: the library builds and loads, exports every
symbol the header declares, the binding's structs match the C layout, and
argument validation happens before any device call."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lagmean.h")


@pytest.fixture(scope="module")
def lm():
    import paper_2208_02682_gb300 as lm
    lm.build()
    lm.api.load()
    return lm


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**\s*(\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("sw_create", "sw_step", "lmean_begin", "lmean_step", "lmean_end", "sw_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lm):
    lib = C.CDLL(lm.api.LIB_PATH)
    for n in declared_functions():
        assert hasattr(lib, n), n
    assert set(lm.api.EXPORTS) == set(declared_functions())


def test_struct_layout_matches_c(tmp_path, lm):
    prog = tmp_path / "sz.c"
    prog.write_text('#include "lagmean.h"\n#include <stdio.h>\n#include <stddef.h>\n'
                    "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n\", sizeof(sw_params),"
                    " sizeof(lm_params), sizeof(lm_result), offsetof(sw_params, dt),"
                    " offsetof(lm_result, on_device), sizeof(sw_server_params), sizeof(sw_job),"
                    " offsetof(sw_job, tag), sizeof(sw_job_done), sizeof(sw_server_stats));"
                    " printf(\"%zu %zu\\n\", sizeof(sl_params), offsetof(sl_params, n_steps));"
                    " printf(\"%zu %zu\\n\", offsetof(sw_params, stepper), offsetof(sw_params, visc)); return 0;}\n")
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", os.path.dirname(HEADER), str(prog), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    api = lm.api
    assert got == [C.sizeof(api.sw_params), C.sizeof(api.lm_params), C.sizeof(api.lm_result),
                   api.sw_params.dt.offset, api.lm_result.on_device.offset,
                   C.sizeof(api.sw_server_params), C.sizeof(api.sw_job), api.sw_job.tag.offset,
                   C.sizeof(api.sw_job_done), C.sizeof(api.sw_server_stats),
                   C.sizeof(api.sl_params), api.sl_params.n_steps.offset,
                   api.sw_params.stepper.offset, api.sw_params.visc.offset]


@pytest.mark.parametrize("field,value", [("N", 48), ("N", 8), ("N", 4096), ("dt", 0.0), ("dt", -1.0),
                                         ("precision", 7), ("model", 3), ("nu8", -1.0),
                                         ("c2", float("nan")), ("reserved", 1),
                                         ("stepper", 3), ("stepper", -1), ("visc", 2)])
def test_invalid_parameters_rejected_before_device_use(lm, field, value):
    p = lm.make_params(64, 1e-3)
    setattr(p, field, value)
    ic = np.zeros((3, 64, 64))
    with pytest.raises(lm.SWError) as ei:
        lm.sw_create(p, ic)
    assert ei.value.code == lm.api.SW_EINVAL
    assert lm.sw_last_error(None)


def test_state_bytes_and_server_validation(lm):
    # the budget unit grows with the grid and halves in FP32; invalid -> 0
    b = [lm.sw_state_bytes(lm.make_params(N, 1e-3, precision="f32")) for N in (64, 128, 256)]
    assert 0 < b[0] < b[1] < b[2]
    assert lm.sw_state_bytes(lm.make_params(64, 1e-3, precision="f64")) > b[0]
    p = lm.make_params(48, 1e-3)
    assert lm.sw_state_bytes(p) == 0
    with pytest.raises(lm.SWError):
        lm.sw_server_create(max_active=0)


def test_null_handle_is_rejected(lm):
    lib = lm.api.load()
    assert lib.sw_step(None, 1) == lm.api.SW_EINVAL
    assert lib.lmean_step(None, 1) == lm.api.SW_EINVAL
    assert lib.lmean_begin(None, None) == lm.api.SW_EINVAL
    assert lib.sw_sync(None) == lm.api.SW_EINVAL
    lib.sw_destroy(None)  # no-op


@pytest.mark.parametrize("case", ["N_not_pow2", "N_too_big", "iters_zero", "too_many_fields", "alias_in",
                                  "alias_out", "null_pos"])
def test_remap_arguments_rejected_before_device_use(lm, case):
    # every case is invalid, so the call returns before touching the (fake)
    # device addresses or launching anything
    lib = lm.api.load()
    DP = lm.api._DP
    fake = [C.cast(C.c_void_p(0x10000 * (k + 1)), DP) for k in range(8)]
    N, iters, nf = 64, 20, 1
    pos_x, pos_y = fake[0], fake[1]
    fin = (DP * 1)(fake[2])
    fout = (DP * 1)(fake[3])
    xi_x = fake[4]
    if case == "N_not_pow2":
        N = 48
    elif case == "N_too_big":
        N = 8192
    elif case == "iters_zero":
        iters = 0
    elif case == "too_many_fields":
        nf = 17
    elif case == "alias_in":
        fout = (DP * 1)(fake[2])
    elif case == "alias_out":
        xi_x = fake[3]
    elif case == "null_pos":
        pos_y = None
    rc = lib.lmean_remap(N, pos_x, pos_y, nf, fin, fout, iters, xi_x, None, None, None)
    assert rc == lm.api.SW_EINVAL
    assert "lmean_remap" in lm.sw_last_error(None)


@pytest.mark.parametrize("case", ["N_not_pow2", "no_fields", "too_many_fields", "alias_pos", "alias_field",
                                  "null_pos"])
def test_lift_arguments_rejected_before_device_use(lm, case):
    # every case is invalid: the call returns before touching the (fake)
    # device addresses or launching anything
    lib = lm.api.load()
    DP = lm.api._DP
    fake = [C.cast(C.c_void_p(0x10000 * (k + 1)), DP) for k in range(6)]
    N, nf = 64, 1
    pos_x, pos_y = fake[0], fake[1]
    fin = (DP * 1)(fake[2])
    fout = (DP * 1)(fake[3])
    if case == "N_not_pow2":
        N = 100
    elif case == "no_fields":
        nf = 0
    elif case == "too_many_fields":
        nf = 17
    elif case == "alias_pos":
        fout = (DP * 1)(fake[0])
    elif case == "alias_field":
        fout = (DP * 1)(fake[2])
    elif case == "null_pos":
        pos_x = None
    assert lib.lmean_lift(N, pos_x, pos_y, nf, fin, fout, None) == lm.api.SW_EINVAL
    assert "lmean_lift" in lm.sw_last_error(None)


def test_spectrum_rejects_null_handle(lm):
    lib = lm.api.load()
    out = np.zeros(4)
    assert lib.sw_spectrum(None, None, 0, out.ctypes.data_as(lm.api._DP), 4) == lm.api.SW_EINVAL


def test_sl_arguments_rejected_before_device_use(lm):
    lib = lm.api.load()
    s = C.c_void_p()
    p = lm.make_sl_params(n_steps=4)
    assert lib.sw_sl_create(None, C.byref(p), C.byref(s)) == lm.api.SW_EINVAL
    assert "sw_sl" in lm.sw_last_error(None)
    assert lib.sw_sl_step(None, 1) == lm.api.SW_EINVAL
    assert lib.sw_sl_end(None, None) == lm.api.SW_EINVAL
    lib.sw_sl_destroy(None)  # no-op


@pytest.mark.parametrize("case", ["short_in", "short_out", "host_array", "wrong_dtype", "cpu_tensor"])
def test_project_static_rejects_bad_buffers_before_any_launch(lm, case):
    # the binding checks shape, dtype and device before it calls the library,
    # so a buffer shorter than N*N never reaches a kernel (no GPU needed here)
    import torch
    N = 64
    good = torch.zeros((N, N), dtype=torch.float64)
    inp, out = good, good
    if case == "short_in":
        inp = torch.zeros((N // 2, N), dtype=torch.float64)
    elif case == "short_out":
        out = torch.zeros((N, N - 1), dtype=torch.float64)
    elif case == "host_array":
        inp = np.zeros((N, N))
    elif case == "wrong_dtype":
        out = torch.zeros((N, N), dtype=torch.float32)
    with pytest.raises(ValueError):
        lm.sw_project_static(inp, out, N)


def test_batch_shape_setter_rejects_null(lm):
    assert lm.api.load().sw_batch_set_shape(None, 0) == lm.api.SW_EINVAL


def test_fma_peak_rejects_bad_arguments(lm):
    lib = lm.api.load()
    import ctypes as C
    t = C.c_double(0.0)
    assert lib.sw_fma_peak(7, 16, C.byref(t), None) == lm.api.SW_EINVAL
    assert lib.sw_fma_peak(lm.api.SW_PREC_FP64, 0, C.byref(t), None) == lm.api.SW_EINVAL
    assert lib.sw_fma_peak(lm.api.SW_PREC_FP32, 16, None, None) == lm.api.SW_EINVAL
    assert "sw_fma_peak" in lm.sw_last_error(None)
