"""Thin Python binding of the C ABI in include/lagmean.h (ctypes).

Same names as the C entry points; this module only marshals arguments.  All
computation happens in liblagmean.so (CUDA, sm_103a).  Loading fails loudly
when the library is missing: there is no CPU fallback.

Host arrays are numpy float64 C-contiguous; device arrays are torch CUDA
float64 tensors (only their data pointers cross the ABI).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblagmean.so")

SW_OK, SW_EINVAL, SW_ENOMEM, SW_EBUSY, SW_ERANGE, SW_ESTATE, SW_ETIMEOUT, SW_ECUDA = range(8)
SW_PREC_FP64, SW_PREC_FP32 = 0, 1
SW_MODEL_SW, SW_MODEL_KINEMATIC, SW_MODEL_EULER2D = 0, 1, 2
LM_ZETA, LM_H, LM_U, LM_V, LM_Q, LM_POS = 1, 2, 4, 8, 16, 32
FIELD_BITS = {"zeta": LM_ZETA, "h": LM_H, "u": LM_U, "v": LM_V, "q": LM_Q}

EXPORTS = ("sw_create", "sw_destroy", "sw_step", "lmean_begin", "lmean_step", "lmean_end",
           "lmean_progress", "sw_get_fields", "sw_set_fields", "sw_diag", "sw_get_state",
           "sw_set_state", "sw_time", "sw_sync", "sw_last_error", "sw_version", "sw_kernel_times",
           "sw_launch_count", "sw_project_static", "sw_batch_create", "sw_batch_step",
           "sw_batch_tune", "sw_batch_set_shape", "sw_batch_launch_count", "sw_batch_last_error", "sw_batch_destroy",
           "sw_server_create", "sw_server_submit", "sw_server_poll", "sw_server_stats_get",
           "sw_server_clock", "sw_server_destroy", "sw_state_bytes", "lmean_remap", "lmean_lift",
           "sw_spectrum", "sw_sl_create", "sw_sl_step", "sw_sl_end", "sw_sl_destroy", "sw_fma_peak")
SW_K_NAMES = ("col_inv", "row_inv", "row_prod", "col_fwd", "update", "phys_q")
SW_K_COUNT = 8


class sw_params(C.Structure):
    _fields_ = [("N", C.c_int32), ("precision", C.c_int32), ("model", C.c_int32),
                ("stepper", C.c_int32), ("dt", C.c_double), ("f0", C.c_double),
                ("c2", C.c_double), ("nu8", C.c_double), ("lm_nu8", C.c_double),
                ("adv_x", C.c_double), ("adv_y", C.c_double), ("visc", C.c_int32),
                ("reserved", C.c_int32)]


class lm_params(C.Structure):
    _fields_ = [("strategy", C.c_int32), ("fields", C.c_int32), ("eulerian", C.c_int32),
                ("scheme", C.c_int32), ("n_steps", C.c_int64)]


_DP = C.POINTER(C.c_double)


class lm_result(C.Structure):
    _fields_ = [("zeta", _DP), ("h", _DP), ("u", _DP), ("v", _DP), ("q", _DP),
                ("pos_x", _DP), ("pos_y", _DP),
                ("e_zeta", _DP), ("e_h", _DP), ("e_u", _DP), ("e_v", _DP), ("e_q", _DP),
                ("on_device", C.c_int32), ("reserved", C.c_int32)]


SL_EULER, SL_TRAPEZOID = 0, 1
SL_LINEAR, SL_CUBIC = 0, 1


class sl_params(C.Structure):
    _fields_ = [("fields", C.c_int32), ("scheme", C.c_int32), ("interp", C.c_int32),
                ("reserved", C.c_int32), ("n_steps", C.c_int64)]


class sw_server_params(C.Structure):
    _fields_ = [("precision", C.c_int32), ("max_active", C.c_int32), ("chunk_steps", C.c_int32),
                ("reserved", C.c_int32), ("hbm_budget", C.c_int64), ("stream", C.c_void_p)]


class sw_job(C.Structure):
    _fields_ = [("params", sw_params), ("lm", lm_params), ("ic_uvh", _DP), ("out", lm_result),
                ("tag", C.c_int64)]


class sw_job_done(C.Structure):
    _fields_ = [("tag", C.c_int64), ("status", C.c_int32), ("reserved", C.c_int32),
                ("t_submit", C.c_double), ("t_admit", C.c_double), ("t_done", C.c_double),
                ("bytes", C.c_int64)]


class sw_server_stats(C.Structure):
    _fields_ = [(n, C.c_int64) for n in ("submitted", "completed", "failed", "active", "queued",
                                         "grid_point_steps", "bytes_in_use", "peak_bytes", "rounds")]


class SWError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"lagmean error {code}: {msg}")
        self.code = code


_lib = None


def load(path: str = LIB_PATH):
    """Load liblagmean.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} not found: build it with paper_2208_02682_gb300.build()")
    lib = C.CDLL(path)
    H = C.c_void_p
    sig = {
        "sw_create": (C.c_int, [C.POINTER(sw_params), _DP, C.c_int, C.c_void_p, C.POINTER(H)]),
        "sw_destroy": (None, [H]),
        "sw_step": (C.c_int, [H, C.c_int64]),
        "lmean_begin": (C.c_int, [H, C.POINTER(lm_params)]),
        "lmean_step": (C.c_int, [H, C.c_int64]),
        "lmean_end": (C.c_int, [H, C.POINTER(lm_result)]),
        "lmean_progress": (C.c_int, [H, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
        "sw_get_fields": (C.c_int, [H, _DP, C.c_int]),
        "sw_set_fields": (C.c_int, [H, _DP, C.c_int]),
        "sw_diag": (C.c_int, [H, _DP]),
        "sw_get_state": (C.c_int, [H, C.c_void_p, C.POINTER(C.c_size_t)]),
        "sw_set_state": (C.c_int, [H, C.c_void_p, C.c_size_t]),
        "sw_time": (C.c_int, [H, _DP]),
        "sw_sync": (C.c_int, [H]),
        "sw_last_error": (C.c_char_p, [H]),
        "sw_kernel_times": (C.c_int, [H, C.c_int64, _DP, C.POINTER(C.c_int64), _DP]),
        "sw_launch_count": (C.c_int, [H, C.POINTER(C.c_int64)]),
        "sw_project_static": (C.c_int, [_DP, _DP, C.c_int, C.c_void_p]),
        "lmean_remap": (C.c_int, [C.c_int, _DP, _DP, C.c_int, C.POINTER(_DP), C.POINTER(_DP), C.c_int, _DP, _DP,
                                  _DP, C.c_void_p]),
        "lmean_lift": (C.c_int, [C.c_int, _DP, _DP, C.c_int, C.POINTER(_DP), C.POINTER(_DP), C.c_void_p]),
        "sw_spectrum": (C.c_int, [C.c_void_p, _DP, C.c_int, _DP, C.c_int]),
        "sw_sl_create": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p)]),
        "sw_sl_step": (C.c_int, [C.c_void_p, C.c_int64]),
        "sw_sl_end": (C.c_int, [C.c_void_p, C.c_void_p]),
        "sw_sl_destroy": (None, [C.c_void_p]),
        "sw_batch_create": (C.c_int, [C.POINTER(H), C.c_int, C.POINTER(H)]),
        "sw_batch_step": (C.c_int, [H, C.c_int64]),
        "sw_batch_tune": (C.c_int, [H, C.c_int, C.POINTER(C.c_int)]),
        "sw_batch_set_shape": (C.c_int, [H, C.c_int]),
        "sw_batch_launch_count": (C.c_int, [H, C.POINTER(C.c_int64)]),
        "sw_batch_last_error": (C.c_char_p, [H]),
        "sw_batch_destroy": (None, [H]),
        "sw_server_create": (C.c_int, [C.POINTER(sw_server_params), C.POINTER(H)]),
        "sw_server_submit": (C.c_int, [H, C.POINTER(sw_job)]),
        "sw_server_poll": (C.c_int, [H, C.POINTER(sw_job_done), C.c_int, C.POINTER(C.c_int), C.c_int]),
        "sw_server_stats_get": (C.c_int, [H, C.POINTER(sw_server_stats)]),
        "sw_server_clock": (C.c_double, [H]),
        "sw_server_destroy": (None, [H]),
        "sw_state_bytes": (C.c_int64, [C.POINTER(sw_params)]),
        "sw_version": (C.c_char_p, []),
        "sw_fma_peak": (C.c_int, [C.c_int, C.c_int, _DP, C.c_void_p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(rc, h):
    if rc != SW_OK:
        msg = load().sw_last_error(h)
        raise SWError(rc, msg.decode() if msg else "")


def _ptr(a):
    """(pointer, on_device) of a numpy float64 array or a torch CUDA tensor."""
    if a is None:
        return None, 0
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be C-contiguous float64")
        return a.ctypes.data_as(_DP), 0
    # torch tensor
    if not a.is_contiguous() or str(a.dtype) != "torch.float64":
        raise ValueError("device tensors must be contiguous float64")
    return C.cast(C.c_void_p(a.data_ptr()), _DP), 1 if a.is_cuda else 0


def make_params(N, dt, precision="f64", model="sw", f0=1.0, c2=1.0, nu8=0.0, lm_nu8=None,
                adv=(0.0, 0.0), stepper="rk4", visc="hyper8") -> sw_params:
    p = sw_params()
    p.N = int(N)
    p.precision = {"f64": SW_PREC_FP64, "f32": SW_PREC_FP32}[precision]
    p.model = {"sw": SW_MODEL_SW, "kinematic": SW_MODEL_KINEMATIC, "euler2d": SW_MODEL_EULER2D}[model]
    p.stepper = {"rk4": 0, "heun": 1, "euler": 2}[stepper]
    p.visc = {"hyper8": 0, "laplace": 1}[visc]
    p.reserved = 0
    p.dt, p.f0, p.c2, p.nu8 = float(dt), float(f0), float(c2), float(nu8)
    p.lm_nu8 = float(nu8 if lm_nu8 is None else lm_nu8)
    p.adv_x, p.adv_y = float(adv[0]), float(adv[1])
    return p


def make_lm_params(strategy, fields=("zeta", "h", "u", "v"), pos=True, eulerian=True,
                   n_steps=1, scheme="coupled") -> lm_params:
    lp = lm_params()
    lp.strategy = int(strategy)
    bits = 0
    for f in fields:
        bits |= FIELD_BITS[f]
    if pos:
        bits |= LM_POS
    lp.fields = bits
    lp.eulerian = 1 if eulerian else 0
    lp.scheme = {"coupled": 0, "xi_first": 1}[scheme]
    lp.n_steps = int(n_steps)
    return lp


# ---- same names as the C ABI --------------------------------------------------
def sw_create(params: sw_params, ic_uvh, stream=None):
    """Create a handle; ic_uvh: (3, N, N) float64 host array or CUDA tensor."""
    lib = load()
    ptr, dev = _ptr(ic_uvh)
    h = C.c_void_p()
    rc = lib.sw_create(C.byref(params), ptr, dev, C.c_void_p(stream or 0), C.byref(h))
    if rc != SW_OK:
        raise SWError(rc, lib.sw_last_error(None).decode())
    return h


def sw_destroy(h):
    load().sw_destroy(h)


def sw_step(h, nsteps):
    _check(load().sw_step(h, int(nsteps)), h)


def lmean_begin(h, lp: lm_params):
    _check(load().lmean_begin(h, C.byref(lp)), h)


def lmean_step(h, nsteps):
    _check(load().lmean_step(h, int(nsteps)), h)


def lmean_progress(h):
    d, r = C.c_int64(), C.c_int64()
    _check(load().lmean_progress(h, C.byref(d), C.byref(r)), h)
    return d.value, r.value


RESULT_KEYS = ("zeta", "h", "u", "v", "q", "pos_x", "pos_y", "e_zeta", "e_h", "e_u", "e_v", "e_q")


def lmean_end(h, out: dict):
    """out: dict key -> array (see RESULT_KEYS); all host or all device."""
    r = lm_result()
    ondev = set()
    for k in RESULT_KEYS:
        a = out.get(k)
        p, d = _ptr(a)
        if a is not None:
            ondev.add(d)
            setattr(r, k, p)
    if len(ondev) > 1:
        raise ValueError("outputs must be all host or all device")
    r.on_device = ondev.pop() if ondev else 0
    r.reserved = 0
    _check(load().lmean_end(h, C.byref(r)), h)
    return out


def sw_get_fields(h, uvh):
    p, d = _ptr(uvh)
    _check(load().sw_get_fields(h, p, d), h)
    return uvh


def sw_set_fields(h, uvh):
    p, d = _ptr(uvh)
    _check(load().sw_set_fields(h, p, d), h)


def sw_diag(h):
    out = (C.c_double * 3)()
    _check(load().sw_diag(h, out), h)
    return tuple(out)


def sw_get_state(h) -> bytes:
    lib = load()
    n = C.c_size_t(0)
    _check(lib.sw_get_state(h, None, C.byref(n)), h)
    buf = C.create_string_buffer(n.value)
    _check(lib.sw_get_state(h, buf, C.byref(n)), h)
    return buf.raw[: n.value]


def sw_set_state(h, blob: bytes):
    buf = C.create_string_buffer(blob, len(blob))
    _check(load().sw_set_state(h, buf, len(blob)), h)


def sw_time(h):
    t = C.c_double()
    _check(load().sw_time(h, C.byref(t)), h)
    return t.value


def sw_sync(h):
    _check(load().sw_sync(h), h)


def sw_kernel_times(h, nsteps):
    """{kernel: (total_ms, launches, total_algorithmic_bytes)} over nsteps
    RK4 steps launched kernel by kernel (advances the state)."""
    ms = (C.c_double * SW_K_COUNT)()
    nl = (C.c_int64 * SW_K_COUNT)()
    by = (C.c_double * SW_K_COUNT)()
    _check(load().sw_kernel_times(h, int(nsteps), ms, nl, by), h)
    return {name: (ms[k], nl[k], by[k]) for k, name in enumerate(SW_K_NAMES) if nl[k] > 0}


def sw_launch_count(h):
    n = C.c_int64()
    _check(load().sw_launch_count(h, C.byref(n)), h)
    return n.value


def _bcheck(rc, b):
    if rc != SW_OK:
        msg = load().sw_batch_last_error(b)
        raise SWError(rc, msg.decode() if msg else "")


def sw_batch_create(handles):
    """Batch of handles stepped in shared launches (see include/lagmean.h)."""
    lib = load()
    arr = (C.c_void_p * len(handles))(*[h.value for h in handles])
    b = C.c_void_p()
    rc = lib.sw_batch_create(arr, len(handles), C.byref(b))
    if rc != SW_OK:
        raise SWError(rc, lib.sw_last_error(None).decode())
    return b


def sw_batch_step(b, nsteps):
    _bcheck(load().sw_batch_step(b, int(nsteps)), b)


def sw_batch_tune(b, trial_steps=8):
    c = C.c_int(-1)
    _bcheck(load().sw_batch_tune(b, int(trial_steps), C.byref(c)), b)
    return c.value


def sw_batch_set_shape(b, choice):
    _bcheck(load().sw_batch_set_shape(b, int(choice)), b)


def sw_batch_launch_count(b):
    n = C.c_int64()
    _bcheck(load().sw_batch_launch_count(b, C.byref(n)), b)
    return n.value


def sw_batch_last_error(b):
    m = load().sw_batch_last_error(b)
    return m.decode() if m else ""


def sw_batch_destroy(b):
    load().sw_batch_destroy(b)


def sw_state_bytes(params: sw_params) -> int:
    return int(load().sw_state_bytes(C.byref(params)))


class Server:
    """Handle of a running sw_server plus the host buffers of its jobs (kept
    alive here until each job completes)."""

    def __init__(self, ptr):
        self.ptr = ptr
        self.pending = {}


def sw_server_create(precision="f32", max_active=16, chunk_steps=32, hbm_budget=150 << 30, stream=None):
    lib = load()
    p = sw_server_params()
    p.precision = {"f64": SW_PREC_FP64, "f32": SW_PREC_FP32}[precision]
    p.max_active, p.chunk_steps, p.reserved = int(max_active), int(chunk_steps), 0
    p.hbm_budget = int(hbm_budget)
    p.stream = stream or 0
    sp = C.c_void_p()
    rc = lib.sw_server_create(C.byref(p), C.byref(sp))
    if rc != SW_OK:
        raise SWError(rc, lib.sw_last_error(None).decode())
    return Server(sp)


def sw_server_submit(s: Server, params: sw_params, lp: lm_params, ic_uvh, out: dict, tag: int):
    """Queue a job; ic_uvh (3, N, N) and the host output arrays in `out` are
    kept referenced until the job is polled as done."""
    ic = np.ascontiguousarray(ic_uvh, dtype=np.float64)
    j = sw_job()
    j.params = params
    j.lm = lp
    j.ic_uvh = ic.ctypes.data_as(_DP)
    r = lm_result()
    for k in RESULT_KEYS:
        a = out.get(k)
        if a is not None:
            p, d = _ptr(a)
            if d:
                raise ValueError("server outputs are host arrays")
            setattr(r, k, p)
    r.on_device = 0
    j.out = r
    j.tag = int(tag)
    rc = load().sw_server_submit(s.ptr, C.byref(j))
    if rc != SW_OK:
        raise SWError(rc, "job rejected")
    s.pending[int(tag)] = (ic, out)


def sw_server_poll(s: Server, max_jobs=256, wait_ms=0):
    buf = (sw_job_done * max_jobs)()
    n = C.c_int(0)
    rc = load().sw_server_poll(s.ptr, buf, max_jobs, C.byref(n), int(wait_ms))
    if rc != SW_OK:
        raise SWError(rc, "poll failed")
    res = []
    for i in range(n.value):
        d = buf[i]
        ic, out = s.pending.pop(int(d.tag), (None, None))
        res.append(dict(tag=d.tag, status=d.status, t_submit=d.t_submit, t_admit=d.t_admit,
                        t_done=d.t_done, bytes=d.bytes, out=out))
    return res


def sw_server_stats_get(s: Server) -> dict:
    st = sw_server_stats()
    load().sw_server_stats_get(s.ptr, C.byref(st))
    return {n: getattr(st, n) for n, _ in sw_server_stats._fields_}


def sw_server_clock(s: Server) -> float:
    return load().sw_server_clock(s.ptr)


def sw_server_destroy(s: Server):
    load().sw_server_destroy(s.ptr)
    s.pending.clear()


def sw_project_static(inp, out, N, stream=None):
    """Allocation-free projection of a device field onto the dealiased box
    (see include/lagmean.h); inp, out: contiguous float64 CUDA tensors of
    shape (N, N) on the current CUDA device (they may be the same tensor).
    Shapes, dtypes and devices are checked before the library is called, so
    a short buffer never reaches a kernel."""
    N = int(N)
    for name, t in (("inp", inp), ("out", out)):
        if isinstance(t, np.ndarray) or not hasattr(t, "is_cuda"):
            raise ValueError(f"sw_project_static: {name} must be a torch CUDA tensor")
        if tuple(t.shape) != (N, N):
            raise ValueError(f"sw_project_static: {name} has shape {tuple(t.shape)}, expected ({N}, {N})")
        if str(t.dtype) != "torch.float64" or not t.is_contiguous():
            raise ValueError(f"sw_project_static: {name} must be contiguous float64")
        if not t.is_cuda:
            raise ValueError(f"sw_project_static: {name} must be on a CUDA device")
    import torch
    cur = torch.cuda.current_device()
    if inp.device.index != cur or out.device.index != cur:
        raise ValueError("sw_project_static: inp and out must be on the current CUDA device")
    pi, _ = _ptr(inp)
    po, _ = _ptr(out)
    lib = load()
    rc = lib.sw_project_static(pi, po, int(N), C.c_void_p(stream or 0))
    if rc != SW_OK:
        raise SWError(rc, lib.sw_last_error(None).decode())
    return out


def lmean_remap(pos_x, pos_y, ftilde, iters=20, xi=True, resid=True, stream=None):
    """Strategy-1 means onto the mean-position grid, Eq. (remap-strat1) (see
    include/lagmean.h).  pos_x, pos_y: Xi^{-1} at the grid points; ftilde: dict
    name -> f~^L; all contiguous float64 CUDA tensors of shape (N, N).
    Returns a dict with the fbar^L fields under the same names, plus
    "xi_x"/"xi_y" (Xi at the grid points) and "resid" when requested."""
    import torch

    N = int(pos_x.shape[-1])
    names = list(ftilde)
    out = {k: torch.empty_like(pos_x) for k in names}
    if xi:
        out["xi_x"] = torch.empty_like(pos_x)
        out["xi_y"] = torch.empty_like(pos_x)
    if resid:
        out["resid"] = torch.empty_like(pos_x)
    px, dx_ = _ptr(pos_x)
    py, dy_ = _ptr(pos_y)
    if not (dx_ and dy_):
        raise ValueError("lmean_remap takes device tensors")
    fin = (_DP * max(1, len(names)))()
    fout = (_DP * max(1, len(names)))()
    for i, k in enumerate(names):
        p, d = _ptr(ftilde[k])
        if not d or tuple(ftilde[k].shape) != (N, N):
            raise ValueError("ftilde fields must be (N, N) float64 CUDA tensors")
        fin[i] = p
        fout[i] = _ptr(out[k])[0]
    opt = [_ptr(out[k])[0] if k in out else None for k in ("xi_x", "xi_y", "resid")]
    lib = load()
    rc = lib.lmean_remap(N, px, py, len(names), fin, fout, int(iters), opt[0], opt[1], opt[2],
                         C.c_void_p(stream or 0))
    if rc != SW_OK:
        raise SWError(rc, lib.sw_last_error(None).decode())
    return out


def lmean_lift(pos_x, pos_y, fields, stream=None):
    """Fields at given positions (see include/lagmean.h): dict name -> f(pos)
    for contiguous float64 CUDA tensors of shape (N, N)."""
    import torch

    N = int(pos_x.shape[-1])
    names = list(fields)
    out = {k: torch.empty_like(pos_x) for k in names}
    px, dx_ = _ptr(pos_x)
    py, dy_ = _ptr(pos_y)
    if not (dx_ and dy_):
        raise ValueError("lmean_lift takes device tensors")
    fin = (_DP * max(1, len(names)))()
    fout = (_DP * max(1, len(names)))()
    for i, k in enumerate(names):
        p, d = _ptr(fields[k])
        if not d or tuple(fields[k].shape) != (N, N):
            raise ValueError("fields must be (N, N) float64 CUDA tensors")
        fin[i] = p
        fout[i] = _ptr(out[k])[0]
    lib = load()
    rc = lib.lmean_lift(N, px, py, len(names), fin, fout, C.c_void_p(stream or 0))
    if rc != SW_OK:
        raise SWError(rc, lib.sw_last_error(None).decode())
    return out


def spectrum_shells(N):
    """Number of shells sw_spectrum fills for an N x N grid."""
    K = (int(N) - 1) // 3
    return int(np.floor(np.sqrt(2.0) * K + 0.5)) + 1


def sw_spectrum(h, field, N):
    """Shell spectrum of a real N x N field (numpy array or CUDA tensor) on the
    handle's 2/3 box; returns a numpy array of spectrum_shells(N) values."""
    p, d = _ptr(field)
    n = spectrum_shells(N)
    out = np.zeros(n)
    _check(load().sw_spectrum(h, p, d, out.ctypes.data_as(_DP), n), h)
    return out


def make_sl_params(fields=("zeta", "h", "u", "v"), pos=True, scheme="trapezoid", interp="cubic",
                   n_steps=1) -> sl_params:
    p = sl_params()
    mask = 0
    for f in fields:
        mask |= FIELD_BITS[f]
    if pos:
        mask |= LM_POS
    p.fields = mask
    p.scheme = {"euler": SL_EULER, "trapezoid": SL_TRAPEZOID}[scheme]
    p.interp = {"linear": SL_LINEAR, "cubic": SL_CUBIC}[interp]
    p.reserved = 0
    p.n_steps = int(n_steps)
    return p


def sw_sl_create(h, p: sl_params):
    """Open a semi-Lagrangian Strategy-1 interval on handle h (App. B; see
    include/lagmean.h); returns the interval."""
    s = C.c_void_p()
    _check(load().sw_sl_create(h, C.byref(p), C.byref(s)), h)
    return (s, h)


def sw_sl_step(s, nsteps):
    _check(load().sw_sl_step(s[0], int(nsteps)), s[1])


def sw_sl_end(s, out: dict):
    """out: dict key -> array among zeta, h, u, v, q, pos_x, pos_y; all host or
    all device.  Frees the interval."""
    r = lm_result()
    ondev = set()
    for k in ("zeta", "h", "u", "v", "q", "pos_x", "pos_y"):
        a = out.get(k)
        p, d = _ptr(a)
        if a is not None:
            ondev.add(d)
            setattr(r, k, p)
    if len(ondev) > 1:
        raise ValueError("outputs must be all host or all device")
    r.on_device = ondev.pop() if ondev else 0
    _check(load().sw_sl_end(s[0], C.byref(r)), s[1])
    return out


def sw_sl_destroy(s):
    load().sw_sl_destroy(s[0])


def sw_fma_peak(precision="f64", trips=4096, stream=None):
    """FMA rate of the CUDA cores in TFLOP/s (see include/lagmean.h)."""
    lib = load()
    t = C.c_double(0.0)
    rc = lib.sw_fma_peak({"f64": SW_PREC_FP64, "f32": SW_PREC_FP32}[precision], int(trips), C.byref(t),
                         C.c_void_p(stream or 0))
    if rc != SW_OK:
        raise SWError(rc, lib.sw_last_error(None).decode())
    return t.value


def sw_last_error(h=None):
    m = load().sw_last_error(h)
    return m.decode() if m else ""


def sw_version():
    return load().sw_version().decode()
