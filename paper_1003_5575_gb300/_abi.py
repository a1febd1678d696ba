"""ctypes binding of librtspeel.so: the C ABI of include/rts_peel.h, same names,
argument marshalling only.  Every step of the path runs in the library's CUDA
kernels; there is no other implementation behind these functions.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librtspeel.so")

RTS_OK = 0
RTS_NOT_CONVERGED = 1
RTS_EINVAL = -1
RTS_ENOMEM = -2
RTS_ECUDA = -3
RTS_ENONFINITE = -4
RTS_PREC_MIXED = 0
RTS_PREC_FP64 = 1

RTS_K_AVERAGE, RTS_K_SUB_AVERAGE, RTS_K_SUBTRACT, RTS_K_SOLVE = 0, 1, 2, 3
RTS_K_PREDICT, RTS_K_GRAD, RTS_K_GRAD_REDUCE, RTS_K_BLOCK_PASS, RTS_K_BLOCK_FIX = 4, 5, 6, 7, 8
RTS_K_OFFSETS = 9
RTS_K_CLASSES = 10
RTS_BLOCK = 64
RTS_BLOCK_AUTO, RTS_BLOCK_FMA, RTS_BLOCK_TENSOR, RTS_BLOCK_TCGEN05 = 0, 1, 2, 3
RTS_SOLVE_AUTO, RTS_SOLVE_LAUNCHES = 0, 1
RTS_GRAD_AUTO, RTS_GRAD_DIRECT = 0, 1
KERNEL_CLASSES = ("average", "sub_average", "subtract", "solve", "predict", "grad", "grad_reduce",
                  "block_pass", "block_fix", "offsets")

EXPORTS = ("rts_peel_init", "rts_peel_set_uvw", "rts_peel_cadence", "rts_peel_cadence_host",
           "rts_peel_cadence_taylor",
           "rts_peel_predict", "rts_peel_rotate_average", "rts_peel_solve", "rts_peel_grad", "rts_peel_offsets",
           "rts_offsets_solve",
           "rts_peel_solve_noalloc", "rts_peel_rel", "rts_peel_phases",
           "rts_peel_shard_begin", "rts_peel_shard_partials", "rts_peel_shard_step",
           "rts_peel_pipeline_submit", "rts_peel_pipeline_wait",
           "rts_peel_timing", "rts_peel_timing_read", "rts_peel_kernels", "rts_barrier_selftest", "rts_fp64_rate",
           "rts_host_alloc", "rts_host_free",
           "rts_peel_last_error", "rts_peel_destroy",
           "rts_grid_init", "rts_grid_run", "rts_grid_last_ms", "rts_grid_last_error", "rts_grid_destroy",
           "rts_integrate_lengths", "rts_integrate_init", "rts_integrate_run", "rts_integrate_last_error",
           "rts_integrate_destroy")


class rts_peel_config(ctypes.Structure):
    _fields_ = [("n_ant", ctypes.c_int32), ("n_chan", ctypes.c_int32), ("n_time", ctypes.c_int32),
                ("n_iter", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("max_sources", ctypes.c_int32),
                ("uvw", ctypes.POINTER(ctypes.c_double)),
                ("freq_hz", ctypes.POINTER(ctypes.c_double)),
                ("sources_per_pass", ctypes.c_int32), ("block_kernel", ctypes.c_int32),
                ("solve_kernel", ctypes.c_int32), ("grad_kernel", ctypes.c_int32),
                ("band_n_chan", ctypes.c_int32), ("band_chan0", ctypes.c_int32)]


class rts_grid_config(ctypes.Structure):
    _fields_ = [("n_pix", ctypes.c_int32), ("bin", ctypes.c_int32), ("r_max", ctypes.c_double),
                ("gcf", ctypes.POINTER(ctypes.c_double)), ("n_tab", ctypes.c_int32),
                ("n_pol", ctypes.c_int32), ("max_vis", ctypes.c_int32)]


class RtsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"rts_peel error {code}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None

_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)
_i32 = ctypes.c_int32


def lib():
    """Load librtspeel.so (raises if it has not been built: there is no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "paper_1003_5575_gb300.build.build() (nvcc, sm_103a)")
            L = ctypes.CDLL(LIB_PATH)
            L.rts_peel_init.restype = ctypes.c_int
            L.rts_peel_init.argtypes = [ctypes.POINTER(rts_peel_config), ctypes.POINTER(_vp)]
            L.rts_peel_set_uvw.restype = ctypes.c_int
            L.rts_peel_set_uvw.argtypes = [_vp, _dp, _vp]
            L.rts_peel_cadence.restype = ctypes.c_int
            L.rts_peel_cadence.argtypes = [_vp, _vp, _vp, _i32, _dp, _vp, _ip, _vp]
            L.rts_peel_cadence_taylor.restype = ctypes.c_int
            L.rts_peel_cadence_taylor.argtypes = [_vp, _vp, _vp, _i32, _dp, _vp, _vp, _ip, _vp]
            L.rts_peel_cadence_host.restype = ctypes.c_int
            L.rts_peel_cadence_host.argtypes = [_vp, _vp, _vp, _i32, _dp, _vp, _ip, _vp, _vp]
            L.rts_peel_predict.restype = ctypes.c_int
            L.rts_peel_predict.argtypes = [_vp, _vp, _i32, _dp, _vp, _i32, _vp]
            L.rts_peel_rotate_average.restype = ctypes.c_int
            L.rts_peel_rotate_average.argtypes = [_vp, _vp, ctypes.c_double, ctypes.c_double, _vp, _vp]
            L.rts_peel_solve.restype = ctypes.c_int
            L.rts_peel_solve.argtypes = [_vp, _vp, ctypes.c_double, _vp, _ip, _vp]
            L.rts_peel_solve_noalloc.restype = ctypes.c_int
            L.rts_peel_solve_noalloc.argtypes = [_vp, _i32, ctypes.c_double, _i32, _i32, _vp, _ip, _vp]
            L.rts_peel_shard_begin.restype = ctypes.c_int
            L.rts_peel_shard_begin.argtypes = [_vp, _vp, _vp, _i32, _dp, _vp, _vp]
            L.rts_peel_shard_partials.restype = ctypes.c_int
            L.rts_peel_shard_partials.argtypes = [_vp, ctypes.POINTER(ctypes.POINTER(ctypes.c_float)),
                                                  ctypes.POINTER(ctypes.c_int64)]
            L.rts_peel_shard_step.restype = ctypes.c_int
            L.rts_peel_shard_step.argtypes = [_vp, _ip, _vp]
            L.rts_peel_rel.restype = ctypes.c_int
            L.rts_peel_rel.argtypes = [_vp, _i32, _dp, _vp]
            L.rts_peel_phases.restype = ctypes.c_int
            L.rts_peel_phases.argtypes = [_vp, ctypes.c_double, ctypes.c_double, _i32, _vp, _i32, _vp, _vp]
            L.rts_peel_pipeline_submit.restype = ctypes.c_int
            L.rts_peel_pipeline_submit.argtypes = [_vp, _vp, _vp, _i32, _dp, _vp, _ip]
            L.rts_peel_pipeline_wait.restype = ctypes.c_int
            L.rts_peel_pipeline_wait.argtypes = [_vp]
            L.rts_peel_grad.restype = ctypes.c_int
            L.rts_peel_grad.argtypes = [_vp, _vp, _i32, _vp, _vp, _vp, _vp, _vp, _vp]
            L.rts_peel_offsets.restype = ctypes.c_int
            L.rts_peel_offsets.argtypes = [_vp, _vp, _i32, _vp, _vp, ctypes.c_double, ctypes.c_double,
                                           _vp, _vp, _vp]
            L.rts_offsets_solve.restype = ctypes.c_int
            L.rts_offsets_solve.argtypes = [_vp, _i32, _vp, _vp]
            L.rts_peel_timing.restype = ctypes.c_int
            L.rts_peel_timing.argtypes = [_vp, _i32]
            L.rts_peel_timing_read.restype = ctypes.c_int
            L.rts_peel_timing_read.argtypes = [_vp, _dp, ctypes.POINTER(ctypes.c_int64),
                                               ctypes.POINTER(ctypes.c_int64)]
            L.rts_barrier_selftest.restype = ctypes.c_int
            L.rts_barrier_selftest.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _ip]
            L.rts_fp64_rate.restype = ctypes.c_int
            L.rts_fp64_rate.argtypes = [_dp]
            L.rts_peel_kernels.restype = ctypes.c_int
            L.rts_peel_kernels.argtypes = [_vp, _ip, _ip]
            L.rts_host_alloc.restype = ctypes.c_int
            L.rts_host_alloc.argtypes = [ctypes.c_uint64, ctypes.POINTER(_vp)]
            L.rts_host_free.restype = ctypes.c_int
            L.rts_host_free.argtypes = [_vp]
            L.rts_peel_last_error.restype = ctypes.c_char_p
            L.rts_peel_last_error.argtypes = [_vp]
            L.rts_peel_destroy.restype = None
            L.rts_peel_destroy.argtypes = [_vp]
            L.rts_grid_init.restype = ctypes.c_int
            L.rts_grid_init.argtypes = [ctypes.POINTER(rts_grid_config), ctypes.POINTER(_vp)]
            L.rts_grid_run.restype = ctypes.c_int
            L.rts_grid_run.argtypes = [_vp, _vp, _vp, _i32, _vp, _vp]
            L.rts_grid_last_ms.restype = ctypes.c_int
            L.rts_grid_last_ms.argtypes = [_vp, _dp, _dp]
            L.rts_grid_last_error.restype = ctypes.c_char_p
            L.rts_grid_last_error.argtypes = [_vp]
            L.rts_grid_destroy.restype = None
            L.rts_grid_destroy.argtypes = [_vp]
            L.rts_integrate_lengths.restype = ctypes.c_int
            L.rts_integrate_lengths.argtypes = [_i32, _dp, _i32, _dp, _ip, _ip]
            L.rts_integrate_init.restype = ctypes.c_int
            L.rts_integrate_init.argtypes = [_i32, ctypes.c_int64, _i32, _ip, _i32, ctypes.POINTER(_vp)]
            L.rts_integrate_run.restype = ctypes.c_int
            L.rts_integrate_run.argtypes = [_vp, _vp, _vp, _vp]
            L.rts_integrate_last_error.restype = ctypes.c_char_p
            L.rts_integrate_last_error.argtypes = [_vp]
            L.rts_integrate_destroy.restype = None
            L.rts_integrate_destroy.argtypes = [_vp]
            _lib = L
    return _lib


def _check(rc: int, handle) -> int:
    if rc < 0:
        msg = lib().rts_peel_last_error(handle)
        raise RtsError(rc, msg.decode() if msg else "")
    return rc


def rts_peel_init(cfg: rts_peel_config):
    h = _vp()
    _check(lib().rts_peel_init(ctypes.byref(cfg), ctypes.byref(h)), None)
    return h


def rts_peel_set_uvw(h, uvw_ptr, stream):
    return _check(lib().rts_peel_set_uvw(h, uvw_ptr, stream), h)


def rts_peel_cadence(h, d_vis, d_resid, n_src, h_src, d_jones, h_status, stream):
    return _check(lib().rts_peel_cadence(h, d_vis, d_resid, n_src, h_src, d_jones, h_status, stream), h)


def rts_peel_cadence_taylor(h, d_vis, d_resid, n_src, h_src, d_gain, d_slope, h_status, stream):
    return _check(lib().rts_peel_cadence_taylor(h, d_vis, d_resid, n_src, h_src, d_gain, d_slope,
                                                h_status, stream), h)


def rts_peel_cadence_host(h, h_vis, h_resid, n_src, h_src, h_jones, h_status, d_work, stream):
    return _check(lib().rts_peel_cadence_host(h, h_vis, h_resid, n_src, h_src, h_jones, h_status,
                                              d_work, stream), h)


def rts_peel_predict(h, d_vis, n_src, h_src, d_jones, accumulate, stream):
    return _check(lib().rts_peel_predict(h, d_vis, n_src, h_src, d_jones, accumulate, stream), h)


def rts_peel_rotate_average(h, d_vis, l, m, d_avg, stream):
    return _check(lib().rts_peel_rotate_average(h, d_vis, l, m, d_avg, stream), h)


def rts_peel_solve(h, d_avg, S, d_jones, h_status, stream):
    return _check(lib().rts_peel_solve(h, d_avg, S, d_jones, h_status, stream), h)


def rts_peel_solve_noalloc(d_avg, n_ant, S, n_iter, precision, d_jones, h_status, stream):
    return _check(lib().rts_peel_solve_noalloc(d_avg, n_ant, S, n_iter, precision, d_jones, h_status,
                                               stream), None)


def rts_peel_shard_begin(h, d_vis, d_resid, n_src, h_src, d_jones, stream):
    return _check(lib().rts_peel_shard_begin(h, d_vis, d_resid, n_src, h_src, d_jones, stream), h)


def rts_peel_shard_partials(h):
    """(device address, float count) of the current block's partial averages."""
    p = ctypes.POINTER(ctypes.c_float)()
    n = ctypes.c_int64()
    _check(lib().rts_peel_shard_partials(h, ctypes.byref(p), ctypes.byref(n)), h)
    return ctypes.cast(p, ctypes.c_void_p).value, n.value


def rts_peel_shard_step(h, h_status, stream) -> int:
    """1 while another exchange of partial averages is needed, 0 when done."""
    return _check(lib().rts_peel_shard_step(h, h_status, stream), h)


def rts_peel_rel(h, n_src, h_rel, stream):
    return _check(lib().rts_peel_rel(h, n_src, h_rel, stream), h)


def rts_peel_phases(h, l, m, n_pair, d_tb, form, d_phase, stream):
    return _check(lib().rts_peel_phases(h, float(l), float(m), n_pair, d_tb, form, d_phase, stream), h)


def rts_peel_pipeline_submit(h, h_vis, h_resid, n_src, h_src, h_jones, h_status):
    return _check(lib().rts_peel_pipeline_submit(h, h_vis, h_resid, n_src, h_src, h_jones, h_status), h)


def rts_peel_pipeline_wait(h):
    return _check(lib().rts_peel_pipeline_wait(h), h)


def rts_peel_grad(h, d_vis, n_src, d_jones, d_src, d_loss, d_gJ, d_gsrc, stream):
    return _check(lib().rts_peel_grad(h, d_vis, n_src, d_jones, d_src, d_loss, d_gJ, d_gsrc, stream), h)


def rts_peel_offsets(h, d_vis, n_src, d_jones, d_src, alpha, nu_ref_hz, d_out, d_offsets, stream):
    return _check(lib().rts_peel_offsets(h, d_vis, n_src, d_jones, d_src, float(alpha), float(nu_ref_hz),
                                         d_out, d_offsets, stream), h)


def rts_offsets_solve(d_out, n_src, d_offsets, stream):
    return _check(lib().rts_offsets_solve(d_out, n_src, d_offsets, stream), None)


def rts_peel_kernels(h):
    """(block_kernel, solve_kernel) resolved by the handle."""
    bk, sk = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().rts_peel_kernels(h, ctypes.byref(bk), ctypes.byref(sk)), h)
    return bk.value, sk.value


def rts_fp64_rate() -> float:
    """Measured FP64 FMA rate of the current device, TFLOP/s."""
    v = ctypes.c_double(0.0)
    _check(lib().rts_fp64_rate(ctypes.byref(v)), None)
    return v.value


def rts_barrier_selftest(n_cta: int, missing: int, rounds: int) -> int:
    """CTAs whose waits all completed (see include/rts_peel.h)."""
    out = ctypes.c_int32()
    _check(lib().rts_barrier_selftest(int(n_cta), int(missing), int(rounds), ctypes.byref(out)), None)
    return out.value


def rts_peel_timing(h, enable: int):
    return _check(lib().rts_peel_timing(h, int(enable)), h)


def rts_peel_timing_read(h):
    """{class: (ms, groups, launches)} since the last rts_peel_timing(h, 1)."""
    ms = (ctypes.c_double * RTS_K_CLASSES)()
    gr = (ctypes.c_int64 * RTS_K_CLASSES)()
    la = (ctypes.c_int64 * RTS_K_CLASSES)()
    _check(lib().rts_peel_timing_read(h, ms, gr, la), h)
    return {name: (ms[i], gr[i], la[i]) for i, name in enumerate(KERNEL_CLASSES)}


def rts_host_alloc(nbytes: int) -> int:
    p = _vp()
    rc = lib().rts_host_alloc(int(nbytes), ctypes.byref(p))
    if rc < 0:
        raise RtsError(rc, rts_peel_last_error(None))
    return p.value


def rts_host_free(ptr: int) -> None:
    rc = lib().rts_host_free(_vp(ptr))
    if rc < 0:
        raise RtsError(rc, "cudaFreeHost failed")


def rts_peel_last_error(h) -> str:
    m = lib().rts_peel_last_error(h)
    return m.decode() if m else ""


def rts_peel_destroy(h) -> None:
    lib().rts_peel_destroy(h)


# ---- gridder (include/rts_grid.h) ---------------------------------------------

def _gcheck(rc: int, handle) -> int:
    if rc < 0:
        msg = lib().rts_grid_last_error(handle)
        raise RtsError(rc, msg.decode() if msg else "")
    return rc


def rts_grid_init(cfg: rts_grid_config):
    h = _vp()
    _gcheck(lib().rts_grid_init(ctypes.byref(cfg), ctypes.byref(h)), None)
    return h


def rts_grid_run(h, d_xy, d_vis, n_vis, d_grid, stream):
    return _gcheck(lib().rts_grid_run(h, d_xy, d_vis, n_vis, d_grid, stream), h)


def rts_grid_last_ms(h):
    a, b = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _gcheck(lib().rts_grid_last_ms(h, ctypes.byref(a), ctypes.byref(b)), h)
    return a.value, b.value


def rts_grid_last_error(h):
    m = lib().rts_grid_last_error(h)
    return m.decode() if m else ""


def rts_grid_destroy(h):
    lib().rts_grid_destroy(h)


# ---- visibility integrator (include/rts_integrate.h) ---------------------------

def _icheck(rc: int, handle) -> int:
    if rc < 0:
        msg = lib().rts_integrate_last_error(handle)
        raise RtsError(rc, msg.decode() if msg else "")
    return rc


def rts_integrate_lengths(n_ant, uvw_ptr, n_cut, cut_ptr, len_for_ptr, len_out_ptr):
    return _icheck(lib().rts_integrate_lengths(n_ant, uvw_ptr, n_cut, cut_ptr, len_for_ptr, len_out_ptr), None)


def rts_integrate_init(n_fine, n_bl, n_chan, len_ptr, n_slot):
    h = _vp()
    _icheck(lib().rts_integrate_init(n_fine, n_bl, n_chan, len_ptr, n_slot, ctypes.byref(h)), None)
    return h


def rts_integrate_run(h, d_fine, d_out, stream):
    return _icheck(lib().rts_integrate_run(h, d_fine, d_out, stream), h)


def rts_integrate_destroy(h):
    lib().rts_integrate_destroy(h)
