"""Thin ctypes binding of the C ABI in ``include/fdas.h``.

Argument marshalling only: every function here forwards to the entry point of
the same name in ``libfdas_gb300.so`` and turns a negative status into
``FdasError``. Device pointers are passed as integers (e.g.
``torch.Tensor.data_ptr()``), host buffers as numpy arrays. There is no CPU
fallback: if the library is missing, loading fails with an error.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

FDAS_OK = 0
FDAS_ERR_INVALID = -1
FDAS_ERR_NOMEM = -2
FDAS_ERR_CUDA = -3
FDAS_ERR_TIMEOUT = -4
FDAS_ERR_OVERFLOW = -5
FDAS_CORR_FFT = 0
FDAS_CORR_GEMM_BF16 = 1
FDAS_CORR_GEMM_FP16 = 2
FDAS_WHITEN_RUNNING = 0
FDAS_WHITEN_BLOCK = 1


class fdas_cand(ctypes.Structure):
    _fields_ = [("r_top", ctypes.c_int32), ("z_idx", ctypes.c_int32),
                ("h", ctypes.c_int32), ("power", ctypes.c_float)]


class fdas_plan_info(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("nb", ctypes.c_int64),
                ("zmax", ctypes.c_int32), ("dz", ctypes.c_int32), ("Z", ctypes.c_int32),
                ("m", ctypes.c_int32), ("L", ctypes.c_int32), ("V", ctypes.c_int32),
                ("S", ctypes.c_int32), ("nharm", ctypes.c_int32), ("n_levels", ctypes.c_int32),
                ("thresholds", ctypes.c_float * 5), ("max_cands", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("plane_floats", ctypes.c_int64),
                ("corr_ctas_per_sm", ctypes.c_int32), ("corr_grid", ctypes.c_int32)]


class fdas_batch_info(ctypes.Structure):
    _fields_ = [("N_max", ctypes.c_int64), ("segment", ctypes.c_int32),
                ("n_lengths", ctypes.c_int32), ("graphs", ctypes.c_int32),
                ("n_tuned", ctypes.c_int32), ("graph_builds", ctypes.c_int64),
                ("graph_launches", ctypes.c_int64), ("hs_block", ctypes.c_int32),
                ("tuned_segment", ctypes.c_int32 * 8), ("tuned_hs_block", ctypes.c_int32 * 8),
                ("tuned_ms", ctypes.c_float * 8), ("n_classes", ctypes.c_int32),
                ("device_bytes", ctypes.c_int64)]


CAND_DTYPE = np.dtype([("r_top", "<i4"), ("z_idx", "<i4"), ("h", "<i4"), ("power", "<f4")])
PEAK_DTYPE = np.dtype([("r_top", "<i4"), ("z_idx", "<i4"), ("h", "<i4"), ("power", "<f4"),
                       ("sigma", "<f4"), ("log10_p", "<f4")])


class FdasError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: status {status} ({detail})")
        self.status = status


_lib = None

_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_SIGS = {
    "fdas_plan_create": [ctypes.POINTER(_P), _I64, _I32, _I32, _I32, _I32, _I32,
                         ctypes.c_float, _I64, _P],
    "fdas_plan_destroy": [_P],
    "fdas_plan_get_info": [_P, ctypes.POINTER(fdas_plan_info)],
    "fdas_search": [_P, _P, _I32, _P, _P],
    "fdas_search_host": [_P, _P, _I32, _P, _P],
    "fdas_search_device": [_P, _P, _I32, _P, _P],
    "fdas_batch_create": [ctypes.POINTER(_P), _I64, _I32, _I32, _I32, _I32, _I32,
                          ctypes.c_float, _I64, _P],
    "fdas_batch_destroy": [_P],
    "fdas_batch_add_class": [_P, _I32, _I32, _I32],
    "fdas_search_batch": [_P, _P, _P, _P, _I32, _P, _P],
    "fdas_plane_debug": [_P, _P],
    "fdas_stage_spectrum": [_P, _P, _P],
    "fdas_stage_whiten": [_P, _P, _P],
    "fdas_stage_plane": [_P, _P, _P],
    "fdas_stage_harmsum": [_P, _P, _P, _P],
    "fdas_template_taps": [_P, _P],
    "fdas_template_bank": [_P, _P],
    "fdas_profile_trial": [_P, _P, _P],
    "fdas_spectrum_noalloc": [_P, _I64, _P, _P],
    "fdas_plan_set_correlation": [_P, _I32],
    "fdas_plan_set_whitening": [_P, _I32],
    "fdas_plan_set_harmsum_block": [_P, _I32],
    "fdas_plan_set_interbin": [_P, _I32],
    "fdas_plan_set_wait_limit": [_P, ctypes.c_uint32],
    "fdas_distill": [_P, _P, _P, _P, _P],
    "fdas_batch_create_tuned": [ctypes.POINTER(_P), _I64, _I32, _I32, _I32, _I32,
                                ctypes.c_float, _I64, _P, _P],
    "fdas_batch_set_graphs": [_P, _I32],
    "fdas_batch_get_info": [_P, ctypes.POINTER(fdas_batch_info)],
    "fdas_host_fresnel": [ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                          ctypes.POINTER(ctypes.c_double)],
}


def library_path() -> str:
    return _build.LIB


def load():
    """Loads the built library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing "
                           "(run __graft_entry__.build() or python -m paper_1511_07343_gb300.build)")
    lib = ctypes.CDLL(path)
    for name, args in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.fdas_strerror.argtypes = [ctypes.c_int]
    lib.fdas_strerror.restype = ctypes.c_char_p
    lib.fdas_last_error.argtypes = []
    lib.fdas_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(status: int, where: str, allow=()):
    if status == FDAS_OK or status in allow:
        return status
    lib = load()
    detail = (lib.fdas_last_error() or b"").decode() or lib.fdas_strerror(status).decode()
    raise FdasError(status, where, detail)


def _ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    raise TypeError(f"cannot pass {type(x)} as a pointer")


def fdas_plan_create(N, zmax, dz, template_width, segment, nharm, sigma=6.0,
                     max_cands=1 << 20, stream=0):
    plan = _P()
    _check(load().fdas_plan_create(ctypes.byref(plan), N, zmax, dz, template_width, segment,
                                   nharm, sigma, max_cands, _ptr(stream) or None),
           "fdas_plan_create")
    return plan.value


def fdas_plan_destroy(plan):
    _check(load().fdas_plan_destroy(plan), "fdas_plan_destroy")


def fdas_plan_get_info(plan) -> fdas_plan_info:
    info = fdas_plan_info()
    _check(load().fdas_plan_get_info(plan, ctypes.byref(info)), "fdas_plan_get_info")
    return info


def fdas_search(plan, d_series, n_trials, h_out, h_counts):
    return _check(load().fdas_search(plan, _ptr(d_series), n_trials, _ptr(h_out),
                                     _ptr(h_counts)), "fdas_search", allow=(FDAS_ERR_OVERFLOW,))


def fdas_search_host(plan, h_series, n_trials, h_out, h_counts):
    return _check(load().fdas_search_host(plan, _ptr(h_series), n_trials, _ptr(h_out),
                                          _ptr(h_counts)), "fdas_search_host",
                  allow=(FDAS_ERR_OVERFLOW,))


def fdas_search_device(plan, d_series, n_trials, d_out, d_counts):
    _check(load().fdas_search_device(plan, _ptr(d_series), n_trials, _ptr(d_out),
                                     _ptr(d_counts)), "fdas_search_device")


def fdas_batch_create(N_max, zmax, dz, template_width, segment, nharm, sigma=6.0,
                      max_cands=1 << 20, stream=0):
    batch = _P()
    _check(load().fdas_batch_create(ctypes.byref(batch), N_max, zmax, dz, template_width, segment,
                                    nharm, sigma, max_cands, _ptr(stream) or None),
           "fdas_batch_create")
    return batch.value


def fdas_batch_create_tuned(N_max, zmax, dz, template_width, nharm, sigma=6.0,
                            max_cands=1 << 20, d_probe=None, stream=0):
    batch = _P()
    _check(load().fdas_batch_create_tuned(ctypes.byref(batch), N_max, zmax, dz, template_width,
                                          nharm, sigma, max_cands, _ptr(d_probe) or None,
                                          _ptr(stream) or None), "fdas_batch_create_tuned")
    return batch.value


def fdas_batch_set_graphs(batch, enable):
    _check(load().fdas_batch_set_graphs(batch, int(bool(enable))), "fdas_batch_set_graphs")


def fdas_batch_get_info(batch) -> fdas_batch_info:
    info = fdas_batch_info()
    _check(load().fdas_batch_get_info(batch, ctypes.byref(info)), "fdas_batch_get_info")
    return info


def fdas_batch_destroy(batch):
    _check(load().fdas_batch_destroy(batch), "fdas_batch_destroy")


def fdas_batch_add_class(batch, zmax, template_width, segment):
    _check(load().fdas_batch_add_class(batch, zmax, template_width, segment),
           "fdas_batch_add_class")


def fdas_search_batch(batch, d_series_list, N_list, d_out, d_counts, zmax_list=None):
    n = len(d_series_list)
    ptrs = (ctypes.c_void_p * n)(*[_ptr(x) for x in d_series_list])
    lens = (ctypes.c_int64 * n)(*[int(v) for v in N_list])
    zs = None
    if zmax_list is not None:
        if len(zmax_list) != n:
            raise ValueError("zmax_list needs one entry per trial")
        zs = (ctypes.c_int32 * n)(*[int(v) for v in zmax_list])
    _check(load().fdas_search_batch(batch, ctypes.cast(ptrs, ctypes.c_void_p),
                                    ctypes.cast(lens, ctypes.c_void_p),
                                    ctypes.cast(zs, ctypes.c_void_p) if zs is not None else None,
                                    n, _ptr(d_out), _ptr(d_counts)), "fdas_search_batch")


def fdas_plane_debug(plan, d_plane):
    _check(load().fdas_plane_debug(plan, _ptr(d_plane)), "fdas_plane_debug")


def fdas_stage_spectrum(plan, d_series, d_spectrum):
    _check(load().fdas_stage_spectrum(plan, _ptr(d_series), _ptr(d_spectrum)),
           "fdas_stage_spectrum")


def fdas_stage_whiten(plan, d_spectrum, d_white):
    _check(load().fdas_stage_whiten(plan, _ptr(d_spectrum), _ptr(d_white)), "fdas_stage_whiten")


def fdas_stage_plane(plan, d_white, d_plane):
    _check(load().fdas_stage_plane(plan, _ptr(d_white), _ptr(d_plane)), "fdas_stage_plane")


def fdas_stage_harmsum(plan, d_plane, d_out, d_count):
    _check(load().fdas_stage_harmsum(plan, _ptr(d_plane), _ptr(d_out), _ptr(d_count)),
           "fdas_stage_harmsum")


def fdas_template_taps(plan, d_taps):
    _check(load().fdas_template_taps(plan, _ptr(d_taps)), "fdas_template_taps")


def fdas_template_bank(plan, d_bank):
    _check(load().fdas_template_bank(plan, _ptr(d_bank)), "fdas_template_bank")


def fdas_profile_trial(plan, d_series):
    ms = np.zeros(5, dtype=np.float32)
    _check(load().fdas_profile_trial(plan, _ptr(d_series), ms.ctypes.data), "fdas_profile_trial")
    return ms


def fdas_distill(plan, d_cands, d_count, d_peaks, d_npeaks):
    _check(load().fdas_distill(plan, _ptr(d_cands), _ptr(d_count), _ptr(d_peaks), _ptr(d_npeaks)),
           "fdas_distill")


def fdas_plan_set_interbin(plan, enable):
    _check(load().fdas_plan_set_interbin(plan, int(bool(enable))), "fdas_plan_set_interbin")


def fdas_plan_set_whitening(plan, mode):
    _check(load().fdas_plan_set_whitening(plan, mode), "fdas_plan_set_whitening")


def fdas_plan_set_harmsum_block(plan, threads):
    _check(load().fdas_plan_set_harmsum_block(plan, threads), "fdas_plan_set_harmsum_block")


def fdas_plan_set_wait_limit(plan, polls):
    _check(load().fdas_plan_set_wait_limit(plan, int(polls)), "fdas_plan_set_wait_limit")


def fdas_plan_set_correlation(plan, mode):
    _check(load().fdas_plan_set_correlation(plan, mode), "fdas_plan_set_correlation")


def fdas_spectrum_noalloc(d_series, N, d_spectrum, stream=0):
    _check(load().fdas_spectrum_noalloc(_ptr(d_series), N, _ptr(d_spectrum), _ptr(stream) or None),
           "fdas_spectrum_noalloc")


def fdas_host_fresnel(x: float):
    c = ctypes.c_double()
    s = ctypes.c_double()
    _check(load().fdas_host_fresnel(x, ctypes.byref(c), ctypes.byref(s)), "fdas_host_fresnel")
    return c.value, s.value


def fdas_strerror(status: int) -> str:
    return load().fdas_strerror(status).decode()


def fdas_last_error() -> str:
    return (load().fdas_last_error() or b"").decode()
