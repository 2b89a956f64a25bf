"""ctypes binding of libcmlbm.so (include/cmlbm.h): argument marshalling only.

Every step of the solver runs in the CUDA kernels behind the C ABI; this module only turns
numpy arrays and torch tensors into pointers.  If the library cannot be built or loaded the
import fails loudly -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

from . import buildlib as _build

LBM_OK, LBM_ERR_ARG, LBM_ERR_CUDA, LBM_ERR_OOM, LBM_ERR_DIVERGED, LBM_ERR_TIMEOUT, LBM_ERR_STATE, \
    LBM_ERR_UNSUPPORTED = range(8)
LBM_FP32, LBM_FP16_DEV, LBM_BF16_DEV = 0, 1, 2
LBM_FORCE_NONE, LBM_FORCE_UNIFORM, LBM_FORCE_KOLMOGOROV, LBM_FORCE_FIELD, LBM_FORCE_SHAN_CHEN = range(5)
LBM_STATS_LEN = 10
LBM_PROFILE_LEN = 4
HEADER = os.path.join(_build.ROOT, "include", "cmlbm.h")


class LbmDesc(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("nu", ctypes.c_double), ("rho0", ctypes.c_double),
        ("walls_y", ctypes.c_int),
        ("mask", ctypes.c_void_p),
        ("storage", ctypes.c_int),
        ("stream", ctypes.c_void_p),
        ("store", ctypes.c_void_p),
        ("slab_z", ctypes.c_int),
    ]


class LbmDomain(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("nu", ctypes.c_double),
        ("force", ctypes.c_double * 3),
        ("walls_y", ctypes.c_int),
        ("mask", ctypes.c_void_p),
    ]


class LbmCgParams(ctypes.Structure):
    _fields_ = [("rho_r0", ctypes.c_double), ("rho_b0", ctypes.c_double), ("nu_r", ctypes.c_double),
                ("nu_b", ctypes.c_double), ("A", ctypes.c_double), ("beta", ctypes.c_double),
                ("g", ctypes.c_double * 3)]


class LbmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{status_name(status)}: {msg}")
        self.status = status


_lib = None
_P = ctypes.c_void_p


def declared_symbols(header: str = HEADER):
    """Names of the entry points declared in include/cmlbm.h."""
    txt = open(header).read()
    return sorted(set(re.findall(r"^LBM_API\s+[\w\s\*]+?\b(lbm_\w+)\s*\(", txt, flags=re.M)))


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        st = ctypes.c_int
        L.lbm_store_bytes.argtypes = [ctypes.POINTER(LbmDesc)]
        L.lbm_store_bytes.restype = ctypes.c_size_t
        L.lbm_create.argtypes = [ctypes.POINTER(LbmDesc), ctypes.POINTER(_P)]
        L.lbm_create.restype = st
        L.lbm_set_force.argtypes = [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_double), _P, _P, _P]
        L.lbm_set_force.restype = st
        L.lbm_set_hermite_orders.argtypes = [_P, ctypes.c_int, ctypes.c_int]
        L.lbm_set_hermite_orders.restype = st
        L.lbm_set_magnetic.argtypes = [_P, ctypes.c_double, ctypes.POINTER(ctypes.c_double), _P, _P, _P]
        L.lbm_set_magnetic.restype = st
        L.lbm_get_magnetic_populations.argtypes = [_P, _P]
        L.lbm_get_magnetic_populations.restype = st
        L.lbm_set_magnetic_populations.argtypes = [_P, _P]
        L.lbm_set_magnetic_populations.restype = st
        L.lbm_magnetic.argtypes = [_P] + [_P] * 6
        L.lbm_magnetic.restype = st
        L.lbm_set_colour_gradient.argtypes = [_P, ctypes.POINTER(LbmCgParams), _P, _P]
        L.lbm_set_colour_gradient.restype = st
        L.lbm_colour_densities.argtypes = [_P, _P, _P]
        L.lbm_colour_densities.restype = st
        L.lbm_get_colour_populations.argtypes = [_P, _P, _P]
        L.lbm_get_colour_populations.restype = st
        L.lbm_set_colour_populations.argtypes = [_P, _P, _P]
        L.lbm_set_colour_populations.restype = st
        L.lbm_set_state.argtypes = [_P, _P, _P, _P, _P]
        L.lbm_set_state.restype = st
        L.lbm_set_populations.argtypes = [_P, _P]
        L.lbm_set_populations.restype = st
        L.lbm_get_populations.argtypes = [_P, _P]
        L.lbm_get_populations.restype = st
        L.lbm_step.argtypes = [_P, ctypes.c_int]
        L.lbm_step.restype = st
        L.lbm_stream_only.argtypes = [_P, ctypes.c_int]
        L.lbm_stream_only.restype = st
        L.lbm_macroscopic.argtypes = [_P, _P, _P, _P, _P]
        L.lbm_macroscopic.restype = st
        L.lbm_stats.argtypes = [_P, ctypes.POINTER(ctypes.c_double)]
        L.lbm_stats.restype = st
        L.lbm_synchronize.argtypes = [_P]
        L.lbm_synchronize.restype = st
        L.lbm_profile.argtypes = [_P, ctypes.c_int]
        L.lbm_profile.restype = st
        L.lbm_profile_read.argtypes = [_P, ctypes.POINTER(ctypes.c_double)]
        L.lbm_profile_read.restype = st
        L.lbm_reduce_fields_noalloc.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P, _P,
                                                _P, _P, _P, ctypes.POINTER(ctypes.c_double), _P]
        L.lbm_reduce_fields_noalloc.restype = st
        L.lbm_batch_create.argtypes = [ctypes.POINTER(LbmDomain), ctypes.c_int, ctypes.c_double, _P, ctypes.POINTER(_P)]
        L.lbm_batch_create.restype = st
        L.lbm_batch_autotune.argtypes = [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
        L.lbm_batch_autotune.restype = st
        L.lbm_batch_set_shape.argtypes = [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.lbm_batch_set_shape.restype = st
        L.lbm_batch_step.argtypes = [_P, ctypes.c_int]
        L.lbm_batch_step.restype = st
        L.lbm_batch_run.argtypes = [_P, ctypes.c_double, ctypes.c_longlong, ctypes.c_int,
                                    ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_int)]
        L.lbm_batch_run.restype = st
        L.lbm_batch_set_state.argtypes = [_P, ctypes.c_int, _P, _P, _P, _P]
        L.lbm_batch_set_state.restype = st
        L.lbm_batch_macroscopic.argtypes = [_P, ctypes.c_int, _P, _P, _P, _P]
        L.lbm_batch_macroscopic.restype = st
        L.lbm_batch_get_populations.argtypes = [_P, ctypes.c_int, _P]
        L.lbm_batch_get_populations.restype = st
        L.lbm_batch_nodes.argtypes = [_P]
        L.lbm_batch_nodes.restype = ctypes.c_longlong
        L.lbm_batch_time.argtypes = [_P]
        L.lbm_batch_time.restype = ctypes.c_longlong
        L.lbm_batch_active.argtypes = [_P]
        L.lbm_batch_active.restype = ctypes.c_int
        L.lbm_batch_last_error.argtypes = [_P]
        L.lbm_batch_last_error.restype = ctypes.c_char_p
        L.lbm_batch_destroy.argtypes = [_P]
        L.lbm_batch_destroy.restype = None
        L.lbm_gemm_bf16.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    _P, ctypes.c_longlong, ctypes.c_longlong, ctypes.c_longlong,
                                    _P, ctypes.c_longlong, ctypes.c_longlong, ctypes.c_longlong,
                                    _P, ctypes.c_longlong, ctypes.c_longlong, ctypes.c_longlong,
                                    ctypes.c_int, ctypes.c_float, ctypes.c_int, _P, _P]
        L.lbm_gemm_bf16.restype = st
        L.lbm_no_create.argtypes = [ctypes.c_int] * 7 + [ctypes.c_ulonglong, _P, ctypes.POINTER(_P)]
        L.lbm_no_create.restype = st
        L.lbm_no_param_count.argtypes = [_P]
        L.lbm_no_param_count.restype = ctypes.c_longlong
        L.lbm_no_params.argtypes = [_P, _P, ctypes.c_int]
        L.lbm_no_params.restype = st
        L.lbm_no_grads.argtypes = [_P, _P]
        L.lbm_no_grads.restype = st
        L.lbm_no_forward.argtypes = [_P, ctypes.c_int, _P, _P]
        L.lbm_no_forward.restype = st
        L.lbm_no_backward.argtypes = [_P, _P]
        L.lbm_no_backward.restype = st
        L.lbm_no_train_step.argtypes = [_P, ctypes.c_int, _P, _P, ctypes.c_float, ctypes.POINTER(ctypes.c_double)]
        L.lbm_no_train_step.restype = st
        L.lbm_no_use_graphs.argtypes = [_P, ctypes.c_int]
        L.lbm_no_use_graphs.restype = st
        L.lbm_no_last_error.argtypes = [_P]
        L.lbm_no_last_error.restype = ctypes.c_char_p
        L.lbm_no_destroy.argtypes = [_P]
        L.lbm_no_destroy.restype = None
        L.lbm_halo_bytes.argtypes = [_P]
        L.lbm_halo_bytes.restype = ctypes.c_size_t
        L.lbm_halo_pack.argtypes = [_P, ctypes.c_int, ctypes.c_int, _P]
        L.lbm_halo_pack.restype = st
        L.lbm_halo_unpack.argtypes = [_P, ctypes.c_int, ctypes.c_int, _P]
        L.lbm_halo_unpack.restype = st
        L.lbm_save.argtypes = [_P, ctypes.c_char_p]
        L.lbm_save.restype = st
        L.lbm_load.argtypes = [_P, ctypes.c_char_p]
        L.lbm_load.restype = st
        L.lbm_parity.argtypes = [_P]
        L.lbm_parity.restype = ctypes.c_int
        L.lbm_time.argtypes = [_P]
        L.lbm_time.restype = ctypes.c_longlong
        L.lbm_last_error.argtypes = [_P]
        L.lbm_last_error.restype = ctypes.c_char_p
        L.lbm_status_string.argtypes = [ctypes.c_int]
        L.lbm_status_string.restype = ctypes.c_char_p
        L.lbm_destroy.argtypes = [_P]
        L.lbm_destroy.restype = None
        _lib = L
    return _lib


def status_name(status: int) -> str:
    return lib().lbm_status_string(int(status)).decode()


def ptr(a):
    """Data pointer of a numpy array or torch tensor (must be contiguous float32/uint8), or None."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if hasattr(a, "ctypes"):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    raise TypeError(f"unsupported array type {type(a)}")
