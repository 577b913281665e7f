"""ctypes loader of libspiir.so: argument types of every C entry point and status codes.

There is no fallback: if the shared library is missing this module raises, and every
compute call goes through the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# SPIIR_LIB_PATH selects another build of the library (for example a bounds-checked debug build)
LIB_PATH = os.environ.get("SPIIR_LIB_PATH") or os.path.join(HERE, "_lib", "libspiir.so")

OK, EINVAL, ECUDA, ENOMEM, EUNSUPPORTED, ETIMEOUT = 0, -1, -2, -3, -4, -5
_NAMES = {EINVAL: "EINVAL", ECUDA: "ECUDA", ENOMEM: "ENOMEM", EUNSUPPORTED: "EUNSUPPORTED", ETIMEOUT: "ETIMEOUT"}


class SpiirError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"{_NAMES.get(code, code)}: {message}")
        self.code = code


_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64
_SZ = ctypes.c_size_t
_D = ctypes.c_double

# name: (restype, argtypes) -- mirrors include/spiir.h
SIGNATURES = {
    "spiir_version": (_I, []),
    "spiir_last_error": (_I, [ctypes.c_char_p, _SZ]),
    "spiir_debug_fail_allocs": (None, [_I]),
    "spiir_debug_fail_alloc_at": (None, [_I]),
    "spiir_device_status": (_I, [_I]),
    "spiir_debug_wait_timeout": (_I, [ctypes.c_uint32, _P]),
    "spiir_bank_create": (_I, [_I, _I, _P, _P, _P, _P, ctypes.POINTER(_P)]),
    "spiir_bank_destroy": (None, [_P]),
    "spiir_bank_info": (_I, [_P, _P, _P, _P, _P]),
    "spiir_bank_reset": (_I, [_P, _P]),
    "spiir_bank_state_bytes": (_I, [_P, ctypes.POINTER(_SZ)]),
    "spiir_bank_get_state": (_I, [_P, _P, _SZ]),
    "spiir_bank_set_state": (_I, [_P, _P, _SZ]),
    "spiir_filter_chunk": (_I, [_P, _P, _I64, _I64, _P, _I64, _P]),
    "spiir_filter_static": (_I, [_I, _I, _P, _P, _P, _P, _P, _I64, _I64, _P, _I64, _P]),
    "spiir_bank_set_shape": (_I, [_P, _I, _I, _I, _I]),
    "spiir_bank_get_shape": (_I, [_P, _P, _P, _P, _P]),
    "spiir_bank_set_delay_bin": (_I, [_P, ctypes.c_int32]),
    "spiir_bank_get_delay_bin": (_I, [_P, _P, _P, _P]),
    "spiir_sky_set_scan_shape": (_I, [_P, _I, _I, _I]),
    "spiir_sky_get_scan_shape": (_I, [_P, _P, _P, _P, _P]),
    "spiir_sky_tables": (_I, [_I, _P, _P, _P, _P, _I, _D, _P, _P, _P]),
    "spiir_sky_create": (_I, [_I, _I, _P, _P, _P, ctypes.POINTER(_P)]),
    "spiir_sky_destroy": (None, [_P]),
    "spiir_sky_info": (_I, [_P, _P, _P, _P]),
    "spiir_coherent_scan": (_I, [_P, _P, _I64, _I, _I64, _P, _P, _P, _P, _P]),
    "spiir_autocorr": (_I, [_I, _P, _I64, _I, _P, _P]),
    "spiir_xi2": (_I, [_I, _I, _P, _I64, _P, _I, _I64, _P, _I64, _P]),
    "spiir_xi2_network": (_I, [_P, _I, _P, _I64, _P, _I64, _P, _P]),
    "spiir_fir_lowpass": (_I, [_I, _I, _D, _P]),
    "spiir_whitening_kernel": (_I, [_I, _P, _D, _I, _P]),
    "spiir_frontend_create": (_I, [_I, _I, _I, _P, _I, _P, _I64, ctypes.POINTER(_P)]),
    "spiir_frontend_destroy": (None, [_P]),
    "spiir_frontend_reset": (_I, [_P, _P]),
    "spiir_frontend_info": (_I, [_P, _P, _P, _P]),
    "spiir_pipeline_run_frontend": (_I, [_P, _P, _P, _I64, _I64, _P, _P, _P, _P, _P]),
    "spiir_frontend_run": (_I, [_P, _P, _I64, _I64, _P, _I64, _P]),
    "spiir_xi2_candidates": (_I, [_P, _I, _P, _I64, _I64, _P, _I, _P, _P, _I, _I, _I, _I, _P, _P, _P, _P]),
    "spiir_select_workspace_bytes": (_I, [_I, _I, _I64, _I, ctypes.POINTER(_SZ)]),
    "spiir_select_candidates": (_I, [_I, _I, _P, _I64, _I64, _I64, ctypes.c_float, _I, _P, _SZ, _P, _I, _P, _P]),
    "spiir_coherent_candidates": (_I, [_P, _I, _P, _I64, _I64, _P, _P, _I, _I, _I, _I, _P, _P, _P, _P]),
    "spiir_impulse_forward": (_I, [_I, _I, _P, _P, _P, _P, _I64, _P, _I, _P, _P]),
    "spiir_impulse_backward": (_I, [_I, _I, _P, _P, _P, _I64, _P, _I, _P, _P, _P, _P, _P, _P]),
    "spiir_batch_create": (_I, [_I, _I, _P, _P, _P, _P, _P, _P, _I, _P, _P, _I64, ctypes.POINTER(_P)]),
    "spiir_batch_destroy": (None, [_P]),
    "spiir_batch_info": (_I, [_P, _P, _P, _P]),
    "spiir_batch_reset": (_I, [_P, _P]),
    "spiir_batch_set_shape": (_I, [_P, _I, _I, _I, _I]),
    "spiir_batch_run": (_I, [_P, _I, _P, _P, _P, _P, _P]),
    "spiir_batch_filter_time": (_I, [_P, ctypes.POINTER(ctypes.c_float)]),
    "spiir_search_create": (_I, [_P, _P, _P, _P, _I, _I64, ctypes.c_float, _I, _I, _I, _I, _I, ctypes.POINTER(_P)]),
    "spiir_search_destroy": (None, [_P]),
    "spiir_search_info": (_I, [_P, _P, _P, _P, _P]),
    "spiir_search_reset": (_I, [_P, _P]),
    "spiir_search_run": (_I, [_P, _P, _I64, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "spiir_pipeline_create": (_I, [_P, _P, _I64, ctypes.POINTER(_P)]),
    "spiir_pipeline_destroy": (None, [_P]),
    "spiir_pipeline_reset": (_I, [_P, _P]),
    "spiir_pipeline_run": (_I, [_P, _P, _I64, _I64, _P, _P, _P, _P, _P]),
    "spiir_pipeline_run_host": (_I, [_P, _P, _I64, _P, _P, _P, _P]),
    "spiir_pipeline_submit_host": (_I, [_P, _P, _I64, _P, _P, _P, _P]),
    "spiir_pipeline_wait": (_I, [_P]),
    "spiir_pipeline_wait_for": (_I, [_P, _D]),
}

_lib = None


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libspiir.so not found at {LIB_PATH}; run __graft_entry__.build() "
                              "or python paper_2011_06787_b300/build.py")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def last_error() -> str:
    buf = ctypes.create_string_buffer(2048)
    lib().spiir_last_error(buf, len(buf))
    return buf.value.decode(errors="replace")


def check(code: int) -> None:
    if code != OK:
        raise SpiirError(code, last_error())
