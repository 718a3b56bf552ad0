"""ctypes binding of libhdfilter (include/hdfilter.h).  Argument marshalling
only: every step of the filter runs in the CUDA library.  Importing this
module loads the library and raises if it has not been built."""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libhdfilter.so")

HDF_OK, HDF_EINVAL, HDF_ENOMEM, HDF_ECUDA, HDF_ETIMEOUT, HDF_EDOMAIN, HDF_EUNSUPPORTED = range(7)
HDF_GUIDE_F32, HDF_GUIDE_BF16 = 0, 1
HDF_COEF_OPT, HDF_COEF_INDICATOR = 0, 1
HDF_SPATIAL_GAUSS, HDF_SPATIAL_BOX, HDF_SPATIAL_YOUNG = 0, 1, 2
HDF_MAX_K, HDF_MAX_RHO, HDF_MAX_S, HDF_MAX_N = 64, 64, 32, 256


class hdf_desc(C.Structure):
    _fields_ = [("H", C.c_int), ("W", C.c_int), ("n", C.c_int), ("rho", C.c_int),
                ("K", C.c_int), ("S", C.c_int), ("sigma_s", C.c_double),
                ("sigma_r", C.c_double), ("guide_dtype", C.c_int), ("coef", C.c_int),
                ("spatial", C.c_int)]


class hdf_stats(C.Structure):
    _fields_ = [("K_eff", C.c_int), ("fallback_pixels", C.c_int), ("device_error", C.c_int),
                ("lloyd_iters_max", C.c_int), ("rounds", C.c_int),
                ("cluster_error", C.c_double), ("rescued_pixels", C.c_int),
                ("nlm_sweeps", C.c_int)]


HDF_BATCH_GRAPH, HDF_BATCH_TIMED, HDF_BATCH_SKIP_CLUSTER = 1, 2, 4


class hdf_tile_trial(C.Structure):
    _fields_ = [("SB", C.c_int), ("planes", C.c_int), ("P", C.c_int), ("TY", C.c_int),
                ("ms", C.c_float), ("chosen", C.c_int)]


class hdf_batch_info(C.Structure):
    _fields_ = [("count", C.c_int), ("graph_state", C.c_int), ("launches_per_run", C.c_int),
                ("nitems", C.c_int), ("ngroups", C.c_int), ("grid_cluster", C.c_int),
                ("grid_tile", C.c_int), ("smem_tile", C.c_size_t), ("device_bytes", C.c_size_t)]


# (name, restype, argtypes) of every exported entry point, in header order.
_P = C.c_void_p
SIGNATURES = [
    ("hdf_create", C.c_int, [C.POINTER(_P), C.POINTER(hdf_desc)]),
    ("hdf_destroy", None, [_P]),
    ("hdf_set_wait_limit", C.c_int, [_P, C.c_double]),
    ("hdf_set_sigmas", C.c_int, [_P, C.c_double, C.c_double, _P]),
    ("hdf_set_stage_timing", C.c_int, [_P, C.c_int]),
    ("hdf_get_stage_times", C.c_int, [_P, _P, C.c_int, C.POINTER(C.c_int)]),
    ("hdf_get_desc", C.c_int, [_P, C.POINTER(hdf_desc)]),
    ("hdf_cluster", C.c_int, [_P, _P, _P]),
    ("hdf_set_centers", C.c_int, [_P, _P, C.c_int, _P]),
    ("hdf_get_centers", C.c_int, [_P, _P, C.POINTER(C.c_int), _P]),
    ("hdf_get_pinv", C.c_int, [_P, _P, _P]),
    ("hdf_get_labels", C.c_int, [_P, _P, _P]),
    ("hdf_apply", C.c_int, [_P, _P, _P, _P, _P]),
    ("hdf_backward", C.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    ("hdf_backward_after_apply", C.c_int, [_P, _P, _P, _P, _P, _P, _P, _P]),
    ("hdf_nlm_guide", C.c_int, [_P, _P, C.c_int, _P, _P]),
    ("hdf_apply_static", C.c_int, [C.POINTER(hdf_desc), _P, C.c_int, _P, _P, _P, _P]),
    ("hdf_scale_guide", C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_int, _P, _P, _P]),
    ("hdf_bruteforce", C.c_int, [C.POINTER(hdf_desc), _P, _P, _P, _P]),
    ("hdf_get_trace", C.c_int, [_P, _P, C.c_int, C.POINTER(C.c_int), _P]),
    ("hdf_get_stats", C.c_int, [_P, C.POINTER(hdf_stats), _P]),
    ("hdf_batch_create", C.c_int, [C.POINTER(_P), C.c_int, C.POINTER(hdf_desc)]),
    ("hdf_batch_destroy", None, [_P]),
    ("hdf_batch_bind", C.c_int, [_P, C.POINTER(_P), C.POINTER(_P), C.POINTER(_P)]),
    ("hdf_batch_set_centers", C.c_int, [_P, C.c_int, _P, C.c_int]),
    ("hdf_batch_run", C.c_int, [_P, C.c_int, _P]),
    ("hdf_batch_tune", C.c_int, [_P, C.c_int, _P]),
    ("hdf_batch_get_tuning", C.c_int, [_P, C.POINTER(hdf_tile_trial), C.c_int, C.POINTER(C.c_int)]),
    ("hdf_batch_set_shape", C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_int]),
    ("hdf_batch_get_times", C.c_int, [_P, C.POINTER(C.c_float), C.c_int, C.POINTER(C.c_int)]),
    ("hdf_batch_get_centers", C.c_int, [_P, C.c_int, _P, C.POINTER(C.c_int)]),
    ("hdf_batch_get_stats", C.c_int, [_P, C.c_int, C.POINTER(hdf_stats)]),
    ("hdf_batch_get_info", C.c_int, [_P, C.POINTER(hdf_batch_info)]),
    ("hdf_probe_peaks", C.c_int, [_P, _P, _P]),
    ("hdf_status_string", C.c_char_p, [C.c_int]),
    ("hdf_last_cuda_error", C.c_char_p, []),
]


class HDFError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = _lib.hdf_status_string(code).decode()
        if code == HDF_ECUDA:
            msg += " (" + _lib.hdf_last_cuda_error().decode() + ")"
        super().__init__(f"{where}: {msg}")


def _load() -> C.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"libhdfilter.so not built ({LIB_PATH}); run "
            "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(LIB_PATH)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()


def check(code: int, where: str) -> None:
    if code != HDF_OK:
        raise HDFError(code, where)


def lib() -> C.CDLL:
    return _lib
