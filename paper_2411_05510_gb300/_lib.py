"""ctypes binding of libssi (the C ABI declared in include/ssi.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Importing this module fails loudly when libssi.so is missing.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libssi.so")

SSI_OK, SSI_E_INVALID, SSI_E_NOMEM, SSI_E_CUDA, SSI_E_TIMEOUT, SSI_E_NOTCONVERGED, SSI_E_BUSY, \
    SSI_E_NOTFOUND = range(8)
STATUS_NAMES = ["SSI_OK", "SSI_E_INVALID", "SSI_E_NOMEM", "SSI_E_CUDA", "SSI_E_TIMEOUT",
                "SSI_E_NOTCONVERGED", "SSI_E_BUSY", "SSI_E_NOTFOUND"]
SSI_PREC_FP32, SSI_PREC_SPLIT_BF16 = 0, 1
SSI_SMALL_FP32, SSI_SMALL_FP64 = 0, 1

POLE_HC_XI, POLE_HC_MPC, POLE_HC_MPD, POLE_HC, POLE_ORDER, POLE_LAG, POLE_VALID, POLE_NOTCONV = \
    1, 2, 4, 8, 16, 32, 64, 128


class SsiPole(ctypes.Structure):
    _fields_ = [("f_hz", ctypes.c_float), ("xi", ctypes.c_float), ("mu_re", ctypes.c_float),
                ("mu_im", ctypes.c_float), ("mpc", ctypes.c_float), ("mpd", ctypes.c_float),
                ("lag", ctypes.c_int32), ("order", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("index", ctypes.c_int32)]


POLE_FIELDS = [f for f, _ in SsiPole._fields_]
POLE_BYTES = ctypes.sizeof(SsiPole)


class SsiStabParams(ctypes.Structure):
    _fields_ = [("xi_max", ctypes.c_double), ("mpc_min", ctypes.c_double),
                ("mpd_max", ctypes.c_double), ("a_f", ctypes.c_double), ("a_xi", ctypes.c_double),
                ("a_mac", ctypes.c_double), ("use_lag_axis", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class SsiClusterParams(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double), ("min_size", ctypes.c_int32),
                ("fcm_max_iter", ctypes.c_int32), ("fcm_m", ctypes.c_double),
                ("fcm_tol", ctypes.c_double)]


class SsiMode(ctypes.Structure):
    _fields_ = [("f_hz", ctypes.c_double), ("xi", ctypes.c_double), ("size", ctypes.c_int32),
                ("medoid_slot", ctypes.c_int32)]


class SsiClusterInfo(ctypes.Structure):
    _fields_ = [("n_candidates", ctypes.c_int32), ("n_kept", ctypes.c_int32),
                ("n_components", ctypes.c_int32), ("n_modes", ctypes.c_int32),
                ("fcm_iterations", ctypes.c_int32), ("fcm_converged", ctypes.c_int32),
                ("physical", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("centroids", (ctypes.c_double * 5) * 2)]


class SsiJobDesc(ctypes.Structure):
    _fields_ = [("Y", ctypes.c_void_p), ("y_on_host", ctypes.c_int32), ("l", ctypes.c_int32),
                ("N", ctypes.c_int64), ("fs", ctypes.c_double), ("n_lags", ctypes.c_int32),
                ("lags", ctypes.POINTER(ctypes.c_int32)), ("n_orders", ctypes.c_int32),
                ("orders", ctypes.POINTER(ctypes.c_int32)), ("k", ctypes.c_int32),
                ("oversample", ctypes.c_int32), ("q", ctypes.c_int32), ("prec", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("stab", SsiStabParams), ("small", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class SsiTuning(ctypes.Structure):
    _fields_ = [("cov_rows_per_split", ctypes.c_int32), ("sketch_splits", ctypes.c_int32),
                ("jacobi_block", ctypes.c_int32), ("qr_chunks_per_cta", ctypes.c_int32),
                ("stage_ms", ctypes.c_double * 4)]


_c = ctypes
_P = ctypes.c_void_p
# name -> (restype, argtypes): the full exported surface of include/ssi.h
PROTOTYPES = {
    "ssi_create": (_c.c_int, [_c.POINTER(_P), _c.c_int, _c.c_size_t]),
    "ssi_destroy": (None, [_P]),
    "ssi_last_error": (_c.c_char_p, []),
    "ssi_version": (_c.c_int, []),
    "ssi_memory_in_use": (_c.c_size_t, [_P]),
    "ssi_set_concurrency": (_c.c_int, [_P, _c.c_int]),
    "ssi_profile": (_c.c_int, [_P, _c.c_int]),
    "ssi_profile_read": (_c.c_int, [_P, _c.POINTER(_c.c_double), _c.POINTER(_c.c_int64), _c.c_int,
                                    _c.POINTER(_c.c_int64)]),
    "ssi_covariances": (_c.c_int, [_P, _P, _c.c_int, _c.c_int64, _c.c_int, _c.c_int, _P, _P]),
    "ssi_cov_stream_create": (_c.c_int, [_P, _c.c_int, _c.c_int, _c.c_int64, _c.c_int64, _c.c_int,
                                         _c.POINTER(_P)]),
    "ssi_cov_stream_push": (_c.c_int, [_P, _P, _c.c_int64, _P]),
    "ssi_cov_stream_covariances": (_c.c_int, [_P, _P, _c.POINTER(_c.c_int64), _P]),
    "ssi_cov_stream_refresh": (_c.c_int, [_P, _P]),
    "ssi_cov_stream_destroy": (_c.c_int, [_P]),
    "ssi_covariances_noalloc": (_c.c_int, [_P, _c.c_int, _c.c_int64, _c.c_int, _P, _P]),
    "ssi_gaussian_omega": (_c.c_int, [_P, _c.c_int, _c.c_int, _c.c_uint64, _P, _P]),
    "ssi_toeplitz_rsvd": (_c.c_int, [_P, _P, _c.c_int, _c.c_int, _c.c_int, _c.c_int, _c.c_int,
                                     _c.c_uint64, _c.c_int, _c.c_int, _P, _P, _P]),
    "ssi_pole_slots": (_c.c_int64, [_c.c_int, _c.POINTER(_c.c_int)]),
    "ssi_realize_batch": (_c.c_int, [_P, _c.c_int, _c.POINTER(_c.c_int), _c.POINTER(_P), _c.c_int,
                                     _c.c_int, _c.POINTER(_c.c_int), _c.c_int, _c.c_double, _c.c_int,
                                     _P, _P, _P]),
    "ssi_stabilize": (_c.c_int, [_P, _c.c_int, _c.c_int, _c.POINTER(_c.c_int), _c.c_int, _P, _P,
                                 _c.POINTER(SsiStabParams), _P]),
    "ssi_cluster": (_c.c_int, [_P, _c.c_int, _c.c_int, _c.POINTER(_c.c_int), _c.c_int, _P, _P,
                               _c.POINTER(SsiClusterParams), _c.POINTER(SsiMode), _c.c_int,
                               _c.POINTER(_c.c_int), _P, _P, _P, _c.POINTER(SsiClusterInfo), _P]),
    "ssi_job_sizes": (_c.c_int, [_c.POINTER(SsiJobDesc), _c.POINTER(_c.c_int64),
                                 _c.POINTER(_c.c_int64)]),
    "ssi_solve": (_c.c_int, [_P, _c.POINTER(SsiJobDesc), _P, _P, _P, _P]),
    "ssi_solve_batch": (_c.c_int, [_P, _c.c_int, _c.POINTER(SsiJobDesc), _c.POINTER(_P),
                                   _c.POINTER(_P), _c.POINTER(_P), _P]),
    "ssi_sync_status": (_c.c_int, [_P, _P]),
    "ssi_autotune": (_c.c_int, [_P, _c.POINTER(SsiJobDesc), _c.POINTER(SsiTuning)]),
    "ssi_tuning_get": (_c.c_int, [_P, _c.POINTER(SsiJobDesc), _c.POINTER(SsiTuning)]),
    "ssi_tuning_set": (_c.c_int, [_P, _c.POINTER(SsiJobDesc), _c.POINTER(SsiTuning)]),
    "ssi_serve_config": (_c.c_int, [_P, _c.c_int, _c.c_int]),
    "ssi_submit": (_c.c_int, [_P, _c.POINTER(SsiJobDesc), _c.POINTER(_c.c_uint64)]),
    "ssi_poll": (_c.c_int, [_P, _c.c_uint64, _c.c_int, _c.POINTER(_P), _c.POINTER(_P),
                            _c.POINTER(_c.c_int64), _c.POINTER(_c.c_double)]),
    "ssi_release": (_c.c_int, [_P, _c.c_uint64]),
    "ssi_rank_rule": (_c.c_int, [_c.c_int64, _c.POINTER(_c.c_double), _c.POINTER(_c.c_int64)]),
    "ssi_lag_rule": (_c.c_int, [_c.c_double, _c.c_double, _c.c_double, _c.POINTER(_c.c_int),
                                _c.POINTER(_c.c_int), _c.POINTER(_c.c_int)]),
    "ssi_time_lag": (_c.c_double, [_c.c_int, _c.c_double]),
}


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"libssi.so not found at {path}: build it with __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in PROTOTYPES.items():
        fn = getattr(lib, name, None)
        if fn is None:
            MISSING.append(name)
            continue
        fn.restype = res
        fn.argtypes = args
    return lib


MISSING: list = []
lib = load()


class SsiError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = lib.ssi_last_error().decode(errors="replace")
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{where}: {name}: {msg}")
        self.status = status


def check(status: int, where: str) -> None:
    if status != SSI_OK:
        raise SsiError(status, where)
