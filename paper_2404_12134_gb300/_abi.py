"""ctypes declarations of the C ABI in include/wetsand.h.

Loads the in-tree ``libwetsand.so``.  There is no fallback: if the library has
not been built, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libwetsand.so")

WTS_OK, WTS_EINVAL, WTS_ENOMEM, WTS_ECUDA, WTS_ETIMEOUT = 0, 1, 2, 3, 4
OP_ANOMALY_SCORE, OP_DTW_ALIGN, OP_DBA_ITERATE, OP_SOFTDTW, OP_PAIRWISE, OP_COMPACT_NAN = 1, 2, 3, 4, 5, 6
OP_SUBDTW = 7
OP_SOFTDTW_LBFGS = 8
OP_SOFTDTW_ADAM = 9
COST_SQEUCLID, COST_L2 = 0, 1

# every symbol declared in include/wetsand.h
EXPORTS = (
    "wts_version", "wts_last_error", "wts_workspace_size", "wts_read_status",
    "wts_profile_enable", "wts_profile_read", "wts_peak_probe",
    "anomaly_score", "dtw_align", "dba_iterate", "wts_pairwise_dtw", "wts_medoid",
    "wts_resample", "wts_euclid_mean", "anomaly_score_noalloc",
    "softdtw_forward", "softdtw_backward", "wts_adam_step", "wts_autotune", "wts_compact_nan",
    "subdtw_align", "wts_segment_workspace_size", "wts_segment", "wts_thresholds", "wts_f2",
    "wts_lbfgs_minimize", "wts_softdtw_barycenter_lbfgs", "wts_pad_last", "wts_select_channel",
    "wts_softdtw_barycenter_adam", "wts_noalloc_read_status",
)


class wts_batch(ctypes.Structure):
    _fields_ = [
        ("data", ctypes.c_void_p),
        ("offsets", ctypes.c_void_p),
        ("offsets_host", ctypes.c_void_p),
        ("T", ctypes.c_int32),
        ("d", ctypes.c_int32),
    ]


class wts_options(ctypes.Structure):
    _fields_ = [
        ("rows_per_thread", ctypes.c_int32),
        ("warps_per_block", ctypes.c_int32),
        ("max_blocks", ctypes.c_int32),
        ("keep_batch_order", ctypes.c_int32),
        ("dir_mode", ctypes.c_int32),
        ("ckpt_bands", ctypes.c_int32),
        ("spin_limit", ctypes.c_int32),
        ("fault_skip_handoff", ctypes.c_int32),
        ("band", ctypes.c_double),
        ("cost_kind", ctypes.c_int32),
        ("score_via_codes", ctypes.c_int32),
        ("store_pairs", ctypes.c_int32),
        ("reserved", ctypes.c_int32 * 3),
    ]


class wts_lbfgs_params(ctypes.Structure):
    _fields_ = [
        ("history", ctypes.c_int32),
        ("max_iter", ctypes.c_int32),
        ("max_fun", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("gtol", ctypes.c_double),
        ("ftol", ctypes.c_double),
        ("c1", ctypes.c_double),
    ]


OBJECTIVE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(ctypes.c_double), ctypes.c_void_p)


class WtsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"wetsand error {code}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None

VP, I32, I64, SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
PB = ctypes.POINTER(wts_batch)
PO = ctypes.POINTER(wts_options)

_SIGS = {
    "wts_version": ([], ctypes.c_int),
    "wts_last_error": ([], ctypes.c_char_p),
    "wts_workspace_size": ([ctypes.c_int, I64, PB, PO, ctypes.POINTER(SZ)], ctypes.c_int),
    "wts_read_status": ([VP, VP, ctypes.POINTER(I32)], ctypes.c_int),
    "wts_profile_enable": ([ctypes.c_int], ctypes.c_int),
    "wts_peak_probe": ([ctypes.c_int, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "wts_profile_read": ([ctypes.c_char_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(I32)], ctypes.c_int),
    "anomaly_score": ([VP, I64, PB, PO, VP, SZ, VP, VP, VP, VP], ctypes.c_int),
    "dtw_align": ([VP, I64, PB, PO, VP, SZ, VP, VP, VP, VP, VP], ctypes.c_int),
    "dba_iterate": ([VP, VP, I64, PB, PO, VP, SZ, VP, VP, VP, VP], ctypes.c_int),
    "subdtw_align": ([VP, I64, PB, PO, VP, SZ, VP, VP, VP, VP, VP, VP, VP], ctypes.c_int),
    "wts_segment_workspace_size": ([I64, I32, PO, ctypes.POINTER(SZ)], ctypes.c_int),
    "wts_segment": ([VP, I64, VP, I64, I32, I64, PO, VP, SZ, VP, I32, VP, VP, VP, ctypes.POINTER(I32)],
                    ctypes.c_int),
    "wts_pairwise_dtw": ([PB, PO, VP, SZ, VP, VP], ctypes.c_int),
    "wts_lbfgs_minimize": ([I64, VP, OBJECTIVE_FN, VP, ctypes.POINTER(wts_lbfgs_params),
                            ctypes.POINTER(ctypes.c_double), ctypes.POINTER(I32), ctypes.POINTER(I32),
                            ctypes.POINTER(I32)], ctypes.c_int),
    "wts_softdtw_barycenter_lbfgs": ([VP, I64, PB, ctypes.c_float, VP, ctypes.POINTER(wts_lbfgs_params), PO, VP, SZ,
                                      VP, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(I32),
                                      ctypes.POINTER(I32), ctypes.POINTER(I32)], ctypes.c_int),
    "wts_thresholds": ([VP, I32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "wts_f2": ([VP, VP, I32, ctypes.c_double, ctypes.POINTER(I32), ctypes.POINTER(I32), ctypes.POINTER(I32),
                ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "wts_medoid": ([VP, I32, VP, VP, VP], ctypes.c_int),
    "wts_resample": ([VP, I64, I32, VP, I64, VP], ctypes.c_int),
    "wts_euclid_mean": ([PB, I64, VP, VP], ctypes.c_int),
    "anomaly_score_noalloc": ([VP, I64, PB, PO, VP, VP, VP, VP], ctypes.c_int),
    "wts_noalloc_read_status": ([VP, ctypes.POINTER(I32)], ctypes.c_int),
    "wts_softdtw_barycenter_adam": ([VP, I64, PB, ctypes.c_float, VP, I32, ctypes.c_float, ctypes.c_float,
                                     ctypes.c_float, ctypes.c_float, PO, VP, SZ, VP, VP], ctypes.c_int),
    "wts_compact_nan": ([PB, VP, SZ, VP, VP, VP], ctypes.c_int),
    "wts_pad_last": ([PB, I64, VP, VP], ctypes.c_int),
    "wts_select_channel": ([PB, I32, VP, VP], ctypes.c_int),
    "wts_autotune": ([ctypes.c_int, VP, I64, PB, VP, SZ, VP, PO, ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
    "softdtw_forward": ([VP, I64, PB, ctypes.c_float, PO, VP, SZ, VP, VP], ctypes.c_int),
    "softdtw_backward": ([VP, I64, PB, ctypes.c_float, VP, PO, VP, SZ, VP, VP], ctypes.c_int),
    "wts_adam_step": ([VP, VP, VP, VP, I64, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                       I32, VP], ctypes.c_int),
}


def load(path: str = LIB_PATH):
    """Load the library and declare every exported function (no CUDA call)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                               f"(there is no CPU fallback)")
        lib = ctypes.CDLL(path)
        for name, (args, res) in _SIGS.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def check(rc: int):
    if rc != WTS_OK:
        raise WtsError(rc, load().wts_last_error().decode())
