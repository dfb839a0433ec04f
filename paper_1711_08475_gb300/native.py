"""ctypes binding of libfpmatch.so (declared in include/fp.h).

Argument marshalling only: every step of the matching path runs in the
library's CUDA kernels.  Loading fails loudly when the library is missing;
there is no other code path.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfpmatch.so")

FP_OK, FP_E_INVAL, FP_E_UNSUPPORTED, FP_E_NOMEM, FP_E_CUDA, FP_E_TIMEOUT, FP_E_OVERFLOW = 0, -1, -2, -3, -4, -5, -6
FP_OCC, FP_OCC_HALVED, FP_COUNT, FP_POS, FP_QGRAM, FP_COUNT_L1 = 0, 1, 2, 3, 4, 5
FP_HAM, FP_LEV = 0, 1
FP_SET_COMMON, FP_SET_RARE, FP_SET_MIXED, FP_SET_CUSTOM = 0, 1, 2, 3
FP_MODE_TILED, FP_MODE_PLAIN, FP_MODE_FUSED = 0, 1, 2


class fp_build_opts(ctypes.Structure):
    _fields_ = [("set", ctypes.c_int32), ("count_bits", ctypes.c_int32), ("pos_bits", ctypes.c_int32),
                ("combined", ctypes.c_int32), ("custom_map", ctypes.POINTER(ctypes.c_int8)),
                ("qgram", ctypes.c_int32)]


class fp_query_opts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("tile_queries", ctypes.c_int32),
                ("words_per_thread", ctypes.c_int32), ("variant", ctypes.c_int32), ("flags", ctypes.c_int32)]


FP_OPT_NO_GRAPH = 1


class fp_learn_opts(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_int32), ("batch", ctypes.c_int32), ("lr", ctypes.c_float),
                ("tau0", ctypes.c_float), ("tau1", ctypes.c_float), ("beta", ctypes.c_float),
                ("seed", ctypes.c_uint64),
                ("init_params", ctypes.POINTER(ctypes.c_float))]


class fp_tune_result(ctypes.Structure):
    _fields_ = [("tile_queries", ctypes.c_int32), ("words_per_thread", ctypes.c_int32), ("variant", ctypes.c_int32),
                ("mode", ctypes.c_int32), ("ms", ctypes.c_float)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class fp_batch(ctypes.Structure):
    _fields_ = [("n_queries", ctypes.c_int64), ("k", ctypes.c_int32), ("metric", ctypes.c_int32)]


class fp_stats(ctypes.Structure):
    _fields_ = [("n_queries", ctypes.c_int64), ("pairs", ctypes.c_int64), ("survivors", ctypes.c_int64),
                ("matches", ctypes.c_int64), ("filter_launches", ctypes.c_int64),
                ("ms_prepare", ctypes.c_float), ("ms_filter", ctypes.c_float), ("ms_verify", ctypes.c_float),
                ("ms_emit", ctypes.c_float), ("ms_total", ctypes.c_float), ("pairs_tested", ctypes.c_int64)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class fp_index_info(ctypes.Structure):
    _fields_ = [("n_words", ctypes.c_int64), ("type", ctypes.c_int32), ("width_bits", ctypes.c_int32),
                ("count_bits", ctypes.c_int32), ("pos_bits", ctypes.c_int32), ("n_pos", ctypes.c_int32),
                ("sigma", ctypes.c_int32), ("bucket_count", ctypes.c_int64 * 256),
                ("device_bytes", ctypes.c_int64), ("qgram", ctypes.c_int32), ("combined", ctypes.c_int32)]


class fp_probe_result(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("sm_count", ctypes.c_int32), ("ops", ctypes.c_double),
                ("seconds", ctypes.c_double), ("ops_per_s", ctypes.c_double),
                ("ops_per_clk_per_sm", ctypes.c_double), ("sm_clock_mhz", ctypes.c_double)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class fp_server_opts(ctypes.Structure):
    _fields_ = [("lanes", ctypes.c_int32), ("max_requests", ctypes.c_int32), ("max_queries", ctypes.c_int64),
                ("max_chars", ctypes.c_int64), ("memory_budget", ctypes.c_int64), ("tile_queries", ctypes.c_int32),
                ("variant", ctypes.c_int32)]


class fp_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("queries", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("reruns", ctypes.c_int64), ("pairs", ctypes.c_int64),
                ("survivors", ctypes.c_int64), ("matches", ctypes.c_int64), ("max_lanes_busy", ctypes.c_int32),
                ("max_requests_per_launch", ctypes.c_int32), ("budget_bytes", ctypes.c_int64),
                ("peak_bytes", ctypes.c_int64), ("in_use_bytes", ctypes.c_int64), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double), ("max_ms", ctypes.c_double),
                ("mean_queue_ms", ctypes.c_double), ("busy_seconds", ctypes.c_double)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


_VP = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int

# name -> (restype, argtypes); every symbol of include/fp.h
SIGNATURES = {
    "fp_build": (ctypes.c_int, [_VP, _VP, _I64, _I32, _I32, ctypes.POINTER(fp_build_opts), _VP, ctypes.POINTER(_VP)]),
    "fp_query": (ctypes.c_int, [_VP, _VP, _VP, _I64, _I32, _I32, _VP, ctypes.POINTER(_VP)]),
    "fp_query_ex": (ctypes.c_int, [_VP, _VP, _VP, _I64, _I32, _I32, ctypes.POINTER(fp_query_opts), _VP,
                                   ctypes.POINTER(_VP)]),
    "fp_query_noalloc": (ctypes.c_int, [_VP, _VP, _VP, _I64, _I32, _I32, _VP, _VP, _I64, ctypes.POINTER(_I64),
                                        _VP]),
    "fp_query_batched": (ctypes.c_int, [_VP, _VP, _VP, _I64, _VP, _I32, ctypes.POINTER(fp_query_opts), _VP,
                                        ctypes.POINTER(_VP)]),
    "fp_plan_create": (ctypes.c_int, [_VP, _I64, _I64, _I32, ctypes.POINTER(fp_query_opts), ctypes.POINTER(_VP)]),
    "fp_plan_run": (ctypes.c_int, [_VP, _VP, _VP, _I64, _VP, _I32, _VP, ctypes.POINTER(_VP)]),
    "fp_plan_free": (None, [_VP]),
    "fp_server_create": (ctypes.c_int, [_VP, ctypes.POINTER(fp_server_opts), ctypes.POINTER(_VP)]),
    "fp_server_submit": (ctypes.c_int, [_VP, _VP, _VP, _I64, _I32, _I32, ctypes.POINTER(_I64)]),
    "fp_server_wait": (ctypes.c_int, [_VP, _I64, _I64, ctypes.POINTER(_VP)]),
    "fp_server_stats_get": (ctypes.c_int, [_VP, ctypes.POINTER(fp_server_stats)]),
    "fp_server_replay": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _I64, _I32, _I32, _I64, _VP, ctypes.POINTER(_VP)]),
    "fp_server_free": (None, [_VP]),
    "fp_mlp_param_count": (ctypes.c_int, []),
    "fp_sample_pairs": (ctypes.c_int, [_VP, _VP, _VP, _I64, _I32, _I32, _I64, ctypes.c_uint64, _VP, _VP, _VP, _VP,
                                       _VP, _VP]),
    "fp_mlp_loss_grad": (ctypes.c_int, [_VP, _I32, ctypes.c_float, ctypes.c_float, _I32, _VP, _VP, _I64, _VP,
                                        ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_I64), _VP]),
    "fp_learn_map": (ctypes.c_int, [_I32, _VP, _VP, _I64, _I32, ctypes.POINTER(fp_learn_opts), _VP, _VP, _VP, _VP]),
    "fp_autotune": (ctypes.c_int, [_VP, _VP, _VP, _I64, _I32, _I32, _I32, _I32, _VP, _VP, _VP, _I32,
                                   ctypes.POINTER(ctypes.c_int32)]),
    "fp_result_csr": (ctypes.c_int, [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP), _I32]),
    "fp_result_stats": (ctypes.c_int, [_VP, ctypes.POINTER(fp_stats)]),
    "fp_result_free": (None, [_VP]),
    "fp_index_info_get": (ctypes.c_int, [_VP, ctypes.POINTER(fp_index_info)]),
    "fp_index_map": (ctypes.c_int, [_VP, _VP]),
    "fp_index_qgrams": (ctypes.c_int, [_VP, _VP, ctypes.POINTER(_I32), ctypes.POINTER(_I32)]),
    "fp_set_symbol_map": (ctypes.c_int, [_VP, _VP]),
    "fp_fingerprint": (ctypes.c_int, [_VP, _VP, _VP, _I64, _VP, _VP]),
    "fp_free": (None, [_VP]),
    "fp_strerror": (ctypes.c_char_p, [_I32]),
    "fp_last_error": (ctypes.c_char_p, []),
    "fp_launch_count": (ctypes.c_int64, []),
    "fp_version": (ctypes.c_char_p, []),
    "fp_probe": (ctypes.c_int, [_I32, _I32, _VP, ctypes.POINTER(fp_probe_result)]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Loads the library (raises if it is not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libfpmatch.so is not built ({path}); run paper_1711_08475_gb300.build.build()")
    L = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


class FpError(RuntimeError):
    def __init__(self, code: int, where: str):
        L = load()
        msg = L.fp_last_error().decode(errors="replace")
        super().__init__(f"{where}: {L.fp_strerror(code).decode()} ({code}): {msg}")
        self.code = code


def check(code: int, where: str):
    if code != FP_OK:
        raise FpError(code, where)
