"""ctypes declarations of the libdcs C ABI (include/dcs.h); argument marshalling only."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("DCS_LIB_PATH", os.path.join(HERE, "libdcs.so"))

CWORDS = 8
MAX_QUBITS = 128
MAX_CHI_FUSED = 32
MAX_CHI = 1024
MAX_CHUNK_LAYERS = 4
PATH_AUTO, PATH_SHARED, PATH_GLOBAL = 0, 1, 2
GEMM_SIMT, GEMM_TENSOR, GEMM_TENSOR_BF16X3 = 0, 1, 2
PREC_FP32, PREC_TF32X3, PREC_BF16X3 = 0, 1, 2

OK, ERR_INVALID, ERR_OOM, ERR_ZERO_PROB, ERR_NUMERICAL, ERR_TIMEOUT, ERR_CUDA, ERR_UNSUPPORTED = range(8)
STATUS_NAMES = ["OK", "INVALID", "OOM", "ZERO_PROB", "NUMERICAL", "TIMEOUT", "CUDA", "UNSUPPORTED"]

COND_NONE, COND_XOR, COND_AND, COND_OR, COND_TABLE = 0, 1, 2, 3, 4
OP_GATE1, OP_GATE2, OP_MEASURE, OP_RESET = 1, 2, 3, 4

FLAG_DRAW_NEAR_THRESHOLD = 1
FLAG_ZERO_PROB = 2
FLAG_NUMERICAL = 4


class dcs_cond(ctypes.Structure):
    _fields_ = [("mask", ctypes.c_uint64 * CWORDS), ("op", ctypes.c_int32),
                ("value", ctypes.c_int32)]


class dcs_op(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("q0", ctypes.c_int32), ("q1", ctypes.c_int32),
                ("cbit", ctypes.c_int32), ("m", ctypes.c_double * 32), ("cond", dcs_cond)]


class dcs_config(ctypes.Structure):
    _fields_ = [("n_qubits", ctypes.c_int32), ("chi_max", ctypes.c_int32),
                ("tol", ctypes.c_double), ("sweeps", ctypes.c_int32),
                ("chunk_k", ctypes.c_int32), ("chunk_layers", ctypes.c_int32),
                ("precision", ctypes.c_int32),
                ("kernel_path", ctypes.c_int32),
                ("n_cbits", ctypes.c_int32), ("n_slots", ctypes.c_int32),
                ("seed", ctypes.c_uint64)]


_c = ctypes
_P = ctypes.c_void_p
SIGNATURES = {
    "dcs_arena_bytes": (_c.c_size_t, [_c.POINTER(dcs_config)]),
    "dcs_create": (_c.c_int, [_c.POINTER(_P), _c.POINTER(dcs_config), _P, _c.c_size_t, _P]),
    "dcs_destroy": (_c.c_int, [_P]),
    "dcs_last_error": (_c.c_char_p, [_P]),
    "dcs_init_state": (_c.c_int, [_P, _c.c_int, _c.c_int, _c.c_uint64]),
    "dcs_fork_shots": (_c.c_int, [_P, _c.c_int]),
    "dcs_apply_layer": (_c.c_int, [_P, _c.POINTER(dcs_op), _c.c_int, _P]),
    "dcs_measure_prob": (_c.c_int, [_P, _c.c_int, _P]),
    "dcs_measure_sample": (_c.c_int, [_P, _c.c_int, _c.c_int, _c.c_uint64]),
    "dcs_collapse": (_c.c_int, [_P, _c.c_int, _c.c_int, _c.POINTER(_c.c_uint8)]),
    "dcs_branch_split": (_c.c_int, [_P, _c.c_int, _c.c_int, _c.c_double]),
    "dcs_branch_topk": (_c.c_int, [_P, _c.c_int]),
    "dcs_branch_keep": (_c.c_int, [_P, _P, _c.c_int]),
    "dcs_topk_select_global": (_c.c_int, [_P, _c.c_int, _c.c_int, _c.c_double, _P]),
    "dcs_set_pruning": (_c.c_int, [_P, _c.c_double]),
    "dcs_get_results": (_c.c_int, [_P, _P, _P, _P, _c.POINTER(_c.c_int), _P]),
    "dcs_get_bonds": (_c.c_int, [_P, _P, _c.POINTER(_c.c_int)]),
    "dcs_export_mps": (_c.c_int, [_P, _c.c_int, _P, _c.POINTER(_c.c_size_t)]),
    "dcs_import_mps": (_c.c_int, [_P, _c.c_int, _P, _c.c_size_t]),
    "dcs_branch_append": (_c.c_int, [_P, _P, _c.c_size_t, _c.c_double, _c.c_double, _P,
                                     _c.c_uint8]),
    "dcs_run_circuit": (_c.c_int, [_P, _c.POINTER(dcs_op), _c.c_int, _c.c_uint64, _c.c_int]),
    "dcs_kernel_launches": (_c.c_uint64, [_P]),
    "dcs_bytes_uploaded": (_c.c_uint64, [_P]),
    "dcs_get_counters": (_c.c_int, [_P, _c.POINTER(_c.c_uint64), _c.POINTER(_c.c_uint64)]),
    "dcs_cgemm": (_c.c_int, [_c.c_int32, _c.c_int32, _c.c_int32, _c.c_int32, _c.c_int32,
                             _P, _c.c_int64, _c.c_int64, _c.c_int64, _c.c_int32,
                             _P, _c.c_int64, _c.c_int64, _c.c_int64, _c.c_int32,
                             _P, _c.c_int64, _c.c_int64, _c.c_int64, _P, _P]),
    "dcs_compress_noalloc": (_c.c_int, [_c.c_int32, _c.c_int32, _c.c_double, _c.c_int32,
                                        _c.POINTER(dcs_op), _c.c_int32, _P, _P, _P, _c.c_int32,
                                        _P, _P, _P, _P, _P]),
}

_lib = None


def load() -> ctypes.CDLL:
    """Load libdcs.so (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libdcs.so is missing at {LIB_PATH}: run paper_2609_26516_b300/build.py")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib
