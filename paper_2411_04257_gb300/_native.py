"""ctypes view of liblshbloom.so (include/lshbloom.h).  Marshalling only."""
from __future__ import annotations

import ctypes as C
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblshbloom.so")

LSHB_OK = 0
STATUS_NAMES = {0: "OK", -1: "ERR_ARG", -2: "ERR_CSR", -3: "ERR_OOM", -4: "ERR_CUDA",
                -5: "ERR_TIMEOUT", -6: "ERR_IO", -7: "ERR_BUSY"}
INSERT_NONDUP, INSERT_ALL = 0, 1
EXEC_PLAIN, EXEC_BATCHED = 0, 1


class Config(C.Structure):
    _fields_ = [
        ("num_perm", C.c_uint32), ("bands", C.c_uint32), ("rows", C.c_uint32),
        ("ngram", C.c_uint32), ("n_expected", C.c_uint64), ("fp_rate", C.c_double),
        ("fp_is_effective", C.c_int32), ("insert_mode", C.c_uint32), ("seed", C.c_uint64),
        ("perm_a", C.POINTER(C.c_uint64)), ("perm_b", C.POINTER(C.c_uint64)),
        ("exec_mode", C.c_uint32), ("device", C.c_int32), ("max_batch_docs", C.c_uint64),
        ("max_batch_tokens", C.c_uint64), ("item_shingles", C.c_uint32),
        ("bloom_layout", C.c_uint32), ("stage_host_inputs", C.c_uint32),
        ("band_key", C.c_uint32), ("reserved", C.c_uint32 * 4),
    ]


class Stats(C.Structure):
    _fields_ = [
        ("num_perm", C.c_uint32), ("bands", C.c_uint32), ("rows", C.c_uint32),
        ("ngram", C.c_uint32), ("k", C.c_uint32), ("insert_mode", C.c_uint32),
        ("exec_mode", C.c_uint32), ("item_shingles", C.c_uint32), ("m_bits", C.c_uint64),
        ("filter_bytes", C.c_uint64), ("docs_seen", C.c_uint64), ("dups_seen", C.c_uint64),
        ("fp_rate", C.c_double), ("fill", C.c_double * 64), ("resolve_rounds", C.c_uint64),
        ("uncertain_docs", C.c_uint64), ("kernel_launches", C.c_uint64),
        ("sig_ms", C.c_double), ("bloom_ms", C.c_double), ("sig_chunks", C.c_uint64),
        ("probe_ms", C.c_double), ("probe_sectors", C.c_uint64),
        ("h2d_ms", C.c_double), ("h2d_bytes", C.c_uint64), ("call_ms", C.c_double),
        ("host_read_bytes", C.c_uint64), ("chunk_docs", C.c_uint64),
        ("pipelined_chunks", C.c_uint64),
    ]


class LSHBloomError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lock = threading.Lock()
_lib = None

_VP = C.c_void_p
_SIGS = {
    "lshbloom_config_default": (None, [C.POINTER(Config)]),
    "lshbloom_create": (C.c_int, [C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint64, C.c_double,
                                  C.POINTER(_VP)]),
    "lshbloom_create_ex": (C.c_int, [C.POINTER(Config), C.POINTER(_VP)]),
    "lshbloom_create_threshold": (C.c_int, [C.c_double, C.c_uint32, C.c_uint64, C.c_double,
                                            C.POINTER(_VP)]),
    "lshbloom_dedup": (C.c_int, [_VP, _VP, _VP, C.c_uint64, _VP]),
    "lshbloom_dedup_async": (C.c_int, [_VP, _VP, _VP, C.c_uint64, _VP, _VP]),
    "lshbloom_dedup_keys": (C.c_int, [_VP, _VP, _VP, C.c_uint64, _VP, _VP]),
    "lshbloom_dedup_from_keys": (C.c_int, [_VP, _VP, C.c_uint64, _VP]),
    "lshbloom_signatures": (C.c_int, [_VP, _VP, _VP, C.c_uint64, _VP]),
    "lshbloom_band_keys": (C.c_int, [_VP, _VP, _VP, C.c_uint64, _VP]),
    "lshbloom_shingle_hashes": (C.c_int, [_VP, _VP, _VP, C.c_uint64, _VP]),
    "lshbloom_band_keys_static": (C.c_int, [_VP, _VP, _VP, C.c_uint64, _VP, _VP]),
    "lshbloom_coefficients": (C.c_int, [_VP, _VP, _VP]),
    "lshbloom_filter_bytes": (C.c_int, [_VP, C.c_uint32, _VP]),
    "lshbloom_reset": (C.c_int, [_VP]),
    "lshbloom_stats": (C.c_int, [_VP, C.POINTER(Stats)]),
    "lshbloom_save": (C.c_int, [_VP, C.c_char_p]),
    "lshbloom_load": (C.c_int, [C.c_char_p, C.c_int32, C.POINTER(_VP)]),
    "lshbloom_optimal_br": (C.c_int, [C.c_double, C.c_uint32, C.POINTER(C.c_uint32),
                                      C.POINTER(C.c_uint32)]),
    "lshbloom_filter_sizing": (C.c_int, [C.c_uint64, C.c_double, C.c_uint32,
                                         C.POINTER(C.c_uint64), C.POINTER(C.c_uint32)]),
    "lshbloom_server_create": (C.c_int, [C.POINTER(_VP), C.c_uint32, C.c_uint64, C.c_uint32,
                                         C.POINTER(_VP)]),
    "lshbloom_server_submit": (C.c_int, [_VP, C.c_uint32, _VP, _VP, C.c_uint64, _VP,
                                         C.POINTER(C.c_uint64)]),
    "lshbloom_server_wait": (C.c_int, [_VP, C.c_uint64, C.c_double, C.POINTER(C.c_double)]),
    "lshbloom_server_destroy": (None, [_VP]),
    "lshbloom_last_error": (C.c_char_p, []),
    "lshbloom_destroy": (None, [_VP]),
}


def lib():
    """The loaded library.  Raises if it has not been built: there is no
    fallback path."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(
                    f"{LIB_PATH} is missing; build it with "
                    "`python -c 'import __graft_entry__ as g; g.build()'`")
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def check(status: int) -> None:
    if status != LSHB_OK:
        msg = lib().lshbloom_last_error()
        raise LSHBloomError(status, msg.decode() if msg else "")


def exported_symbols() -> list[str]:
    return list(_SIGS)
