"""Python view of the LSHBloom CPU oracle -- TEST INFRASTRUCTURE ONLY.

Loads ``liblshb_oracle.so`` (built from ``lshb_oracle.c`` with gcc) through
ctypes and wraps it with numpy arrays.  Only the tests, the smoke check and
the CPU-baseline leg of the benchmark use this module; the product path never
imports it, and it imports nothing from the product package.

Every function here is marshalling only: the arithmetic lives in the C file,
each function of which cites the passage of arxiv 2411.04257 it restates.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lshb_oracle.c")
_SRC_THREADS = os.path.join(_HERE, "lshb_cpu_threads.c")
_LIB = os.path.join(_HERE, "liblshb_oracle.so")
_lock = threading.Lock()
_lib = None

P61 = (1 << 61) - 1


def build(force: bool = False) -> str:
    """Compile the oracle and its threaded driver with gcc (plain -O2, no
    vector intrinsics)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_THREADS))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fvisibility=hidden", "-pthread",
             "-o", tmp, _SRC, _SRC_THREADS, "-lm"],
            check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            u8p, u32p, u64p = (C.POINTER(C.c_uint8), C.POINTER(C.c_uint32),
                               C.POINTER(C.c_uint64))
            sig = {
                "or_sha1": (None, [u8p, C.c_uint64, u8p]),
                "or_shingle_hash": (C.c_uint32, [u32p, C.c_uint32]),
                "or_mix64": (C.c_uint64, [C.c_uint64]),
                "or_coefficients": (None, [C.c_uint64, C.c_uint32, u64p, u64p]),
                "or_perm": (C.c_uint32, [C.c_uint64, C.c_uint64, C.c_uint32]),
                "or_signature": (None, [u32p, C.c_uint64, C.c_uint32, C.c_uint32, u64p, u64p,
                                        u32p]),
                "or_band_keys": (None, [u32p, C.c_uint32, C.c_uint32, u64p]),
                "or_probe_positions": (None, [C.c_uint64, C.c_uint32, C.c_uint64, C.c_uint32,
                                              u64p]),
                "or_probe_positions_blocked": (None, [C.c_uint64, C.c_uint32, C.c_uint64,
                                                      C.c_uint32, u64p]),
                "or_index_set_layout": (C.c_int, [C.c_void_p, C.c_uint32]),
                "or_index_set_band_key": (C.c_int, [C.c_void_p, C.c_uint32]),
                "or_band_keys_mode": (None, [C.POINTER(C.c_uint32), C.c_uint32, C.c_uint32,
                                             C.c_uint32, u64p]),
                "or_index_exact_keys": (C.c_uint64, [C.c_void_p, C.c_uint32, u64p, C.c_uint64]),
                "or_p_from_effective": (C.c_double, [C.c_double, C.c_uint32]),
                "or_effective_from_p": (C.c_double, [C.c_double, C.c_uint32]),
                "or_sizing": (None, [C.c_uint64, C.c_double, u64p, C.POINTER(C.c_uint32)]),
                "or_sizing_blocked": (None, [C.c_uint64, C.c_double, u64p,
                                             C.POINTER(C.c_uint32)]),
                "or_fp_blocked": (C.c_double, [C.c_uint64, C.c_uint64, C.c_uint32]),
                "or_blocked_hit": (C.c_double, [C.c_uint32, C.c_uint32]),
                "or_fp_lsh": (C.c_double, [C.c_double, C.c_uint32, C.c_uint32]),
                "or_fn_lsh": (C.c_double, [C.c_double, C.c_uint32, C.c_uint32]),
                "or_fp_bloom": (C.c_double, [C.c_double, C.c_double, C.c_uint32, C.c_double]),
                "or_fn_bloom": (C.c_double, [C.c_double, C.c_double, C.c_uint32, C.c_double]),
                "or_optimal_br": (None, [C.c_double, C.c_uint32, C.POINTER(C.c_uint32),
                                         C.POINTER(C.c_uint32)]),
                "or_index_create": (C.c_void_p, [C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32,
                                                 C.c_uint64, C.c_uint32, u64p, u64p,
                                                 C.c_uint32]),
                "or_index_destroy": (None, [C.c_void_p]),
                "or_index_dedup": (None, [C.c_void_p, u64p, u32p, C.c_uint64, u8p]),
                "or_index_dedup_keys": (None, [C.c_void_p, u64p, C.c_uint64, u8p]),
                "or_batch_band_keys": (None, [u64p, u32p, C.c_uint64, C.c_uint32, C.c_uint32,
                                              u64p, u64p, C.c_uint32, C.c_uint32, C.c_uint32,
                                              u64p]),
                "ort_batch_band_keys": (C.c_uint32, [u64p, u32p, C.c_uint64, C.c_uint32,
                                                     C.c_uint32, u64p, u64p, C.c_uint32,
                                                     C.c_uint32, C.c_uint32, u64p, C.c_uint32]),
                "ort_index_dedup": (C.c_uint32, [C.c_void_p, u64p, u32p, C.c_uint64, u8p,
                                                 C.c_uint32, C.c_uint32, u64p, u64p, C.c_uint32,
                                                 C.c_uint32, C.c_uint32, C.c_uint32,
                                                 C.c_uint64]),
                "or_index_query_key": (C.c_int, [C.c_void_p, C.c_uint32, C.c_uint64]),
                "or_index_insert_key": (None, [C.c_void_p, C.c_uint32, C.c_uint64]),
                "or_index_insert_keys": (None, [C.c_void_p, C.c_uint32, u64p, C.c_uint64]),
                "or_index_query_keys": (None, [C.c_void_p, C.c_uint32, u64p, C.c_uint64, u8p]),
                "or_index_filter_bytes": (None, [C.c_void_p, C.c_uint32, u8p]),
                "or_index_popcount": (C.c_uint64, [C.c_void_p, C.c_uint32]),
                "or_index_docs_seen": (C.c_uint64, [C.c_void_p]),
                "or_batch_signatures": (None, [u64p, u32p, C.c_uint64, C.c_uint32, C.c_uint32,
                                               u64p, u64p, u32p]),
                "or_batch_shingle_hashes": (None, [u64p, u32p, C.c_uint64, C.c_uint32, u32p,
                                                   u64p]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _p(arr: np.ndarray, ct):
    return arr.ctypes.data_as(C.POINTER(ct))


def _u32(x) -> np.ndarray:
    return np.ascontiguousarray(x, dtype=np.uint32)


def _u64(x) -> np.ndarray:
    return np.ascontiguousarray(x, dtype=np.uint64)


# --- hashing -------------------------------------------------------------

def sha1(data: bytes) -> bytes:
    buf = np.frombuffer(data, dtype=np.uint8).copy() if data else np.zeros(1, np.uint8)
    out = np.zeros(20, np.uint8)
    lib().or_sha1(_p(buf, C.c_uint8), len(data), _p(out, C.c_uint8))
    return out.tobytes()


def shingle_hash(tokens) -> int:
    t = _u32(tokens)
    if t.size == 0:
        t = np.zeros(1, np.uint32)
        return int(lib().or_shingle_hash(_p(t, C.c_uint32), 0))
    return int(lib().or_shingle_hash(_p(t, C.c_uint32), t.size))


def mix64(z: int) -> int:
    return int(lib().or_mix64(z & (2**64 - 1)))


def coefficients(seed: int, P: int):
    a = np.zeros(P, np.uint64)
    b = np.zeros(P, np.uint64)
    lib().or_coefficients(seed, P, _p(a, C.c_uint64), _p(b, C.c_uint64))
    return a, b


def perm(a: int, b: int, h: int) -> int:
    return int(lib().or_perm(a, b, h))


def signature(tokens, n: int, a: np.ndarray, b: np.ndarray) -> np.ndarray:
    t = _u32(tokens)
    P = a.size
    sig = np.zeros(P, np.uint32)
    tt = t if t.size else np.zeros(1, np.uint32)
    lib().or_signature(_p(tt, C.c_uint32), t.size, n, P, _p(_u64(a), C.c_uint64),
                       _p(_u64(b), C.c_uint64), _p(sig, C.c_uint32))
    return sig


def band_keys(sig: np.ndarray, bands: int, rows: int, mode: int = 0) -> np.ndarray:
    """Band keys of one signature: the paper's sums (mode 0) or the weighted
    sums (mode 1)."""
    s = _u32(sig)
    keys = np.zeros(bands, np.uint64)
    if mode == 0:
        lib().or_band_keys(_p(s, C.c_uint32), bands, rows, _p(keys, C.c_uint64))
    else:
        lib().or_band_keys_mode(_p(s, C.c_uint32), bands, rows, mode, _p(keys, C.c_uint64))
    return keys


def probe_positions(key: int, j: int, m: int, k: int) -> np.ndarray:
    q = np.zeros(k, np.uint64)
    lib().or_probe_positions(key, j, m, k, _p(q, C.c_uint64))
    return q


def probe_positions_blocked(key: int, j: int, m: int, k: int) -> np.ndarray:
    q = np.zeros(k, np.uint64)
    lib().or_probe_positions_blocked(key, j, m, k, _p(q, C.c_uint64))
    return q


def batch_signatures(offsets, tokens, n: int, a, b) -> np.ndarray:
    off = _u64(offsets)
    tok = _u32(tokens)
    D = off.size - 1
    P = len(a)
    out = np.zeros((max(D, 0), P), np.uint32)
    tt = tok if tok.size else np.zeros(1, np.uint32)
    if D > 0:
        lib().or_batch_signatures(_p(off, C.c_uint64), _p(tt, C.c_uint32), D, n, P,
                                  _p(_u64(a), C.c_uint64), _p(_u64(b), C.c_uint64),
                                  _p(out, C.c_uint32))
    return out


def host_threads() -> int:
    """Host cores this process may run on."""
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except (AttributeError, OSError):
        return max(1, os.cpu_count() or 1)


def batch_band_keys(offsets, tokens, n: int, a, b, bands: int, rows: int, mode: int = 0,
                    threads: int = 1) -> np.ndarray:
    """Band keys (D x bands) of a CSR batch.  threads > 1 runs the unchanged
    per-document oracle on several threads (lshb_cpu_threads.c)."""
    off = _u64(offsets)
    tok = _u32(tokens)
    D = off.size - 1
    out = np.zeros((max(D, 1), bands), np.uint64)
    tt = tok if tok.size else np.zeros(1, np.uint32)
    aa, bb = _u64(a), _u64(b)
    if D > 0:
        args = (_p(off, C.c_uint64), _p(tt, C.c_uint32), D, n, len(aa), _p(aa, C.c_uint64),
                _p(bb, C.c_uint64), bands, rows, mode, _p(out, C.c_uint64))
        if threads > 1:
            lib().ort_batch_band_keys(*args, threads)
        else:
            lib().or_batch_band_keys(*args)
    return out[:max(D, 0)]


def batch_shingle_hashes(offsets, tokens, n: int):
    off = _u64(offsets)
    tok = _u32(tokens)
    D = off.size - 1
    h = np.zeros(max(tok.size, 1), np.uint32)
    counts = np.zeros(max(D, 1), np.uint64)
    tt = tok if tok.size else np.zeros(1, np.uint32)
    if D > 0:
        lib().or_batch_shingle_hashes(_p(off, C.c_uint64), _p(tt, C.c_uint32), D, n,
                                      _p(h, C.c_uint32), _p(counts, C.c_uint64))
    total = int(counts[:D].sum()) if D > 0 else 0
    return h[:total], counts[:D]


# --- sizing and the error model --------------------------------------------

def p_from_effective(p_eff: float, bands: int) -> float:
    return float(lib().or_p_from_effective(p_eff, bands))


def effective_from_p(p: float, bands: int) -> float:
    return float(lib().or_effective_from_p(p, bands))


def sizing(n: int, p: float):
    m = C.c_uint64()
    k = C.c_uint32()
    lib().or_sizing(n, p, C.byref(m), C.byref(k))
    return int(m.value), int(k.value)


def sizing_blocked(n: int, p: float):
    """(m, k) of the blocked layout: the fewest 256-bit blocks meeting p."""
    m = C.c_uint64()
    k = C.c_uint32()
    lib().or_sizing_blocked(n, p, C.byref(m), C.byref(k))
    return int(m.value), int(k.value)


def fp_blocked(n: int, m: int, k: int) -> float:
    return float(lib().or_fp_blocked(n, m, k))


def blocked_hit(i: int, k: int) -> float:
    return float(lib().or_blocked_hit(i, k))


def fp_lsh(T, b, r):
    return float(lib().or_fp_lsh(T, b, r))


def fn_lsh(T, b, r):
    return float(lib().or_fn_lsh(T, b, r))


def fp_bloom(fpl, p_eff, b, N):
    return float(lib().or_fp_bloom(fpl, p_eff, b, N))


def fn_bloom(fnl, p_eff, b, N):
    return float(lib().or_fn_bloom(fnl, p_eff, b, N))


def optimal_br(T: float, P: int):
    b = C.c_uint32()
    r = C.c_uint32()
    lib().or_optimal_br(T, P, C.byref(b), C.byref(r))
    return int(b.value), int(r.value)


# --- the index --------------------------------------------------------------

class OracleIndex:
    """b Bloom filters fed in stream order (Sec. 4.1, 4.2, 4.4.2)."""

    def __init__(self, P: int, bands: int, rows: int, n_expected: int = 10_000,
                 fp_rate: float = 1e-5, ngram: int = 5, seed: int = 1,
                 insert_all: bool = False, fp_is_effective: bool = False,
                 m: int | None = None, k: int | None = None, a=None, b=None,
                 layout: int = 0, band_key: int = 0):
        p = p_from_effective(fp_rate, bands) if fp_is_effective else fp_rate
        mm, kk = sizing_blocked(n_expected, p) if layout == 1 else sizing(n_expected, p)
        self.m = int(m) if m is not None else mm
        self.k = int(k) if k is not None else kk
        if a is None or b is None:
            a, b = coefficients(seed, P)
        self.a, self.b = _u64(a), _u64(b)
        self.P, self.bands, self.rows, self.ngram = P, bands, rows, ngram
        self.band_key = band_key
        self._h = lib().or_index_create(P, bands, rows, ngram, self.m, self.k,
                                        _p(self.a, C.c_uint64), _p(self.b, C.c_uint64),
                                        1 if insert_all else 0)
        if not self._h:
            raise ValueError("oracle index: bad parameters")
        if layout and lib().or_index_set_layout(self._h, layout) != 0:
            raise ValueError("oracle index: bad layout")
        if band_key and lib().or_index_set_band_key(self._h, band_key) != 0:
            raise ValueError("oracle index: bad band-key mode")

    def close(self):
        if getattr(self, "_h", None):
            lib().or_index_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def dedup(self, offsets, tokens) -> np.ndarray:
        off = _u64(offsets)
        tok = _u32(tokens)
        D = off.size - 1
        flags = np.zeros(max(D, 1), np.uint8)
        tt = tok if tok.size else np.zeros(1, np.uint32)
        if D > 0:
            lib().or_index_dedup(self._h, _p(off, C.c_uint64), _p(tt, C.c_uint32), D,
                                 _p(flags, C.c_uint8))
        return flags[:max(D, 0)]

    def dedup_keys(self, keys) -> np.ndarray:
        """The stream decision alone, fed with band keys (D x bands)."""
        k = _u64(keys).reshape(-1, self.bands)
        D = k.shape[0]
        flags = np.zeros(max(D, 1), np.uint8)
        if D > 0:
            lib().or_index_dedup_keys(self._h, _p(k, C.c_uint64), D, _p(flags, C.c_uint8))
        return flags[:D]

    def dedup_threaded(self, offsets, tokens, threads: int | None = None,
                       block_docs: int = 65536):
        """As dedup, with the band keys of each block of documents computed on
        `threads` threads and the decisions taken in order (the paper's CPU
        design, Sec. 4.4.2).  Returns (flags, threads used)."""
        off = _u64(offsets)
        tok = _u32(tokens)
        D = off.size - 1
        flags = np.zeros(max(D, 1), np.uint8)
        tt = tok if tok.size else np.zeros(1, np.uint32)
        used = 1
        if D > 0:
            used = lib().ort_index_dedup(self._h, _p(off, C.c_uint64), _p(tt, C.c_uint32), D,
                                         _p(flags, C.c_uint8), self.ngram, self.P,
                                         _p(self.a, C.c_uint64), _p(self.b, C.c_uint64),
                                         self.bands, self.rows, self.band_key,
                                         threads or host_threads(), block_docs)
        return flags[:max(D, 0)], int(used)

    def query_key(self, j: int, key: int) -> bool:
        return bool(lib().or_index_query_key(self._h, j, key))

    def insert_key(self, j: int, key: int) -> None:
        lib().or_index_insert_key(self._h, j, key)

    def insert_keys(self, j: int, keys) -> None:
        k = _u64(keys)
        if k.size:
            lib().or_index_insert_keys(self._h, j, _p(k, C.c_uint64), k.size)

    def query_keys(self, j: int, keys) -> np.ndarray:
        k = _u64(keys)
        hit = np.zeros(max(k.size, 1), np.uint8)
        if k.size:
            lib().or_index_query_keys(self._h, j, _p(k, C.c_uint64), k.size,
                                      _p(hit, C.c_uint8))
        return hit[:k.size].astype(bool)

    def filter_bytes(self, j: int) -> np.ndarray:
        out = np.zeros((self.m + 7) // 8, np.uint8)
        lib().or_index_filter_bytes(self._h, j, _p(out, C.c_uint8))
        return out

    def exact_keys(self, j: int) -> np.ndarray:
        """Sorted band keys of band j (exact-set layout)."""
        n = int(lib().or_index_exact_keys(self._h, j, None, 0))
        out = np.zeros(max(n, 1), np.uint64)
        lib().or_index_exact_keys(self._h, j, _p(out, C.c_uint64), n)
        return np.sort(out[:n])

    def popcount(self, j: int) -> int:
        return int(lib().or_index_popcount(self._h, j))

    @property
    def docs_seen(self) -> int:
        return int(lib().or_index_docs_seen(self._h))
