"""GB300 LSHBloom: near-duplicate detection with MinHash LSH bands indexed by
Bloom filters (arxiv 2411.04257), on hand-written sm_103a CUDA kernels.

The Python layer only marshals arguments to the C ABI of liblshbloom.so
(include/lshbloom.h).  Inputs may be numpy arrays (host), or torch tensors on
the host or on the handle's GPU; outputs live where the tokens live.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from ._native import (EXEC_BATCHED, EXEC_PLAIN, INSERT_ALL, INSERT_NONDUP, Config,
                      LSHBloomError, Stats, check, lib)

__all__ = ["LSHBloom", "LSHBloomServer", "LSHBloomError", "optimal_br", "filter_sizing", "lib", "EXEC_PLAIN",
           "EXEC_BATCHED"]


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _arg(x, np_dtype, torch_dtypes):
    """(pointer, keep-alive object, is_cuda) for a 1-D/2-D array argument."""
    if _is_torch(x):
        import torch
        if x.dtype not in [getattr(torch, d) for d in torch_dtypes if hasattr(torch, d)]:
            raise TypeError(f"expected one of {torch_dtypes}, got {x.dtype}")
        if not x.is_contiguous():
            x = x.contiguous()
        return x.data_ptr(), x, x.is_cuda
    a = np.ascontiguousarray(x)
    if a.dtype != np_dtype:
        if a.dtype.kind in "iu" and a.dtype.itemsize == np.dtype(np_dtype).itemsize:
            a = a.view(np_dtype)
        else:
            a = a.astype(np_dtype)
    return a.ctypes.data, a, False


def _out(n_items, row, np_dtype, torch_dtype, like_cuda_tensor):
    if like_cuda_tensor is not None:
        import torch
        shape = (n_items,) if row is None else (n_items, row)
        t = torch.empty(shape, dtype=getattr(torch, torch_dtype), device=like_cuda_tensor.device)
        return t.data_ptr(), t
    shape = (n_items,) if row is None else (n_items, row)
    a = np.empty(shape, dtype=np_dtype)
    return a.ctypes.data, a


def _after_current_stream(t) -> None:
    """The synchronous C calls wait for the legacy default stream only; a CUDA
    tensor made on another torch stream must be complete before the call."""
    import torch
    st = torch.cuda.current_stream(t.device)
    if st.cuda_stream != 0:
        st.synchronize()


_LAYOUTS = {"standard": 0, "blocked": 1, "exact": 2}


class LSHBloom:
    """b Bloom filters, one per LSH band, fed in stream order.

    Parameters follow lshb_config: P permutations, b bands of r rows, n-gram
    size, the number of documents the filters are sized for and their
    false-positive rate (per filter, or effective over all b when
    fp_is_effective)."""

    def __init__(self, P: int = 121, bands: int = 11, rows: int = 11, n_expected: int = 10_000,
                 fp_rate: float = 1e-5, ngram: int = 5, seed: int = 1, insert_all: bool = False,
                 fp_is_effective: bool = False, exec_mode: str = "batched", device: int = -1,
                 max_batch_docs: int = 0, max_batch_tokens: int = 0, item_shingles: int = 0,
                 perm_a=None, perm_b=None, bloom_layout: str = "standard",
                 stage_host_inputs: bool = False, band_key: str = "sum", _handle=None):
        self._h = None
        if _handle is not None:
            self._h = _handle
            return
        cfg = Config()
        lib().lshbloom_config_default(C.byref(cfg))
        cfg.num_perm, cfg.bands, cfg.rows, cfg.ngram = P, bands, rows, ngram
        cfg.n_expected, cfg.fp_rate = n_expected, fp_rate
        cfg.fp_is_effective = 1 if fp_is_effective else 0
        cfg.insert_mode = INSERT_ALL if insert_all else INSERT_NONDUP
        cfg.seed = seed
        cfg.exec_mode = {"plain": EXEC_PLAIN, "batched": EXEC_BATCHED}[exec_mode]
        cfg.device = device
        cfg.max_batch_docs, cfg.max_batch_tokens = max_batch_docs, max_batch_tokens
        cfg.item_shingles = item_shingles
        cfg.bloom_layout = _LAYOUTS[bloom_layout]
        cfg.stage_host_inputs = 1 if stage_host_inputs else 0
        cfg.band_key = {"sum": 0, "weighted": 1}[band_key]
        keep = []
        if perm_a is not None:
            pa = np.ascontiguousarray(perm_a, np.uint64)
            pb = np.ascontiguousarray(perm_b, np.uint64)
            keep += [pa, pb]
            cfg.perm_a = pa.ctypes.data_as(C.POINTER(C.c_uint64))
            cfg.perm_b = pb.ctypes.data_as(C.POINTER(C.c_uint64))
        h = C.c_void_p()
        check(lib().lshbloom_create_ex(C.byref(cfg), C.byref(h)))
        self._h = h

    # -- lifetime ---------------------------------------------------------------
    def close(self) -> None:
        if self._h:
            lib().lshbloom_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self) -> int:
        return self._h.value

    # -- the path ---------------------------------------------------------------
    def _inputs(self, offsets, tokens, sync=True):
        po, ko, co = _arg(offsets, np.uint64, ["uint64", "int64"])
        pt, kt, ct = _arg(tokens, np.uint32, ["uint32", "int32"])
        if sync and (co or ct):
            _after_current_stream(kt if ct else ko)
        D = (ko.shape[0] if hasattr(ko, "shape") else len(ko)) - 1
        like = kt if ct else None
        return po, pt, max(D, 0), like, (ko, kt)

    def dedup(self, offsets, tokens, out=None):
        """uint8 duplicate flags of the batch (Sec. 2.1 decision), inserting it."""
        po, pt, D, like, keep = self._inputs(offsets, tokens)
        if out is None:
            pf, fl = _out(D, None, np.uint8, "uint8", like)
        else:
            pf, fl, _ = _arg(out, np.uint8, ["uint8"])
        check(lib().lshbloom_dedup(self._h, po, pt, D, pf))
        return fl

    def dedup_keys(self, offsets, tokens):
        """(flags, band keys) of the batch: dedup that also returns the keys
        the judgement used."""
        po, pt, D, like, keep = self._inputs(offsets, tokens)
        pf, fl = _out(D, None, np.uint8, "uint8", like)
        pk, keys = _out(D, self.bands, np.uint64, "uint64", like)
        check(lib().lshbloom_dedup_keys(self._h, po, pt, D, pf, pk))
        return fl, keys

    def dedup_from_keys(self, keys):
        """Flags of documents given by their band keys (D x bands, uint64 or
        int64, host or device), judged and inserted in order."""
        pk, kk, ck = _arg(keys, np.uint64, ["uint64", "int64"])
        if ck:
            _after_current_stream(kk)
        D = kk.shape[0] if kk.ndim == 2 else kk.shape[0] // self.bands
        if kk.ndim == 2 and kk.shape[1] != self.bands:
            raise ValueError(f"keys must have {self.bands} columns")
        pf, fl = _out(D, None, np.uint8, "uint8", kk if ck else None)
        check(lib().lshbloom_dedup_from_keys(self._h, pk, D, pf))
        return fl

    def dedup_async(self, offsets, tokens, stream=None):
        """As dedup, device tensors only, ordered on `stream` (torch stream or
        raw cudaStream_t; default the current torch stream)."""
        import torch
        po, pt, D, like, keep = self._inputs(offsets, tokens, sync=False)
        pf, fl = _out(D, None, np.uint8, "uint8", like)
        if stream is None:
            stream = torch.cuda.current_stream()
        sp = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        check(lib().lshbloom_dedup_async(self._h, po, pt, D, pf, C.c_void_p(sp)))
        return fl

    def signatures(self, offsets, tokens):
        po, pt, D, like, keep = self._inputs(offsets, tokens)
        ps, sig = _out(D, self.P, np.uint32, "uint32", like)
        check(lib().lshbloom_signatures(self._h, po, pt, D, ps))
        return sig

    def band_keys(self, offsets, tokens):
        po, pt, D, like, keep = self._inputs(offsets, tokens)
        pk, keys = _out(D, self.bands, np.uint64, "uint64", like)
        check(lib().lshbloom_band_keys(self._h, po, pt, D, pk))
        return keys

    def band_keys_static(self, offsets, tokens, out=None, stream=None):
        """Band keys through lshbloom_band_keys_static: no allocation inside
        the library (device tensors only; `out` may be preallocated)."""
        import torch
        po, pt, D, like, keep = self._inputs(offsets, tokens, sync=False)
        if out is None:
            pk, keys = _out(D, self.bands, np.uint64, "uint64", like)
        else:
            pk, keys, _ = _arg(out, np.uint64, ["uint64", "int64"])
        if stream is None:
            stream = torch.cuda.current_stream()
        sp = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        check(lib().lshbloom_band_keys_static(self._h, po, pt, D, pk, C.c_void_p(sp)))
        return keys

    def shingle_hashes(self, offsets, tokens):
        po, pt, D, like, keep = self._inputs(offsets, tokens)
        ko = keep[0]
        n = int(ko[-1]) - int(ko[0]) if D > 0 else 0
        ph, hs = _out(n, None, np.uint32, "uint32", like)
        check(lib().lshbloom_shingle_hashes(self._h, po, pt, D, ph))
        return hs

    # -- inspection ---------------------------------------------------------------
    def stats(self) -> dict:
        s = Stats()
        check(lib().lshbloom_stats(self._h, C.byref(s)))
        d = {f: getattr(s, f) for f, _ in Stats._fields_ if f != "fill"}
        d["fill"] = list(s.fill)[: s.bands]
        return d

    def _dims(self):
        if not hasattr(self, "_dim_cache"):
            s = self.stats()
            self._dim_cache = (s["num_perm"], s["bands"], s["rows"], s["m_bits"], s["k"],
                               s["filter_bytes"])
        return self._dim_cache

    @property
    def P(self) -> int:
        return self._dims()[0]

    @property
    def bands(self) -> int:
        return self._dims()[1]

    @property
    def rows(self) -> int:
        return self._dims()[2]

    @property
    def m(self) -> int:
        return self._dims()[3]

    @property
    def k(self) -> int:
        return self._dims()[4]

    def coefficients(self):
        P = self.P
        a = np.zeros(P, np.uint64)
        b = np.zeros(P, np.uint64)
        check(lib().lshbloom_coefficients(self._h, a.ctypes.data, b.ctypes.data))
        return a, b

    def filter_bytes(self, band: int) -> np.ndarray:
        """Filter `band` as bytes (bit q at byte q/8, LSB first); for the
        exact-key layout, the band's table of uint64 slots."""
        out = np.zeros(self._dims()[5], np.uint8)
        check(lib().lshbloom_filter_bytes(self._h, band, out.ctypes.data))
        return out

    def exact_keys(self, band: int) -> np.ndarray:
        """Sorted band keys stored in band `band`'s table (exact-key layout):
        the table's cap key slots, then the slot recording the key 2^64-1,
        then 15 padding slots."""
        t = self.filter_bytes(band).view(np.uint64)
        cap = t.size - 16
        keys = t[:cap][t[:cap] != np.uint64(2**64 - 1)]
        if t[cap] == 0:
            keys = np.append(keys, np.uint64(2**64 - 1))
        return np.sort(keys)

    def reset(self) -> None:
        check(lib().lshbloom_reset(self._h))

    def save(self, path: str) -> None:
        check(lib().lshbloom_save(self._h, path.encode()))

    @classmethod
    def from_threshold(cls, T: float, P: int, n_expected: int, p_eff: float) -> "LSHBloom":
        """(b, r) from the Jaccard threshold (Eqs. 1-2), per-filter rate from
        the effective rate over all bands (Sec. 4.3)."""
        h = C.c_void_p()
        check(lib().lshbloom_create_threshold(T, P, n_expected, p_eff, C.byref(h)))
        return cls(_handle=h)

    @classmethod
    def load(cls, path: str, device: int = -1) -> "LSHBloom":
        h = C.c_void_p()
        check(lib().lshbloom_load(path.encode(), device, C.byref(h)))
        return cls(_handle=h)


class LSHBloomServer:
    """Continuous-batching request server over resident indexes
    (lshbloom_server_*).  submit() takes host arrays and returns a ticket;
    wait() returns (flags, latency in microseconds)."""

    def __init__(self, indexes, mem_budget_bytes: int = 1 << 30, max_inflight: int = 32):
        self._indexes = list(indexes)  # keep the handles alive
        arr = (C.c_void_p * len(self._indexes))(*[ix._h.value for ix in self._indexes])
        h = C.c_void_p()
        check(lib().lshbloom_server_create(arr, len(self._indexes), mem_budget_bytes,
                                           max_inflight, C.byref(h)))
        self._h = h
        self._live = {}

    def submit(self, index: int, offsets, tokens) -> int:
        off = np.ascontiguousarray(offsets, dtype=np.uint64)
        tok = np.ascontiguousarray(tokens, dtype=np.uint32)
        D = off.size - 1
        flags = np.zeros(max(D, 1), np.uint8)
        t = C.c_uint64()
        tok_p = tok.ctypes.data if tok.size else np.zeros(1, np.uint32).ctypes.data
        check(lib().lshbloom_server_submit(self._h, index, off.ctypes.data, tok_p, D,
                                           flags.ctypes.data, C.byref(t)))
        self._live[t.value] = (off, tok, flags, D)
        return t.value

    def wait(self, ticket: int, timeout_ms: float = -1.0):
        lat = C.c_double()
        check(lib().lshbloom_server_wait(self._h, ticket, timeout_ms, C.byref(lat)))
        off, tok, flags, D = self._live.pop(ticket)
        return flags[:D], lat.value

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().lshbloom_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def filter_sizing(n_expected: int, fp_rate: float, bloom_layout: str = "standard"):
    """(m bits, k) of one filter as an index of this layout sizes it."""
    m = C.c_uint64()
    k = C.c_uint32()
    check(lib().lshbloom_filter_sizing(n_expected, fp_rate, _LAYOUTS[bloom_layout],
                                       C.byref(m), C.byref(k)))
    return int(m.value), int(k.value)


def optimal_br(T: float, P: int):
    """(b, r) minimising the equal-weight LSH error integrals (Eqs. 1-2)."""
    b = C.c_uint32()
    r = C.c_uint32()
    check(lib().lshbloom_optimal_br(T, P, C.byref(b), C.byref(r)))
    return int(b.value), int(r.value)
