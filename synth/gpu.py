"""Device generator for synth/corpus.py corpora (same bytes, built in HBM)."""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

from . import corpus

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth_gen.cu")
_LIB = os.path.join(_HERE, "libsynth_gen.so")
_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        nvcc = "/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else "nvcc"
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                        "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden", "-shared",
                        "-o", tmp, _SRC], check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Params(C.Structure):
    _fields_ = [("zipf_cdf", C.c_void_p), ("word_hash", C.c_void_p), ("length", C.c_void_p),
                ("mut_thr", C.c_void_p), ("vocab", C.c_uint64), ("dup_thr", C.c_uint64),
                ("window", C.c_uint64), ("fkey", C.c_uint64 * 8)]


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB):
            build()
        L = C.CDLL(_LIB)
        L.synth_doc_lengths.restype = C.c_int
        L.synth_doc_lengths.argtypes = [C.POINTER(_Params), C.c_uint64, C.c_uint64, C.c_void_p,
                                        C.c_void_p]
        L.synth_tokens.restype = C.c_int
        L.synth_tokens.argtypes = [C.POINTER(_Params), C.c_uint64, C.c_uint64, C.c_void_p,
                                   C.c_void_p, C.c_void_p]
        _lib = L
    return _lib


class DeviceCorpus:
    """Tables of one corpus uploaded to a GPU; generates CSR slices there."""

    def __init__(self, spec: corpus.CorpusSpec, device="cuda:0"):
        import torch
        self.spec = spec
        self.device = torch.device(device)
        t = corpus.build_tables(spec)
        self.tables = t
        dev = self.device
        self._zipf = torch.from_numpy(t.zipf_cdf.view(np.int64)).to(dev)
        self._wh = torch.from_numpy(t.word_hash.view(np.int32)).to(dev)
        self._len = torch.from_numpy(t.length.view(np.int32)).to(dev)
        self._mut = torch.from_numpy(t.mut_thr.view(np.int64)).to(dev)
        p = _Params()
        p.zipf_cdf, p.word_hash = self._zipf.data_ptr(), self._wh.data_ptr()
        p.length, p.mut_thr = self._len.data_ptr(), self._mut.data_ptr()
        p.vocab, p.dup_thr, p.window = t.zipf_cdf.size, t.dup_thr, t.window
        for f in range(8):
            p.fkey[f] = corpus.field_key(spec.seed, f) if f > 0 else 0
        self._p = p

    def generate(self, d0: int, D: int, stream=None):
        """(offsets int64[D+1] from 0, tokens int32[T]) on the device."""
        import torch
        L = _load()
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        sp = C.c_void_p(s.cuda_stream)
        lens = torch.empty(D, dtype=torch.int64, device=self.device)
        if L.synth_doc_lengths(C.byref(self._p), d0, D, lens.data_ptr(), sp) != 0:
            raise RuntimeError("synth_doc_lengths failed")
        offsets = torch.zeros(D + 1, dtype=torch.int64, device=self.device)
        torch.cumsum(lens, 0, out=offsets[1:])
        T = int(offsets[-1].item())
        tokens = torch.empty(max(T, 1), dtype=torch.int32, device=self.device)[:T]
        if L.synth_tokens(C.byref(self._p), d0, D, offsets.data_ptr(), tokens.data_ptr(), sp) != 0:
            raise RuntimeError("synth_tokens failed")
        return offsets, tokens
