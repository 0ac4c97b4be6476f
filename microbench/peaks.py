"""Measured peaks for the rooflines of the LSHBloom kernels (see peaks.cu).

measure(device) returns, on one GPU:
  gather_dram, gather_l2:
           random 32-byte-sector reads over a 4 GiB buffer (far larger than
           L2) and over a 64 MiB one (L2-resident), as GB/s of the sectors
           addressed (32 B each), per load form; random 4-byte atomic ORs
           (sectors/s); whole sectors read by 8 lanes;
  issue:   operations per second of mad.wide.u32, mad.lo.u32 and four ALU
           operations (eight independent chains per thread, all SMs);
  ceiling: shingles/s and perm-hashes/s of the library's SHA-1 window hash
           and MinHash fold (P = 121) without memory traffic.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
_SRC = os.path.join(_HERE, "peaks.cu")
_LIB = os.path.join(_HERE, "libpeaks.so")
_CSRC = os.path.join(_ROOT, "paper_2411_04257_gb300", "csrc")
_lib = None

GATHER_MODES = {0: "ld.global.nc", 1: "ld.global.cg", 2: "ld.relaxed.gpu", 3: "ld.global.nc.L2::64B",
                4: "ld.global.cv", 5: "ld.global.nc.L1::no_allocate", 6: "atom.or (random RMW)",
                7: "8 lanes x 4 B = one whole sector"}
ISSUE_KINDS = {0: "mad.wide.u32", 1: "mad.lo.u32", 2: "min.u32", 3: "add.u32", 4: "lop3 (xor3)",
               5: "shf.r.wrap"}
CEILING_KINDS = {0: "fold (P=121, PPL=4)", 1: "sha1 5-gram windows", 2: "sha1 + fold"}


def _deps():
    hs = [os.path.join(_CSRC, f) for f in ("sig_kernels.cuh", "lshb_device.cuh", "lshb_internal.h")]
    return max(os.path.getmtime(p) for p in [_SRC] + hs)


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < _deps():
        nvcc = "/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else "nvcc"
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                        "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
                        "-shared", "-I", _CSRC, "-I", os.path.join(_ROOT, "include"),
                        "-o", tmp, _SRC], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        L.mb_gather.restype = C.c_float
        L.mb_gather.argtypes = [C.c_void_p, C.c_uint64, C.c_uint64, C.c_uint64, C.c_int,
                                C.c_uint64]
        L.mb_issue.restype = C.c_float
        L.mb_issue.argtypes = [C.c_int, C.c_uint64, C.c_uint64]
        L.mb_ceiling.restype = C.c_float
        L.mb_ceiling.argtypes = [C.c_int, C.c_uint64, C.c_uint64, C.c_void_p, C.c_void_p]
        L.mb_ceiling_occupancy.restype = C.c_int
        L.mb_ceiling_occupancy.argtypes = [C.c_int]
        _lib = L
    return _lib


def _best(f, reps=3):
    best = None
    for _ in range(reps):
        ms = f()
        if ms <= 0:
            raise RuntimeError("microbenchmark launch failed")
        best = ms if best is None else min(best, ms)
    return best


def _gather(L, sms, device, log2_sectors, per):
    import torch
    nsect = 1 << log2_sectors
    buf = torch.zeros(nsect * 8, dtype=torch.int32, device=f"cuda:{device}")
    threads = sms * 2048
    out = {"buffer_bytes": nsect * 32}
    for mode, name in GATHER_MODES.items():
        L.mb_gather(buf.data_ptr(), nsect - 1, threads, 8, mode, 7)          # warm-up
        ms = _best(lambda: L.mb_gather(buf.data_ptr(), nsect - 1, threads, per, mode, 1))
        acc = threads * per
        sectors = acc / 8 if mode == 7 else acc                          # mode 7: 8 lanes per sector
        out[name] = {"sectors_per_s": sectors / (ms / 1e3),
                     "gbs": sectors * 32 / (ms / 1e3) / 1e9, "ms": ms}
    del buf
    torch.cuda.empty_cache()
    return out


def measure(device: int = 0, quick: bool = False) -> dict:
    """All peaks on `device` (the current CUDA device must be `device`):
    random sectors over a 4 GiB buffer (DRAM) and over a 64 MiB one (L2)."""
    import numpy as np
    import torch
    L = lib()
    props = torch.cuda.get_device_properties(device)
    sms = props.multi_processor_count
    out = {"sms": sms, "issue": {}, "ceiling": {}}
    per = 128 if quick else 512
    out["gather_dram"] = _gather(L, sms, device, 27, per)
    out["gather_l2"] = _gather(L, sms, device, 21, per)
    blocks = sms * 8
    iters = 2000 if quick else 20000
    for kind, name in ISSUE_KINDS.items():
        L.mb_issue(kind, blocks, 10)
        ms = _best(lambda: L.mb_issue(kind, blocks, iters))
        ops = blocks * 256 * iters * 8
        out["issue"][name] = {"ops_per_s": ops / (ms / 1e3),
                              "per_sm_per_clk_at_2070": ops / (ms / 1e3) / sms / 2.07e9}
    a = np.arange(1, 122, dtype=np.uint64) * np.uint64(0x1234567) + np.uint64(99)
    b = np.arange(0, 121, dtype=np.uint64) * np.uint64(0x7654321) + np.uint64(5)
    steps = 200 if quick else 2000
    for kind, name in CEILING_KINDS.items():
        nb = max(1, L.mb_ceiling_occupancy(kind)) * sms
        L.mb_ceiling(kind, nb, 5, a.ctypes.data, b.ctypes.data)
        ms = _best(lambda: L.mb_ceiling(kind, nb, steps, a.ctypes.data, b.ctypes.data))
        shingles = nb * 2 * steps * 32
        out["ceiling"][name] = {"shingles_per_s": shingles / (ms / 1e3),
                                "perm_hashes_per_s": shingles * 121 / (ms / 1e3)
                                if kind != 1 else None,
                                "blocks": nb}
    return out


if __name__ == "__main__":
    import json
    import sys
    print(json.dumps(measure(quick="--quick" in sys.argv), indent=1))
