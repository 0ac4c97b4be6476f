"""The C ABI library builds for sm_103a, loads without a GPU, and exports every
function include/lshbloom.h declares (no compute call is made here)."""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lshbloom.h")


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"LSHB_API\s+[\w\s\*]+?\b(lshbloom_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def built():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2411_04257_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("lshbloom_create", "lshbloom_dedup", "lshbloom_destroy", "lshbloom_create_ex",
                 "lshbloom_dedup_async", "lshbloom_save", "lshbloom_load", "lshbloom_stats",
                 "lshbloom_last_error"):
        assert must in names
    # every declaration carries a comment that cites the paper or states its role
    text = open(HEADER).read()
    assert "Sec. 4.1" in text and "Sec. 2.1" in text


def test_library_exports_every_declared_symbol(built):
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (lshbloom_\w+)", out))
    assert set(_declared()) <= exported, set(_declared()) - exported
    assert exported <= set(_declared()), exported - set(_declared())


def test_library_loads_and_binding_matches(built):
    import ctypes

    from paper_2411_04257_gb300 import _native
    lib = _native.lib()
    for name in _declared():
        assert hasattr(lib, name)
    assert set(_native.exported_symbols()) == set(_declared())
    # config_default is pure host code: defaults are the 10k-document workload's
    cfg = _native.Config()
    lib.lshbloom_config_default(ctypes.byref(cfg))
    assert (cfg.num_perm, cfg.bands, cfg.rows, cfg.ngram) == (121, 11, 11, 5)
    assert lib.lshbloom_last_error() == b""


def test_struct_layouts_match_header(built):
    """ctypes layouts agree with the C structs (compiled probe of sizeof)."""
    import ctypes

    from paper_2411_04257_gb300 import _native
    src = os.path.join(os.environ.get("TMPDIR", "/tmp"), f"lshb_probe_{os.getpid()}.c")
    exe = src[:-2]
    with open(src, "w") as f:
        f.write('#include "lshbloom.h"\n#include <stdio.h>\n#include <stddef.h>\n'
                'int main(void){printf("%zu %zu %zu %zu\\n", sizeof(lshb_config), '
                'sizeof(lshb_stats), offsetof(lshb_config, exec_mode), '
                'offsetof(lshb_stats, fill));return 0;}\n')
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", exe, src], check=True)
    vals = list(map(int, subprocess.run([exe], capture_output=True, text=True,
                                        check=True).stdout.split()))
    os.unlink(src)
    os.unlink(exe)
    assert vals == [ctypes.sizeof(_native.Config), ctypes.sizeof(_native.Stats),
                    _native.Config.exec_mode.offset, _native.Stats.fill.offset]


def test_filter_sizing_matches_the_oracle(built, oracle):
    """lshbloom_filter_sizing (host only) equals the oracle's sizing for both
    Bloom layouts; the two implement the blocked model independently."""
    import paper_2411_04257_gb300 as L
    cases = [(39_000_000, 1e-5), (1_000_000, 1e-3), (1600, 1e-4), (100_000, 1e-5), (10_000, 0.3),
             (5, 0.01), (1, 0.5), (123_457, 0.0123), (39_000_000, 1 - (1 - 1e-10) ** (1 / 42))]
    for n, p in cases:
        assert L.filter_sizing(n, p, "standard") == oracle.sizing(n, p)
        assert L.filter_sizing(n, p, "blocked") == oracle.sizing_blocked(n, p)
    for bad in ((0, 0.1), (10, 0.0), (10, 1.0)):
        with pytest.raises(L.LSHBloomError):
            L.filter_sizing(*bad)


def test_invalid_configurations_are_refused_before_any_device_work(built):
    """lshbloom_create_ex validates the whole configuration first: each
    violated rule gives LSHB_ERR_ARG and a message naming it, on a host with
    or without a GPU."""
    import numpy as np

    import paper_2411_04257_gb300 as L
    bad = [
        (dict(P=0), "num_perm"), (dict(P=2000), "num_perm"), (dict(bands=0), "bands"),
        (dict(bands=65, rows=1, P=128), "bands"), (dict(rows=0), "rows"),
        (dict(P=100, bands=11, rows=11), "exceeds num_perm"), (dict(ngram=0), "ngram"),
        (dict(ngram=65), "ngram"), (dict(n_expected=0), "n_expected"),
        (dict(fp_rate=0.0), "fp_rate"), (dict(fp_rate=1.0), "fp_rate"),
        (dict(item_shingles=8), "item_shingles"), (dict(fp_rate=1e-25), "exceeds 64"),
        (dict(perm_a=np.ones(121, np.uint64), perm_b=np.full(121, 2**61, np.uint64)), "perm_b"),
        (dict(perm_a=np.zeros(121, np.uint64), perm_b=np.zeros(121, np.uint64)), "perm_a"),
    ]
    for kw, word in bad:
        P = kw.pop("P", 121)
        bands = kw.pop("bands", 11)
        rows = kw.pop("rows", 11)
        with pytest.raises(L.LSHBloomError) as e:
            L.LSHBloom(P, bands, rows, **kw)
        assert e.value.status == -1 and word in str(e.value), (kw, str(e.value))
    with pytest.raises(KeyError):
        L.LSHBloom(121, 11, 11, bloom_layout="striped")


def test_optimal_br_matches_the_oracle_on_the_host(built, oracle):
    """lshbloom_optimal_br is host code: (b, r) for thresholds and permutation
    counts equal the oracle's tuner (Eqs. 1-2), including the paper's 9 bands
    at T = 0.8, P = 128 and 42 x 6 at T = 0.5, P = 256."""
    import paper_2411_04257_gb300 as L
    assert L.optimal_br(0.8, 128) == (9, 13)
    assert L.optimal_br(0.5, 256) == (42, 6)
    for T in (0.3, 0.5, 0.65, 0.8, 0.9):
        for P in (32, 64, 121, 128, 200):
            assert L.optimal_br(T, P) == oracle.optimal_br(T, P), (T, P)
