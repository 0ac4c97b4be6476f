"""lshbloom_band_keys_static: band keys for callers that cannot let the library
allocate device memory (a fixed-budget memory pool owns the GPU, or a
latency-critical loop cannot afford cudaMalloc's device-wide synchronisation).

With more than 256 permutations the entry point keeps its signature scratch in
an array compiled into the library; with fewer the signature kernel writes the
keys itself.  Its keys must equal those of lshbloom_band_keys, bit for bit, on
two calls in a row (the second call reuses the array the first one filled),
and those of the CPU oracle; a successful call must leave the device's free
memory unchanged; a batch larger than the array, however large, must be
refused before any kernel runs.  This file is collected last so a failure here
leaves every other test already run; it also passes alone."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

STATIC_BYTES = 16 << 20


@pytest.fixture(scope="module")
def lshb():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2411_04257_gb300 as L
    L.lib()
    return L


def _batch_host(n, seed, median=300):
    from synth import corpus
    spec = corpus.CorpusSpec(n_docs=n, seed=seed, length_median=median, length_min=0,
                             length_max=4000, dup_frac=0.2)
    return corpus.generate(spec)


def _to_dev(off, tok):
    return (torch.from_numpy(off.view(np.int64)).cuda(),
            torch.from_numpy(tok.view(np.int32)).cuda())


def _static_call(lshb, ix, off, tok, out):
    """Direct C-ABI call with caller-owned device output on torch's stream."""
    D = off.numel() - 1
    stream = torch.cuda.current_stream()
    return lshb.lib().lshbloom_band_keys_static(ctypes.c_void_p(ix.handle), off.data_ptr(),
                                                 tok.data_ptr(), D, out.data_ptr(),
                                                 ctypes.c_void_p(stream.cuda_stream))


def _static_keys(lshb, ix, off, tok):
    D = off.numel() - 1
    out = torch.empty((D, ix.bands), dtype=torch.int64, device="cuda")
    lshb._native.check(_static_call(lshb, ix, off, tok, out))
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint64)


CASES = [
    # (P, bands, rows, ngram, exec_mode): one pass, the fused kernel writes keys
    (121, 11, 11, 5, "batched"),
    (256, 42, 6, 5, "batched"),
    (121, 11, 11, 3, "batched"),        # run-time n-gram size
    (121, 11, 11, 5, "plain"),          # a handle made for the one-kernel-per-stage form
    # several passes: the signature matrix lives in the fixed array
    (300, 30, 10, 5, "batched"),
    (1024, 64, 16, 7, "batched"),
]


@pytest.mark.parametrize("P,bands,rows,ngram,mode", CASES)
def test_static_keys_match_band_keys_twice(lshb, oracle, P, bands, rows, ngram, mode):
    ix = lshb.LSHBloom(P, bands, rows, ngram=ngram, exec_mode=mode)
    n_max = min(3000, STATIC_BYTES // (4 * P))
    a, b = ix.coefficients()
    # a large batch, then a smaller different one: stale rows must not leak
    for n, seed in [(n_max, 1), (n_max * 2 // 5, 2)]:
        off_h, tok_h = _batch_host(n, seed)
        off, tok = _to_dev(off_h, tok_h)
        want = ix.band_keys(off, tok).cpu().numpy().view(np.uint64)
        got = _static_keys(lshb, ix, off, tok)
        assert got.shape == want.shape
        assert np.array_equal(got, want)
        # the oracle, on the first documents of the batch
        k = 60
        sig = oracle.batch_signatures(off_h[:k + 1], tok_h, ngram, a, b)
        ref = np.stack([oracle.band_keys(sig[d], bands, rows) for d in range(k)])
        assert np.array_equal(got[:k], ref)
    ix.close()


@pytest.mark.parametrize("P,bands,rows", [(121, 11, 11), (300, 30, 10)])
def test_static_keys_allocate_nothing(lshb, P, bands, rows):
    """After one call (which loads the kernels it uses), a second call leaves
    the device's free memory exactly where it was."""
    ix = lshb.LSHBloom(P, bands, rows)
    off_h, tok_h = _batch_host(min(2000, STATIC_BYTES // (4 * P)), 4)
    off, tok = _to_dev(off_h, tok_h)
    out = torch.empty((off.numel() - 1, bands), dtype=torch.int64, device="cuda")
    lshb._native.check(_static_call(lshb, ix, off, tok, out))
    torch.cuda.synchronize()
    first = out.clone()
    free0, _ = torch.cuda.mem_get_info()
    lshb._native.check(_static_call(lshb, ix, off, tok, out))
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.equal(out, first)
    ix.close()


def test_static_keys_reject_oversize_and_bad_offsets(lshb):
    ix = lshb.LSHBloom(300, 30, 10)
    limit = STATIC_BYTES // (4 * 300)
    tok = torch.zeros(1, dtype=torch.int32, device="cuda")
    # stats() itself launches a popcount per band: measure its own share first
    l0 = ix.stats()["kernel_launches"]
    l1 = ix.stats()["kernel_launches"]
    # one past the limit, and a count whose byte size wraps around 2^64
    for D in (limit + 1, 1 << 62):
        off = torch.zeros(2, dtype=torch.int64, device="cuda")
        out = torch.empty(1, dtype=torch.int64, device="cuda")
        st = lshb.lib().lshbloom_band_keys_static(ctypes.c_void_p(ix.handle), off.data_ptr(),
                                                   tok.data_ptr(), D, out.data_ptr(), None)
        assert st == -1, (D, st)
        assert "fixed array" in lshb.lib().lshbloom_last_error().decode()
    assert ix.stats()["kernel_launches"] - l1 == l1 - l0, "a refused call launched a kernel"
    off_h, tok_h = _batch_host(50, 3)
    off2, tok2 = _to_dev(off_h, tok_h)
    bad = off2.clone()
    bad[10] = bad[11] + 1
    with pytest.raises(lshb.LSHBloomError) as e:
        _static_keys(lshb, ix, bad, tok2)
    assert e.value.status == -2
    # still usable afterwards
    assert np.array_equal(_static_keys(lshb, ix, off2, tok2),
                          ix.band_keys(off2, tok2).cpu().numpy().view(np.uint64))
    ix.close()
