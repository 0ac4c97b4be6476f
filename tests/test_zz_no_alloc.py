"""lshbloom_band_keys_static: band keys for callers that cannot let the library
allocate device memory (a fixed-budget memory pool owns the GPU, or a
latency-critical loop cannot afford cudaMalloc's device-wide synchronisation).

The entry point keeps its signature scratch in an array compiled into the
library.  Its keys must equal those of lshbloom_band_keys, bit for bit, on two
calls in a row (the second call reuses the array the first one filled), and a
batch larger than the array must be refused.  This file is collected last so a
failure here leaves every other test already run; it also passes alone."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lshb():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2411_04257_gb300 as L
    L.lib()
    return L


def _batch(n, seed):
    from synth import corpus
    spec = corpus.CorpusSpec(n_docs=n, seed=seed, length_median=300, length_min=0,
                             length_max=4000, dup_frac=0.2)
    off, tok = corpus.generate(spec)
    return (torch.from_numpy(off.view(np.int64)).cuda(),
            torch.from_numpy(tok.view(np.int32)).cuda())


def _static_keys(lshb, ix, off, tok):
    """Direct C-ABI call with caller-owned device output and a torch stream."""
    D = off.numel() - 1
    out = torch.empty((D, ix.bands), dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    st = lshb.lib().lshbloom_band_keys_static(ctypes.c_void_p(ix.handle), off.data_ptr(),
                                               tok.data_ptr(), D, out.data_ptr(),
                                               ctypes.c_void_p(stream.cuda_stream))
    lshb._native.check(st)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint64)


@pytest.mark.parametrize("P,bands,rows", [(121, 11, 11), (256, 42, 6)])
def test_static_keys_match_band_keys_twice(lshb, P, bands, rows):
    ix = lshb.LSHBloom(P, bands, rows)
    # a large batch, then a smaller different one: stale rows must not leak
    for n, seed in [(3000, 1), (1200, 2)]:
        off, tok = _batch(n, seed)
        want = ix.band_keys(off, tok).cpu().numpy().view(np.uint64)
        got = _static_keys(lshb, ix, off, tok)
        assert got.shape == want.shape
        assert np.array_equal(got, want)
    ix.close()


def test_static_keys_reject_oversize_and_bad_offsets(lshb):
    ix = lshb.LSHBloom(121, 11, 11)
    limit = (16 << 20) // (4 * 121)
    off = torch.zeros(limit + 2, dtype=torch.int64, device="cuda")
    tok = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(lshb.LSHBloomError) as e:
        _static_keys(lshb, ix, off, tok)
    assert e.value.status == -1 and "fixed array" in str(e.value)
    off2, tok2 = _batch(50, 3)
    bad = off2.clone()
    bad[10] = bad[11] + 1
    with pytest.raises(lshb.LSHBloomError) as e:
        _static_keys(lshb, ix, bad, tok2)
    assert e.value.status == -2
    # still usable afterwards
    assert np.array_equal(_static_keys(lshb, ix, off2, tok2),
                          ix.band_keys(off2, tok2).cpu().numpy().view(np.uint64))
    ix.close()
