"""Bit-exact parity at the workloads' full sizes, in the launch configuration
bench.py times (batched form, whole batch per call, default chunking).

For every document the oracle computes the band keys (shingling, SHA-1,
MinHash, band sums: Sec. 2.2, Sec. 4.1) from its tokens; those are per
document, so the host's cores share the documents (the unchanged
single-threaded oracle on each thread).  The keys the GPU judged with must
equal them for every document.  The oracle then replays the stream decision
(Sec. 2.1, Sec. 4.2, Sec. 4.4.2) from its own keys, one document after the
other, and the GPU's flags must equal its flags for every document and the
GPU's filters its filters, byte for byte.  The CPU tests check that this
replay equals the oracle's one-document loop."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

P, BANDS, ROWS, NGRAM = 121, 11, 11, 5


@pytest.fixture(scope="module")
def lshb():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2411_04257_gb300 as L
    L.lib()
    return L


def _check_exact(lshb, oracle, spec, n_expected, calls=1):
    """Deduplicate `spec` in `calls` calls on the GPU and on the oracle;
    compare every band key, every flag and every filter byte."""
    from synth import gpu as sgpu
    gen = sgpu.DeviceCorpus(spec)
    ix = lshb.LSHBloom(P, BANDS, ROWS, n_expected=n_expected, fp_rate=1e-5)
    ref = oracle.OracleIndex(P, BANDS, ROWS, n_expected=n_expected, fp_rate=1e-5)
    assert (ix.m, ix.k) == (ref.m, ref.k)
    threads = oracle.host_threads()
    per = spec.n_docs // calls
    flags = []
    for c in range(calls):
        off, tok = gen.generate(c * per, per)
        torch.cuda.synchronize()
        f, k = ix.dedup_keys(off, tok)
        torch.cuda.synchronize()
        off_h = off.cpu().numpy().view(np.uint64)
        tok_h = tok.cpu().numpy().view(np.uint32)
        got_keys = k.cpu().numpy().view(np.uint64)
        got = f.cpu().numpy()
        del off, tok, f, k
        want_keys = oracle.batch_band_keys(off_h, tok_h, NGRAM, ref.a, ref.b, BANDS, ROWS,
                                           threads=threads)
        del tok_h
        bad = np.nonzero((got_keys != want_keys).any(axis=1))[0]
        assert bad.size == 0, f"call {c}: band keys differ for {bad.size} documents: {bad[:8]}"
        want = ref.dedup_keys(want_keys)
        diff = np.nonzero(got != want)[0]
        assert diff.size == 0, f"call {c}: flags differ for {diff.size} documents: {diff[:8]}"
        flags.append(got)
    for j in range(BANDS):
        assert np.array_equal(ix.filter_bytes(j), ref.filter_bytes(j)), f"filter {j} differs"
    ref.close()
    return ix, np.concatenate(flags), gen


def test_pes2o_shaped_1m(lshb, oracle):
    from synth import corpus
    spec = corpus.pes2o_shaped(n_docs=1_000_000)
    ix, flags, gen = _check_exact(lshb, oracle, spec, 39_000_000)
    assert 100_000 < flags.sum() < 200_000
    # the plain form agrees on the whole batch
    off, tok = gen.generate(0, spec.n_docs)
    ixp = lshb.LSHBloom(P, BANDS, ROWS, n_expected=39_000_000, fp_rate=1e-5, exec_mode="plain")
    assert np.array_equal(ixp.dedup(off, tok).cpu().numpy(), flags)
    ixp.close()
    # and so does the batch from page-locked host memory (the bench's e2e leg:
    # 19.7 GB of tokens read in place by the kernels), filters included
    h_off = torch.empty(off.shape, dtype=off.dtype, pin_memory=True)
    h_tok = torch.empty(tok.shape, dtype=tok.dtype, pin_memory=True)
    h_off.copy_(off)
    h_tok.copy_(tok)
    del off, tok
    torch.cuda.empty_cache()
    ixh = lshb.LSHBloom(P, BANDS, ROWS, n_expected=39_000_000, fp_rate=1e-5)
    assert np.array_equal(np.asarray(ixh.dedup(h_off, h_tok)), flags)
    st = ixh.stats()
    assert st["host_read_bytes"] == h_tok.numel() * 4 and st["h2d_bytes"] == 0
    for j in range(BANDS):
        assert np.array_equal(ixh.filter_bytes(j), ix.filter_bytes(j))
    ixh.close()
    ix.close()


def test_pareto_batched_8m(lshb, oracle):
    from synth import corpus
    spec = corpus.pareto_batched(n_docs=8_000_000)
    ix, flags, _ = _check_exact(lshb, oracle, spec, 39_000_000)
    assert flags.sum() > 300_000
    ix.close()


def test_billion_stream_prefix_three_calls(lshb, oracle):
    """First 3M documents of the billion-document stream (sources within a
    1M-document window), generated per call on the device, filters sized for
    n = 1e9 (11 x 3 GB), three calls continuing one stream."""
    from synth import corpus
    spec = corpus.billion_stream(n_docs=3_000_000)
    ix, flags, _ = _check_exact(lshb, oracle, spec, 1_000_000_000, calls=3)
    assert flags.sum() > 20_000
    ix.close()


def test_chunk_autotuner_keeps_the_results(lshb):
    """Calls of at least 2^22 documents tune the batched form's chunk size: the
    first runs with 2^21 documents per chunk, the next four try 2^18 .. 2^21,
    later ones keep the fastest.  Chunking never changes a result: with the
    index cleared before each call, every call gives the same flags."""
    from synth import corpus
    from synth import gpu as sgpu
    n = 1 << 22
    spec = corpus.pareto_batched(n_docs=n)
    off, tok = sgpu.DeviceCorpus(spec).generate(0, n)
    ix = lshb.LSHBloom(P, BANDS, ROWS, n_expected=39_000_000, fp_rate=1e-5)
    first, chunks = None, []
    for _ in range(6):
        ix.reset()
        f = ix.dedup(off, tok).cpu().numpy()
        chunks.append(ix.stats()["chunk_docs"])
        if first is None:
            first = f
        else:
            assert np.array_equal(f, first)
    cands = [1 << 18, 1 << 19, 1 << 20, 1 << 21]
    assert chunks[:4] == [1 << 21, 1 << 18, 1 << 19, 1 << 20]
    assert chunks[4] in cands and chunks[5] == chunks[4]
    assert first.sum() > 100_000
    ix.close()
