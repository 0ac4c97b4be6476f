"""The oracle's stream decision fed with precomputed band keys, and its
threaded driver, against the oracle's own one-document-at-a-time loop.

The full-size parity tests compute every document's band keys with the
oracle on many threads and then replay the stream decision (Sec. 2.1,
Sec. 4.2, Sec. 4.4.2) from those keys.  That is only the oracle if the
split changes nothing: flags, filter bits and exact key sets must equal
or_index_dedup's on the same documents, for every layout, both insert
rules and both band-key modes, whatever the block size and thread count."""
import numpy as np
import pytest

from synth import corpus


@pytest.fixture(scope="module")
def batch():
    spec = corpus.CorpusSpec(n_docs=2500, seed=11, length_median=150, length_min=0,
                             length_max=2500, dup_frac=0.3, dup_lo=0.0, dup_hi=0.1)
    return corpus.generate(spec)


def _same_index(O, x, y, layout, bands):
    for j in range(bands):
        if layout == 2:
            assert np.array_equal(x.exact_keys(j), y.exact_keys(j))
        else:
            assert np.array_equal(x.filter_bytes(j), y.filter_bytes(j))


@pytest.mark.parametrize("layout", [0, 1, 2])
@pytest.mark.parametrize("insert_all", [False, True])
@pytest.mark.parametrize("band_key", [0, 1])
def test_replay_from_keys_equals_dedup(oracle, batch, layout, insert_all, band_key):
    off, tok = batch
    mk = lambda: oracle.OracleIndex(121, 11, 11, n_expected=2500, fp_rate=1e-3,
                                    layout=layout, insert_all=insert_all, band_key=band_key)
    ref, rep, thr = mk(), mk(), mk()
    want = ref.dedup(off, tok)
    keys = oracle.batch_band_keys(off, tok, 5, ref.a, ref.b, 11, 11, band_key)
    assert keys.shape == (2500, 11)
    assert np.array_equal(rep.dedup_keys(keys), want)
    got, used = thr.dedup_threaded(off, tok, threads=3, block_docs=777)
    assert used == 3
    assert np.array_equal(got, want)
    assert want.sum() > 50
    _same_index(oracle, ref, rep, layout, 11)
    _same_index(oracle, ref, thr, layout, 11)
    for ix in (ref, rep, thr):
        assert ix.docs_seen == 2500
        ix.close()


def test_threaded_keys_equal_single_thread(oracle, batch):
    off, tok = batch
    a, b = oracle.coefficients(3, 64)
    one = oracle.batch_band_keys(off, tok, 3, a, b, 8, 8, 0, threads=1)
    many = oracle.batch_band_keys(off, tok, 3, a, b, 8, 8, 0, threads=5)
    assert np.array_equal(one, many)
    sig = oracle.batch_signatures(off[:41], tok, 3, a, b)
    assert np.array_equal(one[:40], np.stack([oracle.band_keys(s, 8, 8) for s in sig[:40]]))


def test_replay_split_across_calls(oracle, batch):
    """Replaying the keys in several calls continues one stream."""
    off, tok = batch
    ref = oracle.OracleIndex(121, 11, 11, n_expected=2500, fp_rate=1e-3)
    want = ref.dedup(off, tok)
    keys = oracle.batch_band_keys(off, tok, 5, ref.a, ref.b, 11, 11)
    rep = oracle.OracleIndex(121, 11, 11, n_expected=2500, fp_rate=1e-3)
    got = np.concatenate([rep.dedup_keys(keys[:1]), rep.dedup_keys(keys[1:1000]),
                          rep.dedup_keys(keys[1000:1000]), rep.dedup_keys(keys[1000:])])
    assert np.array_equal(got, want)
    _same_index(oracle, ref, rep, 0, 11)
