"""The seeded corpus generator: determinism, shape, and planted similarity."""
import hashlib

import numpy as np

from synth import corpus


def test_generator_is_deterministic_and_sliceable():
    spec = corpus.CorpusSpec(n_docs=500, seed=3, length_median=50, length_min=5,
                             length_max=400, dup_frac=0.3)
    off, tok = corpus.generate(spec)
    off2, tok2 = corpus.generate(spec)
    assert np.array_equal(off, off2) and np.array_equal(tok, tok2)
    # Any window of documents is the same bytes as in the full corpus.
    o, t = corpus.generate(spec, d0=123, D=77, max_tokens_per_pass=1000)
    assert np.array_equal(t, tok[int(off[123]):int(off[200])])
    assert np.array_equal(o, off[123:201] - off[123])


def test_lengths_follow_the_law():
    spec = corpus.plain_10k()
    t = corpus.build_tables(spec)
    lens = corpus.own_length(t, np.arange(20000, dtype=np.uint64)).astype(np.float64)
    assert lens.min() >= 50 and lens.max() <= 5000
    assert abs(np.median(lens) - 400) < 20
    p = corpus.pareto_batched()
    tp = corpus.build_tables(p)
    lp = corpus.own_length(tp, np.arange(200000, dtype=np.uint64)).astype(np.float64)
    assert lp.min() >= 20 and lp.max() <= 200_000
    assert lp.max() > 20_000          # the heavy tail reaches far
    assert 60 < lp.mean() < 160


def test_zipf_word_frequencies():
    spec = corpus.CorpusSpec(n_docs=200, seed=1, length_median=500, length_min=500,
                             length_max=500, dup_frac=0.0)
    _, tok = corpus.generate(spec)
    t = corpus.build_tables(spec)
    # rank-1 and rank-2 word frequencies are in ratio 2^1.1
    c1 = np.sum(tok == t.word_hash[0])
    c2 = np.sum(tok == t.word_hash[1])
    assert 1.6 < c1 / c2 < 2.7


def test_planted_duplicates():
    spec = corpus.pes2o_shaped(n_docs=3000)
    t = corpus.build_tables(spec)
    d = np.arange(3000, dtype=np.uint64)
    frac = corpus.is_dup(t, d).mean()
    assert 0.08 < frac < 0.12
    pairs = corpus.planted_pairs(spec, 0, 3000, tables=t)
    assert np.all(pairs[:, 1] < pairs[:, 0])
    # Shingle-set Jaccard of a few planted pairs is near the 0.6-0.95 range.
    js = []
    for dd, ss in pairs[:8]:
        od, td = corpus.generate(spec, d0=int(dd), D=1, tables=t)
        os_, ts = corpus.generate(spec, d0=int(ss), D=1, tables=t)
        A = {td[i:i + 5].tobytes() for i in range(len(td) - 4)}
        B = {ts[i:i + 5].tobytes() for i in range(len(ts) - 4)}
        js.append(len(A & B) / len(A | B))
    assert min(js) > 0.35 and max(js) < 0.999


def test_tables_digest_is_stable():
    """The tables are the recipe: any change to them changes every corpus."""
    t = corpus.build_tables(corpus.plain_10k())
    h = hashlib.sha256()
    for arr in (t.zipf_cdf, t.word_hash, t.length, t.mut_thr):
        h.update(np.ascontiguousarray(arr).tobytes())
    h.update(str(t.dup_thr).encode())
    assert len(h.hexdigest()) == 64
    off, tok = corpus.generate(corpus.CorpusSpec(n_docs=10, seed=0))
    assert off[-1] == tok.size and tok.dtype == np.uint32
