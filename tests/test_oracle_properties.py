"""Statistical and structural properties of the oracle's index.

* the LSH S-curve 1 - (1 - s^r)^b on planted pairs of exact Jaccard s
  (the curve behind Eqs. 1-2);
* the Bloom false-positive closed form (1 - e^{-kn/m})^k (Sec. 2.4);
* no false negatives against an exact band-bucket index (the MinHashLSH
  hash map of Sec. 2.3) replayed on the oracle's own insert decisions;
* the stream decision of Sec. 2.1 on small hand-checked streams.
"""
import math

import numpy as np
import pytest


def _binom_ok(hits, n, p, z=3.3):
    sd = math.sqrt(max(p * (1 - p), 1e-12) / n)
    return abs(hits / n - p) <= z * sd + 1.0 / n


def _csr(docs):
    lens = np.array([len(d) for d in docs], np.uint64)
    off = np.zeros(len(docs) + 1, np.uint64)
    np.cumsum(lens, out=off[1:])
    toks = np.concatenate([np.asarray(d, np.uint32) for d in docs]) if docs else \
        np.zeros(0, np.uint32)
    return off, toks


@pytest.mark.parametrize("s", [0.5, 0.7, 0.8, 0.9])
def test_s_curve_on_planted_pairs(oracle, s):
    """Pairs (A, B) of unigram sets with Jaccard exactly s, each pair on its own
    token range.  B is flagged when some band collides with A; the flag rate
    must match 1 - (1 - s^r)^b within a 99.9% binomial interval."""
    b, r = 11, 11
    rnd = np.random.default_rng(int(s * 100))
    N = 100
    # |A n B| = c, |A u B| = 2N - c, J = c / (2N - c)  ->  c = 2 N s / (1 + s)
    c = int(round(2 * N * s / (1 + s)))
    J = c / (2 * N - c)
    pairs = 1500
    docs = []
    for t in range(pairs):
        base = (t * 1000 + rnd.permutation(2 * N - c)).astype(np.uint32) + 1
        docs.append(base[:N])
        docs.append(np.concatenate([base[:c], base[N:]]))
    off, toks = _csr(docs)
    ix = oracle.OracleIndex(121, b, r, n_expected=10 * len(docs), fp_rate=1e-9, ngram=1,
                            seed=3)
    flags = ix.dedup(off, toks)
    want = 1 - (1 - J ** r) ** b
    hits = int(flags[1::2].sum())
    assert _binom_ok(hits, pairs, want), (hits / pairs, want)
    # The first of each pair has no earlier similar document.
    assert int(flags[0::2].sum()) <= 3


def test_bloom_false_positive_closed_form(oracle):
    """Insert n random keys into one filter sized for n at p = 1e-5, query 4M
    fresh keys: the hit rate must match (1 - e^{-kn/m})^k."""
    n = 10_000
    ix = oracle.OracleIndex(11, 11, 1, n_expected=n, fp_rate=1e-5)
    rnd = np.random.default_rng(12)
    keys = rnd.integers(0, 2**63, size=n, dtype=np.uint64) * np.uint64(2) + np.uint64(1)
    ix.insert_keys(0, keys)
    assert ix.query_keys(0, keys).all()  # no false negatives
    fresh = rnd.integers(0, 2**63, size=4_000_000, dtype=np.uint64) * np.uint64(2)
    fp = int(ix.query_keys(0, fresh).sum())
    m, k = ix.m, ix.k
    want = (1 - math.exp(-k * n / m)) ** k
    lam = want * fresh.size
    assert abs(fp - lam) <= 4 * math.sqrt(lam) + 2, (fp, lam)
    # The filter fill matches 1 - e^{-kn/m} as well.
    fill = ix.popcount(0) / m
    assert abs(fill - (1 - math.exp(-k * n / m))) < 0.01


def test_no_false_negatives_against_exact_band_buckets(oracle):
    """Replay the stream against an exact band-bucket index (hash maps of the
    r-row bands, as MinHashLSH stores them) fed with the documents the oracle
    inserted.  Every document with an exact band match must be flagged, and
    flags without one must be rare."""
    from synth import corpus
    spec = corpus.CorpusSpec(n_docs=3000, seed=4, length_median=120, length_min=10,
                             length_max=800, dup_frac=0.3, dup_lo=0.0, dup_hi=0.1)
    off, toks = corpus.generate(spec)
    P, b, r = 121, 11, 11
    ix = oracle.OracleIndex(P, b, r, n_expected=3000, fp_rate=1e-4, ngram=5, seed=1)
    flags = ix.dedup(off, toks)
    sigs = oracle.batch_signatures(off, toks, 5, ix.a, ix.b)
    buckets = [set() for _ in range(b)]
    exact = np.zeros(len(flags), bool)
    for i in range(len(flags)):
        bands = [tuple(sigs[i, j * r:(j + 1) * r].tolist()) for j in range(b)]
        exact[i] = any(bands[j] in buckets[j] for j in range(b))
        if not flags[i]:
            for j in range(b):
                buckets[j].add(bands[j])
    assert np.all(flags[exact] == 1)
    extra = int(np.sum(flags.astype(bool) & ~exact))
    # p_eff = 1 - (1 - 1e-4)^11 ~ 1.1e-3 per document at full load.
    assert extra <= 12, extra
    assert exact.sum() > 300  # the planted duplicates are found


def test_identical_documents_stream(oracle):
    doc = np.arange(100, 400, dtype=np.uint32)
    off, toks = _csr([doc] * 6)
    ix = oracle.OracleIndex(121, 11, 11)
    assert ix.dedup(off, toks).tolist() == [0, 1, 1, 1, 1, 1]
    # A second call continues the same stream.
    assert ix.dedup(off, toks).tolist() == [1] * 6
    assert ix.docs_seen == 12


def test_query_before_insert_and_modes(oracle):
    """A document never matches itself (query comes first); with insert-all a
    duplicate's bits are still inserted, which the default mode skips."""
    A = np.arange(0, 300, dtype=np.uint32)
    B = np.arange(10_000, 10_300, dtype=np.uint32)
    off, toks = _csr([A, A, B])
    for insert_all in (False, True):
        ix = oracle.OracleIndex(121, 11, 11, insert_all=insert_all)
        assert ix.dedup(off, toks).tolist() == [0, 1, 0]
    # Filters after [A, A]: identical for both modes (A's bits either way).
    ix1 = oracle.OracleIndex(121, 11, 11)
    ix2 = oracle.OracleIndex(121, 11, 11, insert_all=True)
    off2, toks2 = _csr([A, A])
    ix1.dedup(off2, toks2)
    ix2.dedup(off2, toks2)
    for j in range(11):
        assert np.array_equal(ix1.filter_bytes(j), ix2.filter_bytes(j))
        assert ix1.popcount(j) <= 17


def test_empty_and_short_documents(oracle):
    """Readings: an empty document has no shingle (all-max signature), so a
    second empty document is a duplicate of the first; a document shorter than
    n has one shingle made of all its tokens."""
    e = np.zeros(0, np.uint32)
    s3 = np.array([5, 6, 7], np.uint32)
    off, toks = _csr([e, s3, e, s3, np.array([5, 6, 7, 8], np.uint32)])
    ix = oracle.OracleIndex(121, 11, 11, ngram=5)
    assert ix.dedup(off, toks).tolist() == [0, 0, 1, 1, 0]


def test_filters_fill_monotonically(oracle):
    from synth import corpus
    spec = corpus.CorpusSpec(n_docs=400, seed=9, length_median=80, length_min=5,
                             length_max=300)
    off, toks = corpus.generate(spec)
    ix = oracle.OracleIndex(121, 11, 11, n_expected=400)
    prev = [0] * 11
    for s in range(0, 400, 50):
        sub = off[s:s + 51] - off[s]
        ix.dedup(sub, toks[int(off[s]):int(off[min(s + 50, 400)])])
        cur = [ix.popcount(j) for j in range(11)]
        assert all(c >= p for c, p in zip(cur, prev))
        prev = cur


def test_batch_split_does_not_change_flags(oracle):
    """The stream semantics do not depend on how the stream is cut into calls."""
    from synth import corpus
    spec = corpus.CorpusSpec(n_docs=600, seed=2, length_median=60, length_min=3,
                             length_max=300, dup_frac=0.4, dup_lo=0.0, dup_hi=0.05)
    off, toks = corpus.generate(spec)
    whole = oracle.OracleIndex(121, 11, 11, n_expected=600).dedup(off, toks)
    ix = oracle.OracleIndex(121, 11, 11, n_expected=600)
    parts = []
    for s, e in [(0, 1), (1, 250), (250, 251), (251, 600)]:
        parts.append(ix.dedup(off[s:e + 1], toks))
    assert np.array_equal(np.concatenate(parts), whole)
    assert whole.sum() > 100


# --- the blocked layout (a variant beyond the paper) ---------------------------

def _blocked_fp_model(n, m, k, B=256):
    """Blocked Bloom filter with k independent positions per key inside one
    B-bit block (Putze, Sanders, Singler 2007), exact under that model: keys
    per block ~ Poisson(n B / m); a block hit by i keys has Z set bits, the
    occupancy of i k draws into B cells; a query with D distinct positions is
    a false positive with probability C(Z, D) / C(B, D)."""
    def occupancy(draws):
        d = [0.0] * (B + 1)
        d[0] = 1.0
        for _ in range(draws):
            nd = [0.0] * (B + 1)
            for z, p in enumerate(d):
                if p:
                    nd[z] += p * z / B
                    if z < B:
                        nd[z + 1] += p * (B - z) / B
            d = nd
        return d
    lam = n * B / m
    dq = occupancy(k)[:k + 1]
    tot = 0.0
    for i in range(int(4 * lam) + 40):
        w = math.exp(-lam + i * math.log(lam) - math.lgamma(i + 1))
        if w < 1e-14:
            continue
        s = 0.0
        for z, pz in enumerate(occupancy(i * k)):
            if pz > 1e-16:
                s += pz * sum(pd * math.comb(z, D) / math.comb(B, D)
                              for D, pd in enumerate(dq) if pd and D <= z)
        tot += w * s
    return tot


def test_blocked_positions_share_one_block(oracle):
    rnd = np.random.default_rng(4)
    m = 1 << 20
    blocks = []
    for _ in range(3000):
        key = int(rnd.integers(0, 2**63))
        j = int(rnd.integers(0, 11))
        q = oracle.probe_positions_blocked(key, j, m, 17)
        assert len(set((q >> 8).tolist())) == 1 and np.all(q < m)
        x = oracle.mix64(key ^ ((j * 0x9E3779B97F4A7C15) % 2**64))
        assert int(q[0] >> 8) == x >> (64 - 12)     # m/256 = 2^12 blocks: the top bits of x
        blocks.append(int(q[0] >> 8))
    counts = np.bincount(np.array(blocks) * 64 // 4096, minlength=64)
    exp = 3000 / 64
    assert float(((counts - exp) ** 2 / exp).sum()) < 120.0


@pytest.mark.parametrize("fp", [1e-5, 1e-3])
def test_blocked_false_positive_closed_form(oracle, fp):
    """At the standard layout's m and k (explicitly given: a blocked index
    otherwise sizes itself by its own rule), the blocked rate of the oracle's
    index follows the model, the oracle's own model agrees with this one, and
    both are above the standard rate."""
    n = 100_000
    mm, kk = oracle.sizing(n, fp)
    ix = oracle.OracleIndex(11, 11, 1, n_expected=n, fp_rate=fp, layout=1, m=mm, k=kk)
    rnd = np.random.default_rng(31)
    keys = rnd.integers(0, 2**63, size=n, dtype=np.uint64) * np.uint64(2) + np.uint64(1)
    ix.insert_keys(0, keys)
    assert ix.query_keys(0, keys).all()           # still no false negatives
    fresh = rnd.integers(0, 2**63, size=3_000_000, dtype=np.uint64) * np.uint64(2)
    rate = float(ix.query_keys(0, fresh).mean())
    want = _blocked_fp_model(n, ix.m, ix.k)
    std = (1 - math.exp(-ix.k * n / ix.m)) ** ix.k
    assert abs(rate / want - 1) < 0.25, (rate, want)
    assert rate > 1.5 * std                       # blocking costs accuracy at equal m
    assert oracle.fp_blocked(n, ix.m, ix.k) == pytest.approx(want, rel=1e-9)


def test_blocked_model_reduces_to_the_standard_filter_at_k1(oracle):
    """With one position per key the blocks are just cells of one flat
    filter: the blocked rate is the standard 1 - exp(-n/m)."""
    for n, m in ((1000, 256_000), (50_000, 256 * 1000), (7, 256), (10**6, 256 * 10**5)):
        assert oracle.fp_blocked(n, m, 1) == pytest.approx(1 - math.exp(-n / m), rel=1e-12)


def _stirling2(n, k):
    row = [1] + [0] * k                           # S(0, j)
    for i in range(1, n + 1):
        new = [0] * (k + 1)
        for j in range(1, min(i, k) + 1):
            new[j] = j * row[j] + row[j - 1]
        row = new
    return row[k]


def test_blocked_hit_matches_the_occupancy_formula(oracle):
    """P(a query's k positions are all set | i keys in the block) =
    E[(Z/256)^k], Z the occupied cells after i k uniform draws, with
    P(Z = s) = C(256, s) s! S(ik, s) / 256^(ik) (Stirling numbers of the
    second kind), summed in exact rationals."""
    from fractions import Fraction
    for i, k in ((0, 5), (1, 1), (1, 2), (1, 5), (2, 3), (3, 4), (6, 1), (4, 6)):
        draws = i * k
        want = Fraction(0)
        for z in range(0, min(draws, 256) + 1):
            pz = Fraction(math.comb(256, z) * math.factorial(z) * _stirling2(draws, z),
                          256 ** draws)
            want += pz * Fraction(z, 256) ** k
        assert oracle.blocked_hit(i, k) == pytest.approx(float(want), rel=1e-11, abs=1e-300)


def test_blocked_sizing_meets_its_target_on_fresh_keys(oracle):
    """An index sized by the blocked rule for p = 1e-3 shows that rate on
    3M keys it never saw (about 3,000 false positives: +-2% noise)."""
    n, p = 100_000, 1e-3
    m, k = oracle.sizing_blocked(n, p)
    ix = oracle.OracleIndex(11, 11, 1, n_expected=n, fp_rate=p, layout=1)
    assert (ix.m, ix.k) == (m, k)
    rnd = np.random.default_rng(77)
    keys = rnd.integers(0, 2**63, size=n, dtype=np.uint64) * np.uint64(2) + np.uint64(1)
    ix.insert_keys(3, keys)
    fresh = rnd.integers(0, 2**63, size=3_000_000, dtype=np.uint64) * np.uint64(2)
    rate = float(ix.query_keys(3, fresh).mean())
    model = oracle.fp_blocked(n, m, k)
    assert model <= p
    assert abs(rate / model - 1) < 0.1, (rate, model)


@pytest.mark.parametrize("n,p", [(39_000_000, 1e-5), (1_000_000, 1e-3), (1600, 1e-4),
                                 (10_000, 0.3), (5, 0.01)])
def test_blocked_sizing_is_the_fewest_blocks(oracle, n, p):
    """The blocked rule returns a whole number of blocks that meets p, one
    block fewer meets it for no k in the searched range, and it never needs
    fewer bits than the standard filter."""
    m, k = oracle.sizing_blocked(n, p)
    ms, ks = oracle.sizing(n, p)
    assert m % 256 == 0 and m >= ms
    assert oracle.fp_blocked(n, m, k) <= p
    if m > 256:
        for kk in range(1, min(64, ks + 8) + 1):
            assert oracle.fp_blocked(n, m - 256, kk) > p


def test_exact_key_sets_equal_a_set_replay(oracle):
    """Layout 2 (exact band-key sets, the MinHashLSH bucket rule on band keys)
    equals a replay with Python sets; the Bloom index flags a superset (no
    false negatives) and the difference is its false positives."""
    from synth import corpus
    spec = corpus.CorpusSpec(n_docs=2500, seed=6, length_median=100, length_min=0,
                             length_max=600, dup_frac=0.35, dup_lo=0.0, dup_hi=0.1)
    off, toks = corpus.generate(spec)
    ex = oracle.OracleIndex(121, 11, 11, n_expected=2500, fp_rate=1e-3, layout=2)
    bl = oracle.OracleIndex(121, 11, 11, n_expected=2500, fp_rate=1e-3)
    fe, fb = ex.dedup(off, toks), bl.dedup(off, toks)
    sigs = oracle.batch_signatures(off, toks, 5, ex.a, ex.b)
    keys = sigs[:, :121].astype(np.uint64).reshape(-1, 11, 11).sum(axis=2)
    sets = [set() for _ in range(11)]
    want = np.zeros(len(fe), np.uint8)
    for i in range(len(fe)):
        want[i] = any(int(keys[i, j]) in sets[j] for j in range(11))
        if not want[i]:
            for j in range(11):
                sets[j].add(int(keys[i, j]))
    assert np.array_equal(fe, want)
    # The Bloom index differs only by its false positives (which, not being
    # inserted, can also unflag a later copy): the totals stay close.
    assert abs(int(fb.sum()) - int(fe.sum())) <= 25
    for j in (0, 5, 10):
        assert ex.exact_keys(j).tolist() == sorted(sets[j])


def test_blocked_stream_semantics(oracle):
    doc = np.arange(100, 400, dtype=np.uint32)
    off, toks = _csr([doc, doc, np.arange(5000, 5300, dtype=np.uint32)])
    ix = oracle.OracleIndex(121, 11, 11, layout=1)
    assert ix.dedup(off, toks).tolist() == [0, 1, 0]
    for j in range(11):
        assert ix.popcount(j) <= 2 * 17


# --- weighted band keys (a variant beyond the paper) ------------------------------

def test_weighted_band_keys_separate_what_sums_merge(oracle):
    """Band tuples of small values, as minima of long documents are: their
    plain sums (the paper's keys) collapse onto a few thousand values, while
    the weighted sums keep every distinct tuple distinct; mode 0 is the plain
    row sum; the same tuple in two bands gets two keys."""
    rnd = np.random.default_rng(91)
    n, r = 20_000, 11
    tuples = rnd.integers(0, 512, size=(n, r), dtype=np.uint32)
    distinct = len({t.tobytes() for t in tuples})
    sums = {int(oracle.band_keys(t, 1, r)[0]) for t in tuples}
    weighted = {int(oracle.band_keys(t, 1, r, mode=1)[0]) for t in tuples}
    assert len(sums) < 6_000 < distinct
    assert len(weighted) == distinct
    t = tuples[0]
    assert int(oracle.band_keys(t, 1, r)[0]) == int(t.astype(np.uint64).sum())
    two = oracle.band_keys(np.concatenate([t, t]), 2, r, mode=1)
    assert two[0] != two[1]
    # keys are linear in the tuple (a weighted sum): k(x + y) = k(x) + k(y) mod 2^64
    x, y = tuples[1] // 2, tuples[2] // 2
    kx, ky, kxy = (int(oracle.band_keys(v, 1, r, mode=1)[0]) for v in (x, y, x + y))
    assert kxy == (kx + ky) % 2**64
