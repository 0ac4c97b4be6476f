"""GPU path against the CPU oracle, element by element, through the C ABI.

Everything here is integer work, so the bar is bit-exact: shingle hashes,
signatures, band keys, duplicate flags and the final filter bits."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lshb():
    import paper_2411_04257_gb300 as L
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    L.lib()
    return L


@pytest.fixture(scope="module")
def corpus():
    from synth import corpus as C
    return C


def _dev(off, tok):
    return (torch.from_numpy(np.ascontiguousarray(off).view(np.int64)).cuda(),
            torch.from_numpy(np.ascontiguousarray(tok).view(np.int32)).cuda())


def _csr(docs):
    lens = np.array([len(d) for d in docs], np.uint64)
    off = np.zeros(len(docs) + 1, np.uint64)
    np.cumsum(lens, out=off[1:])
    tok = np.concatenate([np.asarray(d, np.uint32) for d in docs]) if docs else np.zeros(0, np.uint32)
    return off, tok


def _small_corpus(corpus, n=700, seed=5, **kw):
    args = dict(n_docs=n, seed=seed, length_median=150, length_min=0, length_max=3000,
                dup_frac=0.3, dup_lo=0.0, dup_hi=0.08)
    args.update(kw)
    return corpus.generate(corpus.CorpusSpec(**args))


@pytest.mark.parametrize("ngram", [5, 1, 3, 7, 14])
def test_shingle_hashes(lshb, oracle, corpus, ngram):
    off, tok = _small_corpus(corpus, n=300, length_min=0)
    ix = lshb.LSHBloom(121, 11, 11, ngram=ngram)
    got = ix.shingle_hashes(*_dev(off, tok)).cpu().numpy().view(np.uint32)
    want, counts = oracle.batch_shingle_hashes(off, tok, ngram)
    pos = 0
    for d in range(len(off) - 1):
        base = int(off[d])
        c = int(counts[d])
        assert np.array_equal(got[base:base + c], want[pos:pos + c]), d
        pos += c


@pytest.mark.parametrize("P,ngram", [(121, 5), (128, 5), (64, 5), (32, 1), (256, 5), (200, 5),
                                     (48, 7), (121, 1), (121, 3)])
def test_signatures(lshb, oracle, corpus, P, ngram):
    off, tok = _small_corpus(corpus, n=400)
    ix = lshb.LSHBloom(P, 8, 4, ngram=ngram, seed=11)
    a, b = ix.coefficients()
    oa, ob = oracle.coefficients(11, P)
    assert np.array_equal(a, oa) and np.array_equal(b, ob)
    got = ix.signatures(*_dev(off, tok)).cpu().numpy().view(np.uint32)
    want = oracle.batch_signatures(off, tok, ngram, a, b)
    bad = np.nonzero((got != want).any(axis=1))[0]
    assert bad.size == 0, f"signature rows differ: {bad[:10]}"


MERSENNE = (1 << 61) - 1


def _residue_coefficients(oracle, off, tok, P, seed):
    """Coefficients under which, for every permutation i, one chosen shingle
    of one chosen document lands on a residue tau < 2^32 (mostly 0-3):
    b_i = (tau - a_i h) mod p.  With a_i >= 2^40 the integer a h + b is many
    times p, so the Mersenne fold of a h + b + 1 lands at or above 2^61, the
    case whose final conditional subtraction is rarest (probability ~2^-29 on
    random data).  Returns (a, b, which documents, fraction in that case)."""
    hashes, counts = oracle.batch_shingle_hashes(off, tok, 5)
    starts = np.concatenate([[0], np.cumsum(counts.astype(np.int64))])
    rnd = np.random.default_rng(seed)
    docs = [d for d in range(len(counts)) if counts[d] > 0]
    a = np.zeros(P, np.uint64)
    b = np.zeros(P, np.uint64)
    hit_docs, in_case = [], 0
    for i in range(P):
        d = int(docs[rnd.integers(len(docs))])
        h = int(hashes[starts[d] + rnd.integers(int(counts[d]))])
        ai = int(rnd.integers(1 << 40, MERSENNE - 1))
        tau = int(rnd.choice([0, 1, 2, 3, int(rnd.integers(0, 1 << 32))]))
        bi = (tau - ai * h) % MERSENNE
        a[i], b[i] = ai, bi
        y = ai * h + bi + 1
        in_case += ((y & MERSENNE) + (y >> 61)) >= (1 << 61)
        hit_docs.append(d)
    return a, b, sorted(set(hit_docs)), in_case / P


@pytest.mark.parametrize("P", [121, 64, 256])
def test_signatures_at_constructed_residues(lshb, oracle, corpus, P):
    """Both signature kernels (per document, and the batched form with
    64-shingle items, so the residues fall in split documents too) on
    coefficients that put shingles on residues 0-3 through the rare branch
    of the modular reduction.  Compared with the oracle's exact arithmetic."""
    off, tok = _small_corpus(corpus, n=300, seed=21, length_median=400, length_max=6000)
    a, b, hit, frac = _residue_coefficients(oracle, off, tok, P, seed=P)
    assert frac > 0.6                                # the test reaches the case
    want = oracle.batch_signatures(off, tok, 5, a, b)
    rows = 8 if P >= 88 else 4
    ix = lshb.LSHBloom(P, 11, rows, perm_a=a, perm_b=b)
    got = ix.signatures(*_dev(off, tok)).cpu().numpy().view(np.uint32)
    bad = np.nonzero((got != want).any(axis=1))[0]
    assert bad.size == 0, f"signature rows differ: {bad[:10]}"
    assert (want[hit] <= 3).any()
    keys_want = want[:, :11 * rows].astype(np.uint64).reshape(-1, 11, rows).sum(axis=2)
    ixb = lshb.LSHBloom(P, 11, rows, perm_a=a, perm_b=b, exec_mode="batched", item_shingles=64,
                        n_expected=1000)
    _, keys = ixb.dedup_keys(*_dev(off, tok))
    assert np.array_equal(keys.cpu().numpy().view(np.uint64), keys_want)


def test_single_shingle_minimum_of_all_ones(lshb, oracle):
    """Documents of exactly n tokens have one shingle, so its permuted value is
    the signature entry.  Coefficients put that value on 2^32 - 1 (residues
    2^32 - 1 and 2^33 - 1) for half of the permutations: the entry must be
    2^32 - 1, which an accumulation of value + 1 would wrap to 0."""
    rnd = np.random.default_rng(4)
    docs = [rnd.integers(0, 2**32, size=5, dtype=np.uint64).astype(np.uint32) for _ in range(64)]
    docs += [rnd.integers(0, 2**32, size=3, dtype=np.uint64).astype(np.uint32) for _ in range(8)]
    off, tok = _csr(docs)
    hashes, counts = oracle.batch_shingle_hashes(off, tok, 5)
    assert np.all(counts == 1)
    P = 64
    a = rnd.integers(1 << 40, MERSENNE - 1, size=P, dtype=np.uint64)
    b = rnd.integers(0, MERSENNE, size=P, dtype=np.uint64)
    for i in range(0, P, 2):                       # permutation i sends doc i's shingle to -1
        h = int(hashes[i % len(docs)])
        tau = (1 << 32) - 1 if i % 4 == 0 else (1 << 33) - 1
        b[i] = (tau - int(a[i]) * h) % MERSENNE
    want = oracle.batch_signatures(off, tok, 5, a, b)
    assert (want == 0xFFFFFFFF).sum() >= P // 2
    for mode in ("batched", "plain"):
        ix = lshb.LSHBloom(P, 8, 4, perm_a=a, perm_b=b, exec_mode=mode)
        got = ix.signatures(*_dev(off, tok)).cpu().numpy().view(np.uint32)
        assert np.array_equal(got, want), mode
        sig = want.astype(np.uint64)[:, :32].reshape(-1, 8, 4).sum(axis=2)
        _, keys = ix.dedup_keys(*_dev(off, tok))
        assert np.array_equal(keys.cpu().numpy().view(np.uint64), sig), mode


@pytest.mark.parametrize("exec_mode", ["batched", "plain"])
def test_band_keys(lshb, oracle, corpus, exec_mode):
    off, tok = _small_corpus(corpus, n=500)
    ix = lshb.LSHBloom(121, 11, 11, exec_mode=exec_mode)
    got = ix.band_keys(*_dev(off, tok)).cpu().numpy().view(np.uint64)
    sig = oracle.batch_signatures(off, tok, 5, *oracle.coefficients(1, 121))
    want = np.stack([oracle.band_keys(s, 11, 11) for s in sig])
    assert np.array_equal(got, want)


@pytest.mark.parametrize("exec_mode", ["batched", "plain"])
def test_weighted_band_keys(lshb, oracle, corpus, exec_mode, tmp_path):
    """Weighted band keys (beyond the paper): keys of both signature kernels
    and of the batched kernel, then flags and filters over a save/load
    continuation, against the oracle's weighted mode."""
    off, tok = _small_corpus(corpus, n=900, dup_frac=0.4)
    ix = lshb.LSHBloom(121, 11, 11, n_expected=900, band_key="weighted", exec_mode=exec_mode,
                       max_batch_docs=300)
    sig = oracle.batch_signatures(off, tok, 5, *oracle.coefficients(1, 121))
    want_keys = np.stack([oracle.band_keys(g, 11, 11, mode=1) for g in sig])
    assert np.array_equal(ix.band_keys(*_dev(off, tok)).cpu().numpy().view(np.uint64), want_keys)
    ref = oracle.OracleIndex(121, 11, 11, n_expected=900, band_key=1)
    f1, k1 = ix.dedup_keys(*_dev(off[:451], tok))
    assert np.array_equal(k1.cpu().numpy().view(np.uint64), want_keys[:450])
    path = str(tmp_path / "weighted.lshb")
    ix.save(path)
    ix2 = lshb.LSHBloom.load(path)
    got = np.concatenate([f1.cpu().numpy(), ix2.dedup(*_dev(off[450:], tok)).cpu().numpy()])
    want = ref.dedup(off, tok)
    assert np.array_equal(got, want) and want.sum() > 50
    for j in range(11):
        assert np.array_equal(ix2.filter_bytes(j), ref.filter_bytes(j)), f"filter {j}"


def _check_dedup(lshb, oracle, off, tok, calls=None, device_inputs=True, **kw):
    kw.setdefault("n_expected", max(len(off) - 1, 1))
    okw = {k: v for k, v in kw.items() if k in ("n_expected", "fp_rate", "ngram", "seed",
                                                  "insert_all", "fp_is_effective")}
    if "band_key" in kw:
        okw["band_key"] = {"sum": 0, "weighted": 1}[kw["band_key"]]
    ix = lshb.LSHBloom(121, 11, 11, **kw)
    ref = oracle.OracleIndex(121, 11, 11, **okw)
    D = len(off) - 1
    cuts = calls or [0, D]
    got = []
    for s, e in zip(cuts[:-1], cuts[1:]):
        o = off[s:e + 1]
        if device_inputs:
            got.append(ix.dedup(*_dev(o, tok)).cpu().numpy())
        else:
            got.append(np.asarray(ix.dedup(o, tok)))
    got = np.concatenate(got) if got else np.zeros(0, np.uint8)
    want = ref.dedup(off, tok)
    bad = np.nonzero(got != want)[0]
    assert bad.size == 0, f"{bad.size} flags differ, first {bad[:10]}"
    for j in range(11):
        assert np.array_equal(ix.filter_bytes(j), ref.filter_bytes(j)), f"filter {j}"
    st = ix.stats()
    assert st["docs_seen"] == D and st["dups_seen"] == int(want.sum())
    return want, st


@pytest.mark.parametrize("exec_mode", ["batched", "plain"])
@pytest.mark.parametrize("insert_all", [False, True])
def test_dedup_plain_10k_workload(lshb, oracle, corpus, exec_mode, insert_all):
    """The 10,000-document workload (Zipf 50k words, lognormal median 400,
    20% near-duplicates), one call, at its own sizing (n=10k, p=1e-5)."""
    off, tok = corpus.generate(corpus.plain_10k())
    want, st = _check_dedup(lshb, oracle, off, tok, n_expected=10_000, fp_rate=1e-5,
                            exec_mode=exec_mode, insert_all=insert_all)
    # 5-30% substitutions give shingle Jaccard 0.09-0.63, mostly below the
    # ~0.8 threshold of b = r = 11: few are flagged, and all of them exactly.
    assert want.sum() >= 10


@pytest.mark.parametrize("item", [64, 1024, 0])
def test_batched_split_documents_heavy_tail(lshb, oracle, corpus, item):
    """Pareto(1.2) lengths up to 40,000 tokens: with 64-shingle items the long
    documents are split over hundreds of warps and merged by atomicMin; 0
    lets the autotuner pick."""
    spec = corpus.CorpusSpec(n_docs=2500, seed=13, vocab=20_000, length_law="pareto",
                             pareto_alpha=1.2, length_min=20, length_max=40_000, dup_frac=0.3,
                             dup_lo=0.0, dup_hi=0.05)
    off, tok = corpus.generate(spec)
    want, st = _check_dedup(lshb, oracle, off, tok, exec_mode="batched", item_shingles=item)
    assert want.sum() > 100
    assert st["item_shingles"] in (64, 128, 256, 512, 1024)
    if item:
        assert st["item_shingles"] == item


def test_dedup_many_calls_and_small_chunks(lshb, oracle, corpus):
    off, tok = _small_corpus(corpus, n=1500, dup_frac=0.5)
    _check_dedup(lshb, oracle, off, tok, calls=[0, 1, 2, 100, 101, 700, 1500],
                 max_batch_docs=97, max_batch_tokens=5000)


@pytest.mark.parametrize("insert_all", [False, True])
@pytest.mark.parametrize("inputs", ["device", "host_staged"])
def test_pipelined_chunks_match_oracle(lshb, oracle, corpus, insert_all, inputs):
    """Short documents over many chunks.  The first call runs its chunks one
    after the other and measures a Bloom stage that outweighs the signatures,
    so later calls pipeline them: the next chunk's signatures (in the other
    of two signature slots) run while this chunk's Bloom stage does.  Flags
    and every filter byte equal the oracle's over the whole stream."""
    off, tok = _small_corpus(corpus, n=12000, seed=21, length_median=40, length_min=5,
                             length_max=400, dup_frac=0.4)
    want, st = _check_dedup(lshb, oracle, off, tok, calls=[0, 3000, 7000, 12000],
                            device_inputs=inputs == "device", max_batch_docs=1000,
                            insert_all=insert_all, stage_host_inputs=inputs == "host_staged")
    assert want.sum() > 1000
    assert st["pipelined_chunks"] >= 7, st["pipelined_chunks"]


def test_pipelined_chunks_keys_out(lshb, oracle, corpus):
    """lshbloom_dedup_keys on a pipelined handle: each chunk's keys leave its
    signature slot row-major; keys and flags equal the oracle's."""
    off, tok = _small_corpus(corpus, n=6000, seed=22, length_median=40, length_min=5,
                             length_max=400, dup_frac=0.4)
    ix = lshb.LSHBloom(121, 11, 11, n_expected=6000, max_batch_docs=500)
    ref = oracle.OracleIndex(121, 11, 11, n_expected=6000)
    want_keys = oracle.batch_band_keys(off, tok, 5, ref.a, ref.b, 11, 11)
    want = ref.dedup_keys(want_keys)
    first = ix.dedup(*_dev(off[:2001], tok)).cpu().numpy()
    o2 = off[2000:] - off[2000]
    flags, keys = ix.dedup_keys(o2, tok[int(off[2000]):])
    assert ix.stats()["pipelined_chunks"] >= 7
    assert np.array_equal(keys.view(np.uint64), want_keys[2000:])
    assert np.array_equal(np.concatenate([first, np.asarray(flags)]), want)
    for j in (0, 10):
        assert np.array_equal(ix.filter_bytes(j), ref.filter_bytes(j))
    ix.close()


@pytest.mark.parametrize("stage", [True, False])
def test_dedup_host_inputs(lshb, oracle, corpus, stage):
    """Pageable host arrays: staged through device buffers (forced), or read in
    place where the device reads pageable host memory (else staged)."""
    off, tok = _small_corpus(corpus, n=900)
    for mode in ("batched", "plain"):
        want, st = _check_dedup(lshb, oracle, off, tok, device_inputs=False, max_batch_docs=200,
                                exec_mode=mode, stage_host_inputs=stage)
        if stage:
            assert st["host_read_bytes"] == 0 and st["h2d_bytes"] == int(tok.nbytes)
        else:
            assert st["host_read_bytes"] + st["h2d_bytes"] == int(tok.nbytes)


@pytest.mark.parametrize("exec_mode", ["batched", "plain"])
def test_pinned_host_inputs_read_in_place(lshb, oracle, corpus, exec_mode):
    """Page-locked host tensors: the kernels read the tokens through their
    device mapping.  Flags over several calls and chunks, the final filters,
    signatures and band keys all equal the oracle's."""
    off, tok = _small_corpus(corpus, n=1200)
    h_off = torch.from_numpy(off.view(np.int64)).pin_memory()
    h_tok = torch.from_numpy(tok.view(np.int32)).pin_memory()
    ix = lshb.LSHBloom(121, 11, 11, n_expected=1200, exec_mode=exec_mode, max_batch_docs=300)
    ref = oracle.OracleIndex(121, 11, 11, n_expected=1200)
    got = np.concatenate([np.asarray(ix.dedup(h_off[:601], h_tok)),
                          np.asarray(ix.dedup(h_off[600:], h_tok))])
    want = ref.dedup(off, tok)
    assert np.array_equal(got, want) and want.sum() > 20
    st = ix.stats()
    assert st["host_read_bytes"] == int(tok.nbytes) and st["h2d_bytes"] == 0
    for j in range(11):
        assert np.array_equal(ix.filter_bytes(j), ref.filter_bytes(j)), f"filter {j}"
    sig = np.asarray(ix.signatures(h_off[:401], h_tok)).view(np.uint32)
    osig = oracle.batch_signatures(off[:401], tok, 5, *oracle.coefficients(1, 121))
    assert np.array_equal(sig, osig)
    keys = np.asarray(ix.band_keys(h_off, h_tok)).view(np.uint64)
    osig = oracle.batch_signatures(off, tok, 5, *oracle.coefficients(1, 121))
    assert np.array_equal(keys, osig[:, :121].astype(np.uint64).reshape(-1, 11, 11).sum(axis=2))


def test_identical_documents(lshb, oracle):
    doc = np.arange(1000, 1600, dtype=np.uint32)
    off, tok = _csr([doc] * 3000)
    want, st = _check_dedup(lshb, oracle, off, tok)
    assert want.tolist() == [0] + [1] * 2999


def test_duplicate_chains_in_one_batch(lshb, oracle):
    """d_{i+1} is a near-copy of d_i: long dependence chains inside one call
    force many resolution sweeps (or the in-order fallback)."""
    rnd = np.random.default_rng(3)
    docs = [rnd.integers(0, 1 << 30, size=400).astype(np.uint32)]
    for i in range(300):
        nxt = docs[-1].copy()
        nxt[rnd.integers(0, 400, size=6)] = rnd.integers(0, 1 << 30, size=6)
        docs.append(nxt)
    off, tok = _csr(docs)
    for insert_all in (False, True):
        _check_dedup(lshb, oracle, off, tok, insert_all=insert_all, fp_rate=1e-3)


def test_empty_short_and_long_documents(lshb, oracle):
    rnd = np.random.default_rng(9)
    docs = [np.zeros(0, np.uint32), np.array([1, 2, 3], np.uint32), np.zeros(0, np.uint32),
            np.array([1, 2, 3], np.uint32), np.array([7], np.uint32),
            rnd.integers(0, 1 << 31, size=200_000).astype(np.uint32),
            np.array([7], np.uint32), np.array([1, 2, 3, 4], np.uint32)]
    docs += [rnd.integers(0, 50, size=rnd.integers(0, 12)).astype(np.uint32) for _ in range(400)]
    docs.append(docs[5].copy())
    off, tok = _csr(docs)
    want, _ = _check_dedup(lshb, oracle, off, tok, n_expected=1000)
    assert want[2] == 1 and want[3] == 1 and want[6] == 1 and want[-1] == 1


@pytest.mark.parametrize("exec_mode", ["batched", "plain"])
def test_blocked_layout(lshb, oracle, corpus, exec_mode, tmp_path):
    """The 256-bit blocked filter layout against the oracle's blocked mode:
    flags and every filter bit, then a save/load continuation."""
    off, tok = _small_corpus(corpus, n=1600, dup_frac=0.4)
    ix = lshb.LSHBloom(121, 11, 11, n_expected=1600, fp_rate=1e-4, bloom_layout="blocked",
                       exec_mode=exec_mode, max_batch_docs=700)
    ref = oracle.OracleIndex(121, 11, 11, n_expected=1600, fp_rate=1e-4, layout=1)
    got = ix.dedup(*_dev(off[:1001], tok)).cpu().numpy()
    path = str(tmp_path / "blocked.lshb")
    ix.save(path)
    ix2 = lshb.LSHBloom.load(path)
    got = np.concatenate([got, ix2.dedup(*_dev(off[1000:], tok)).cpu().numpy()])
    want = ref.dedup(off, tok)
    assert np.array_equal(got, want)
    assert want.sum() > 100
    for j in range(11):
        fb = ix2.filter_bytes(j)
        assert np.array_equal(fb, ref.filter_bytes(j))


@pytest.mark.parametrize("exec_mode", ["batched", "plain"])
def test_exact_key_index(lshb, oracle, corpus, exec_mode):
    """Exact band-key sets (the MinHashLSH bucket rule on band keys) against the
    oracle's exact mode: flags, and every band's key set."""
    off, tok = _small_corpus(corpus, n=1800, dup_frac=0.4)
    ix = lshb.LSHBloom(121, 11, 11, n_expected=1800, bloom_layout="exact", exec_mode=exec_mode,
                       max_batch_docs=800)
    ref = oracle.OracleIndex(121, 11, 11, n_expected=1800, layout=2)
    got = np.concatenate([ix.dedup(*_dev(off[:901], tok)).cpu().numpy(),
                          ix.dedup(*_dev(off[900:], tok)).cpu().numpy()])
    want = ref.dedup(off, tok)
    assert np.array_equal(got, want)
    for j in range(11):
        assert np.array_equal(ix.exact_keys(j), ref.exact_keys(j))
    st = ix.stats()
    # 4096 key slots, the slot of the key 2^64-1 and 15 padding slots
    assert st["k"] == 1 and st["filter_bytes"] == (4096 + 16) * 8


@pytest.mark.parametrize("ngram", [1, 7])
def test_dedup_other_ngrams(lshb, oracle, corpus, ngram):
    off, tok = _small_corpus(corpus, n=800)
    _check_dedup(lshb, oracle, off, tok, ngram=ngram)


@pytest.mark.parametrize("P", [300, 1024])
def test_signatures_several_passes(lshb, oracle, corpus, P):
    """More than 256 permutations: the signature runs in passes of up to 256
    (two and four passes here), each folding every shingle again."""
    off, tok = _small_corpus(corpus, n=250)
    ix = lshb.LSHBloom(P, 16, 8, seed=3)
    a, b = ix.coefficients()
    got = ix.signatures(*_dev(off, tok)).cpu().numpy().view(np.uint32)
    want = oracle.batch_signatures(off, tok, 5, a, b)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("exec_mode", ["batched", "plain"])
def test_dedup_many_bands_and_passes(lshb, oracle, corpus, exec_mode):
    """The largest band count (64 bands of 4 rows) on P = 300 (two signature
    passes): flags and all 64 filters against the oracle."""
    off, tok = _small_corpus(corpus, n=900, dup_frac=0.4)
    ix = lshb.LSHBloom(300, 64, 4, n_expected=900, fp_rate=1e-4, exec_mode=exec_mode,
                       max_batch_docs=400)
    ref = oracle.OracleIndex(300, 64, 4, n_expected=900, fp_rate=1e-4)
    got = np.concatenate([ix.dedup(*_dev(off[:451], tok)).cpu().numpy(),
                          ix.dedup(*_dev(off[450:], tok)).cpu().numpy()])
    want = ref.dedup(off, tok)
    assert np.array_equal(got, want) and want.sum() > 50
    for j in range(64):
        assert np.array_equal(ix.filter_bytes(j), ref.filter_bytes(j)), f"filter {j}"


@pytest.mark.parametrize("ngram", [13, 14, 64])
def test_long_ngrams_around_the_document_length(lshb, oracle, ngram):
    """n = 13 (the largest single-block SHA-1 message), 14 (two blocks) and 64
    (five blocks), on documents of 0 .. 3n tokens, so that shorter-than-n,
    exactly-n and longer documents all occur."""
    rnd = np.random.default_rng(ngram)
    lens = list(range(0, 3 * ngram + 2)) + list(rnd.integers(0, 400, size=60))
    docs = [rnd.integers(0, 2**32, size=int(L), dtype=np.uint64).astype(np.uint32) for L in lens]
    docs += [docs[-1].copy(), docs[ngram].copy()]           # exact copies
    off, tok = _csr(docs)
    ix = lshb.LSHBloom(121, 11, 11, ngram=ngram, n_expected=len(docs))
    a, b = ix.coefficients()
    got = ix.signatures(*_dev(off, tok)).cpu().numpy().view(np.uint32)
    assert np.array_equal(got, oracle.batch_signatures(off, tok, ngram, a, b))
    flags = ix.dedup(*_dev(off, tok)).cpu().numpy()
    want = oracle.OracleIndex(121, 11, 11, ngram=ngram, n_expected=len(docs)).dedup(off, tok)
    assert np.array_equal(flags, want) and want[-2:].tolist() == [1, 1]


def test_largest_probe_count(lshb, oracle, corpus):
    """p = 1e-18 per filter sizes k = 60 probes per key (the limit is 64)."""
    off, tok = _small_corpus(corpus, n=700)
    want, st = _check_dedup(lshb, oracle, off, tok, n_expected=700, fp_rate=1e-18)
    assert st["k"] == oracle.sizing(700, 1e-18)[1] and 56 <= st["k"] <= 64


def test_sizing_matches_oracle(lshb, oracle):
    for n, p, eff in [(10_000, 1e-5, False), (39_000_000, 1e-5, False), (1234, 0.01, False),
                      (10_000, 1e-10, True), (5_000, 1e-3, True)]:
        ix = lshb.LSHBloom(121, 11, 11, n_expected=n, fp_rate=p, fp_is_effective=eff)
        pp = oracle.p_from_effective(p, 11) if eff else p
        assert (ix.m, ix.k) == oracle.sizing(n, pp), (n, p)
        ix.close()


def test_save_load_continues_the_stream(lshb, oracle, corpus, tmp_path):
    off, tok = _small_corpus(corpus, n=1000, dup_frac=0.4)
    ix = lshb.LSHBloom(121, 11, 11, n_expected=1000)
    a = ix.dedup(*_dev(off[:501], tok)).cpu().numpy()
    path = str(tmp_path / "ix.lshb")
    ix.save(path)
    ix.close()
    ix2 = lshb.LSHBloom.load(path)
    b = ix2.dedup(*_dev(off[500:], tok)).cpu().numpy()
    ref = oracle.OracleIndex(121, 11, 11, n_expected=1000)
    want = ref.dedup(off, tok)
    assert np.array_equal(np.concatenate([a, b]), want)
    assert ix2.stats()["docs_seen"] == 1000


def test_reset_and_errors(lshb, corpus):
    off, tok = _small_corpus(corpus, n=50)
    ix = lshb.LSHBloom(121, 11, 11)
    f1 = ix.dedup(*_dev(off, tok)).cpu().numpy()
    ix.reset()
    f2 = ix.dedup(*_dev(off, tok)).cpu().numpy()
    assert np.array_equal(f1, f2)
    bad = off.copy()
    bad[10] = bad[11] + 1
    with pytest.raises(lshb.LSHBloomError) as e:
        ix.dedup(*_dev(bad, tok))
    assert e.value.status == -2
    assert ix.stats()["docs_seen"] == 50
    with pytest.raises(lshb.LSHBloomError):
        lshb.LSHBloom(121, 12, 11)
    assert ix.dedup(*_dev(off[:1], tok)).numel() == 0


@pytest.mark.parametrize("layout,band_key", [("standard", "weighted"), ("blocked", "sum"),
                                             ("blocked", "weighted"), ("exact", "sum"),
                                             ("exact", "weighted")])
@pytest.mark.parametrize("insert_all", [False, True])
@pytest.mark.parametrize("exec_mode", ["batched", "plain"])
def test_option_combinations(lshb, oracle, corpus, layout, band_key, insert_all, exec_mode):
    """Every filter layout with both band-key modes, both insert rules and
    both forms, over two calls: flags and the final index equal the oracle's."""
    off, tok = _small_corpus(corpus, n=700, seed=31, dup_frac=0.4)
    lay = {"standard": 0, "blocked": 1, "exact": 2}[layout]
    ix = lshb.LSHBloom(121, 11, 11, n_expected=700, fp_rate=1e-4, bloom_layout=layout,
                       band_key=band_key, insert_all=insert_all, exec_mode=exec_mode)
    ref = oracle.OracleIndex(121, 11, 11, n_expected=700, fp_rate=1e-4, layout=lay,
                             band_key=1 if band_key == "weighted" else 0, insert_all=insert_all)
    got = np.concatenate([ix.dedup(*_dev(off[:351], tok)).cpu().numpy(),
                          ix.dedup(*_dev(off[350:], tok)).cpu().numpy()])
    want = ref.dedup(off, tok)
    assert np.array_equal(got, want) and want.sum() > 30
    for j in (0, 5, 10):
        fb = ix.filter_bytes(j)
        if layout == "exact":
            assert np.array_equal(ix.exact_keys(j), ref.exact_keys(j))
        else:
            assert np.array_equal(fb, ref.filter_bytes(j))


def _chain_keys(n, bands=4):
    """Document i shares one band key with document i-1 only (band 0 and band 1
    alternately): under the insert-non-duplicates rule every decision depends
    on the previous one, a chain of n documents."""
    i = np.arange(n, dtype=np.uint64)
    keys = np.zeros((n, bands), np.uint64)
    keys[:, 0] = (i + np.uint64(1)) // np.uint64(2)
    keys[:, 1] = i // np.uint64(2) + np.uint64(10**6)
    for j in range(2, bands):
        keys[:, j] = i * np.uint64(bands) + np.uint64(j) + np.uint64(10**9)
    return keys


@pytest.mark.parametrize("layout,lay", [("standard", 0), ("blocked", 1), ("exact", 2)])
@pytest.mark.parametrize("insert_all", [False, True])
def test_dedup_from_keys_matches_oracle(lshb, oracle, layout, lay, insert_all):
    """lshbloom_dedup_from_keys on arbitrary 64-bit band keys: equal keys, keys
    a multiple of 2^58 apart in one band and across bands, 2^64 - 1, and a
    2,000-document dependency chain (more than the 64 Jacobi sweeps, so the
    in-order finish runs), in chunks of 1,000 documents, from host and device
    memory; flags and the final index equal the oracle's replay of the keys."""
    from test_oracle_exact_keys import constructed, random_keys
    keys = np.concatenate([constructed(), random_keys(3000, 9), _chain_keys(2000)])
    kw = dict(n_expected=6000, fp_rate=1e-3, insert_all=insert_all)
    ix = lshb.LSHBloom(8, 4, 2, bloom_layout=layout, max_batch_docs=1000, **kw)
    ref = oracle.OracleIndex(8, 4, 2, layout=lay, **kw)
    assert (ix.m, ix.k) == (ref.m, ref.k) or layout == "exact"
    got = np.concatenate([
        np.asarray(ix.dedup_from_keys(keys[:8])),
        ix.dedup_from_keys(torch.from_numpy(keys[8:2500].view(np.int64)).cuda()).cpu().numpy(),
        np.asarray(ix.dedup_from_keys(keys[2500:]))])
    want = ref.dedup_keys(keys)
    diff = np.nonzero(got != want)[0]
    assert diff.size == 0, diff[:10]
    assert 0 < want.sum() < want.size
    for j in range(4):
        if layout == "exact":
            assert np.array_equal(ix.exact_keys(j), ref.exact_keys(j))
        else:
            assert np.array_equal(ix.filter_bytes(j), ref.filter_bytes(j))
    st = ix.stats()
    assert st["docs_seen"] == keys.shape[0]
    if not insert_all:
        assert st["resolve_rounds"] > 64          # the chain outlasted the sweeps
    ix.close()


@pytest.mark.parametrize("exec_mode", ["batched", "plain"])
def test_dedup_keys_host_buffers_several_chunks(lshb, oracle, corpus, exec_mode):
    """lshbloom_dedup_keys with host offsets, tokens, flags and keys, over
    chunks of 300 documents: the batched form keeps the keys band-major on the
    device and hands them back row-major; keys and flags equal the oracle's."""
    off, tok = _small_corpus(corpus, n=1000, seed=12)
    ix = lshb.LSHBloom(121, 11, 11, n_expected=1000, exec_mode=exec_mode, max_batch_docs=300)
    flags, keys = ix.dedup_keys(off, tok)
    ref = oracle.OracleIndex(121, 11, 11, n_expected=1000)
    want_keys = oracle.batch_band_keys(off, tok, 5, ref.a, ref.b, 11, 11)
    assert isinstance(keys, np.ndarray) and keys.shape == (1000, 11)
    assert np.array_equal(keys.view(np.uint64), want_keys)
    assert np.array_equal(np.asarray(flags), ref.dedup_keys(want_keys))
    for j in (0, 10):
        assert np.array_equal(ix.filter_bytes(j), ref.filter_bytes(j))
    ix.close()
