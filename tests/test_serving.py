"""Serving: continuous batching over resident indexes.

A request's flags must be exactly those it gets when the same requests are
run alone, one lshbloom_dedup call after another in submission order on fresh
indexes — whatever else shares the GPU with it, and however admission by
memory budget interleaves them."""
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


def _requests(n_req=60, seed=3, max_docs=300):
    """Requests cut from one corpus with many near-duplicates, so documents of
    one request duplicate documents of earlier requests."""
    from synth import corpus
    rnd = np.random.default_rng(seed)
    sizes = np.maximum(1, np.exp(rnd.uniform(0, np.log(max_docs), n_req)).astype(int))
    spec = corpus.CorpusSpec(n_docs=int(sizes.sum()), seed=seed, length_median=250, length_min=0,
                             length_max=3000, dup_frac=0.35, dup_lo=0.0, dup_hi=0.05)
    off, tok = corpus.generate(spec)
    reqs, d = [], 0
    for s in sizes:
        o = off[d:d + s + 1].copy()
        reqs.append((int(rnd.integers(0, 4)), o, tok))
        d += s
    return reqs


def _sequential(lshb, reqs, **kw):
    ixs = [lshb.LSHBloom(121, 11, 11, n_expected=5000, fp_rate=1e-4, **kw) for _ in range(4)]
    out = [np.asarray(ixs[i].dedup(o, tok)) for i, o, tok in reqs]
    return out, ixs


def _served(lshb, reqs, budget=1 << 28, inflight=16, **kw):
    ixs = [lshb.LSHBloom(121, 11, 11, n_expected=5000, fp_rate=1e-4, **kw) for _ in range(4)]
    srv = lshb.LSHBloomServer(ixs, mem_budget_bytes=budget, max_inflight=inflight)
    tickets = []
    for i, o, tok in reqs:
        # each request gets its own rebased copy, as a client would send it
        lo, hi = int(o[0]), int(o[-1])
        tickets.append(srv.submit(i, o - o[0], tok[lo:hi].copy()))
    res = [srv.wait(t) for t in tickets]
    srv.close()
    return [f for f, _ in res], [lat for _, lat in res], ixs


def test_served_equals_alone(lshb):
    reqs = _requests()
    want, ref_ixs = _sequential(lshb, reqs)
    got, lat, ixs = _served(lshb, reqs)
    for k, (g, w) in enumerate(zip(got, want)):
        assert np.array_equal(g, w), f"request {k} differs"
    assert sum(int(w.sum()) for w in want) > 50
    for a, b in zip(ixs, ref_ixs):
        for j in range(11):
            assert np.array_equal(a.filter_bytes(j), b.filter_bytes(j))
    assert all(x > 0 for x in lat)


def test_served_matches_oracle(lshb, oracle):
    reqs = _requests(n_req=25, seed=8, max_docs=120)
    got, _, _ = _served(lshb, reqs)
    refs = [oracle.OracleIndex(121, 11, 11, n_expected=5000, fp_rate=1e-4) for _ in range(4)]
    for (i, o, tok), g in zip(reqs, got):
        assert np.array_equal(g, refs[i].dedup(o, tok))


def test_tight_budget_serialises_but_agrees(lshb):
    """Requests copied into the budget (staged host inputs), at most one or
    two of the largest in flight: same flags as plain sequential calls."""
    reqs = _requests(n_req=30, seed=5)
    want, _ = _sequential(lshb, reqs, exec_mode="plain")
    biggest = max(int(o[-1] - o[0]) * 4 + len(o) * 8 + (len(o) - 1) * 97 + 1024
                  for _, o, _ in reqs)
    got, _, _ = _served(lshb, reqs, budget=biggest + 4096, inflight=3, stage_host_inputs=True)
    for g, w in zip(got, want):
        assert np.array_equal(g, w)


def test_served_staged_equals_in_place(lshb):
    """The same requests with their tokens copied into the budget and read in
    place (where the device can) give the same flags and filters."""
    reqs = _requests(n_req=40, seed=12)
    a, _, ia = _served(lshb, reqs, stage_host_inputs=True)
    b, _, ib = _served(lshb, reqs)
    for g, w in zip(a, b):
        assert np.array_equal(g, w)
    for x, y in zip(ia, ib):
        for j in range(11):
            assert np.array_equal(x.filter_bytes(j), y.filter_bytes(j))


def test_oversize_request_and_timeouts(lshb):
    ix = lshb.LSHBloom(121, 11, 11, stage_host_inputs=True)
    srv = lshb.LSHBloomServer([ix], mem_budget_bytes=1 << 16, max_inflight=2)
    off = np.array([0, 100_000], np.uint64)
    tok = np.arange(100_000, dtype=np.uint32)
    with pytest.raises(lshb.LSHBloomError) as e:     # 400 KB of tokens to copy
        srv.submit(0, off, tok)
    assert e.value.status == -7
    many = np.arange(0, 2001, dtype=np.uint64)       # 2000 one-token documents:
    with pytest.raises(lshb.LSHBloomError) as e:     # 176 KB of band keys alone
        srv.submit(0, many, np.arange(2000, dtype=np.uint32))
    assert e.value.status == -7
    bad = np.array([0, 5, 3], np.uint64)
    with pytest.raises(lshb.LSHBloomError) as e:
        srv.submit(0, bad, np.arange(5, dtype=np.uint32))
    assert e.value.status == -2
    t = srv.submit(0, np.array([0, 50, 120], np.uint64), np.arange(120, dtype=np.uint32))
    try:
        flags, lat = srv.wait(t, timeout_ms=0.0)
    except lshb.LSHBloomError as err:   # still running: a host-side timeout, then done
        assert err.status == -5
        flags, lat = srv.wait(t)
    assert flags.tolist() == [0, 0] and lat > 0
    srv.close()
    ix.close()


@pytest.mark.parametrize("layout,band_key", [("blocked", "weighted"), ("exact", "sum")])
def test_served_other_layouts_equal_alone(lshb, layout, band_key):
    """The server drives the Bloom stage of any layout and band-key mode: each
    request's flags equal plain sequential calls on indexes of that kind."""
    reqs = _requests(n_req=30, seed=17)
    kw = dict(bloom_layout=layout, band_key=band_key)
    want, _ = _sequential(lshb, reqs, **kw)
    got, _, _ = _served(lshb, reqs, **kw)
    for g, w in zip(got, want):
        assert np.array_equal(g, w)
