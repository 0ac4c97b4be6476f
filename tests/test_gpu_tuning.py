"""(b, r) from a Jaccard threshold and the p_eff interface (Eqs. 1-2, Sec. 4.3,
Sec. 4.5): the library's tuner (Gauss-Legendre quadrature) against the
oracle's (Simpson), and an index created the paper's way."""
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


def test_optimal_br_matches_oracle(lshb, oracle):
    for T in (0.3, 0.5, 0.7, 0.8, 0.9):
        for P in (32, 64, 128, 256):
            assert lshb.optimal_br(T, P) == oracle.optimal_br(T, P), (T, P)
    assert lshb.optimal_br(0.8, 128)[0] == 9      # the paper's example (Sec. 4.5)
    assert lshb.optimal_br(0.5, 256) == (42, 6)   # Table 1 settings


def test_threshold_index_sizing_and_parity(lshb, oracle):
    ix = lshb.LSHBloom.from_threshold(0.5, 256, 39_000_000, 1e-10)
    st = ix.stats()
    assert (st["bands"], st["rows"], st["num_perm"]) == (42, 6, 256)
    p = oracle.p_from_effective(1e-10, 42)
    assert abs(st["fp_rate"] - p) <= 1e-12 * p
    assert (st["m_bits"], st["k"]) == oracle.sizing(39_000_000, p)
    assert abs(42 * st["m_bits"] / 8 / 1e9 - 11.4) < 0.1     # the 11 GB of Sec. 5.4.1
    ix.close()
    # a small stream through a threshold-built index equals the oracle's
    from synth import corpus
    off, tok = corpus.generate(corpus.CorpusSpec(n_docs=600, seed=21, length_median=150,
                                                 length_min=0, length_max=2000, dup_frac=0.3,
                                                 dup_lo=0.0, dup_hi=0.2))
    ix = lshb.LSHBloom.from_threshold(0.5, 256, 600, 1e-6)
    got = ix.dedup(torch.from_numpy(off.view(np.int64)).cuda(),
                   torch.from_numpy(tok.view(np.int32)).cuda()).cpu().numpy()
    ref = oracle.OracleIndex(256, 42, 6, n_expected=600, fp_rate=1e-6, fp_is_effective=True)
    assert np.array_equal(got, ref.dedup(off, tok))
    for j in (0, 17, 41):
        assert np.array_equal(ix.filter_bytes(j), ref.filter_bytes(j))
