"""Pins of the CPU oracle to things other than itself.

Each test checks one oracle function against an independent source: a
library routine (hashlib, Python big integers, numpy), a published test
vector, a number the paper prints, or a closed form.  A plausible slip in the
oracle (a dropped term, a wrong sign, a transposed operand, a wrong modulus)
fails at least one of them.
"""
import hashlib
import json
import math
import os
import random

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden")
P61 = (1 << 61) - 1


def _golden(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


# --- SHA-1 (FIPS 180-4) against hashlib ------------------------------------

@pytest.mark.parametrize("length", [0, 1, 3, 4, 20, 52, 55, 56, 57, 63, 64, 65, 100, 119, 120,
                                    127, 128, 129, 300])
def test_sha1_matches_hashlib(oracle, length):
    rnd = random.Random(length)
    msg = bytes(rnd.getrandbits(8) for _ in range(length))
    assert oracle.sha1(msg) == hashlib.sha1(msg).digest()


def test_sha1_fips_examples(oracle):
    # FIPS 180-4 / FIPS 180-2 Appendix A example messages.
    assert oracle.sha1(b"abc").hex() == "a9993e364706816aba3e25717850c26c9cd0d89d"
    assert oracle.sha1(
        b"abcdbcdecdefdefgefghfghighijhijkijkljklmklmnlmnomnopnopq").hex() == \
        "84983e441c3bd26ebaae4aa1f95129e5e54670f1"


@pytest.mark.parametrize("n", [1, 2, 5, 7, 13, 14, 26, 40])
def test_shingle_hash_is_sha1_prefix(oracle, n):
    """Sec. 4.1/4.3 reading: SHA-1 of the little-endian token bytes, first four
    digest bytes as a little-endian uint32."""
    rnd = np.random.default_rng(n)
    for _ in range(20):
        toks = rnd.integers(0, 2**32, size=n, dtype=np.uint64).astype(np.uint32)
        want = int.from_bytes(hashlib.sha1(toks.astype("<u4").tobytes()).digest()[:4], "little")
        assert oracle.shingle_hash(toks) == want


# --- SplitMix64 published vector and coefficient ranges ---------------------

def test_splitmix64_published_vector(oracle):
    g = _golden("splitmix64.json")
    st = g["seed"]
    got = []
    for _ in range(5):
        st = (st + 0x9E3779B97F4A7C15) % 2**64
        got.append(oracle.mix64(st))
    assert got == g["outputs"]


def test_coefficients_follow_the_stream(oracle):
    """a_i = 1 + x mod (p-2), b_i = x' mod p from the SplitMix64 stream."""
    g = _golden("splitmix64.json")
    a, b = oracle.coefficients(g["seed"], 2)
    outs = g["outputs"]
    assert int(a[0]) == 1 + outs[0] % (P61 - 1)
    assert int(b[0]) == outs[1] % P61
    assert int(a[1]) == 1 + outs[2] % (P61 - 1)
    assert int(b[1]) == outs[3] % P61
    a, b = oracle.coefficients(1, 512)
    assert np.all(a >= 1) and np.all(a <= P61 - 2)
    assert np.all(b <= P61 - 1)
    assert len(set(a.tolist())) == 512


# --- the permutation (a h + b) mod (2^61 - 1), low 32 bits -----------------

def test_perm_against_big_integers(oracle):
    rnd = random.Random(7)
    cases = [(1, 0, 0), (1, 0, 2**32 - 1), (P61 - 2, P61 - 1, 2**32 - 1), (P61 - 2, 0, 1),
             (2**32, 0, 2**32 - 1), (2**61 - 3, 2**61 - 2, 2**31), (12345, P61 - 1, 1)]
    for _ in range(3000):
        cases.append((rnd.randrange(1, P61 - 1), rnd.randrange(0, P61), rnd.getrandbits(32)))
    for a, b, h in cases:
        assert oracle.perm(a, b, h) == ((a * h + b) % P61) & 0xFFFFFFFF


def test_perm_mersenne_identities(oracle):
    """Closed forms of the Mersenne modulus: 2^61 = 1 (mod p), so a = 2^s
    rotates h inside 61 bits; a = p - 1 = -1 maps h to p - h."""
    rnd = random.Random(3)
    for _ in range(500):
        h = rnd.getrandbits(32)
        s = rnd.randrange(0, 61)
        rot = ((h << s) | (h >> (61 - s))) & P61 if s else h
        assert oracle.perm(1 << s, 0, h) == rot & 0xFFFFFFFF
        assert oracle.perm(P61 - 1, 0, h) == ((P61 - h) % P61) & 0xFFFFFFFF


def test_perm_hits_the_reduction_boundary(oracle):
    """Inputs chosen so a h + b lands exactly on multiples of p and next to them."""
    rnd = random.Random(11)
    for _ in range(300):
        h = rnd.getrandbits(32) | 1
        a = rnd.randrange(1, P61 - 1)
        for want in (0, 1, P61 - 1, P61 - 2, 2**32 - 1, 2**32):
            # b = want - a h (mod p) makes the residue exactly `want`.
            b = (want - a * h) % P61
            assert oracle.perm(a, b, h) == want & 0xFFFFFFFF


# --- signatures and band keys ----------------------------------------------

def _shingle_set_hashes(tokens, n):
    toks = np.asarray(tokens, np.uint32)
    L = toks.size
    if L == 0:
        return set()
    w = n if L >= n else L
    out = set()
    for s in range(0, max(L - n + 1, 1) if L >= n else 1):
        b = toks[s:s + w].astype("<u4").tobytes()
        out.add(int.from_bytes(hashlib.sha1(b).digest()[:4], "little"))
    return out


def test_signature_with_identity_permutation_is_min_sha1(oracle):
    """a = 1, b = 0 is the identity on h < 2^32, so every signature entry is the
    smallest SHA-1-derived shingle hash (computed here with hashlib)."""
    rnd = np.random.default_rng(5)
    for L in [0, 1, 3, 4, 5, 6, 17, 200]:
        toks = rnd.integers(0, 1000, size=L).astype(np.uint32)
        a = np.ones(4, np.uint64)
        b = np.zeros(4, np.uint64)
        sig = oracle.signature(toks, 5, a, b)
        hs = _shingle_set_hashes(toks, 5)
        want = min(hs) if hs else 0xFFFFFFFF
        assert np.all(sig == want), L


def test_signature_is_a_set_function(oracle):
    """Sec. 2.2: the signature depends only on the shingle set.  Repeating the
    document (adding only shingles already present, plus the seam windows)
    and reordering whole shingle-preserving blocks must keep a signature built
    only over the shared set."""
    a, b = oracle.coefficients(9, 64)
    toks = np.arange(40, dtype=np.uint32)
    s1 = oracle.signature(toks, 1, a, b)
    s2 = oracle.signature(toks[::-1].copy(), 1, a, b)      # same unigram set
    s3 = oracle.signature(np.concatenate([toks, toks]), 1, a, b)
    assert np.array_equal(s1, s2) and np.array_equal(s1, s3)


def test_signature_brute_force_tiny(oracle):
    """Definition written out with hashlib and Python big integers."""
    a, b = oracle.coefficients(2, 16)
    rnd = np.random.default_rng(8)
    for L in [1, 2, 4, 5, 6, 9, 30]:
        toks = rnd.integers(0, 50, size=L).astype(np.uint32)
        hs = _shingle_set_hashes(toks, 5)
        want = [min(((int(a[i]) * h + int(b[i])) % P61) & 0xFFFFFFFF for h in hs)
                for i in range(16)]
        assert oracle.signature(toks, 5, a, b).tolist() == want


def test_minhash_collision_rate_is_jaccard(oracle):
    """Sec. 2.2: P(sig_i(A) = sig_i(B)) = J(A, B).  Sets of distinct unigrams with
    exact Jaccard J; the mean equality rate over 4000 set pairs x 32 perms
    must sit inside a 99.9% interval of J."""
    a, b = oracle.coefficients(21, 32)
    rnd = np.random.default_rng(1)
    for N, c in [(60, 40), (60, 15)]:
        J = c / (2 * N - c)
        eq = 0
        tot = 0
        for t in range(1500):
            base = rnd.choice(2**31, size=2 * N - c, replace=False).astype(np.uint32)
            A = base[:N]
            B = np.concatenate([base[:c], base[N:]])
            sa = oracle.signature(A, 1, a, b)
            sb = oracle.signature(B, 1, a, b)
            eq += int(np.sum(sa == sb))
            tot += 32
        rate = eq / tot
        # Per-perm equalities within one pair are independent given the pair.
        sd = math.sqrt(J * (1 - J) / tot)
        assert abs(rate - J) < 3.3 * sd + 2e-3, (N, c, rate, J)


def test_band_keys_are_row_sums(oracle):
    rnd = np.random.default_rng(4)
    sig = rnd.integers(0, 2**32, size=121, dtype=np.uint64).astype(np.uint32)
    keys = oracle.band_keys(sig, 11, 11)
    want = sig[:121].astype(np.uint64).reshape(11, 11).sum(axis=1)
    assert np.array_equal(keys, want)
    # The all-max signature of an empty document: each key is r (2^32 - 1).
    full = np.full(121, 0xFFFFFFFF, np.uint32)
    assert np.all(oracle.band_keys(full, 11, 11) == 11 * 0xFFFFFFFF)
    # Only the first b*r rows take part.
    keys2 = oracle.band_keys(np.concatenate([sig[:110], np.zeros(11, np.uint32)]), 10, 11)
    assert np.array_equal(keys2, want[:10])


# --- probe positions ---------------------------------------------------------

def test_probe_positions_power_of_two_m_is_a_shift(oracle):
    """With m = 2^s the multiply-high range reduction is the top s bits."""
    rnd = random.Random(2)
    for _ in range(200):
        key = rnd.getrandbits(64)
        j = rnd.randrange(0, 50)
        s = rnd.randrange(8, 40)
        q = oracle.probe_positions(key, j, 1 << s, 17)
        x = oracle.mix64(key ^ ((j * 0x9E3779B97F4A7C15) % 2**64))
        y = oracle.mix64(x ^ 0x6A09E667F3BCC909) | 1
        want = [(((x + u * y) % 2**64) >> (64 - s)) for u in range(17)]
        assert q.tolist() == want


def test_probe_positions_range_and_uniformity(oracle):
    m = 239872
    counts = np.zeros(64, np.int64)
    rnd = random.Random(5)
    for _ in range(4000):
        q = oracle.probe_positions(rnd.getrandbits(64), rnd.randrange(11), m, 17)
        assert np.all(q < m)
        np.add.at(counts, (q * 64 // m).astype(np.int64), 1)
    exp = 4000 * 17 / 64
    chi2 = float(((counts - exp) ** 2 / exp).sum())
    assert chi2 < 120.0  # 63 dof, p ~ 1e-5


# --- sizing and the numbers the paper prints --------------------------------

def test_sizing_reproduces_the_10B_doc_example(oracle):
    g = _golden("paper_numbers.json")["index_10B_docs"]
    p = oracle.p_from_effective(g["p_eff"], g["bands"])
    m, k = oracle.sizing(g["n"], p)
    gb = g["bands"] * m / 8 / 1e9
    assert abs(gb - g["gigabytes"]) <= g["tolerance_gb"]


def test_sizing_reproduces_the_pes2o_index(oracle):
    g = _golden("paper_numbers.json")["pes2o_index"]
    b, r = oracle.optimal_br(g["T"], g["P"])
    p = oracle.p_from_effective(g["p_eff"], b)
    m, _ = oracle.sizing(g["n"], p)
    assert abs(b * m / 8 / 1e9 - g["gigabytes"]) <= g["tolerance_gb"]


def test_sizing_reproduces_table2(oracle):
    g = _golden("paper_numbers.json")["table2"]
    for row in g["rows"]:
        pe = 1.0 / row["N"] if row["p_eff"] == "1/N" else row["p_eff"]
        p = oracle.p_from_effective(pe, g["bands"])
        m, _ = oracle.sizing(row["N"], p)
        tb = g["bands"] * m / 8 / 1e12
        assert abs(tb - row["terabytes"]) <= g["tolerance_tb"] + 0.005, row


def test_sizing_closed_form_and_rounding(oracle):
    for n, p in [(10_000, 1e-5), (39_000_000, 1e-5), (1, 0.5), (12345, 1e-3)]:
        m, k = oracle.sizing(n, p)
        exact = -n * math.log(p) / math.log(2) ** 2
        assert m % 256 == 0 and exact <= m < exact + 257
        assert k == max(1, round(m / n * math.log(2)))
    # The 10k-document plain workload: k = 17, 239,872 bits.
    assert oracle.sizing(10_000, 1e-5) == (239872, 17)


def test_effective_rate_round_trip(oracle):
    for pe, b in [(1e-5, 11), (1e-10, 9), (0.01, 42)]:
        p = oracle.p_from_effective(pe, b)
        assert abs(oracle.effective_from_p(p, b) - pe) < 1e-6 * pe + 1e-16
        assert abs(p - (1 - (1 - pe) ** (1 / b))) < 1e-18 + 1e-9 * p


def test_optimal_bands_match_the_paper(oracle):
    g = _golden("paper_numbers.json")["bands_for_T08_P128"]
    b, r = oracle.optimal_br(g["T"], g["P"])
    assert b == g["bands"] and b * r <= g["P"]


def test_lsh_error_integrals_closed_forms(oracle):
    """Eqs. 1-2: with b = r = 1 the integrands are t and 1 - t."""
    for T in [0.2, 0.5, 0.8]:
        assert abs(oracle.fp_lsh(T, 1, 1) - T * T / 2) < 1e-12
        assert abs(oracle.fn_lsh(T, 1, 1) - (1 - T) ** 2 / 2) < 1e-12
        # b = 1, r = 2: integral of t^2 and of 1 - t^2.
        assert abs(oracle.fp_lsh(T, 1, 2) - T ** 3 / 3) < 1e-12
        assert abs(oracle.fn_lsh(T, 1, 2) - ((1 - T) - (1 - T ** 3) / 3)) < 1e-12
    # Eqs. 3-4 reduce to the LSH terms when p_eff = 0 and N is infinite.
    assert oracle.fp_bloom(0.1, 0.0, 11, float("inf")) == 0.1
    assert oracle.fn_bloom(0.1, 0.0, 11, float("inf")) == 0.1
    assert abs(oracle.fp_bloom(0.1, 1e-3, 10, 2.0**32) - (0.1 + 0.9 * (1e-3 + 10 / 2**32))) < 1e-15
