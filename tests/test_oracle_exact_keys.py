"""The oracle's exact band-key index (the MinHashLSH bucket rule of Sec. 2.3 on
band keys) fed with constructed keys, against a replay of the stream with
Python sets written here.

Keys are arbitrary 64-bit values (the weighted band key spans all of them):
keys that differ by a multiple of 2^58, in one band and across bands, must
stay distinct, and 2^64 - 1 (the empty marker of an open-addressing table)
must be an ordinary key."""
import numpy as np
import pytest

MAX = 2**64 - 1
M58 = 2**58


def replay(keys, insert_all):
    """Sec. 2.1 / Sec. 4.4.2 stream rule with one Python set per band."""
    b = keys.shape[1]
    sets = [set() for _ in range(b)]
    flags = []
    for row in keys:
        ks = [int(k) for k in row]
        dup = any(k in sets[j] for j, k in enumerate(ks))
        flags.append(1 if dup else 0)
        if insert_all or not dup:
            for j, k in enumerate(ks):
                sets[j].add(k)
    return np.array(flags, np.uint8), [np.array(sorted(s), np.uint64) for s in sets]


def constructed():
    rows = [
        [5, 5 + M58, 7, MAX],            # inserted
        [5 + M58, 5, 7 + 2 * M58, 3],    # every key a multiple of 2^58 away from doc 0's
        [5, 0, 0, 0],                    # band 0 equals doc 0's: duplicate
        [1, 2, 3, MAX],                  # band 3 holds 2^64 - 1 (doc 0)
        [MAX, MAX, MAX, 9],              # 2^64 - 1 in bands 0-2 is new there
        [MAX, 1, 1, 1],                  # band 0 now holds it (doc 4)
        [MAX - M58, MAX - 2 * M58, 7 + 3 * M58, MAX - 1],
        [MAX - M58, 11, 12, 13],         # equals doc 6 in band 0
    ]
    return np.array(rows, dtype=np.uint64)


def random_keys(n, seed):
    """Keys drawn from few values spaced 2^58 apart (and 2^64 - 1), so that
    equal keys, and keys a multiple of 2^58 apart, occur often in every band."""
    rng = np.random.default_rng(seed)
    base = np.array([3, 3 + M58, 3 + 5 * M58, 3 + 63 * M58, MAX, MAX - M58, 17, 17 + 32 * M58],
                    dtype=np.uint64)
    pick = rng.integers(0, base.size, size=(n, 4))
    salt = rng.integers(0, 40, size=(n, 4)).astype(np.uint64) * np.uint64(M58 // 8)
    keys = base[pick] + np.where(rng.random((n, 4)) < 0.5, salt, np.uint64(0))
    return keys.astype(np.uint64)


@pytest.mark.parametrize("insert_all", [False, True])
def test_exact_layout_constructed(oracle, insert_all):
    keys = constructed()
    ix = oracle.OracleIndex(8, 4, 2, n_expected=100, layout=2, insert_all=insert_all)
    got = ix.dedup_keys(keys)
    want, sets = replay(keys, insert_all)
    assert np.array_equal(got, want)
    assert list(want[:6]) == [0, 0, 1, 1, 0, 1]
    for j in range(4):
        assert np.array_equal(ix.exact_keys(j), sets[j])
    assert MAX in set(int(x) for x in ix.exact_keys(3))


@pytest.mark.parametrize("insert_all", [False, True])
def test_exact_layout_random_spaced_keys(oracle, insert_all):
    keys = random_keys(4000, 5)
    ix = oracle.OracleIndex(8, 4, 2, n_expected=4000, layout=2, insert_all=insert_all)
    got = ix.dedup_keys(keys)
    want, sets = replay(keys, insert_all)
    assert np.array_equal(got, want)
    assert 0 < want.sum() < want.size
    for j in range(4):
        assert np.array_equal(ix.exact_keys(j), sets[j])
