"""Seeded synthetic corpora shaped like the paper's workloads.

This module holds none of the deduplication method's arithmetic.  It makes
CSR batches of uint32 word hashes (``offsets`` uint64[D+1], ``tokens``
uint32[T]) that stand in for the paper's corpora (peS2o and the AdaParse
derived sets are not available): Zipf-distributed words, lognormal or Pareto
document lengths, and planted near-duplicates that copy an earlier document
and substitute a fraction of its tokens.

Every value is a pure function of (seed, field, doc, position) through a
counter-based SplitMix64 mix (Steele, Lea, Flood, OOPSLA 2014), and every
distribution is sampled by an integer comparison against a table built once
on the host in float64.  The CUDA generator in ``synth/synth_gen.cu`` reads
the same tables and the same counters, so the two produce identical bytes;
the tests check that.

Recipe (all fields drawn independently):
  * word id w = first Zipf-CDF entry above rng(TOK, c, pos); token value
    = low 32 bits of mix64(w ^ vocab_key)
  * own length of doc d = length_table[rng(LEN, d, 0) >> 48] (65536
    equiprobable quantiles of the length law, clipped and rounded)
  * doc d > 0 is a near-duplicate when rng(DUP, d, 0) < dup_frac * 2^64; its
    source is d - 1 - rng(SRC, d, 0) mod min(d, window)
  * a near-duplicate takes its root's length; its token at pos is a fresh
    word when rng(MUTPOS, d, pos) < mut_threshold[d], otherwise its source's
    token at pos (followed down the chain, at most 64 links)
"""
from __future__ import annotations

import dataclasses
import math
import statistics

import numpy as np

M64 = (1 << 64) - 1
MAX_CHAIN = 64
LEN_TABLE_BITS = 16
MUT_TABLE_BITS = 10

FIELD_LEN, FIELD_DUP, FIELD_SRC, FIELD_MUT, FIELD_MUTPOS, FIELD_TOK, FIELD_VOCAB = range(1, 8)

_C1 = np.uint64(0xBF58476D1CE4E5B9)
_C2 = np.uint64(0x94D049BB133111EB)
_GOLD = np.uint64(0x9E3779B97F4A7C15)
_FKEY = 0xD1B54A32D192ED03


def _mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser on a uint64 array (wrapping arithmetic)."""
    z = z.astype(np.uint64, copy=True)
    z ^= z >> np.uint64(30)
    z *= _C1
    z ^= z >> np.uint64(27)
    z *= _C2
    z ^= z >> np.uint64(31)
    return z


def _mix_int(z: int) -> int:
    z &= M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def field_key(seed: int, field: int) -> int:
    return _mix_int((seed ^ (field * _FKEY)) & M64)


def rng(seed: int, field: int, i: np.ndarray, j) -> np.ndarray:
    """Counter-based 64-bit draw: mix(key + mix(i * GOLD + j))."""
    with np.errstate(over="ignore"):
        i = np.asarray(i, dtype=np.uint64)
        j = np.asarray(j, dtype=np.uint64)
        inner = _mix(i * _GOLD + j)
        return _mix(np.uint64(field_key(seed, field)) + inner)


@dataclasses.dataclass(frozen=True)
class CorpusSpec:
    n_docs: int
    seed: int = 0
    vocab: int = 50_000
    zipf_s: float = 1.1
    length_law: str = "lognormal"       # "lognormal" | "pareto" | "fixed"
    length_median: float = 400.0        # lognormal median (or fixed length)
    length_sigma: float = 1.0           # lognormal sigma
    pareto_alpha: float = 1.2
    length_min: int = 50
    length_max: int = 5000
    dup_frac: float = 0.20
    dup_mode: str = "mutate"            # "mutate" (rate range) | "jaccard" (target range)
    dup_lo: float = 0.05
    dup_hi: float = 0.30
    ngram: int = 5                      # only used to turn a Jaccard target into a rate
    window: int = 0                     # 0: any earlier doc is a possible source


# The workloads, by what they are.
def plain_10k(seed: int = 0) -> CorpusSpec:
    """10,000 docs, Zipf(1.1) over 50k words, lognormal median 400 (clip
    50-5000), 20% near-duplicates with 5-30% of tokens substituted."""
    return CorpusSpec(n_docs=10_000, seed=seed)


def pes2o_shaped(n_docs: int = 1_000_000, seed: int = 0) -> CorpusSpec:
    """peS2o-shaped: lognormal median 3,000 tokens (clip 200-60,000), Zipf(1.1)
    over 200k words, 10% near-duplicates at Jaccard 0.6-0.95."""
    return CorpusSpec(n_docs=n_docs, seed=seed, vocab=200_000, length_median=3000.0,
                      length_min=200, length_max=60_000, dup_frac=0.10, dup_mode="jaccard",
                      dup_lo=0.6, dup_hi=0.95)


def pareto_batched(n_docs: int = 8_000_000, seed: int = 0) -> CorpusSpec:
    """Heavy-tailed lengths Pareto(alpha=1.2, min 20, clip 200,000), 15%
    near-duplicates at Jaccard 0.6-0.95, Zipf(1.1) over 200k words."""
    return CorpusSpec(n_docs=n_docs, seed=seed, vocab=200_000, length_law="pareto",
                      pareto_alpha=1.2, length_min=20, length_max=200_000, dup_frac=0.15,
                      dup_mode="jaccard", dup_lo=0.6, dup_hi=0.95)


def billion_stream(n_docs: int = 1_000_000_000, seed: int = 0) -> CorpusSpec:
    """Lognormal median 300 tokens (clip 20-20,000), 5% near-duplicates within
    a 1M-document window at Jaccard 0.6-0.95."""
    return CorpusSpec(n_docs=n_docs, seed=seed, vocab=200_000, length_median=300.0,
                      length_min=20, length_max=20_000, dup_frac=0.05, dup_mode="jaccard",
                      dup_lo=0.6, dup_hi=0.95, window=1_000_000)


def serving_requests(seed: int = 0) -> CorpusSpec:
    """Request documents: lognormal median 1,000 tokens (clip 50-20,000), 10%
    near-duplicates at Jaccard 0.6-0.95."""
    return CorpusSpec(n_docs=0, seed=seed, vocab=200_000, length_median=1000.0,
                      length_min=50, length_max=20_000, dup_frac=0.10, dup_mode="jaccard",
                      dup_lo=0.6, dup_hi=0.95)


@dataclasses.dataclass
class Tables:
    zipf_cdf: np.ndarray      # uint64[V], strictly a threshold table
    word_hash: np.ndarray     # uint32[V]
    length: np.ndarray        # uint32[2^16]
    mut_thr: np.ndarray       # uint64[2^10]
    dup_thr: int
    window: int
    seed: int


def _to_u64_threshold(x: np.ndarray) -> np.ndarray:
    y = np.minimum(np.asarray(x, np.float64) * 2.0**64, 2.0**64 - 4096.0)
    return np.maximum(y, 0.0).astype(np.uint64)


def build_tables(spec: CorpusSpec) -> Tables:
    V = int(spec.vocab)
    ranks = np.arange(1, V + 1, dtype=np.float64)
    w = ranks ** (-float(spec.zipf_s))
    cdf = np.cumsum(w) / w.sum()
    zipf = _to_u64_threshold(cdf)
    zipf[-1] = np.uint64(M64)
    vkey = np.uint64(field_key(spec.seed, FIELD_VOCAB))
    word_hash = (_mix(np.arange(V, dtype=np.uint64) ^ vkey) & np.uint64(0xFFFFFFFF)).astype(
        np.uint32)

    nl = 1 << LEN_TABLE_BITS
    u = (np.arange(nl, dtype=np.float64) + 0.5) / nl
    if spec.length_law == "lognormal":
        nd = statistics.NormalDist()
        z = np.array([nd.inv_cdf(float(x)) for x in u])
        L = np.exp(math.log(spec.length_median) + spec.length_sigma * z)
    elif spec.length_law == "pareto":
        L = spec.length_min * (1.0 - u) ** (-1.0 / spec.pareto_alpha)
    elif spec.length_law == "fixed":
        L = np.full(nl, float(spec.length_median))
    else:
        raise ValueError(spec.length_law)
    L = np.clip(np.rint(L), spec.length_min, spec.length_max).astype(np.uint32)

    nm = 1 << MUT_TABLE_BITS
    v = spec.dup_lo + (spec.dup_hi - spec.dup_lo) * (np.arange(nm) + 0.5) / nm
    if spec.dup_mode == "mutate":
        q = v
    elif spec.dup_mode == "jaccard":
        q = 1.0 - (2.0 * v / (1.0 + v)) ** (1.0 / spec.ngram)
    else:
        raise ValueError(spec.dup_mode)
    mut = _to_u64_threshold(q)
    dup_thr = int(_to_u64_threshold(np.array([spec.dup_frac]))[0])
    return Tables(zipf, word_hash, L, mut, dup_thr, int(spec.window), int(spec.seed))


# --- document-level draws ----------------------------------------------------

def is_dup(t: Tables, d: np.ndarray) -> np.ndarray:
    d = np.asarray(d, np.uint64)
    return (d > 0) & (rng(t.seed, FIELD_DUP, d, 0) < np.uint64(t.dup_thr))


def source(t: Tables, d: np.ndarray) -> np.ndarray:
    d = np.asarray(d, np.uint64)
    span = np.maximum(d, np.uint64(1))
    if t.window > 0:
        span = np.minimum(span, np.uint64(t.window))
    r = rng(t.seed, FIELD_SRC, d, 0)
    with np.errstate(over="ignore"):
        return d - np.uint64(1) - (r % span)


def mut_threshold(t: Tables, d: np.ndarray) -> np.ndarray:
    r = rng(t.seed, FIELD_MUT, np.asarray(d, np.uint64), 0)
    return t.mut_thr[(r >> np.uint64(64 - MUT_TABLE_BITS)).astype(np.int64)]


def own_length(t: Tables, d: np.ndarray) -> np.ndarray:
    r = rng(t.seed, FIELD_LEN, np.asarray(d, np.uint64), 0)
    return t.length[(r >> np.uint64(64 - LEN_TABLE_BITS)).astype(np.int64)]


def root(t: Tables, d: np.ndarray) -> np.ndarray:
    cur = np.asarray(d, np.uint64).copy()
    for _ in range(MAX_CHAIN):
        dup = is_dup(t, cur)
        if not dup.any():
            break
        cur = np.where(dup, source(t, cur), cur)
    return cur


def doc_lengths(t: Tables, d0: int, D: int) -> np.ndarray:
    d = np.arange(d0, d0 + D, dtype=np.uint64)
    return own_length(t, root(t, d)).astype(np.uint64)


def fresh_token(t: Tables, c: np.ndarray, pos: np.ndarray) -> np.ndarray:
    r = rng(t.seed, FIELD_TOK, c, pos)
    idx = np.searchsorted(t.zipf_cdf, r, side="right")
    idx = np.minimum(idx, t.zipf_cdf.size - 1)
    return t.word_hash[idx]


def tokens_at(t: Tables, d: np.ndarray, pos: np.ndarray) -> np.ndarray:
    cur = np.asarray(d, np.uint64).copy()
    pos = np.asarray(pos, np.uint64)
    done = np.zeros(cur.shape, bool)
    for _ in range(MAX_CHAIN):
        dup = is_dup(t, cur) & ~done
        if not dup.any():
            break
        idx = np.nonzero(dup)[0]
        mutated = rng(t.seed, FIELD_MUTPOS, cur[idx], pos[idx]) < mut_threshold(t, cur[idx])
        done[idx[mutated]] = True
        keep = idx[~mutated]
        cur[keep] = source(t, cur[keep])
    return fresh_token(t, cur, pos)


def generate(spec: CorpusSpec, d0: int = 0, D: int | None = None,
             tables: Tables | None = None, max_tokens_per_pass: int = 1 << 24):
    """CSR batch for documents d0 .. d0+D-1 of the corpus: (offsets, tokens)."""
    t = tables if tables is not None else build_tables(spec)
    if D is None:
        D = spec.n_docs - d0
    lens = doc_lengths(t, d0, D)
    offsets = np.zeros(D + 1, np.uint64)
    np.cumsum(lens, out=offsets[1:])
    T = int(offsets[-1])
    tokens = np.empty(T, np.uint32)
    # Fill in passes of whole documents to bound temporary memory.
    i = 0
    while i < D:
        j = int(np.searchsorted(offsets, offsets[i] + np.uint64(max_tokens_per_pass),
                                side="right")) - 1
        j = max(j, i + 1)
        j = min(j, D)
        lo, hi = int(offsets[i]), int(offsets[j])
        if hi > lo:
            seg_lens = lens[i:j].astype(np.int64)
            docs = np.repeat(np.arange(d0 + i, d0 + j, dtype=np.uint64), seg_lens)
            starts = np.repeat(offsets[i:j] - offsets[i], seg_lens)
            pos = np.arange(hi - lo, dtype=np.uint64) - starts
            tokens[lo:hi] = tokens_at(t, docs, pos)
        i = j
    return offsets, tokens


def planted_pairs(spec: CorpusSpec, d0: int, D: int, tables: Tables | None = None):
    """(doc, source) of the planted near-duplicates among d0 .. d0+D-1."""
    t = tables if tables is not None else build_tables(spec)
    d = np.arange(d0, d0 + D, dtype=np.uint64)
    dup = is_dup(t, d)
    return np.stack([d[dup], source(t, d[dup])], axis=1)
