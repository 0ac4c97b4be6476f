/*
 * LSHBloom CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded restatement of what the LSHBloom
 * deduplication path computes (arxiv 2411.04257).  It exists so that the
 * GPU path can be checked against something obviously correct.  Only the
 * test suite, the smoke check and the CPU-baseline leg of the benchmark may
 * load it; the product path never calls it.  It shares no code with the
 * CUDA library: SHA-1, SplitMix64, the Mersenne reduction, the probe hash
 * and the sizing formulae are all written out again here, from their
 * published definitions.
 *
 * Each function names the passage of the paper it follows.  Where the paper
 * is silent the function states the reading it takes; those readings are
 * conventions shared by specification, not by code.
 *
 * Integer results are exact.  The only floating point is in the sizing
 * formula (Sec. 4.5) and in the LSH error integrals (Eqs. 1-4).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_API __attribute__((visibility("default")))

typedef unsigned __int128 u128;

/* ------------------------------------------------------------------------ */
/* SHA-1, FIPS 180-4 Sec. 6.1 (the "universal hash" of Sec. 4.1).            */
/* ------------------------------------------------------------------------ */

static uint32_t or_rotl(uint32_t x, int s) { return (x << s) | (x >> (32 - s)); }

static void or_sha1_block(uint32_t H[5], const uint8_t blk[64]) {
    uint32_t W[80];
    for (int t = 0; t < 16; ++t)
        W[t] = ((uint32_t)blk[4 * t] << 24) | ((uint32_t)blk[4 * t + 1] << 16) |
               ((uint32_t)blk[4 * t + 2] << 8) | (uint32_t)blk[4 * t + 3];
    for (int t = 16; t < 80; ++t)
        W[t] = or_rotl(W[t - 3] ^ W[t - 8] ^ W[t - 14] ^ W[t - 16], 1);
    uint32_t a = H[0], b = H[1], c = H[2], d = H[3], e = H[4];
    for (int t = 0; t < 80; ++t) {
        uint32_t f, K;
        if (t < 20) {        /* Ch */
            f = (b & c) ^ (~b & d);
            K = 0x5a827999u;
        } else if (t < 40) { /* Parity */
            f = b ^ c ^ d;
            K = 0x6ed9eba1u;
        } else if (t < 60) { /* Maj */
            f = (b & c) ^ (b & d) ^ (c & d);
            K = 0x8f1bbcdcu;
        } else {             /* Parity */
            f = b ^ c ^ d;
            K = 0xca62c1d6u;
        }
        uint32_t T = or_rotl(a, 5) + f + e + K + W[t];
        e = d;
        d = c;
        c = or_rotl(b, 30);
        b = a;
        a = T;
    }
    H[0] += a; H[1] += b; H[2] += c; H[3] += d; H[4] += e;
}

/* Full SHA-1 of an arbitrary byte string; digest is the 20-byte big-endian
 * concatenation H0..H4 (FIPS 180-4 Sec. 6.1.2). */
OR_API void or_sha1(const uint8_t *msg, uint64_t len, uint8_t digest[20]) {
    uint32_t H[5] = {0x67452301u, 0xefcdab89u, 0x98badcfeu, 0x10325476u, 0xc3d2e1f0u};
    uint64_t full = len / 64;
    for (uint64_t i = 0; i < full; ++i) or_sha1_block(H, msg + 64 * i);
    /* Padding (Sec. 5.1.1): 0x80, zeros, 64-bit big-endian bit length. */
    uint8_t tail[128];
    memset(tail, 0, sizeof tail);
    uint64_t rem = len - 64 * full;
    memcpy(tail, msg + 64 * full, rem);
    tail[rem] = 0x80;
    uint64_t tail_len = (rem + 1 + 8 <= 64) ? 64 : 128;
    uint64_t bits = len * 8;
    for (int i = 0; i < 8; ++i) tail[tail_len - 1 - i] = (uint8_t)(bits >> (8 * i));
    for (uint64_t off = 0; off < tail_len; off += 64) or_sha1_block(H, tail + off);
    for (int i = 0; i < 5; ++i) {
        digest[4 * i + 0] = (uint8_t)(H[i] >> 24);
        digest[4 * i + 1] = (uint8_t)(H[i] >> 16);
        digest[4 * i + 2] = (uint8_t)(H[i] >> 8);
        digest[4 * i + 3] = (uint8_t)(H[i]);
    }
}

/* Shingle base hash, Sec. 4.1 (SHA1 as the universal hash under each
 * signature value) with Sec. 4.3 (32-bit hash values).  Reading: the shingle
 * is the byte string of its tokens, each token a little-endian uint32; the
 * hash is the first four digest bytes read as a little-endian uint32. */
OR_API uint32_t or_shingle_hash(const uint32_t *tok, uint32_t len) {
    uint8_t buf[4 * 256];
    uint8_t *msg = buf;
    uint8_t *heap = NULL;
    if (len > 256) msg = heap = (uint8_t *)malloc(4 * (size_t)len);
    for (uint32_t i = 0; i < len; ++i) {
        msg[4 * i + 0] = (uint8_t)(tok[i]);
        msg[4 * i + 1] = (uint8_t)(tok[i] >> 8);
        msg[4 * i + 2] = (uint8_t)(tok[i] >> 16);
        msg[4 * i + 3] = (uint8_t)(tok[i] >> 24);
    }
    uint8_t dg[20];
    or_sha1(msg, 4 * (uint64_t)len, dg);
    free(heap);
    return (uint32_t)dg[0] | ((uint32_t)dg[1] << 8) | ((uint32_t)dg[2] << 16) |
           ((uint32_t)dg[3] << 24);
}

/* ------------------------------------------------------------------------ */
/* SplitMix64 (Steele, Lea, Flood, OOPSLA 2014).                             */
/* ------------------------------------------------------------------------ */

OR_API uint64_t or_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

static uint64_t or_splitmix_next(uint64_t *state) {
    *state += 0x9e3779b97f4a7c15ull;
    return or_mix64(*state);
}

#define OR_P61 ((1ull << 61) - 1)

/* Permutation coefficients.  The paper relies on a MinHash package for them
 * (Sec. 5.1.2) and fixes no generator.  Reading: a SplitMix64 stream from
 * `seed`, drawn in the order a_0, b_0, a_1, b_1, ...; a_i = 1 + x mod (p-2)
 * lies in [1, p-2] and b_i = x' mod p lies in [0, p-1], p = 2^61 - 1. */
OR_API void or_coefficients(uint64_t seed, uint32_t P, uint64_t *a, uint64_t *b) {
    uint64_t st = seed;
    for (uint32_t i = 0; i < P; ++i) {
        a[i] = 1 + or_splitmix_next(&st) % (OR_P61 - 1);
        b[i] = or_splitmix_next(&st) % OR_P61;
    }
}

/* One MinHash permutation value, Sec. 2.2 / Sec. 4.1: the universal hash
 * (a*h + b) mod (2^61 - 1) taken exactly on the full product, truncated to
 * its low 32 bits (the 32-bit hash values of Sec. 4.3). */
OR_API uint32_t or_perm(uint64_t a, uint64_t b, uint32_t h) {
    u128 x = (u128)a * (u128)h + (u128)b;
    uint64_t v = (uint64_t)(x % (u128)OR_P61);
    return (uint32_t)(v & 0xffffffffull);
}

/* Shingles of a document, Sec. 2.2 (a document as its set of word n-grams).
 * A document of L tokens has the L-n+1 windows tok[s..s+n-1].  Readings for
 * the cases the paper leaves open: 0 < L < n gives one window of all L
 * tokens; L = 0 gives no shingle.  Returns the number of windows and, for
 * window s, its start and length. */
static uint64_t or_num_shingles(uint64_t L, uint32_t n) {
    if (L == 0) return 0;
    if (L < n) return 1;
    return L - n + 1;
}

/* MinHash signature, Sec. 2.2 and Sec. 4.1: sig_i is the minimum over the
 * document's shingles of permutation i of the shingle hash.  With no
 * shingle, every entry keeps its start value 2^32 - 1. */
OR_API void or_signature(const uint32_t *tok, uint64_t L, uint32_t n, uint32_t P,
                         const uint64_t *a, const uint64_t *b, uint32_t *sig) {
    for (uint32_t i = 0; i < P; ++i) sig[i] = 0xffffffffu;
    uint64_t S = or_num_shingles(L, n);
    uint32_t w = (L < n) ? (uint32_t)L : n;
    for (uint64_t s = 0; s < S; ++s) {
        uint32_t h = or_shingle_hash(tok + s, w);
        for (uint32_t i = 0; i < P; ++i) {
            uint32_t v = or_perm(a[i], b[i], h);
            if (v < sig[i]) sig[i] = v;
        }
    }
}

/* Band keys, Sec. 4.1: the band of rows j*r .. j*r+r-1 is reduced to the sum
 * of its signature values modulo N.  Reading: N = 2^64 (the low half of the
 * add-with-carry sum of Sec. 4.4.1); with 32-bit values and r < 2^32 the sum
 * never wraps, so the key is the exact sum. */
OR_API void or_band_keys(const uint32_t *sig, uint32_t bands, uint32_t rows, uint64_t *keys) {
    for (uint32_t j = 0; j < bands; ++j) {
        uint64_t s = 0;
        for (uint32_t t = 0; t < rows; ++t) s += sig[j * rows + t];
        keys[j] = s;
    }
}

/* Weighted band key, a variant beyond the paper: sum_t c_{j,t} x_t mod 2^64
 * with c_{j,t} the SplitMix64 output number (j << 10) + t + 1 of seed 0 (the
 * finaliser of (j << 10 + t + 1) times the golden gamma), made odd.  Mode 0 is
 * the paper's plain sum (or_band_keys). */
OR_API void or_band_keys_mode(const uint32_t *sig, uint32_t bands, uint32_t rows, uint32_t mode,
                              uint64_t *keys) {
    if (mode == 0) {
        or_band_keys(sig, bands, rows, keys);
        return;
    }
    for (uint32_t j = 0; j < bands; ++j) {
        uint64_t s = 0;
        for (uint32_t t = 0; t < rows; ++t) {
            const uint64_t idx = ((uint64_t)j << 10) + t + 1;
            const uint64_t c = or_mix64(idx * 0x9e3779b97f4a7c15ull) | 1ull;
            s += c * sig[j * rows + t];
        }
        keys[j] = s;
    }
}

/* Probe positions of a band key in its band's Bloom filter, Sec. 2.4 (k hash
 * functions into a bit array of m bits).  The paper names no hash family.
 * Reading: Kirsch-Mitzenmacher double hashing (ESA 2006) on SplitMix64
 * finalisers, with Lemire's multiply-high range reduction (2019):
 *   x = mix64(key ^ (j * 0x9e3779b97f4a7c15)),
 *   y = mix64(x ^ 0x6a09e667f3bcc909) | 1,
 *   q_u = floor((x + u*y mod 2^64) * m / 2^64),  u = 0..k-1. */
OR_API void or_probe_positions(uint64_t key, uint32_t j, uint64_t m, uint32_t k, uint64_t *q) {
    uint64_t x = or_mix64(key ^ ((uint64_t)j * 0x9e3779b97f4a7c15ull));
    uint64_t y = or_mix64(x ^ 0x6a09e667f3bcc909ull) | 1ull;
    for (uint32_t u = 0; u < k; ++u) {
        uint64_t g = x + (uint64_t)u * y;
        q[u] = (uint64_t)(((u128)g * (u128)m) >> 64);
    }
}

/* Blocked layout (a variant beyond the paper, after Putze, Sanders and
 * Singler's cache-efficient Bloom filters, 2007): all k bits of a key lie in
 * one 256-bit block of the m-bit filter (m is a multiple of 256), each bit an
 * independent byte of a SplitMix64 word.  With x and y as above:
 * block = floor(x * (m/256) / 2^64), w_t = mix64(y + t * 0x9e3779b97f4a7c15),
 * q_u = 256 block + (byte u mod 8 of w_{floor(u/8)}). */
OR_API void or_probe_positions_blocked(uint64_t key, uint32_t j, uint64_t m, uint32_t k,
                                       uint64_t *q) {
    uint64_t x = or_mix64(key ^ ((uint64_t)j * 0x9e3779b97f4a7c15ull));
    uint64_t y = or_mix64(x ^ 0x6a09e667f3bcc909ull) | 1ull;
    uint64_t nblocks = m / 256;
    uint64_t block = (uint64_t)(((u128)x * (u128)nblocks) >> 64);
    for (uint32_t u = 0; u < k; ++u) {
        uint64_t w = or_mix64(y + (uint64_t)(u / 8) * 0x9e3779b97f4a7c15ull);
        q[u] = 256 * block + ((w >> (8 * (u % 8))) & 255);
    }
}

/* ------------------------------------------------------------------------ */
/* Sizing, Sec. 4.5 and Sec. 4.3.                                            */
/* ------------------------------------------------------------------------ */

/* Per-filter false-positive rate that gives an effective rate p_eff over b
 * independent filters, Sec. 4.3: p = 1 - (1 - p_eff)^(1/b). */
OR_API double or_p_from_effective(double p_eff, uint32_t bands) {
    return 1.0 - pow(1.0 - p_eff, 1.0 / (double)bands);
}

/* Effective rate of b filters each at rate p, Sec. 4.3: 1 - (1 - p)^b. */
OR_API double or_effective_from_p(double p, uint32_t bands) {
    return 1.0 - pow(1.0 - p, (double)bands);
}

/* Bits per filter, Sec. 4.5: m = -n ln p / (ln 2)^2 (natural log).
 * Reading: rounded up to a whole number of bits, then up to a multiple of
 * 256 bits (one 32-byte memory sector).  Hash count, which the paper leaves
 * to the filter package: k = max(1, round((m / n) ln 2)). */
OR_API void or_sizing(uint64_t n, double p, uint64_t *m_bits, uint32_t *k) {
    double mr = -(double)n * log(p) / (log(2.0) * log(2.0));
    uint64_t m = (uint64_t)ceil(mr);
    m = (m + 255) / 256 * 256;
    if (m == 0) m = 256;
    double kr = (double)m / (double)n * log(2.0);
    long kk = lround(kr);
    if (kk < 1) kk = 1;
    *m_bits = m;
    *k = (uint32_t)kk;
}

/* ------------------------------------------------------------------------ */
/* Blocked layout (a design beyond the paper): every key's k positions lie   */
/* in one 256-bit block, drawn uniformly with replacement inside it.  Its    */
/* false-positive model and the sizing that meets a target rate with it.     */
/* ------------------------------------------------------------------------ */

/* One occupancy step: after one more uniform draw over 256 cells, the count
 * of occupied cells moves from z-1 to z with probability (256-(z-1))/256 and
 * stays at z with probability z/256. */
static void or_occupancy_step(double *P) {
    for (int z = 256; z >= 1; --z) P[z] = P[z] * z / 256.0 + P[z - 1] * (257 - z) / 256.0;
    P[0] = 0.0;
}

typedef struct {
    uint32_t k;
    double occ[257];   /* law of the set-bit count after len * k draws */
    double hit[257];   /* P(query all set | z set bits) */
    double *g;         /* g[i] = P(query all set | i keys in the block) */
    uint32_t len, cap;
} or_blocked_model;

static void or_blocked_model_init(or_blocked_model *M, uint32_t k) {
    double q[257];
    memset(q, 0, sizeof(q));
    q[0] = 1.0;
    for (uint32_t u = 0; u < k; ++u) or_occupancy_step(q);   /* distinct cells of a query */
    for (int z = 0; z <= 256; ++z) {
        double s = 0.0;
        for (int d = 1; d <= 256 && d <= (int)k; ++d) {
            if (q[d] == 0.0) continue;
            double r = 1.0;                                   /* C(z, d) / C(256, d) */
            for (int j = 0; j < d; ++j) r *= (double)(z - j) / (double)(256 - j);
            if (z < d) r = 0.0;
            s += q[d] * r;
        }
        M->hit[z] = s;
    }
    memset(M->occ, 0, sizeof(M->occ));
    M->occ[0] = 1.0;
    M->k = k;
    M->g = NULL;
    M->len = M->cap = 0;
}

static double or_blocked_model_g(or_blocked_model *M, uint32_t i) {
    while (M->len <= i) {
        if (M->len == M->cap) {
            M->cap = M->cap ? 2 * M->cap : 256;
            M->g = (double *)realloc(M->g, sizeof(double) * M->cap);
        }
        double s = 0.0;
        for (int z = 0; z <= 256; ++z) s += M->occ[z] * M->hit[z];
        M->g[M->len++] = s;
        for (uint32_t u = 0; u < M->k; ++u) or_occupancy_step(M->occ);
    }
    return M->g[i];
}

/* Block loads Poisson(256 n / m); the rate is the load-weighted g. */
static double or_blocked_model_fp(or_blocked_model *M, uint64_t n, uint64_t m) {
    if (n == 0) return 0.0;
    const double lam = 256.0 * (double)n / (double)m;
    const double spread = 12.0 * sqrt(lam) + 30.0;
    const double lo_r = floor(lam - spread), hi_r = ceil(lam + spread);
    const uint32_t lo = lo_r < 0.0 ? 0u : (uint32_t)lo_r, hi = (uint32_t)hi_r;
    double s = 0.0;
    for (uint32_t i = lo; i <= hi; ++i) {
        const double w = exp(-lam + (double)i * log(lam) - lgamma((double)i + 1.0));
        s += w * or_blocked_model_g(M, i);
    }
    return s;
}

/* P(a query's k positions are all set | i keys in its block). */
OR_API double or_blocked_hit(uint32_t i, uint32_t k) {
    or_blocked_model M;
    or_blocked_model_init(&M, k);
    double g = or_blocked_model_g(&M, i);
    free(M.g);
    return g;
}

/* False-positive rate of one blocked filter of m bits holding n keys. */
OR_API double or_fp_blocked(uint64_t n, uint64_t m, uint32_t k) {
    or_blocked_model M;
    or_blocked_model_init(&M, k);
    double fp = or_blocked_model_fp(&M, n, m);
    free(M.g);
    return fp;
}

/* Sizing of the blocked layout: over k = 1 .. min(64, k_std + 8), the fewest
 * 256-bit blocks whose model rate is at most p; the fewest blocks overall win
 * (ties: the smaller k).  The rate falls as blocks are added, so each k is a
 * bracket (from half the standard layout's blocks, doubling) and a bisection. */
OR_API void or_sizing_blocked(uint64_t n, double p, uint64_t *m_bits, uint32_t *k_out) {
    uint64_t m0;
    uint32_t k0;
    or_sizing(n, p, &m0, &k0);
    const uint64_t B0 = m0 / 256;
    const uint32_t kmax = k0 + 8 > 64 ? 64 : k0 + 8;
    uint64_t bestB = UINT64_MAX;
    uint32_t bestk = k0;
    for (uint32_t k = 1; k <= kmax; ++k) {
        or_blocked_model M;
        or_blocked_model_init(&M, k);
        uint64_t lo = B0 / 2 ? B0 / 2 : 1, hi = B0 ? B0 : 1;
        int ok = 1;
        while (or_blocked_model_fp(&M, n, 256 * hi) > p) {
            lo = hi;
            hi *= 2;
            if (hi > (B0 << 24)) { ok = 0; break; }
        }
        if (ok) {
            while (lo > 1 && or_blocked_model_fp(&M, n, 256 * lo) <= p) { hi = lo; lo /= 2; }
            if (or_blocked_model_fp(&M, n, 256 * lo) <= p) hi = lo;
            while (hi - lo > 1) {
                const uint64_t mid = lo + (hi - lo) / 2;
                if (or_blocked_model_fp(&M, n, 256 * mid) <= p) hi = mid;
                else lo = mid;
            }
            if (hi < bestB) { bestB = hi; bestk = k; }
        }
        free(M.g);
    }
    *m_bits = 256 * bestB;
    *k_out = bestk;
}

/* ------------------------------------------------------------------------ */
/* LSH error model, Eqs. 1-4 (Sec. 4.3), and the (b, r) choice of Sec. 4.3   */
/* and Sec. 4.5 (minimise the two LSH error integrals over b*r <= P).        */
/* ------------------------------------------------------------------------ */

/* Composite Simpson rule with 2000 panels: the integrands are smooth
 * polynomials in t of degree <= b*r. */
static double or_simpson(double (*f)(double, uint32_t, uint32_t), double lo, double hi,
                         uint32_t b, uint32_t r) {
    const int N = 2000;
    double hstep = (hi - lo) / N;
    double s = f(lo, b, r) + f(hi, b, r);
    for (int i = 1; i < N; ++i) s += f(lo + i * hstep, b, r) * ((i & 1) ? 4.0 : 2.0);
    return s * hstep / 3.0;
}

static double or_fp_integrand(double t, uint32_t b, uint32_t r) {
    return 1.0 - pow(1.0 - pow(t, (double)r), (double)b);
}

static double or_fn_integrand(double t, uint32_t b, uint32_t r) {
    return pow(1.0 - pow(t, (double)r), (double)b);
}

/* Eq. 1: FP_lsh = integral_0^T 1 - (1 - t^r)^b dt. */
OR_API double or_fp_lsh(double T, uint32_t b, uint32_t r) {
    return or_simpson(or_fp_integrand, 0.0, T, b, r);
}

/* Eq. 2: FN_lsh = integral_T^1 1 - (1 - (1 - t^r)^b) dt. */
OR_API double or_fn_lsh(double T, uint32_t b, uint32_t r) {
    return or_simpson(or_fn_integrand, T, 1.0, b, r);
}

/* Eq. 3: FP_bloom = FP_lsh + (1 - FP_lsh)(p_eff + b/N). */
OR_API double or_fp_bloom(double fp_lsh, double p_eff, uint32_t b, double N) {
    return fp_lsh + (1.0 - fp_lsh) * (p_eff + (double)b / N);
}

/* Eq. 4: FN_bloom = (1 - (p_eff + b/N)) FN_lsh. */
OR_API double or_fn_bloom(double fn_lsh, double p_eff, uint32_t b, double N) {
    return (1.0 - (p_eff + (double)b / N)) * fn_lsh;
}

/* (b, r) with b*r <= P minimising FP_lsh + FN_lsh with equal weights (the
 * tuning the paper adopts, Sec. 4.3).  Ties keep the first (smallest b). */
OR_API void or_optimal_br(double T, uint32_t P, uint32_t *b_out, uint32_t *r_out) {
    double best = 1e300;
    uint32_t bb = 1, rr = 1;
    for (uint32_t b = 1; b <= P; ++b) {
        for (uint32_t r = 1; b * r <= P; ++r) {
            double e = 0.5 * or_fp_lsh(T, b, r) + 0.5 * or_fn_lsh(T, b, r);
            if (e < best) {
                best = e;
                bb = b;
                rr = r;
            }
        }
    }
    *b_out = bb;
    *r_out = rr;
}

/* ------------------------------------------------------------------------ */
/* The index: b Bloom filters, Sec. 4.1, and the stream decision, Sec. 2.1.  */
/* ------------------------------------------------------------------------ */

typedef struct {
    uint32_t P, bands, rows, ngram, k, insert_all;
    uint32_t layout;     /* 0: standard filter (Sec. 2.4), 1: 256-bit blocked variant,
                            2: exact band-key sets */
    void *sets;          /* layout 2: one or_keyset per band */
    uint32_t band_key;   /* 0: the paper's sum, 1: weighted sum (or_band_keys_mode) */
    uint64_t m;          /* bits per filter */
    uint64_t words;      /* 64-bit words per filter */
    uint64_t *a, *b;     /* permutation coefficients */
    uint64_t *filt;      /* bands * words, bit q of filter j is bit q%64 of word q/64 */
    uint64_t docs_seen;
} or_index;

OR_API or_index *or_index_create(uint32_t P, uint32_t bands, uint32_t rows, uint32_t ngram,
                                 uint64_t m, uint32_t k, const uint64_t *a, const uint64_t *b,
                                 uint32_t insert_all) {
    if (P == 0 || bands == 0 || rows == 0 || (uint64_t)bands * rows > P || ngram == 0 ||
        m == 0 || k == 0)
        return NULL;
    or_index *ix = (or_index *)calloc(1, sizeof(or_index));
    ix->P = P; ix->bands = bands; ix->rows = rows; ix->ngram = ngram;
    ix->m = m; ix->k = k; ix->insert_all = insert_all;
    ix->words = (m + 63) / 64;
    ix->a = (uint64_t *)malloc(sizeof(uint64_t) * P);
    ix->b = (uint64_t *)malloc(sizeof(uint64_t) * P);
    memcpy(ix->a, a, sizeof(uint64_t) * P);
    memcpy(ix->b, b, sizeof(uint64_t) * P);
    ix->filt = (uint64_t *)calloc((size_t)bands * ix->words, sizeof(uint64_t));
    if (!ix->filt) {
        free(ix->a); free(ix->b); free(ix);
        return NULL;
    }
    return ix;
}

/* Exact band-key sets (layout 2): the bucket rule of MinHashLSH (Sec. 2.3)
 * applied to band keys, i.e. the index without Bloom false positives.  One
 * open-addressing set per band, doubled when half full. */
typedef struct {
    uint64_t *slot; /* ~0 = empty */
    uint64_t cap, used;
    int has_max;    /* the key 2^64 - 1, which the empty marker cannot hold */
} or_keyset;

static uint64_t or_set_home(uint64_t key, uint64_t cap) { return or_mix64(key) & (cap - 1); }

static int or_set_contains(const or_keyset *s, uint64_t key) {
    if (key == ~0ull) return s->has_max;
    for (uint64_t i = or_set_home(key, s->cap);; i = (i + 1) & (s->cap - 1)) {
        if (s->slot[i] == key) return 1;
        if (s->slot[i] == ~0ull) return 0;
    }
}

static void or_set_add(or_keyset *s, uint64_t key);

static void or_set_grow(or_keyset *s) {
    or_keyset t;
    t.cap = s->cap * 2;
    t.used = 0;
    t.has_max = s->has_max;
    t.slot = (uint64_t *)malloc(sizeof(uint64_t) * t.cap);
    memset(t.slot, 0xff, sizeof(uint64_t) * t.cap);
    for (uint64_t i = 0; i < s->cap; ++i)
        if (s->slot[i] != ~0ull) or_set_add(&t, s->slot[i]);
    free(s->slot);
    *s = t;
}

static void or_set_add(or_keyset *s, uint64_t key) {
    if (key == ~0ull) {
        s->has_max = 1;
        return;
    }
    if (2 * (s->used + 1) > s->cap) or_set_grow(s);
    for (uint64_t i = or_set_home(key, s->cap);; i = (i + 1) & (s->cap - 1)) {
        if (s->slot[i] == key) return;
        if (s->slot[i] == ~0ull) {
            s->slot[i] = key;
            s->used++;
            return;
        }
    }
}

/* Select the layout of an empty index: 0 standard filter, 1 blocked filter,
 * 2 exact band-key sets. */
OR_API int or_index_set_layout(or_index *ix, uint32_t layout) {
    if (layout > 2 || (layout == 1 && ix->m % 256 != 0)) return -1;
    ix->layout = layout;
    if (layout == 2 && !ix->sets) {
        ix->sets = calloc(ix->bands, sizeof(or_keyset));
        or_keyset *s = (or_keyset *)ix->sets;
        for (uint32_t j = 0; j < ix->bands; ++j) {
            s[j].cap = 1024;
            s[j].slot = (uint64_t *)malloc(sizeof(uint64_t) * 1024);
            memset(s[j].slot, 0xff, sizeof(uint64_t) * 1024);
        }
    }
    return 0;
}

/* Band-key mode of an index (before its first document). */
OR_API int or_index_set_band_key(or_index *ix, uint32_t mode) {
    if (mode > 1) return -1;
    ix->band_key = mode;
    return 0;
}

/* Keys of band j of an exact index (unordered); returns how many. */
OR_API uint64_t or_index_exact_keys(const or_index *ix, uint32_t j, uint64_t *out, uint64_t cap) {
    if (ix->layout != 2) return 0;
    const or_keyset *s = (const or_keyset *)ix->sets + j;
    uint64_t n = 0;
    for (uint64_t i = 0; i < s->cap; ++i)
        if (s->slot[i] != ~0ull) {
            if (n < cap) out[n] = s->slot[i];
            n++;
        }
    if (s->has_max) {
        if (n < cap) out[n] = ~0ull;
        n++;
    }
    return n;
}

static void or_index_positions(const or_index *ix, uint64_t key, uint32_t j, uint64_t *q) {
    if (ix->layout == 1) or_probe_positions_blocked(key, j, ix->m, ix->k, q);
    else or_probe_positions(key, j, ix->m, ix->k, q);
}

OR_API void or_index_destroy(or_index *ix) {
    if (!ix) return;
    if (ix->sets) {
        or_keyset *s = (or_keyset *)ix->sets;
        for (uint32_t j = 0; j < ix->bands; ++j) free(s[j].slot);
        free(ix->sets);
    }
    free(ix->a); free(ix->b); free(ix->filt); free(ix);
}

static int or_get_bit(const or_index *ix, uint32_t j, uint64_t q) {
    return (int)((ix->filt[(uint64_t)j * ix->words + (q >> 6)] >> (q & 63)) & 1ull);
}

static void or_set_bit(or_index *ix, uint32_t j, uint64_t q) {
    ix->filt[(uint64_t)j * ix->words + (q >> 6)] |= 1ull << (q & 63);
}

/* The stream of documents is processed strictly in order (Sec. 4.4.2: index
 * writes stay sequential so each document is judged against the ones before
 * it; Sec. 2.1 defines the decision against D_seen = {d_j | j < i}).
 * For document i with band keys keys[0 .. bands-1]:
 *   - its band keys are probed in their filters (Sec. 4.2); a band hits when
 *     all k probed bits are set (Sec. 2.4); the document is a duplicate when
 *     any band hits;
 *   - then it is inserted (Sec. 4.1): every probed bit is set.  Reading of
 *     Sec. 4.4.2: by default only documents found not to be duplicates are
 *     inserted; insert_all inserts every document.
 * The query comes before the insert, so a document never matches itself.
 * q is scratch for bands * k positions.  Returns the duplicate flag. */
static int or_index_judge(or_index *ix, const uint64_t *keys, uint64_t *q) {
    int dup = 0;
    if (ix->layout == 2) {
        or_keyset *sets = (or_keyset *)ix->sets;
        for (uint32_t j = 0; j < ix->bands; ++j)
            if (or_set_contains(&sets[j], keys[j])) dup = 1;
        if (ix->insert_all || !dup)
            for (uint32_t j = 0; j < ix->bands; ++j) or_set_add(&sets[j], keys[j]);
        ix->docs_seen++;
        return dup;
    }
    for (uint32_t j = 0; j < ix->bands; ++j) {
        uint64_t *qj = q + (uint64_t)j * ix->k;
        or_index_positions(ix, keys[j], j, qj);
        int all_set = 1;
        for (uint32_t u = 0; u < ix->k; ++u)
            if (!or_get_bit(ix, j, qj[u])) all_set = 0;
        if (all_set) dup = 1;
    }
    if (ix->insert_all || !dup) {
        for (uint32_t j = 0; j < ix->bands; ++j)
            for (uint32_t u = 0; u < ix->k; ++u)
                or_set_bit(ix, j, q[(uint64_t)j * ix->k + u]);
    }
    ix->docs_seen++;
    return dup;
}

/* A batch of D documents: signature (Sec. 2.2, 4.1), band keys (Sec. 4.1),
 * then the stream decision above, one document after the other. */
OR_API void or_index_dedup(or_index *ix, const uint64_t *offsets, const uint32_t *tokens,
                           uint64_t D, uint8_t *flags) {
    uint32_t *sig = (uint32_t *)malloc(sizeof(uint32_t) * ix->P);
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * ix->bands);
    uint64_t *q = (uint64_t *)malloc(sizeof(uint64_t) * ix->k * ix->bands);
    for (uint64_t i = 0; i < D; ++i) {
        uint64_t L = offsets[i + 1] - offsets[i];
        or_signature(tokens + offsets[i], L, ix->ngram, ix->P, ix->a, ix->b, sig);
        or_band_keys_mode(sig, ix->bands, ix->rows, ix->band_key, keys);
        flags[i] = (uint8_t)or_index_judge(ix, keys, q);
    }
    free(sig); free(keys); free(q);
}

/* The same stream decision fed with band keys already computed (row i of
 * keys holds document i's bands keys[i*bands .. i*bands + bands-1]): the
 * order-dependent half of the path, replayed alone.  A document's keys depend
 * on that document only, so a caller may compute them in any order (or in
 * parallel, with or_batch_band_keys) and get the flags of or_index_dedup. */
OR_API void or_index_dedup_keys(or_index *ix, const uint64_t *keys, uint64_t D, uint8_t *flags) {
    uint64_t *q = (uint64_t *)malloc(sizeof(uint64_t) * ix->k * ix->bands);
    for (uint64_t i = 0; i < D; ++i)
        flags[i] = (uint8_t)or_index_judge(ix, keys + i * ix->bands, q);
    free(q);
}

/* Bloom filter alone (Sec. 2.4), for the false-positive closed-form pin:
 * query first, then insert, of a raw 64-bit key in filter 0. */
OR_API int or_index_query_key(const or_index *ix, uint32_t j, uint64_t key) {
    uint64_t q[256];
    if (ix->k > 256) return -1;
    or_index_positions(ix, key, j, q);
    for (uint32_t u = 0; u < ix->k; ++u)
        if (!or_get_bit(ix, j, q[u])) return 0;
    return 1;
}

OR_API void or_index_insert_key(or_index *ix, uint32_t j, uint64_t key) {
    uint64_t q[256];
    if (ix->k > 256) return;
    or_index_positions(ix, key, j, q);
    for (uint32_t u = 0; u < ix->k; ++u) or_set_bit(ix, j, q[u]);
}

/* The same two operations over arrays of keys, in array order. */
OR_API void or_index_insert_keys(or_index *ix, uint32_t j, const uint64_t *keys, uint64_t n) {
    for (uint64_t i = 0; i < n; ++i) or_index_insert_key(ix, j, keys[i]);
}

OR_API void or_index_query_keys(const or_index *ix, uint32_t j, const uint64_t *keys, uint64_t n,
                                uint8_t *hit) {
    for (uint64_t i = 0; i < n; ++i) hit[i] = (uint8_t)or_index_query_key(ix, j, keys[i]);
}

/* Copy out filter j as bytes, bit q at byte q/8, bit q%8 (LSB first). */
OR_API void or_index_filter_bytes(const or_index *ix, uint32_t j, uint8_t *out) {
    uint64_t nbytes = (ix->m + 7) / 8;
    const uint64_t *w = ix->filt + (uint64_t)j * ix->words;
    for (uint64_t i = 0; i < nbytes; ++i) out[i] = (uint8_t)(w[i >> 3] >> (8 * (i & 7)));
}

OR_API uint64_t or_index_popcount(const or_index *ix, uint32_t j) {
    uint64_t c = 0;
    const uint64_t *w = ix->filt + (uint64_t)j * ix->words;
    for (uint64_t i = 0; i < ix->words; ++i) c += (uint64_t)__builtin_popcountll(w[i]);
    return c;
}

OR_API uint64_t or_index_docs_seen(const or_index *ix) { return ix->docs_seen; }

/* Batch helpers for tests: signatures and band keys of a CSR batch. */
OR_API void or_batch_signatures(const uint64_t *offsets, const uint32_t *tokens, uint64_t D,
                                uint32_t n, uint32_t P, const uint64_t *a, const uint64_t *b,
                                uint32_t *sig_out) {
    for (uint64_t i = 0; i < D; ++i)
        or_signature(tokens + offsets[i], offsets[i + 1] - offsets[i], n, P, a, b,
                     sig_out + i * P);
}

OR_API void or_batch_shingle_hashes(const uint64_t *offsets, const uint32_t *tokens, uint64_t D,
                                    uint32_t n, uint32_t *h_out, uint64_t *counts) {
    uint64_t o = 0;
    for (uint64_t i = 0; i < D; ++i) {
        uint64_t L = offsets[i + 1] - offsets[i];
        uint64_t S = or_num_shingles(L, n);
        uint32_t w = (L < n) ? (uint32_t)L : n;
        for (uint64_t s = 0; s < S; ++s) h_out[o++] = or_shingle_hash(tokens + offsets[i] + s, w);
        counts[i] = S;
    }
}

/* Band keys of a CSR batch (Sec. 2.2, Sec. 4.1): signature then band keys,
 * per document; keys_out is D x bands, row-major. */
OR_API void or_batch_band_keys(const uint64_t *offsets, const uint32_t *tokens, uint64_t D,
                               uint32_t n, uint32_t P, const uint64_t *a, const uint64_t *b,
                               uint32_t bands, uint32_t rows, uint32_t mode, uint64_t *keys_out) {
    uint32_t *sig = (uint32_t *)malloc(sizeof(uint32_t) * P);
    for (uint64_t i = 0; i < D; ++i) {
        or_signature(tokens + offsets[i], offsets[i + 1] - offsets[i], n, P, a, b, sig);
        or_band_keys_mode(sig, bands, rows, mode, keys_out + i * bands);
    }
    free(sig);
}
