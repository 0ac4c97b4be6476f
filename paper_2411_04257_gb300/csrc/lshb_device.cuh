// Device primitives of the LSHBloom path: the shingle hash (SHA-1, FIPS
// 180-4), the exact (a*h + b) mod (2^61 - 1) permutation truncated to 32
// bits, the SplitMix64 finaliser, and the Bloom probe sequence.
#pragma once

#include <cstdint>

#define LSHB_FULL_MASK 0xffffffffu

namespace lshb {

constexpr uint64_t kP61 = (1ull << 61) - 1;
constexpr uint64_t kGolden = 0x9e3779b97f4a7c15ull;
constexpr uint64_t kProbeSalt = 0x6a09e667f3bcc909ull;

// SplitMix64 finaliser (Steele, Lea, Flood 2014).
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint32_t rotl32(uint32_t x, int s) { return __funnelshift_l(x, x, s); }

// Byte reversal: a little-endian token word read as a big-endian SHA-1 word.
__device__ __forceinline__ uint32_t bswap32(uint32_t x) { return __byte_perm(x, 0, 0x0123); }

// One SHA-1 round group (FIPS 180-4 Sec. 4.1.1 and 6.1.2).  t is a
// compile-time constant after unrolling, so the function choice folds away.
__device__ __forceinline__ void sha1_step(int t, uint32_t w, uint32_t &a, uint32_t &b, uint32_t &c,
                                          uint32_t &d, uint32_t &e) {
    uint32_t f, K;
    if (t < 20) {
        f = (b & c) | (~b & d);
        K = 0x5a827999u;
    } else if (t < 40) {
        f = b ^ c ^ d;
        K = 0x6ed9eba1u;
    } else if (t < 60) {
        f = (b & c) | (d & (b | c));
        K = 0x8f1bbcdcu;
    } else {
        f = b ^ c ^ d;
        K = 0xca62c1d6u;
    }
    const uint32_t T = rotl32(a, 5) + f + e + K + w;
    e = d;
    d = c;
    c = rotl32(b, 30);
    b = a;
    a = T;
}

// Compress one 16-word block into H (a 16-word ring for the schedule).
__device__ __forceinline__ void sha1_compress(uint32_t H[5], uint32_t W[16]) {
    uint32_t a = H[0], b = H[1], c = H[2], d = H[3], e = H[4];
#pragma unroll
    for (int t = 0; t < 80; ++t) {
        uint32_t w;
        if (t < 16) {
            w = W[t];
        } else {
            w = rotl32(W[(t + 13) & 15] ^ W[(t + 8) & 15] ^ W[(t + 2) & 15] ^ W[t & 15], 1);
            W[t & 15] = w;
        }
        sha1_step(t, w, a, b, c, d, e);
    }
    H[0] += a; H[1] += b; H[2] += c; H[3] += d; H[4] += e;
}

// First digest word of SHA-1 over NW big-endian words (4*NW <= 55 bytes, one
// padded block).  Only H0 is needed: the shingle hash is its first 4 bytes.
template <int NW>
__device__ __forceinline__ uint32_t sha1_h0_one_block(const uint32_t (&m)[NW]) {
    static_assert(NW >= 1 && NW <= 13, "single-block message");
    uint32_t W[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) W[i] = 0u;
#pragma unroll
    for (int i = 0; i < NW; ++i) W[i] = m[i];
    W[NW] = 0x80000000u;
    W[15] = 32u * NW;
    uint32_t a = 0x67452301u, b = 0xefcdab89u, c = 0x98badcfeu, d = 0x10325476u, e = 0xc3d2e1f0u;
#pragma unroll
    for (int t = 0; t < 80; ++t) {
        uint32_t w;
        if (t < 16) {
            w = W[t];
        } else {
            w = rotl32(W[(t + 13) & 15] ^ W[(t + 8) & 15] ^ W[(t + 2) & 15] ^ W[t & 15], 1);
            W[t & 15] = w;
        }
        sha1_step(t, w, a, b, c, d, e);
    }
    return 0x67452301u + a;
}

// First digest word of SHA-1 over `nw` little-endian tokens at `tok` (any
// length; padding per FIPS 180-4 Sec. 5.1.1).
__device__ __forceinline__ uint32_t sha1_h0_tokens(const uint32_t *tok, uint32_t nw) {
    uint32_t H[5] = {0x67452301u, 0xefcdab89u, 0x98badcfeu, 0x10325476u, 0xc3d2e1f0u};
    const uint32_t total = nw + 1 + 2;               // words incl. 0x80 marker and length
    const uint32_t blocks = (total + 15) / 16;
    for (uint32_t blk = 0; blk < blocks; ++blk) {
        uint32_t W[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const uint32_t g = blk * 16 + i;
            uint32_t v = 0u;
            if (g < nw) v = bswap32(__ldg(tok + g));
            else if (g == nw) v = 0x80000000u;
            if (blk == blocks - 1 && i == 15) v = 32u * nw;
            W[i] = v;
        }
        sha1_compress(H, W);
    }
    return H[0];
}

__device__ __forceinline__ uint32_t shingle_hash_from_h0(uint32_t h0) { return bswap32(h0); }

// Band key j of a signature band row[0 .. rows): the paper's sum (mode 0) or
// the weighted sum with odd weights mix64(G ((j << 10) + t + 1)) | 1 (mode 1,
// beyond the paper), mod 2^64.
__host__ __device__ __forceinline__ uint64_t band_key_of(const uint32_t *row, uint32_t rows,
                                                         uint32_t j, uint32_t mode) {
    uint64_t s = 0;
    if (mode == 0) {
        for (uint32_t t = 0; t < rows; ++t) s += row[t];
    } else {
        for (uint32_t t = 0; t < rows; ++t)
            s += (mix64(kGolden * (((uint64_t)j << 10) + t + 1)) | 1ull) * row[t];
    }
    return s;
}

// Probe sequence of one band key (library convention).  Standard layout:
// Kirsch-Mitzenmacher double hashing over the m bits.  Blocked layout (the
// variant beyond the paper): one 256-bit block per key, each position an
// independent byte of a SplitMix64 word.
// The exact-key layout has a single "position" per band: the key itself.
constexpr uint64_t kExactTag = ~1ull;

struct ProbeSeq {
    uint64_t x, y, m, base;  // base: first bit of the key's block, ~0 standard, kExactTag exact
    __device__ __forceinline__ ProbeSeq(uint64_t key, uint32_t band, uint64_t m_bits,
                                        uint32_t layout) {
        m = m_bits;
        if (layout == 2) {
            x = key;
            y = 0;
            base = kExactTag;
            return;
        }
        x = mix64(key ^ ((uint64_t)band * kGolden));
        y = mix64(x ^ kProbeSalt) | 1ull;
        base = layout == 1 ? (__umul64hi(x, m_bits >> 8) << 8) : ~0ull;
    }
    __device__ __forceinline__ uint64_t pos(uint32_t u) const {
        if (base == kExactTag) return x;
        if (base != ~0ull) {
            const uint64_t w = mix64(y + (uint64_t)(u >> 3) * kGolden);
            return base + ((w >> (8 * (u & 7))) & 255);
        }
        return __umul64hi(x + (uint64_t)u * y, m);
    }
};

}  // namespace lshb
