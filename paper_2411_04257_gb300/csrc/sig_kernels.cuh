// Signature-stage kernels: warp-cooperative shingling, SHA-1 shingle hash,
// MinHash minimum over a pass of up to 32*PPL permutations, band-key epilogue.
//
// Layout: one warp per document (or per shingle range of one).  Each step the
// 32 lanes hash 32 consecutive shingles (one SHA-1 each) into a per-warp
// shared-memory slot; then every lane folds all 32 hashes, read back as
// broadcast 128-bit loads, into the PPL permutations it owns: lane l owns
// permutations l, l+32, ..., with their coefficients in registers.  The inner
// loop is a few integer instructions per (shingle, permutation), the loop body
// is small enough to stay in the instruction cache, and no cross-lane
// reduction is needed at the end of a document.
#pragma once

#include "lshb_device.cuh"
#include "lshb_internal.h"

namespace lshb {

template <int PPL>
struct LaneCoef {
    uint32_t a0[PPL], a1[PPL];
    uint64_t b0[PPL], b1[PPL];  // 64-bit addends of the wide multiplies (b0 carries a +1, see below)
    uint32_t eight;             // 8, read from memory so that the multiply by it stays a multiply

    __device__ __forceinline__ void load(const PermSlice &c, uint32_t npc, int lane) {
#pragma unroll
        for (int t = 0; t < PPL; ++t) {
            const uint32_t i = lane + 32 * t;
            const bool on = i < npc;
            a0[t] = on ? c.a0[i] : 0u;
            a1[t] = on ? c.a1[i] : 0u;
            b0[t] = on ? (uint64_t)c.b0[i] + 1ull : 1ull;
            b1[t] = on ? c.b1[i] : 0u;
        }
        eight = 8u + (c.a1[0] >> 31);  // a1 < 2^29
    }
};

// ((a*h + b) mod (2^61 - 1)) mod 2^32, exact, for a = a1:a0, b = b1:b0 < 2^61 - 1
// and h < 2^32.  With x = a h + b, work on x + 1 (the +1 rides in b0):
//   t = a0 h + b0 + 1 < 2^64,  V = a1 h + b1 + (t >> 32) < 2^61,
//   x + 1 = V 2^32 + (t mod 2^32);
// 2^61 = 1 (mod p) folds it to s = (V mod 2^29) 2^32 + (t mod 2^32) + (V >> 29),
// 1 <= s < 2^61 + 2^32, s = x + 1 (mod p).  Then x mod p = s - 1 - p [s >= 2^61],
// whose low 32 bits are s_lo - 1 + (s >> 61) since 2^61 = 0 (mod 2^32).
// Two wide multiplies and ALU work.  V < 2^61, so V >> 29 fits in 32 bits and
// is taken with one funnel shift of V's two halves instead of a 64-bit shift
// (4.6% faster signature kernel, measured); the rest is left to the compiler,
// whose split between the IMAD and ALU pipes measured faster than
// hand-placing the 64-bit adds on the IMAD pipe.
__device__ __forceinline__ uint32_t perm_lo32w(uint32_t h, uint32_t a0, uint32_t a1, uint64_t b0,
                                               uint64_t b1) {
    const uint64_t t = (uint64_t)a0 * h + b0;
    const uint64_t V = (uint64_t)a1 * h + b1 + (t >> 32);
    const uint32_t vlo = (uint32_t)V, vhi = (uint32_t)(V >> 32);
    const uint32_t q = __funnelshift_r(vlo, vhi, 29);  // V >> 29
    const uint64_t s = (((uint64_t)(vlo & 0x1fffffffu) << 32) | (uint32_t)t) + q;
    return (uint32_t)s - 1u + (uint32_t)(s >> 61);
}

// Fast form of perm_lo32w: s_lo - 1 without the (s >> 61) term.  That term
// is nonzero only when s >= 2^61, and s = (V mod 2^29) 2^32 + (t mod 2^32) +
// (V >> 29) with V >> 29 < 2^32 reaches 2^61 only if V mod 2^29 = 2^29 - 1
// (probability 2^-29 per value).  `guard` keeps the maximum of
// (8 V) mod 2^32 = (V mod 2^29) << 3, which equals 0xfffffff8 exactly for
// such a V: a range whose guard stays below it has every value exact, and one
// whose guard reaches it is recomputed with perm_lo32w.  This saves the mask,
// the 64-bit add and the final shift-and-add of the exact form on the ALU
// pipe, which bounds the kernel.
//
// V = a1 h + b1 + (t >> 32) by a wide multiply and a 64-bit add, V >> 29 by
// one funnel shift of its halves, and the guard's 8 V by a multiply with a
// run-time 8: that keeps it one multiply-add on the FMA pipe, which has room
// (measured 6% faster than the same guard as min(-8 V - 8) with literal
// constants, and faster than any mix with a form taking 8 V from a third wide
// multiply-add).
constexpr uint32_t kGuardTrip = 0xfffffff8u;

__device__ __forceinline__ uint32_t perm_lo32_fast(uint32_t h, uint32_t a0, uint32_t a1,
                                                   uint64_t b0, uint64_t b1, uint32_t eight,
                                                   uint32_t &guard) {
    const uint64_t t = (uint64_t)a0 * h + b0;
    const uint64_t V = (uint64_t)a1 * h + b1 + (t >> 32);
    const uint32_t vlo = (uint32_t)V, vhi = (uint32_t)(V >> 32);
    guard = max(guard, vlo * eight);
    return (uint32_t)t + __funnelshift_r(vlo, vhi, 29) - 1u;
}

template <int PPL, bool FAST>
__device__ __forceinline__ void fold4(uint32_t (&mn)[PPL], const LaneCoef<PPL> &c, uint4 hv,
                                      uint32_t &guard) {
#pragma unroll
    for (int t = 0; t < PPL; ++t) {
        uint32_t m = mn[t];
        if constexpr (FAST) {
            m = min(m, perm_lo32_fast(hv.x, c.a0[t], c.a1[t], c.b0[t], c.b1[t], c.eight, guard));
            m = min(m, perm_lo32_fast(hv.y, c.a0[t], c.a1[t], c.b0[t], c.b1[t], c.eight, guard));
            m = min(m, perm_lo32_fast(hv.z, c.a0[t], c.a1[t], c.b0[t], c.b1[t], c.eight, guard));
            m = min(m, perm_lo32_fast(hv.w, c.a0[t], c.a1[t], c.b0[t], c.b1[t], c.eight, guard));
        } else {
            m = min(m, perm_lo32w(hv.x, c.a0[t], c.a1[t], c.b0[t], c.b1[t]));
            m = min(m, perm_lo32w(hv.y, c.a0[t], c.a1[t], c.b0[t], c.b1[t]));
            m = min(m, perm_lo32w(hv.z, c.a0[t], c.a1[t], c.b0[t], c.b1[t]));
            m = min(m, perm_lo32w(hv.w, c.a0[t], c.a1[t], c.b0[t], c.b1[t]));
        }
        mn[t] = m;
    }
}

// Hash of the NG-token shingle starting at lane `lane` of a 32-token step,
// from that step's tokens (ta, one per lane) and the next step's (tb): the
// window is assembled with shuffles.
template <int NG>
__device__ __forceinline__ uint32_t window_hash_regs(uint32_t ta, uint32_t tb, int lane) {
    uint32_t w[NG];
    w[0] = bswap32(ta);
#pragma unroll
    for (int k = 1; k < NG; ++k) {
        const uint32_t v = lane >= k ? ta : tb;
        w[k] = bswap32(__shfl_sync(LSHB_FULL_MASK, v, (lane + k) & 31));
    }
    return bswap32(sha1_h0_one_block<NG>(w));
}

// Token i of a document of L tokens, 0 past its end.
__device__ __forceinline__ uint32_t token_or_zero(const uint32_t *tk, uint64_t i, uint64_t L) {
    return i < L ? __ldg(tk + i) : 0u;
}

// Hash of shingle s0+lane of a document of L >= n tokens.  For NG > 0 the
// window is assembled with shuffles from two coalesced loads; lanes past the
// last shingle return an unspecified value.
template <int NG>
__device__ __forceinline__ uint32_t window_hash(const uint32_t *tk, uint64_t L, uint64_t S,
                                                uint64_t s0, int lane, uint32_t n) {
    if constexpr (NG > 0) {
        return window_hash_regs<NG>(token_or_zero(tk, s0 + lane, L),
                                    token_or_zero(tk, s0 + 32 + lane, L), lane);
    } else {
        uint64_t s = s0 + lane;
        if (s >= S) s = S - 1;
        return bswap32(sha1_h0_tokens(tk + s, n));
    }
}

// Number of shingles of a document of L tokens (a shorter-than-n document has
// one shingle of all its tokens; an empty one has none).
__device__ __forceinline__ uint64_t shingle_count(uint64_t L, uint32_t n) {
    return L == 0 ? 0 : (L < n ? 1 : L - n + 1);
}

// Fold shingles [s_begin, s_end) of one document into the lane's minima.
// hbuf is the warp's 32-entry, 16-byte aligned shared slot.  When `hashes` is
// given the shingle hashes are read from it (plain form) instead of computed.
template <int NG, int PPL, bool FAST>
__device__ __forceinline__ void fold_pass(uint32_t (&mn)[PPL], const LaneCoef<PPL> &cf,
                                          const uint32_t *tk, uint64_t L, uint32_t n,
                                          uint64_t s_begin, uint64_t s_end,
                                          const uint32_t *hashes, uint32_t *hbuf, int lane,
                                          uint32_t &guard) {
    const uint64_t S = shingle_count(L, n);
    if (L < n) {
        // one short shingle of all L tokens (only when the range covers it)
        if (s_begin == 0 && s_end > 0 && L > 0) {
            uint32_t h = hashes ? __ldg(hashes) : bswap32(sha1_h0_tokens(tk, (uint32_t)L));
            const uint4 hv = make_uint4(h, h, h, h);
            fold4<PPL, false>(mn, cf, hv, guard);
        }
        return;
    }
    // For NG > 0 each step loads the next step's 32 tokens, which also hold
    // the NG-1 tokens the current windows run into: one coalesced load per
    // step, issued a whole step before its tokens are hashed.
    uint32_t ta = 0u;
    if constexpr (NG > 0) ta = hashes ? 0u : token_or_zero(tk, s_begin + lane, L);
    for (uint64_t s0 = s_begin; s0 < s_end; s0 += 32) {
        const uint32_t cnt = (uint32_t)min((uint64_t)32, s_end - s0);
        uint32_t h;
        if (hashes) {
            h = (s0 + lane < s_end) ? __ldg(hashes + s0 + lane) : 0u;
        } else if constexpr (NG > 0) {
            const uint32_t tn = token_or_zero(tk, s0 + 32 + lane, L);
            h = window_hash_regs<NG>(ta, tn, lane);
            ta = tn;
        } else {
            h = window_hash<NG>(tk, L, S, s0, lane, n);
        }
        // lanes past the range repeat the first hash of the step: a repeat
        // leaves every minimum unchanged.
        const uint32_t h0 = __shfl_sync(LSHB_FULL_MASK, h, 0);
        if ((uint32_t)lane >= cnt) h = h0;
        __syncwarp();
        hbuf[lane] = h;
        __syncwarp();
        const uint4 *hv4 = reinterpret_cast<const uint4 *>(hbuf);
        const uint32_t groups = (cnt + 3) >> 2;
        for (uint32_t g = 0; g < groups; ++g) fold4<PPL, FAST>(mn, cf, hv4[g], guard);
    }
}

// The exact pass, kept out of line: inlined next to the fast pass it raised
// the persistent kernel from 95 to 122 registers (8 instead of 10 blocks per
// SM) and measured 14% slower; called, it costs a stack frame on a path that
// a range takes with probability about (shingles x permutations) / 2^29.
template <int NG, int PPL>
__device__ __noinline__ void fold_exact(uint32_t (&mn)[PPL], const LaneCoef<PPL> &cf,
                                        const uint32_t *tk, uint64_t L, uint32_t n,
                                        uint64_t s_begin, uint64_t s_end,
                                        const uint32_t *hashes, uint32_t *hbuf, int lane) {
    uint32_t guard = 0u;
#pragma unroll
    for (int t = 0; t < PPL; ++t) mn[t] = 0xffffffffu;
    fold_pass<NG, PPL, false>(mn, cf, tk, L, n, s_begin, s_end, hashes, hbuf, lane, guard);
}

// The lane's minima over shingles [s_begin, s_end) (all-ones when the range
// is empty): the fast pass, and, in the rare case that its guard tripped in
// some lane, the whole range again in exact arithmetic.  Called by all 32
// lanes of the warp with the same range.
template <int NG, int PPL>
__device__ __forceinline__ void fold_range(uint32_t (&mn)[PPL], const LaneCoef<PPL> &cf,
                                           const uint32_t *tk, uint64_t L, uint32_t n,
                                           uint64_t s_begin, uint64_t s_end,
                                           const uint32_t *hashes, uint32_t *hbuf, int lane) {
    uint32_t guard = 0u;
#pragma unroll
    for (int t = 0; t < PPL; ++t) mn[t] = 0xffffffffu;
    fold_pass<NG, PPL, true>(mn, cf, tk, L, n, s_begin, s_end, hashes, hbuf, lane, guard);
    if (__any_sync(LSHB_FULL_MASK, guard == kGuardTrip))
        fold_exact<NG, PPL>(mn, cf, tk, L, n, s_begin, s_end, hashes, hbuf, lane);
}

// Write the pass minima (sig_out) and, for a single full pass, band keys.
template <int PPL>
__device__ __forceinline__ void sig_epilogue(const SigArgs &A, uint64_t d, uint32_t (&mn)[PPL],
                                             uint32_t *sigbuf, int lane) {
    if (A.sig_out) {
        uint32_t *row = A.sig_out + d * A.P + A.p0;
#pragma unroll
        for (int t = 0; t < PPL; ++t)
            if (lane + 32 * t < (int)A.npc) row[lane + 32 * t] = mn[t];
    }
    if (A.keys_out) {
        __syncwarp();
#pragma unroll
        for (int t = 0; t < PPL; ++t) sigbuf[lane + 32 * t] = mn[t];
        __syncwarp();
        for (uint32_t j = lane; j < A.bands; j += 32)
            A.keys_out[d * A.bands + j] = band_key_of(sigbuf + j * A.rows, A.rows, j, A.band_key);
        __syncwarp();
    }
}

template <int PPL>
struct SigSmem {
    uint4 hbuf[kSigThreads / 32][8];          // 32 hashes per warp
    uint32_t sig[kSigThreads / 32][32 * PPL];
};

// Fused signature kernel: shingling + SHA-1 + MinHash (+ band keys), warp per
// document.  `hashes` in SigArgs switches it to the plain form's second stage.
template <int NG, int PPL>
__global__ void __launch_bounds__(kSigThreads) k_sig(const __grid_constant__ SigArgs A) {
    __shared__ SigSmem<PPL> sm;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const uint64_t nwarps = (uint64_t)gridDim.x * (kSigThreads / 32);
    const uint32_t n = NG > 0 ? (uint32_t)NG : A.ngram;
    LaneCoef<PPL> cf;
    cf.load(A.c, A.npc, lane);
    uint32_t *hbuf = reinterpret_cast<uint32_t *>(sm.hbuf[wib]);
    for (uint64_t d = (uint64_t)blockIdx.x * (kSigThreads / 32) + wib; d < A.D; d += nwarps) {
        const uint64_t o0 = A.offsets[d], o1 = A.offsets[d + 1];
        const uint64_t L = o1 - o0;
        const uint32_t *tk = A.tokens + (o0 - A.tok_base);
        const uint32_t *hs = A.hashes ? A.hashes + (o0 - A.tok_base) : nullptr;
        uint32_t mn[PPL];
        fold_range<NG, PPL>(mn, cf, tk, L, n, 0, shingle_count(L, n), hs, hbuf, lane);
        sig_epilogue<PPL>(A, d, mn, sm.sig[wib], lane);
    }
}

// Plain form, stage 1: shingle hashes to global memory.
template <int NG>
__global__ void __launch_bounds__(kSigThreads) k_shingle_hash(const __grid_constant__ SigArgs A) {
    const int lane = threadIdx.x & 31;
    const uint64_t nwarps = (uint64_t)gridDim.x * (kSigThreads / 32);
    const uint32_t n = NG > 0 ? (uint32_t)NG : A.ngram;
    for (uint64_t d = (uint64_t)blockIdx.x * (kSigThreads / 32) + (threadIdx.x >> 5); d < A.D;
         d += nwarps) {
        const uint64_t o0 = A.offsets[d], o1 = A.offsets[d + 1];
        const uint64_t L = o1 - o0;
        const uint32_t *tk = A.tokens + (o0 - A.tok_base);
        uint32_t *out = A.hash_out + (o0 - A.tok_base);
        if (L >= n) {
            const uint64_t S = L - n + 1;
            for (uint64_t s0 = 0; s0 < L; s0 += 32) {
                uint32_t h = 0u;
                if (s0 < S) h = window_hash<NG>(tk, L, S, s0, lane, n);
                if (s0 + lane < S) out[s0 + lane] = h;
                else if (s0 + lane < L) out[s0 + lane] = 0u;
            }
        } else if (L > 0) {
            for (uint64_t s = lane; s < L; s += 32) out[s] = 0u;
            __syncwarp();
            if (lane == 0) out[0] = bswap32(sha1_h0_tokens(tk, (uint32_t)L));
        }
    }
}

}  // namespace lshb
