// Signature-stage kernels: warp-cooperative shingling, SHA-1 shingle hash,
// MinHash minimum over a pass of PC permutations, band-key epilogue.
//
// Layout: one warp per document (plain form).  Lane l hashes shingle s0+l of
// each 32-shingle step and folds it into its own PC running minima; the
// coefficients are constant-bank operands (the kernel parameter), so the hot
// loop is IMAD.WIDE + ALU work on registers only.  At the end of a document
// the 32 lanes' minima are reduced across the warp.
#pragma once

#include "lshb_device.cuh"
#include "lshb_internal.h"

namespace lshb {

template <int PC>
struct SigOcc {
    // Register cap: the PC minima stay live across the SHA-1 of the next step,
    // which needs about 30 more; below these caps ptxas spills.
    static constexpr int kMaxRegs = PC >= 96 ? 200 : 128;
};

// Fold one shingle hash into the PC running minima.
template <int PC>
__device__ __forceinline__ void fold_perms(uint32_t (&mn)[PC], uint32_t h, const PermSlice &c) {
#pragma unroll
    for (int i = 0; i < PC; ++i) mn[i] = min(mn[i], perm_lo32(h, c.a0[i], c.a1[i], c.b0[i], c.b1[i]));
}

// Minimum across the warp, every lane ends with the full result.
template <int PC>
__device__ __forceinline__ void warp_min_all(uint32_t (&mn)[PC]) {
#pragma unroll
    for (int i = 0; i < PC; ++i) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) mn[i] = min(mn[i], __shfl_xor_sync(LSHB_FULL_MASK, mn[i], off));
    }
}

// Hash of shingle s0+lane of a document of L tokens (L >= n).  For NG > 0 the
// window is assembled with shuffles from two coalesced loads; lanes past the
// last shingle return an unspecified value.
template <int NG>
__device__ __forceinline__ uint32_t window_hash(const uint32_t *tk, uint64_t L, uint64_t S,
                                                uint64_t s0, int lane, uint32_t n) {
    if constexpr (NG > 0) {
        const uint64_t ia = s0 + lane;
        const uint32_t ta = ia < L ? __ldg(tk + ia) : 0u;
        uint32_t tb = 0u;
        if constexpr (NG > 1) {
            const uint64_t ib = s0 + 32 + lane;
            if (lane < NG - 1 && ib < L) tb = __ldg(tk + ib);
        }
        uint32_t w[NG];
        w[0] = bswap32(ta);
#pragma unroll
        for (int k = 1; k < NG; ++k) {
            const uint32_t v = lane >= k ? ta : tb;
            w[k] = bswap32(__shfl_sync(LSHB_FULL_MASK, v, (lane + k) & 31));
        }
        return bswap32(sha1_h0_one_block<NG>(w));
    } else {
        uint64_t s = s0 + lane;
        if (s >= S) s = S - 1;
        return bswap32(sha1_h0_tokens(tk + s, n));
    }
}

// Write the pass minima and (single full pass) the band keys.
template <int PC>
__device__ __forceinline__ void sig_epilogue(const SigArgs &A, uint64_t d, uint32_t (&mn)[PC],
                                             uint32_t *smw, int lane) {
    if (A.sig_out) {
        uint32_t *row = A.sig_out + d * A.P + A.p0;
#pragma unroll
        for (int i = 0; i < PC; ++i)
            if ((i & 31) == lane && i < (int)A.npc) row[i] = mn[i];
    }
    if (A.keys_out) {
#pragma unroll
        for (int i = 0; i < PC; ++i)
            if ((i & 31) == lane) smw[i] = mn[i];
        __syncwarp();
        for (uint32_t j = lane; j < A.bands; j += 32) {
            uint64_t s = 0;
            for (uint32_t t = 0; t < A.rows; ++t) s += smw[j * A.rows + t];
            A.keys_out[d * A.bands + j] = s;
        }
        __syncwarp();
    }
}

template <int NG, int PC>
__global__ void __maxnreg__(SigOcc<PC>::kMaxRegs)
k_sig_fused(const __grid_constant__ SigArgs A) {
    __shared__ uint32_t sm[kSigThreads / 32][PC];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const uint64_t nwarps = (uint64_t)gridDim.x * (kSigThreads / 32);
    const uint32_t n = NG > 0 ? (uint32_t)NG : A.ngram;
    for (uint64_t d = (uint64_t)blockIdx.x * (kSigThreads / 32) + wib; d < A.D; d += nwarps) {
        const uint64_t o0 = A.offsets[d], o1 = A.offsets[d + 1];
        const uint64_t L = o1 - o0;
        const uint32_t *tk = A.tokens + (o0 - A.tok_base);
        uint32_t mn[PC];
#pragma unroll
        for (int i = 0; i < PC; ++i) mn[i] = 0xffffffffu;
        if (L >= n) {
            const uint64_t S = L - n + 1;
            for (uint64_t s0 = 0; s0 < S; s0 += 32) {
                uint32_t h = window_hash<NG>(tk, L, S, s0, lane, n);
                const uint32_t h0 = __shfl_sync(LSHB_FULL_MASK, h, 0);
                if (s0 + lane >= S) h = h0;  // a repeat of a real shingle leaves the minima unchanged
                fold_perms<PC>(mn, h, A.c);
            }
        } else if (L > 0) {
            const uint32_t h = bswap32(sha1_h0_tokens(tk, (uint32_t)L));
            fold_perms<PC>(mn, h, A.c);
        }
        warp_min_all<PC>(mn);
        sig_epilogue<PC>(A, d, mn, sm[wib], lane);
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

// Plain form, stage 2: MinHash minima over precomputed shingle hashes.
template <int PC>
__global__ void __maxnreg__(SigOcc<PC>::kMaxRegs)
k_minhash_hashes(const __grid_constant__ SigArgs A) {
    __shared__ uint32_t sm[kSigThreads / 32][PC];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const uint64_t nwarps = (uint64_t)gridDim.x * (kSigThreads / 32);
    for (uint64_t d = (uint64_t)blockIdx.x * (kSigThreads / 32) + wib; d < A.D; d += nwarps) {
        const uint64_t o0 = A.offsets[d], o1 = A.offsets[d + 1];
        const uint64_t L = o1 - o0;
        const uint64_t S = L == 0 ? 0 : (L < A.ngram ? 1 : L - A.ngram + 1);
        const uint32_t *hs = A.hashes + (o0 - A.tok_base);
        uint32_t mn[PC];
#pragma unroll
        for (int i = 0; i < PC; ++i) mn[i] = 0xffffffffu;
        if (S > 0) {
            const uint32_t hfirst = __ldg(hs);
            for (uint64_t s0 = 0; s0 < S; s0 += 32) {
                const uint32_t h = (s0 + lane < S) ? __ldg(hs + s0 + lane) : hfirst;
                fold_perms<PC>(mn, h, A.c);
            }
        }
        warp_min_all<PC>(mn);
        sig_epilogue<PC>(A, d, mn, sm[wib], lane);
    }
}

}  // namespace lshb
