// Device side of the batched form: the per-chunk parameter block, the item
// bookkeeping kernels (counts, scan, item -> document map) and the persistent
// fused kernel k_batched (SHA-1 + MinHash over a work queue of (document,
// shingle range) items, then the band keys of each document).
#pragma once

#include "bloom_kernels.cuh"
#include "lshb_internal.h"
#include "segment.h"
#include "sig_kernels.cuh"

namespace lshb {

constexpr int kBatchThreads = 64;
constexpr uint32_t kItemCandidates[] = {64, 128, 256, 512, 1024};

struct DynParams {
    const uint64_t *offsets;  // D+1
    const uint32_t *tokens;   // document d at tokens[offsets[d] - tok_base]
    uint64_t tok_base;
    uint64_t D;
    uint64_t n_items;         // written on the device by the scan
    const Segment *segs;      // nseg > 0: the launch covers these batches instead
    uint32_t nseg;
    uint32_t active_blocks;   // persistent-kernel blocks that take items (0: all); the
                              // others return at once and leave their SM slots free
};

// Where document d of a launch lives: its offsets (indexed by `local`), its
// token base and its band keys (band j at keys[j * key_sj]).
struct DocRef {
    const uint64_t *offsets;
    const uint32_t *tokens;
    uint64_t tok_base, local;
    uint64_t *keys;
    uint64_t key_sj;
};

// A single-batch launch writes the keys band-major (band j of document d at
// keys[j * key_rows + d], so the band-by-band Bloom kernels read them
// coalesced); a multi-batch launch writes each batch's keys row-major.
__device__ __forceinline__ DocRef doc_ref(const DynParams &dp, uint64_t *keys, uint64_t key_rows,
                                          uint32_t bands, uint64_t d) {
    DocRef r;
    if (dp.nseg == 0) {
        r.offsets = dp.offsets;
        r.tokens = dp.tokens;
        r.tok_base = dp.tok_base;
        r.local = d;
        r.keys = keys + d;
        r.key_sj = key_rows;
        return r;
    }
    uint32_t lo = 0, hi = dp.nseg - 1;  // last segment with doc0 <= d
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (dp.segs[mid].doc0 <= d) lo = mid; else hi = mid - 1;
    }
    const Segment &sg = dp.segs[lo];
    r.offsets = sg.offsets;
    r.tokens = sg.tokens;
    r.tok_base = sg.tok_base;
    r.local = d - sg.doc0;
    r.keys = sg.keys_out + r.local * bands;
    r.key_sj = 1;
    return r;
}

struct BatchArgs {
    DynParams *dyn;
    uint32_t item_shingles, ngram, P, npc, bands, rows, band_key;
    uint32_t *item_count;      // D
    uint64_t *item_start;      // D+1
    uint64_t *block_sums;      // scan partials
    uint32_t *item_doc;        // n_items
    uint64_t item_cap;         // capacity of item_doc
    uint32_t *pending;         // D: items of the document not finished yet
    uint32_t *sig_partial;     // D x P: merged minima of split documents
    unsigned long long *queue;
    uint64_t *keys;            // single-batch launches: bands x key_rows, band-major
    uint64_t key_rows;         // row length of keys (the chunk capacity)
    uint64_t *cand;            // D: cleared for the Bloom stage (nullptr: left alone)
    uint8_t *prehit;           // D: cleared for the Bloom stage (nullptr: left alone)
    uint32_t *error;
    PermSlice c;
};

__device__ __forceinline__ uint64_t items_of(uint64_t L, uint32_t n, uint32_t item) {
    const uint64_t S = shingle_count(L, n);
    return S == 0 ? 1 : (S + item - 1) / item;
}

// Per document: item count, pending counter, cleared Bloom-stage flags and,
// for a document split over several items, a signature row of 2^32-1.
__global__ void k_batch_prepare(const __grid_constant__ BatchArgs A) {
    const DynParams dp = *A.dyn;
    for (uint64_t d = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; d < dp.D;
         d += (uint64_t)gridDim.x * blockDim.x) {
        const DocRef r = doc_ref(dp, A.keys, A.key_rows, A.bands, d);
        const uint64_t L = r.offsets[r.local + 1] - r.offsets[r.local];
        const uint64_t it = items_of(L, A.ngram, A.item_shingles);
        A.item_count[d] = (uint32_t)it;
        A.pending[d] = (uint32_t)it;
        if (A.cand) A.cand[d] = 0;
        if (A.prehit) A.prehit[d] = 0;
        if (it > 1) {
            uint32_t *row = A.sig_partial + d * A.P;
            for (uint32_t p = 0; p < A.P; ++p) row[p] = 0xffffffffu;
        }
    }
}

// Band-major keys (bands x rows) of the first D documents to row-major
// (D x bands), for callers that asked for the keys.
__global__ void k_keys_row_major(const uint64_t *__restrict__ src, uint64_t rows, uint64_t D,
                                 uint32_t bands, uint64_t *__restrict__ dst) {
    const uint64_t n = D * bands;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t d = i / bands;
        const uint32_t j = (uint32_t)(i - d * bands);
        dst[i] = src[(uint64_t)j * rows + d];
    }
}

// Exclusive scan of item counts into item_start (D+1 entries), three phases.
constexpr int kScanBlock = 1024;

__device__ __forceinline__ uint64_t block_exclusive_scan(uint64_t v, uint64_t *tot) {
    __shared__ uint64_t warp_sums[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint64_t x = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint64_t y = __shfl_up_sync(LSHB_FULL_MASK, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) warp_sums[w] = x;
    __syncthreads();
    if (w == 0) {
        uint64_t s = warp_sums[lane];
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint64_t y = __shfl_up_sync(LSHB_FULL_MASK, s, off);
            if (lane >= off) s += y;
        }
        warp_sums[lane] = s;  // inclusive over warps
    }
    __syncthreads();
    const uint64_t before = (w > 0 ? warp_sums[w - 1] : 0) + x - v;
    if (tot) *tot = warp_sums[31];
    __syncthreads();
    return before;
}

__global__ void __launch_bounds__(kScanBlock) k_scan_reduce(const __grid_constant__ BatchArgs A) {
    const uint64_t D = A.dyn->D;
    const uint64_t i = (uint64_t)blockIdx.x * kScanBlock + threadIdx.x;
    uint64_t tot = 0;
    block_exclusive_scan(i < D ? A.item_count[i] : 0, &tot);
    if (threadIdx.x == 0) A.block_sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanBlock) k_scan_top(const __grid_constant__ BatchArgs A,
                                                         uint32_t nb) {
    __shared__ uint64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint32_t base = 0; base < nb; base += kScanBlock) {
        const uint32_t i = base + threadIdx.x;
        uint64_t tot = 0;
        const uint64_t ex = block_exclusive_scan(i < nb ? A.block_sums[i] : 0, &tot);
        if (i < nb) A.block_sums[i] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        A.dyn->n_items = carry;
        if (carry > A.item_cap) atomicOr(A.error, kErrQueue);
    }
}

__global__ void __launch_bounds__(kScanBlock) k_scan_down(const __grid_constant__ BatchArgs A) {
    const uint64_t D = A.dyn->D;
    const uint64_t i = (uint64_t)blockIdx.x * kScanBlock + threadIdx.x;
    const uint64_t ex = block_exclusive_scan(i < D ? A.item_count[i] : 0, nullptr);
    if (i < D) A.item_start[i] = A.block_sums[blockIdx.x] + ex;
    if (i == 0) A.item_start[D] = A.dyn->n_items;
}

__global__ void k_expand(const __grid_constant__ BatchArgs A) {
    const uint64_t D = A.dyn->D;
    const uint64_t cap = A.item_cap;
    for (uint64_t d = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; d < D;
         d += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t s = A.item_start[d], n = A.item_count[d];
        for (uint64_t t = 0; t < n && s + t < cap; ++t) A.item_doc[s + t] = (uint32_t)d;
    }
}

// The persistent kernel.  Every warp pops items until the queue is drained;
// nothing waits on another warp, so the kernel cannot stall.
template <int NG, int PPL>
__global__ void __launch_bounds__(kBatchThreads) k_batched(const __grid_constant__ BatchArgs A) {
    __shared__ SigSmem<PPL> sm;
    const DynParams dp = *A.dyn;
    if (dp.active_blocks && blockIdx.x >= dp.active_blocks) return;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const uint32_t n = NG > 0 ? (uint32_t)NG : A.ngram;
    LaneCoef<PPL> cf;
    cf.load(A.c, A.npc, lane);
    uint32_t *hbuf = reinterpret_cast<uint32_t *>(sm.hbuf[wib]);
    uint32_t *sigbuf = sm.sig[wib];
    const uint64_t n_items = min(dp.n_items, A.item_cap);
    for (;;) {
        unsigned long long it = 0;
        if (lane == 0) it = atomicAdd(A.queue, 1ull);
        it = __shfl_sync(LSHB_FULL_MASK, it, 0);
        if (it >= n_items) break;
        const uint64_t d = A.item_doc[it];
        const uint64_t ibeg = A.item_start[d];
        const uint64_t icnt = A.item_start[d + 1] - ibeg;
        if (d >= dp.D || it < ibeg || it - ibeg >= icnt) {
            if (lane == 0) atomicOr(A.error, kErrQueue);
            continue;
        }
        const DocRef r = doc_ref(dp, A.keys, A.key_rows, A.bands, d);
        const uint64_t o0 = r.offsets[r.local];
        const uint64_t L = r.offsets[r.local + 1] - o0;
        const uint32_t *tk = r.tokens + (o0 - r.tok_base);
        const uint64_t S = shingle_count(L, n);
        const uint64_t s_begin = (it - ibeg) * A.item_shingles;
        const uint64_t s_end = min(S, s_begin + A.item_shingles);
        uint32_t mn[PPL];
        fold_range<NG, PPL>(mn, cf, tk, L, n, s_begin, s_end, nullptr, hbuf, lane);
        if (icnt > 1) {
            uint32_t *row = A.sig_partial + d * A.P;
#pragma unroll
            for (int t = 0; t < PPL; ++t)
                if (lane + 32 * t < (int)A.npc) atomicMin(row + lane + 32 * t, mn[t]);
            __threadfence();
            __syncwarp();
            uint32_t last = 0;
            if (lane == 0) last = atomicSub(A.pending + d, 1u) == 1u;
            last = __shfl_sync(LSHB_FULL_MASK, last, 0);
            if (!last) continue;
            __threadfence();
#pragma unroll
            for (int t = 0; t < PPL; ++t)
                if (lane + 32 * t < (int)A.npc) mn[t] = __ldcg(row + lane + 32 * t);
        }
        // band keys of this document (Sec. 4.1)
        __syncwarp();
#pragma unroll
        for (int t = 0; t < PPL; ++t) sigbuf[lane + 32 * t] = mn[t];
        __syncwarp();
        for (uint32_t j = lane; j < A.bands; j += 32)
            r.keys[j * r.key_sj] = band_key_of(sigbuf + j * A.rows, A.rows, j, A.band_key);
        __syncwarp();
    }
}

}  // namespace lshb
