// Bloom-stage kernel arguments, device helpers and launch wrappers.
#pragma once

#include "lshb_device.cuh"
#include "lshb_internal.h"

namespace lshb {

constexpr uint32_t kErrTableFull = 1u;   // resolution table overflowed
constexpr uint32_t kErrQueue = 2u;       // persistent kernel work-queue inconsistency

// Every kernel of the stage walks (band, document) pairs band by band: a 2-D
// grid of (document blocks, bands), dispatched in that order, so the blocks
// resident at any moment work on one band's filter (116.8 MB at n = 39M,
// p = 1e-5: it stays in the 129 MB L2) and on that band's sketch.
constexpr int kBloomThreads = 256;

// Block sizes chosen so that every kernel of the stage fits beside the
// persistent signature kernel in one freed block slot of an SM (10,240
// registers with that kernel at 9 of its 10 blocks per SM): the batched form
// runs the Bloom stage of one chunk while the next chunk's signatures are
// computed.  The probe kernel (60 registers) takes 128-thread blocks, the
// status/compaction kernels 256 instead of 1024.
constexpr int kProbeThreads = 128;
constexpr int kStatusThreads = 256;

struct BloomArgs {
    uint64_t D;
    const uint64_t *D_dev;      // when set, the batch size is read from device memory
    uint32_t bands, k;
    uint32_t layout;            // 0 standard filter, 1 256-bit blocked filter, 2 exact key sets
    uint64_t m_bits, words_per_filter;
    uint64_t exact_cap;         // exact layout: slots of each band's key table (power of two)
    uint32_t *filters;          // bands x words_per_filter
    const uint64_t *keys;       // band j of document d at keys[d * key_sd + j * key_sj]
    uint64_t key_sd, key_sj;    // row-major (bands, 1) or band-major (1, row length)
    uint64_t *miss;             // bands x mstride, band-major: bit u = probe u found a clear bit
    uint64_t mstride;           // row stride of miss (>= D)
    uint32_t *sketch;           // bands x (sketch_cells / 16) words of 2-bit cells
    uint64_t sketch_cells;      // cells per band, a multiple of 16
    uint8_t *status;            // D: 1 duplicate whatever the order, 2 uncertain, 0 not duplicate
    uint64_t *cand;             // D: candidate bands
    uint8_t *prehit;            // D
    uint32_t *error;            // device error word
    // Passes over one slice of each band's filter: only positions in filter
    // words [word_lo, word_hi) are handled.  The insert runs one pass per
    // slice; the probe can (the first pass writes the miss masks, later ones
    // OR into them, the last one records the documents with a band that
    // missed nothing) but runs as one pass.
    uint64_t word_lo, word_hi;
    uint32_t first_pass, last_pass;
};

// Bytes of a band's filter one insert pass covers: the slice stays in the
// 129 MB L2 while the pass's atomic ORs land in it, instead of each OR
// dragging a line in from DRAM and writing a dirty one back.  Measured on the
// 8M-document Pareto batch (2^20-document chunks, 116.8 MB filters): the
// Bloom stage outside the probes takes 36.4 ms with one pass, 28.8 ms with
// 64 MB slices, 31.6 ms with 32 MB slices.  Probes are not sliced: a probe
// pass recomputes every key's positions whatever its slice, and 64 MB slices
// made the probes 26 ms against 22 ms in one pass (32 MB: 51 ms).
constexpr uint64_t kSliceBytes = 64ull << 20;

// Resolution table of the candidate bits of the uncertain documents: one
// open-addressing segment per band (keys are positions inside that band's
// filter, or the band key itself in the exact layout; ~0 = empty), so a key
// is identified by (band, position) exactly.  After each segment one more
// slot stands for the position 2^64 - 1 (0 there = present), which only the
// exact layout's 64-bit keys can take.
struct ResolveTable {
    uint64_t *keys;
    uint64_t seg_base[kMaxBands];   // first slot of band j's segment
    uint32_t seg_mask[kMaxBands];   // segment capacity - 1 (power of two)
    uint32_t *first_fixed;          // earliest order-independent setter per slot
    uint32_t *first;                // earliest inserted setter per slot, this sweep
    uint32_t *slots;                // nu x bands x k slot ids (~0 = none)
    uint8_t *ins;                   // nu: inserted in the current sweep
    uint8_t *udup;                  // nu: duplicate in the current sweep
    uint32_t *ctl;                  // sweep control: [0] changed, [1] done, [2] sweeps run
};

constexpr uint32_t kNone = 0xffffffffu;

__device__ __forceinline__ uint64_t batch_docs(const BloomArgs &A) {
    return A.D_dev ? *A.D_dev : A.D;
}

__device__ __forceinline__ uint64_t band_key(const BloomArgs &A, uint64_t d, uint32_t j) {
    return A.keys[d * A.key_sd + (uint64_t)j * A.key_sj];
}

// Sketch cell of position `pos` in its band's sketch: multiplicative hash,
// then Lemire's range reduction to the band's cell count.
__device__ __forceinline__ uint64_t sketch_cell(uint64_t pos, uint64_t cells) {
    return __umul64hi((pos + 1) * kGolden, cells);
}

// Mark one missing position in band j's sketch: the first mark sets the
// cell's low bit, any later mark its high bit (both in one word).
__device__ __forceinline__ void sketch_mark(const BloomArgs &A, uint32_t j, uint64_t pos) {
    const uint64_t c = sketch_cell(pos, A.sketch_cells);
    uint32_t *w = A.sketch + (uint64_t)j * (A.sketch_cells >> 4) + (c >> 4);
    const uint32_t sh = 2u * (uint32_t)(c & 15);
    const uint32_t old = atomicOr(w, 1u << sh);
    if ((old >> sh) & 1u) atomicOr(w, 2u << sh);
}

// Whether a position of band j was marked at least twice.
__device__ __forceinline__ bool sketch_twice(const BloomArgs &A, uint32_t j, uint64_t pos) {
    const uint64_t c = sketch_cell(pos, A.sketch_cells);
    const uint32_t w = __ldg(A.sketch + (uint64_t)j * (A.sketch_cells >> 4) + (c >> 4));
    return (w >> (2u * (uint32_t)(c & 15) + 1u)) & 1u;
}

// Exact-key layout: the band's table of uint64 keys (empty = ~0), linear
// probing from mix64(key); the table is never more than half full.  The key
// 2^64 - 1 cannot be stored in a slot, so slot `cap` records it (0 = present).
__device__ __forceinline__ bool exact_contains(const uint64_t *T, uint64_t cap, uint64_t key) {
    if (key == ~0ull) return __ldg(T + cap) == 0ull;
    uint64_t s = mix64(key) & (cap - 1);
    for (uint64_t i = 0; i < cap; ++i) {
        const uint64_t v = __ldg(T + s);
        if (v == key) return true;
        if (v == ~0ull) return false;
        s = (s + 1) & (cap - 1);
    }
    return false;
}

__device__ __forceinline__ bool exact_insert(uint64_t *T, uint64_t cap, uint64_t key) {
    if (key == ~0ull) {
        T[cap] = 0ull;
        return true;
    }
    uint64_t s = mix64(key) & (cap - 1);
    for (uint64_t i = 0; i < cap; ++i) {
        const unsigned long long prev =
            atomicCAS((unsigned long long *)(T + s), ~0ull, (unsigned long long)key);
        if (prev == ~0ull || prev == key) return true;
        s = (s + 1) & (cap - 1);
    }
    return false;
}

// Probe one band key against its filter F (pre-batch bits): the mask of
// probes that found a clear bit; each such position is marked in the band's
// sketch.  For k <= KMAX all k loads are issued before any is used, then all
// first-level marks, then the second level: one memory round trip per phase
// instead of one per probe (positions are recomputed per phase: a few integer
// operations, fewer registers).
template <int KMAX>
__device__ __forceinline__ uint64_t probe_key(const BloomArgs &A, uint32_t j, uint64_t key) {
    const uint32_t *F = A.filters + (uint64_t)j * A.words_per_filter;
    if (A.layout == 2) {
        if (exact_contains(reinterpret_cast<const uint64_t *>(F), A.exact_cap, key)) return 0;
        sketch_mark(A, j, key);
        return 1;
    }
    const ProbeSeq ps(key, j, A.m_bits, A.layout);
    uint64_t miss = 0;
    if (A.k <= (uint32_t)KMAX) {
        uint32_t w[KMAX];
        uint32_t in = 0;  // probes whose word lies in this pass's slice
#pragma unroll
        for (int u = 0; u < KMAX; ++u) {
            const uint64_t wi = ps.pos(u) >> 5;
            const bool here = u < (int)A.k && wi >= A.word_lo && wi < A.word_hi;
            in |= (uint32_t)here << u;
            w[u] = here ? __ldg(F + wi) : 0xffffffffu;
        }
#pragma unroll
        for (int u = 0; u < KMAX; ++u)
            if (((in >> u) & 1u) && !((w[u] >> (ps.pos(u) & 31)) & 1u)) miss |= 1ull << u;
        uint32_t *S = A.sketch + (uint64_t)j * (A.sketch_cells >> 4);
#pragma unroll
        for (int u = 0; u < KMAX; ++u) {
            w[u] = 0;
            if ((miss >> u) & 1ull) {
                const uint64_t c = sketch_cell(ps.pos(u), A.sketch_cells);
                w[u] = atomicOr(S + (c >> 4), 1u << (2u * (uint32_t)(c & 15)));
            }
        }
#pragma unroll
        for (int u = 0; u < KMAX; ++u) {
            if ((miss >> u) & 1ull) {
                const uint64_t c = sketch_cell(ps.pos(u), A.sketch_cells);
                const uint32_t sh = 2u * (uint32_t)(c & 15);
                if ((w[u] >> sh) & 1u) atomicOr(S + (c >> 4), 2u << sh);
            }
        }
        return miss;
    } else {
        for (uint32_t u0 = 0; u0 < A.k; u0 += 8) {
            uint32_t w[8];
            uint32_t in = 0;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const uint64_t wi = ps.pos(u0 + i) >> 5;
                const bool here = u0 + i < A.k && wi >= A.word_lo && wi < A.word_hi;
                in |= (uint32_t)here << i;
                w[i] = here ? __ldg(F + wi) : 0xffffffffu;
            }
#pragma unroll
            for (int i = 0; i < 8; ++i)
                if (((in >> i) & 1u) && !((w[i] >> (ps.pos(u0 + i) & 31)) & 1u))
                    miss |= 1ull << (u0 + i);
        }
    }
    uint64_t mm = miss;
    while (mm) {
        const uint32_t u = __ffsll((long long)mm) - 1;
        mm &= mm - 1;
        sketch_mark(A, j, ps.pos(u));
    }
    return miss;
}

// Launch wrappers (bloom_kernels.cu).  dcap bounds the documents of the
// batch when A.D_dev is set (the grid is sized for it).
cudaError_t launch_probe(const BloomArgs &a, uint64_t dcap, cudaStream_t s);
cudaError_t launch_classify(const BloomArgs &a, uint64_t dcap, uint32_t *block_counts,
                            uint32_t *total, uint32_t *ulist, cudaStream_t s);
cudaError_t launch_count_keys(const BloomArgs &a, const uint32_t *ulist, uint32_t nu,
                              unsigned long long *band_counts, cudaStream_t s);
cudaError_t launch_resolve_setup(const BloomArgs &a, const uint32_t *ulist, uint32_t nu,
                                 const ResolveTable &t, int insert_all, cudaStream_t s);
cudaError_t launch_resolve_sweep(const BloomArgs &a, const uint32_t *ulist, uint32_t nu,
                                 const ResolveTable &t, uint64_t table_slots, int insert_all,
                                 cudaStream_t s);
cudaError_t launch_resolve_in_order(const BloomArgs &a, const uint32_t *ulist, uint32_t nu,
                                    const ResolveTable &t, uint64_t table_slots,
                                    uint32_t settled, cudaStream_t s);
cudaError_t launch_finalize_insert(const BloomArgs &a, const uint32_t *ulist, uint32_t nu,
                                   const ResolveTable &t, int insert_all, uint8_t *flags,
                                   uint8_t *insd, unsigned long long *dup_count, cudaStream_t s);
cudaError_t launch_popcount(const uint32_t *words, uint64_t n, unsigned long long *out,
                            cudaStream_t s);
cudaError_t launch_count_occupied(const uint64_t *slots, uint64_t n, unsigned long long *out,
                                  cudaStream_t s);

}  // namespace lshb
