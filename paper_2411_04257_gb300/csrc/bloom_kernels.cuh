// Bloom-stage kernel arguments and launch wrappers.
#pragma once

#include "lshb_device.cuh"
#include "lshb_internal.h"

namespace lshb {

constexpr uint32_t kErrTableFull = 1u;   // resolution table overflowed
constexpr uint32_t kErrQueue = 2u;       // persistent kernel work-queue inconsistency

struct BloomArgs {
    uint64_t D;
    const uint64_t *D_dev;      // when set, the batch size is read from device memory
    uint32_t bands, k;
    uint32_t layout;            // 0 standard filter, 1 256-bit blocked filter, 2 exact key sets
    uint64_t m_bits, words_per_filter;
    uint32_t *filters;          // bands x words_per_filter
    const uint64_t *keys;       // D x bands
    uint64_t *miss;             // D x bands: bit u set when probe u found a clear bit
    uint32_t *sketch1, *sketch2;
    uint32_t sketch_bits_log2;
    uint8_t *status;            // D: 1 duplicate whatever the order, 2 uncertain, 0 not duplicate
    uint64_t *cand;             // D: candidate bands
    uint8_t *prehit;            // D
    uint32_t *error;            // device error word
};

struct ResolveTable {
    uint64_t *keys;             // global bit ids, ~0 = empty
    uint32_t mask;              // capacity - 1 (power of two)
    uint32_t *first_fixed;      // earliest order-independent setter per slot
    uint32_t *first;            // earliest inserted setter per slot, this sweep
    uint32_t *slots;            // nu x bands x k slot ids (~0 = none)
    uint8_t *ins;               // nu: inserted in the current sweep
    uint8_t *udup;              // nu: duplicate in the current sweep
    uint32_t *changed;
};

__device__ __forceinline__ uint64_t sketch_index(uint64_t g, uint32_t log2n) {
    return (g * kGolden) >> (64 - log2n);
}

// Probe one band key against its filter F (pre-batch bits): returns the mask
// of probes that found a clear bit, and marks each such bit in the two-level
// sketch (first mark sets sketch1, any later mark sets sketch2).
// For k <= KMAX all k sector loads are issued before any is used, then all
// first-level sketch atomics, then the second level: one memory round trip
// per phase instead of one per probe.  Positions are recomputed per phase
// (three integer operations) rather than held in registers.
template <int KMAX>
__device__ __forceinline__ uint64_t probe_band_unrolled(const uint32_t *F, const ProbeSeq &ps,
                                                        uint32_t j, uint32_t k, uint64_t m,
                                                        uint32_t *sk1, uint32_t *sk2,
                                                        uint32_t sk_log2) {
    uint32_t w[KMAX];
#pragma unroll
    for (int u = 0; u < KMAX; ++u)
        w[u] = (u < (int)k) ? __ldg(F + (ps.pos(u) >> 5)) : 0xffffffffu;
    uint64_t miss = 0;
#pragma unroll
    for (int u = 0; u < KMAX; ++u)
        if (!((w[u] >> (ps.pos(u) & 31)) & 1u)) miss |= 1ull << u;
    uint32_t old[KMAX];
#pragma unroll
    for (int u = 0; u < KMAX; ++u) {
        old[u] = 0;
        if ((miss >> u) & 1ull) {
            const uint64_t si = sketch_index((uint64_t)j * m + ps.pos(u), sk_log2);
            old[u] = atomicOr(sk1 + (si >> 5), 1u << (si & 31));
        }
    }
#pragma unroll
    for (int u = 0; u < KMAX; ++u) {
        if ((miss >> u) & 1ull) {
            const uint64_t si = sketch_index((uint64_t)j * m + ps.pos(u), sk_log2);
            const uint32_t bit = 1u << (si & 31);
            if (old[u] & bit) atomicOr(sk2 + (si >> 5), bit);
        }
    }
    return miss;
}

// Exact-key layout: the band's table of uint64 keys (empty = ~0), linear
// probing from mix64(key); the table is never more than half full.
__device__ __forceinline__ bool exact_contains(const uint64_t *T, uint64_t cap, uint64_t key) {
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
    uint64_t s = mix64(key) & (cap - 1);
    for (uint64_t i = 0; i < cap; ++i) {
        const unsigned long long prev =
            atomicCAS((unsigned long long *)(T + s), ~0ull, (unsigned long long)key);
        if (prev == ~0ull || prev == key) return true;
        s = (s + 1) & (cap - 1);
    }
    return false;
}

// Sketch mark of one missing position (first mark sketch1, later ones sketch2).
__device__ __forceinline__ void sketch_mark(uint64_t g, uint32_t *sk1, uint32_t *sk2,
                                            uint32_t sk_log2) {
    const uint64_t si = sketch_index(g, sk_log2);
    const uint32_t bit = 1u << (si & 31);
    const uint32_t old = atomicOr(sk1 + (si >> 5), bit);
    if (old & bit) atomicOr(sk2 + (si >> 5), bit);
}

// Compact form (few registers): loads in groups of 8, atomics one by one.
// Used where the probe is a small phase of a register-heavy kernel.
// words_per_filter (uint32 words) sizes the exact-key table: words/2 slots.
__device__ __forceinline__ uint64_t probe_band(const uint32_t *F, uint64_t words_per_filter,
                                               uint64_t key, uint32_t j, uint32_t k, uint64_t m,
                                               uint32_t layout, uint32_t *sk1, uint32_t *sk2,
                                               uint32_t sk_log2) {
    if (layout == 2) {
        if (exact_contains(reinterpret_cast<const uint64_t *>(F), words_per_filter / 2, key)) return 0;
        sketch_mark((uint64_t)j * m + key, sk1, sk2, sk_log2);
        return 1;
    }
    const ProbeSeq ps(key, j, m, layout);
    uint64_t miss = 0;
    for (uint32_t u0 = 0; u0 < k; u0 += 8) {
        uint64_t q[8];
        uint32_t w[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            q[i] = ps.pos(u0 + i);
            w[i] = (u0 + i < k) ? __ldg(F + (q[i] >> 5)) : 0xffffffffu;
        }
#pragma unroll
        for (int i = 0; i < 8; ++i)
            if (!((w[i] >> (q[i] & 31)) & 1u)) miss |= 1ull << (u0 + i);
    }
    uint64_t mm = miss;
    while (mm) {
        const uint32_t u = __ffsll((long long)mm) - 1;
        mm &= mm - 1;
        const uint64_t si = sketch_index((uint64_t)j * m + ps.pos(u), sk_log2);
        const uint32_t bit = 1u << (si & 31);
        const uint32_t old = atomicOr(sk1 + (si >> 5), bit);
        if (old & bit) atomicOr(sk2 + (si >> 5), bit);
    }
    return miss;
}

cudaError_t launch_probe_mark(const BloomArgs &a, cudaStream_t s);
cudaError_t launch_classify(const BloomArgs &a, uint32_t *block_counts, uint32_t *total,
                            uint32_t *ulist, cudaStream_t s);
cudaError_t launch_count_keys(const BloomArgs &a, const uint32_t *ulist, uint32_t nu,
                              unsigned long long *count, cudaStream_t s);
cudaError_t launch_resolve_setup(const BloomArgs &a, const uint32_t *ulist, uint32_t nu,
                                 const ResolveTable &t, int insert_all, cudaStream_t s);
cudaError_t launch_resolve_iteration(const BloomArgs &a, const uint32_t *ulist, uint32_t nu,
                                     const ResolveTable &t, int insert_all, cudaStream_t s);
cudaError_t launch_resolve_sequential(const BloomArgs &a, const uint32_t *ulist, uint32_t nu,
                                      const ResolveTable &t, cudaStream_t s);
cudaError_t launch_finalize_insert(const BloomArgs &a, const uint32_t *ulist, uint32_t nu,
                                   const ResolveTable &t, int insert_all, uint8_t *flags,
                                   uint8_t *insd, unsigned long long *dup_count, cudaStream_t s);
cudaError_t launch_popcount(const uint32_t *words, uint64_t n, unsigned long long *out,
                            cudaStream_t s);
cudaError_t launch_count_occupied(const uint64_t *slots, uint64_t n, unsigned long long *out,
                                  cudaStream_t s);

}  // namespace lshb
