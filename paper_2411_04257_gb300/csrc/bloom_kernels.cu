// Bloom stage of the LSHBloom path: probe each band key in its filter
// (Sec. 4.2), decide each document exactly as the sequential stream would
// (Sec. 2.1, Sec. 4.4.2), and insert the documents that the insert rule
// admits (Sec. 4.1).
//
// The batch is judged in parallel.  A band of document d hits when each of its
// k probed bits is set before the batch or by an inserted document d' < d of
// the batch.  The kernels below find that without a sort:
//   1. probe_mark   reads the pre-batch bits; records, per (doc, band), which
//                   probes found a clear bit ("missing"); marks each missing
//                   bit in a two-level sketch (seen once / seen twice);
//   2. classify     a band whose every missing bit was marked twice is a
//                   candidate (some other document may set those bits); a
//                   document with a band with no missing bit is a duplicate
//                   whatever the order; one with neither is not a duplicate;
//                   the rest are "uncertain";
//   3. resolve      uncertain documents only: their candidate bits go into a
//                   hash table; every inserting document records itself as a
//                   setter with atomicMin; uncertain documents iterate
//                   ins <- not dup(ins) (a Jacobi sweep) until nothing changes,
//                   which is the unique sequential answer because document d
//                   depends only on documents before it;
//   4. insert       atomicOr of the missing bits of inserted documents.
// Sketch collisions only add candidates; they never drop one, so the result
// is exact.
#include "bloom_kernels.cuh"

namespace lshb {

__global__ void k_probe_mark(const __grid_constant__ BloomArgs A) {
    const uint64_t n = A.D * A.bands;
    for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t j = (uint32_t)(idx % A.bands);
        const uint32_t *F = A.filters + (uint64_t)j * A.words_per_filter;
        if (A.k <= 24 && A.layout != 2) {
            const ProbeSeq ps(A.keys[idx], j, A.m_bits, A.layout);
            A.miss[idx] = probe_band_unrolled<24>(F, ps, j, A.k, A.m_bits, A.sketch1, A.sketch2,
                                                  A.sketch_bits_log2);
        } else {
            A.miss[idx] = probe_band(F, A.words_per_filter, A.keys[idx], j, A.k, A.m_bits, A.layout,
                                     A.sketch1, A.sketch2, A.sketch_bits_log2);
        }
    }
}

__device__ __forceinline__ uint64_t batch_docs(const BloomArgs &A) {
    return A.D_dev ? *A.D_dev : A.D;
}

__global__ void k_classify(const __grid_constant__ BloomArgs A) {
    const uint64_t n = batch_docs(A) * A.bands;
    for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t d = idx / A.bands;
        const uint32_t j = (uint32_t)(idx % A.bands);
        const uint64_t miss = A.miss[idx];
        if (miss == 0) {
            A.prehit[d] = 1;
            continue;
        }
        const ProbeSeq ps(A.keys[idx], j, A.m_bits, A.layout);
        bool all = true;
        uint64_t mm = miss;
        while (mm && all) {
            const uint32_t u = __ffsll((long long)mm) - 1;
            mm &= mm - 1;
            const uint64_t g = (uint64_t)j * A.m_bits + ps.pos(u);
            const uint64_t si = sketch_index(g, A.sketch_bits_log2);
            all = (__ldg(A.sketch2 + (si >> 5)) >> (si & 31)) & 1u;
        }
        if (all) atomicOr((unsigned long long *)(A.cand + d), 1ull << j);
    }
}

// Status per document and the per-block count of uncertain documents.
// status: 1 = duplicate whatever the order, 2 = uncertain, 0 = not duplicate.
__global__ void __launch_bounds__(1024) k_status(const __grid_constant__ BloomArgs A,
                                                 uint32_t *block_counts) {
    __shared__ uint32_t warp_cnt[32];
    const uint64_t d = (uint64_t)blockIdx.x * 1024 + threadIdx.x;
    uint8_t st = 0;
    if (d < batch_docs(A)) {
        st = A.prehit[d] ? 1 : (A.cand[d] ? 2 : 0);
        A.status[d] = st;
    }
    const uint32_t bal = __ballot_sync(LSHB_FULL_MASK, st == 2);
    if ((threadIdx.x & 31) == 0) warp_cnt[threadIdx.x >> 5] = __popc(bal);
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t s = 0;
        for (int w = 0; w < 32; ++w) s += warp_cnt[w];
        block_counts[blockIdx.x] = s;
    }
}

// Exclusive scan of the block counts (one block; nb up to a few thousand) and
// the total in counters[0].
__global__ void __launch_bounds__(1024) k_scan_counts(uint32_t *block_counts, uint32_t nb,
                                                      uint32_t *total) {
    __shared__ uint32_t part[1024];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint32_t base = 0; base < nb; base += 1024) {
        const uint32_t i = base + threadIdx.x;
        const uint32_t v = i < nb ? block_counts[i] : 0u;
        part[threadIdx.x] = v;
        __syncthreads();
        for (uint32_t off = 1; off < 1024; off <<= 1) {
            const uint32_t add = threadIdx.x >= off ? part[threadIdx.x - off] : 0u;
            __syncthreads();
            part[threadIdx.x] += add;
            __syncthreads();
        }
        if (i < nb) block_counts[i] = carry + part[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += part[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

// Uncertain documents in increasing index order.
__global__ void __launch_bounds__(1024) k_compact(const __grid_constant__ BloomArgs A,
                                                  const uint32_t *block_offsets, uint32_t *ulist) {
    __shared__ uint32_t warp_pre[32];
    const uint64_t d = (uint64_t)blockIdx.x * 1024 + threadIdx.x;
    const bool u = d < batch_docs(A) && A.status[d] == 2;
    const uint32_t bal = __ballot_sync(LSHB_FULL_MASK, u);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) warp_pre[w] = __popc(bal);
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t s = 0;
        for (int i = 0; i < 32; ++i) {
            const uint32_t c = warp_pre[i];
            warp_pre[i] = s;
            s += c;
        }
    }
    __syncthreads();
    if (u) ulist[block_offsets[blockIdx.x] + warp_pre[w] + __popc(bal & ((1u << lane) - 1))] =
        (uint32_t)d;
}

// ---- exact resolution of uncertain documents --------------------------------

constexpr uint64_t kEmpty = ~0ull;
constexpr uint32_t kNone = 0xffffffffu;

__device__ __forceinline__ uint32_t ht_find(const uint64_t *keys, uint32_t mask, uint64_t g) {
    uint32_t s = (uint32_t)(mix64(g) & mask);
    for (uint32_t i = 0; i <= mask; ++i) {
        const uint64_t k = keys[s];
        if (k == g) return s;
        if (k == kEmpty) return kNone;
        s = (s + 1) & mask;
    }
    return kNone;
}

__device__ __forceinline__ bool ht_insert(uint64_t *keys, uint32_t mask, uint64_t g) {
    uint32_t s = (uint32_t)(mix64(g) & mask);
    for (uint32_t i = 0; i <= mask; ++i) {
        const unsigned long long prev =
            atomicCAS((unsigned long long *)(keys + s), (unsigned long long)kEmpty,
                      (unsigned long long)g);
        if (prev == kEmpty || prev == g) return true;
        s = (s + 1) & mask;
    }
    return false;
}

// Number of candidate bits of the uncertain documents (sizes the table).
__global__ void k_count_keys(const __grid_constant__ BloomArgs A, const uint32_t *ulist,
                             uint32_t nu, unsigned long long *count) {
    const uint64_t n = (uint64_t)nu * A.bands;
    unsigned long long local = 0;
    for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t d = ulist[idx / A.bands];
        const uint32_t j = (uint32_t)(idx % A.bands);
        if ((A.cand[d] >> j) & 1ull) local += __popcll(A.miss[d * A.bands + j]);
    }
    if (local) atomicAdd(count, local);
}

__global__ void k_rk_insert(const __grid_constant__ BloomArgs A, const uint32_t *ulist, uint32_t nu,
                            ResolveTable T) {
    const uint64_t n = (uint64_t)nu * A.bands;
    for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t d = ulist[idx / A.bands];
        const uint32_t j = (uint32_t)(idx % A.bands);
        if (!((A.cand[d] >> j) & 1ull)) continue;
        const ProbeSeq ps(A.keys[d * A.bands + j], j, A.m_bits, A.layout);
        uint64_t mm = A.miss[d * A.bands + j];
        while (mm) {
            const uint32_t u = __ffsll((long long)mm) - 1;
            mm &= mm - 1;
            const uint64_t g = (uint64_t)j * A.m_bits + ps.pos(u);
            if (!ht_insert(T.keys, T.mask, g)) atomicOr(A.error, kErrTableFull);
        }
    }
}

// Fixed setters: documents whose insertion does not depend on the order.
// NONDUP mode: status 0; INSERT_ALL mode: every document.
__global__ void k_fixed_setters(const __grid_constant__ BloomArgs A, ResolveTable T,
                                int insert_all) {
    const uint64_t n = A.D * A.bands;
    for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t d = idx / A.bands;
        if (!insert_all && A.status[d] != 0) continue;
        const uint32_t j = (uint32_t)(idx % A.bands);
        uint64_t mm = A.miss[idx];
        if (!mm) continue;
        const ProbeSeq ps(A.keys[idx], j, A.m_bits, A.layout);
        while (mm) {
            const uint32_t u = __ffsll((long long)mm) - 1;
            mm &= mm - 1;
            const uint64_t g = (uint64_t)j * A.m_bits + ps.pos(u);
            const uint32_t s = ht_find(T.keys, T.mask, g);
            if (s != kNone) atomicMin(T.first_fixed + s, (uint32_t)d);
        }
    }
}

// Table slot of every missing bit of every uncertain document (all bands).
__global__ void k_cache_slots(const __grid_constant__ BloomArgs A, const uint32_t *ulist,
                              uint32_t nu, ResolveTable T) {
    const uint64_t n = (uint64_t)nu * A.bands;
    for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t d = ulist[idx / A.bands];
        const uint32_t j = (uint32_t)(idx % A.bands);
        const uint64_t miss = A.miss[d * A.bands + j];
        const ProbeSeq ps(A.keys[d * A.bands + j], j, A.m_bits, A.layout);
        uint32_t *out = T.slots + idx * A.k;
        for (uint32_t u = 0; u < A.k; ++u) {
            uint32_t s = kNone;
            if ((miss >> u) & 1ull) s = ht_find(T.keys, T.mask, (uint64_t)j * A.m_bits + ps.pos(u));
            out[u] = s;
        }
    }
}

__global__ void k_iter_reset(ResolveTable T) {
    for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s <= T.mask;
         s += (uint64_t)gridDim.x * blockDim.x)
        T.first[s] = T.first_fixed[s];
}

__global__ void k_iter_setters(const __grid_constant__ BloomArgs A, const uint32_t *ulist,
                               uint32_t nu, ResolveTable T) {
    const uint64_t n = (uint64_t)nu * A.bands;
    for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t ui = (uint32_t)(idx / A.bands);
        if (!T.ins[ui]) continue;
        const uint32_t d = ulist[ui];
        const uint32_t *sl = T.slots + idx * A.k;
        for (uint32_t u = 0; u < A.k; ++u)
            if (sl[u] != kNone) atomicMin(T.first + sl[u], d);
    }
}

__device__ __forceinline__ bool uncertain_is_dup(const BloomArgs &A, const ResolveTable &T,
                                                 uint32_t ui, uint32_t d) {
    const uint64_t cand = A.cand[d];
    for (uint32_t j = 0; j < A.bands; ++j) {
        if (!((cand >> j) & 1ull)) continue;
        const uint32_t *sl = T.slots + ((uint64_t)ui * A.bands + j) * A.k;
        bool all = true;
        for (uint32_t u = 0; u < A.k && all; ++u) {
            const uint32_t s = sl[u];
            if (s != kNone) all = T.first[s] < d;
        }
        if (all) return true;
    }
    return false;
}

__global__ void k_iter_eval(const __grid_constant__ BloomArgs A, const uint32_t *ulist, uint32_t nu,
                            ResolveTable T, int insert_all) {
    for (uint32_t ui = blockIdx.x * blockDim.x + threadIdx.x; ui < nu; ui += gridDim.x * blockDim.x) {
        const uint32_t d = ulist[ui];
        const bool dup = uncertain_is_dup(A, T, ui, d);
        T.udup[ui] = dup;
        const uint8_t ins = insert_all ? 1 : (dup ? 0 : 1);
        if (ins != T.ins[ui]) {
            T.ins[ui] = ins;
            atomicOr(T.changed, 1u);
        }
    }
}

// In-order pass over the uncertain documents (one thread): the sequential
// definition itself, used when the Jacobi sweep has not settled.
__global__ void k_sequential(const __grid_constant__ BloomArgs A, const uint32_t *ulist, uint32_t nu,
                             ResolveTable T) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    for (uint64_t s = 0; s <= T.mask; ++s) T.first[s] = T.first_fixed[s];
    for (uint32_t ui = 0; ui < nu; ++ui) {
        const uint32_t d = ulist[ui];
        const bool dup = uncertain_is_dup(A, T, ui, d);
        T.udup[ui] = dup;
        T.ins[ui] = dup ? 0 : 1;
        if (!dup) {
            const uint32_t *sl = T.slots + (uint64_t)ui * A.bands * A.k;
            for (uint64_t t = 0; t < (uint64_t)A.bands * A.k; ++t)
                if (sl[t] != kNone && T.first[sl[t]] > d) T.first[sl[t]] = d;
        }
    }
}

// Flags and insert decisions of every document.
__global__ void k_finalize(const __grid_constant__ BloomArgs A, const uint32_t *ulist, uint32_t nu,
                           ResolveTable T, int insert_all, uint8_t *flags, uint8_t *insd,
                           unsigned long long *dup_count) {
    for (uint64_t d = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; d < A.D;
         d += (uint64_t)gridDim.x * blockDim.x) {
        const uint8_t st = A.status[d];
        uint8_t dup = st == 1;
        if (st == 2) {
            // ulist is sorted: find d's position.
            uint32_t lo = 0, hi = nu;
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                if (ulist[mid] < d) lo = mid + 1; else hi = mid;
            }
            dup = (lo < nu && ulist[lo] == d) ? T.udup[lo] : 0;
        }
        flags[d] = dup;
        insd[d] = insert_all ? 1 : (dup ? 0 : 1);
        if (dup) atomicAdd(dup_count, 1ull);
    }
}

__global__ void k_insert(const __grid_constant__ BloomArgs A, const uint8_t *insd) {
    const uint64_t n = A.D * A.bands;
    for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t d = idx / A.bands;
        if (!insd[d]) continue;
        uint64_t mm = A.miss[idx];
        if (!mm) continue;
        const uint32_t j = (uint32_t)(idx % A.bands);
        uint32_t *F = A.filters + (uint64_t)j * A.words_per_filter;
        if (A.layout == 2) {
            if (!exact_insert(reinterpret_cast<uint64_t *>(F), A.words_per_filter / 2, A.keys[idx]))
                atomicOr(A.error, kErrTableFull);
            continue;
        }
        const ProbeSeq ps(A.keys[idx], j, A.m_bits, A.layout);
        while (mm) {
            const uint32_t u = __ffsll((long long)mm) - 1;
            mm &= mm - 1;
            const uint64_t q = ps.pos(u);
            atomicOr(F + (q >> 5), 1u << (q & 31));
        }
    }
}

__global__ void k_popcount(const uint32_t *__restrict__ w, uint64_t n, unsigned long long *out) {
    unsigned long long c = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        c += __popc(w[i]);
    for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(LSHB_FULL_MASK, c, off);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

// ---- launch wrappers --------------------------------------------------------

static int grid_for(uint64_t n, int threads) {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    const uint64_t want = (n + threads - 1) / threads;
    const uint64_t cap = (uint64_t)sms * 16;
    return (int)(want == 0 ? 1 : (want < cap ? want : cap));
}

cudaError_t launch_popcount(const uint32_t *words, uint64_t n, unsigned long long *out,
                            cudaStream_t s) {
    k_popcount<<<grid_for(n, 256), 256, 0, s>>>(words, n, out); count_launch();
    return cudaGetLastError();
}

__global__ void k_count_occupied(const uint64_t *__restrict__ slots, uint64_t n,
                                 unsigned long long *out) {
    unsigned long long c = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        c += slots[i] != ~0ull;
    for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(LSHB_FULL_MASK, c, off);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

cudaError_t launch_count_occupied(const uint64_t *slots, uint64_t n, unsigned long long *out,
                                  cudaStream_t s) {
    k_count_occupied<<<grid_for(n, 256), 256, 0, s>>>(slots, n, out); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_probe_mark(const BloomArgs &a, cudaStream_t s) {
    k_probe_mark<<<grid_for(a.D * a.bands, 256), 256, 0, s>>>(a); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_classify(const BloomArgs &a, uint32_t *block_counts, uint32_t *total,
                            uint32_t *ulist, cudaStream_t s) {
    k_classify<<<grid_for(a.D * a.bands, 256), 256, 0, s>>>(a); count_launch();
    const uint32_t nb = (uint32_t)((a.D + 1023) / 1024);
    k_status<<<nb, 1024, 0, s>>>(a, block_counts); count_launch();
    k_scan_counts<<<1, 1024, 0, s>>>(block_counts, nb, total); count_launch();
    k_compact<<<nb, 1024, 0, s>>>(a, block_counts, ulist); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_count_keys(const BloomArgs &a, const uint32_t *ulist, uint32_t nu,
                              unsigned long long *count, cudaStream_t s) {
    k_count_keys<<<grid_for((uint64_t)nu * a.bands, 256), 256, 0, s>>>(a, ulist, nu, count); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_resolve_setup(const BloomArgs &a, const uint32_t *ulist, uint32_t nu,
                                 const ResolveTable &t, int insert_all, cudaStream_t s) {
    k_rk_insert<<<grid_for((uint64_t)nu * a.bands, 256), 256, 0, s>>>(a, ulist, nu, t); count_launch();
    k_fixed_setters<<<grid_for(a.D * a.bands, 256), 256, 0, s>>>(a, t, insert_all); count_launch();
    k_cache_slots<<<grid_for((uint64_t)nu * a.bands, 128), 128, 0, s>>>(a, ulist, nu, t); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_resolve_iteration(const BloomArgs &a, const uint32_t *ulist, uint32_t nu,
                                     const ResolveTable &t, int insert_all, cudaStream_t s) {
    k_iter_reset<<<grid_for((uint64_t)t.mask + 1, 256), 256, 0, s>>>(t); count_launch();
    if (!insert_all) k_iter_setters<<<grid_for((uint64_t)nu * a.bands, 256), 256, 0, s>>>(a, ulist, nu, t); count_launch();
    k_iter_eval<<<grid_for(nu, 256), 256, 0, s>>>(a, ulist, nu, t, insert_all); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_resolve_sequential(const BloomArgs &a, const uint32_t *ulist, uint32_t nu,
                                      const ResolveTable &t, cudaStream_t s) {
    k_sequential<<<1, 1, 0, s>>>(a, ulist, nu, t); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_finalize_insert(const BloomArgs &a, const uint32_t *ulist, uint32_t nu,
                                   const ResolveTable &t, int insert_all, uint8_t *flags,
                                   uint8_t *insd, unsigned long long *dup_count, cudaStream_t s) {
    k_finalize<<<grid_for(a.D, 256), 256, 0, s>>>(a, ulist, nu, t, insert_all, flags, insd,
                                                   dup_count); count_launch();
    k_insert<<<grid_for(a.D * a.bands, 256), 256, 0, s>>>(a, insd); count_launch();
    return cudaGetLastError();
}

}  // namespace lshb
