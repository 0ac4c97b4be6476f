// Bloom stage of the LSHBloom path: probe each band key in its filter
// (Sec. 4.2), decide each document exactly as the sequential stream would
// (Sec. 2.1, Sec. 4.4.2), and insert the documents that the insert rule
// admits (Sec. 4.1).
//
// The batch is judged in parallel.  A band of document d hits when each of its
// k probed bits is set before the batch or by an inserted document d' < d of
// the batch.  The kernels below find that without a sort:
//   1. probe     reads the pre-batch bits; records, per (band, doc), which
//                probes found a clear bit ("missing"); marks each missing bit
//                in the band's sketch of 2-bit cells (seen once / twice);
//   2. classify  a band whose every missing bit was marked twice is a
//                candidate (some other document may set those bits); a
//                document with a band with no missing bit is a duplicate
//                whatever the order; one with neither is not a duplicate;
//                the rest are "uncertain";
//   3. resolve   uncertain documents only: their candidate bits go into a
//                hash table with one segment per band; every inserting
//                document records itself as a setter with atomicMin;
//                uncertain documents iterate ins <- not dup(ins) (a Jacobi
//                sweep) until nothing changes.  Document d depends only on
//                documents before it, so the fixed point is unique and is
//                the sequential answer; after t sweeps the first t uncertain
//                documents are final, and an in-order pass (one warp) can
//                finish from there;
//   4. insert    atomicOr of the missing bits of inserted documents.
// Sketch collisions only add candidates; they never drop one, so the result
// is exact.  Every (band, document) kernel runs band by band (a 2-D grid with
// the band as its slow index): the filter and sketch of one band stay in L2
// while its documents are processed.
#include "bloom_kernels.cuh"

namespace lshb {

// ---- probe and classification ----------------------------------------------------

__global__ void __launch_bounds__(kProbeThreads) k_probe(const __grid_constant__ BloomArgs A) {
    const uint64_t d = (uint64_t)blockIdx.x * kProbeThreads + threadIdx.x;
    const uint32_t j = blockIdx.y;
    if (d >= batch_docs(A)) return;
    uint64_t miss = probe_key<24>(A, j, band_key(A, d, j));
    uint64_t *mp = A.miss + (uint64_t)j * A.mstride + d;
    if (!A.first_pass) miss |= *mp;
    *mp = miss;
    if (A.last_pass && !miss) A.prehit[d] = 1;
}

__global__ void __launch_bounds__(kBloomThreads) k_classify(const __grid_constant__ BloomArgs A) {
    const uint64_t d = (uint64_t)blockIdx.x * kBloomThreads + threadIdx.x;
    const uint32_t j = blockIdx.y;
    if (d >= batch_docs(A)) return;
    uint64_t mm = A.miss[(uint64_t)j * A.mstride + d];
    if (!mm) return;
    const ProbeSeq ps(band_key(A, d, j), j, A.m_bits, A.layout);
    bool all = true;
    while (mm && all) {
        const uint32_t u = __ffsll((long long)mm) - 1;
        mm &= mm - 1;
        all = sketch_twice(A, j, ps.pos(u));
    }
    if (all) atomicOr((unsigned long long *)(A.cand + d), 1ull << j);
}

// Status per document and the per-block count of uncertain documents.
// status: 1 = duplicate whatever the order, 2 = uncertain, 0 = not duplicate.
__global__ void __launch_bounds__(kStatusThreads) k_status(const __grid_constant__ BloomArgs A,
                                                           uint32_t *block_counts) {
    __shared__ uint32_t warp_cnt[kStatusThreads / 32];
    const uint64_t d = (uint64_t)blockIdx.x * kStatusThreads + threadIdx.x;
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
        for (int w = 0; w < kStatusThreads / 32; ++w) s += warp_cnt[w];
        block_counts[blockIdx.x] = s;
    }
}

// Exclusive scan of the block counts (one block; nb up to several thousand)
// and the total in *total.  Each thread takes kScanPer consecutive counts, so
// a 2^21-document batch (8,192 counts) takes four rounds of the block scan.
constexpr int kScanPer = 8;

__global__ void __launch_bounds__(kStatusThreads) k_scan_counts(uint32_t *block_counts,
                                                                uint32_t nb, uint32_t *total) {
    __shared__ uint32_t part[kStatusThreads];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint32_t base = 0; base < nb; base += kStatusThreads * kScanPer) {
        const uint32_t i0 = base + threadIdx.x * kScanPer;
        uint32_t v[kScanPer];
        uint32_t sum = 0;
#pragma unroll
        for (int k = 0; k < kScanPer; ++k) {
            v[k] = i0 + k < nb ? block_counts[i0 + k] : 0u;
            sum += v[k];
        }
        part[threadIdx.x] = sum;
        __syncthreads();
        for (uint32_t off = 1; off < kStatusThreads; off <<= 1) {
            const uint32_t add = threadIdx.x >= off ? part[threadIdx.x - off] : 0u;
            __syncthreads();
            part[threadIdx.x] += add;
            __syncthreads();
        }
        uint32_t run = carry + part[threadIdx.x] - sum;
#pragma unroll
        for (int k = 0; k < kScanPer; ++k) {
            if (i0 + k < nb) block_counts[i0 + k] = run;
            run += v[k];
        }
        __syncthreads();
        if (threadIdx.x == kStatusThreads - 1) carry += part[kStatusThreads - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

// Uncertain documents in increasing index order.
__global__ void __launch_bounds__(kStatusThreads) k_compact(const __grid_constant__ BloomArgs A,
                                                            const uint32_t *block_offsets,
                                                            uint32_t *ulist) {
    __shared__ uint32_t warp_pre[kStatusThreads / 32];
    const uint64_t d = (uint64_t)blockIdx.x * kStatusThreads + threadIdx.x;
    const bool u = d < batch_docs(A) && A.status[d] == 2;
    const uint32_t bal = __ballot_sync(LSHB_FULL_MASK, u);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) warp_pre[w] = __popc(bal);
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t s = 0;
        for (int i = 0; i < kStatusThreads / 32; ++i) {
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

__device__ __forceinline__ uint32_t ht_find(const ResolveTable &T, uint32_t j, uint64_t pos) {
    const uint64_t base = T.seg_base[j];
    const uint32_t mask = T.seg_mask[j];
    if (pos == ~0ull) {
        const uint64_t s = base + mask + 1;
        return T.keys[s] == 0ull ? (uint32_t)s : kNone;
    }
    uint32_t s = (uint32_t)(mix64(pos) & mask);
    for (uint32_t i = 0; i <= mask; ++i) {
        const uint64_t k = T.keys[base + s];
        if (k == pos) return (uint32_t)(base + s);
        if (k == ~0ull) return kNone;
        s = (s + 1) & mask;
    }
    return kNone;
}

__device__ __forceinline__ bool ht_insert(const ResolveTable &T, uint32_t j, uint64_t pos) {
    const uint64_t base = T.seg_base[j];
    const uint32_t mask = T.seg_mask[j];
    if (pos == ~0ull) {
        T.keys[base + mask + 1] = 0ull;
        return true;
    }
    uint32_t s = (uint32_t)(mix64(pos) & mask);
    for (uint32_t i = 0; i <= mask; ++i) {
        const unsigned long long prev = atomicCAS((unsigned long long *)(T.keys + base + s),
                                                  ~0ull, (unsigned long long)pos);
        if (prev == ~0ull || prev == pos) return true;
        s = (s + 1) & mask;
    }
    return false;
}

// Candidate bits of the uncertain documents, per band (sizes the segments).
__global__ void __launch_bounds__(kBloomThreads) k_count_keys(const __grid_constant__ BloomArgs A,
                                                              const uint32_t *ulist, uint32_t nu,
                                                              unsigned long long *band_counts) {
    __shared__ unsigned long long part[kBloomThreads / 32];
    const uint32_t ui = blockIdx.x * kBloomThreads + threadIdx.x;
    const uint32_t j = blockIdx.y;
    unsigned long long c = 0;
    if (ui < nu) {
        const uint32_t d = ulist[ui];
        if ((A.cand[d] >> j) & 1ull) c = __popcll(A.miss[(uint64_t)j * A.mstride + d]);
    }
    for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(LSHB_FULL_MASK, c, off);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long s = 0;
        for (int w = 0; w < kBloomThreads / 32; ++w) s += part[w];
        if (s) atomicAdd(band_counts + j, s);
    }
}

__global__ void __launch_bounds__(kBloomThreads) k_rk_insert(const __grid_constant__ BloomArgs A,
                                                             const uint32_t *ulist, uint32_t nu,
                                                             const __grid_constant__ ResolveTable T) {
    const uint32_t ui = blockIdx.x * kBloomThreads + threadIdx.x;
    const uint32_t j = blockIdx.y;
    if (ui >= nu) return;
    const uint32_t d = ulist[ui];
    if (!((A.cand[d] >> j) & 1ull)) return;
    const ProbeSeq ps(band_key(A, d, j), j, A.m_bits, A.layout);
    uint64_t mm = A.miss[(uint64_t)j * A.mstride + d];
    while (mm) {
        const uint32_t u = __ffsll((long long)mm) - 1;
        mm &= mm - 1;
        if (!ht_insert(T, j, ps.pos(u))) atomicOr(A.error, kErrTableFull);
    }
}

// Fixed setters: documents whose insertion does not depend on the order.
// NONDUP mode: status 0; INSERT_ALL mode: every document.
__global__ void __launch_bounds__(kBloomThreads) k_fixed_setters(
    const __grid_constant__ BloomArgs A, const __grid_constant__ ResolveTable T, int insert_all) {
    const uint64_t d = (uint64_t)blockIdx.x * kBloomThreads + threadIdx.x;
    const uint32_t j = blockIdx.y;
    if (d >= A.D) return;
    if (!insert_all && A.status[d] != 0) return;
    uint64_t mm = A.miss[(uint64_t)j * A.mstride + d];
    if (!mm) return;
    const ProbeSeq ps(band_key(A, d, j), j, A.m_bits, A.layout);
    while (mm) {
        const uint32_t u = __ffsll((long long)mm) - 1;
        mm &= mm - 1;
        const uint32_t s = ht_find(T, j, ps.pos(u));
        if (s != kNone) atomicMin(T.first_fixed + s, (uint32_t)d);
    }
}

// Table slot of every missing bit of every uncertain document (all bands).
__global__ void __launch_bounds__(kBloomThreads) k_cache_slots(const __grid_constant__ BloomArgs A,
                                                               const uint32_t *ulist, uint32_t nu,
                                                               const __grid_constant__ ResolveTable T) {
    const uint32_t ui = blockIdx.x * kBloomThreads + threadIdx.x;
    const uint32_t j = blockIdx.y;
    if (ui >= nu) return;
    const uint32_t d = ulist[ui];
    const uint64_t miss = A.miss[(uint64_t)j * A.mstride + d];
    const ProbeSeq ps(band_key(A, d, j), j, A.m_bits, A.layout);
    uint32_t *out = T.slots + ((uint64_t)ui * A.bands + j) * A.k;
    for (uint32_t u = 0; u < A.k; ++u)
        out[u] = ((miss >> u) & 1ull) ? ht_find(T, j, ps.pos(u)) : kNone;
}

// Sweep control.  A sweep runs only while the previous one changed an insert
// decision; the host enqueues sweeps in groups and reads ctl once per group.
__device__ __forceinline__ bool sweeps_done(const ResolveTable &T) {
    return __ldcg(T.ctl + 1) != 0u;
}

__global__ void k_sweep_begin(const __grid_constant__ ResolveTable T) {
    if (T.ctl[1]) return;
    if (T.ctl[2] > 0 && T.ctl[0] == 0) {
        T.ctl[1] = 1u;
        return;
    }
    T.ctl[0] = 0u;
    T.ctl[2] += 1u;
}

__global__ void k_iter_reset(const __grid_constant__ ResolveTable T, uint64_t table_slots,
                             int forced) {
    if (!forced && sweeps_done(T)) return;
    for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < table_slots;
         s += (uint64_t)gridDim.x * blockDim.x)
        T.first[s] = T.first_fixed[s];
}

// Setters of the current sweep (uncertain documents ui < n_set with ins set),
// one (document, band) per thread.
__global__ void __launch_bounds__(kBloomThreads) k_iter_setters(const __grid_constant__ BloomArgs A,
                                                                const uint32_t *ulist, uint32_t n_set,
                                                                const __grid_constant__ ResolveTable T,
                                                                int forced) {
    if (!forced && sweeps_done(T)) return;
    const uint32_t ui = blockIdx.x * kBloomThreads + threadIdx.x;
    if (ui >= n_set || !T.ins[ui]) return;
    const uint32_t d = ulist[ui];
    const uint32_t *sl = T.slots + ((uint64_t)ui * A.bands + blockIdx.y) * A.k;
    for (uint32_t u = 0; u < A.k; ++u)
        if (sl[u] != kNone) atomicMin(T.first + sl[u], d);
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
                            const __grid_constant__ ResolveTable T, int insert_all) {
    if (sweeps_done(T)) return;
    for (uint32_t ui = blockIdx.x * blockDim.x + threadIdx.x; ui < nu; ui += gridDim.x * blockDim.x) {
        const uint32_t d = ulist[ui];
        const bool dup = uncertain_is_dup(A, T, ui, d);
        T.udup[ui] = dup;
        const uint8_t ins = insert_all ? 1 : (dup ? 0 : 1);
        if (ins != T.ins[ui]) {
            T.ins[ui] = ins;
            T.ctl[0] = 1u;
        }
    }
}

// The sequential definition, resumed at uncertain document `settled` (the
// earlier ones are final): one warp takes the remaining documents in order;
// its lanes split each document's probed slots.  `first` holds the fixed
// setters and the settled documents' insertions when it starts.
__global__ void __launch_bounds__(32) k_in_order(const __grid_constant__ BloomArgs A,
                                                 const uint32_t *ulist, uint32_t nu,
                                                 const __grid_constant__ ResolveTable T,
                                                 uint32_t settled) {
    const uint32_t lane = threadIdx.x;
    const uint32_t nslots = A.bands * A.k;
    for (uint32_t ui = settled; ui < nu; ++ui) {
        const uint32_t d = ulist[ui];
        const uint64_t cand = A.cand[d];
        const uint32_t *sl = T.slots + (uint64_t)ui * nslots;
        bool dup = false;
        for (uint32_t j = 0; j < A.bands && !dup; ++j) {
            if (!((cand >> j) & 1ull)) continue;
            bool all = true;
            for (uint32_t u = lane; u < A.k; u += 32) {
                const uint32_t s = sl[j * A.k + u];
                if (s != kNone && __ldcg(T.first + s) >= d) all = false;
            }
            dup = __all_sync(LSHB_FULL_MASK, all);
        }
        if (lane == 0) {
            T.udup[ui] = dup;
            T.ins[ui] = dup ? 0 : 1;
        }
        if (!dup) {
            uint32_t sink = 0;
            for (uint32_t t = lane; t < nslots; t += 32)
                if (sl[t] != kNone) sink |= atomicMin(T.first + sl[t], d);
            __threadfence();
            if (sink == 0x7fffffffu) T.ctl[3] = sink;  // keeps the returning atomics
        }
        __syncwarp();
    }
}

// Flags and insert decisions of every document.
__global__ void k_finalize(const __grid_constant__ BloomArgs A, const uint32_t *ulist, uint32_t nu,
                           const __grid_constant__ ResolveTable T, int insert_all, uint8_t *flags,
                           uint8_t *insd, unsigned long long *dup_count) {
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

__global__ void __launch_bounds__(kBloomThreads) k_insert(const __grid_constant__ BloomArgs A,
                                                          const uint8_t *insd) {
    const uint64_t d = (uint64_t)blockIdx.x * kBloomThreads + threadIdx.x;
    const uint32_t j = blockIdx.y;
    if (d >= A.D || !insd[d]) return;
    uint64_t mm = A.miss[(uint64_t)j * A.mstride + d];
    if (!mm) return;
    uint32_t *F = A.filters + (uint64_t)j * A.words_per_filter;
    if (A.layout == 2) {
        if (!exact_insert(reinterpret_cast<uint64_t *>(F), A.exact_cap, band_key(A, d, j)))
            atomicOr(A.error, kErrTableFull);
        return;
    }
    const ProbeSeq ps(band_key(A, d, j), j, A.m_bits, A.layout);
    while (mm) {
        const uint32_t u = __ffsll((long long)mm) - 1;
        mm &= mm - 1;
        const uint64_t q = ps.pos(u);
        const uint64_t wi = q >> 5;
        if (wi >= A.word_lo && wi < A.word_hi) atomicOr(F + wi, 1u << (q & 31));
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

__global__ void k_count_occupied(const uint64_t *__restrict__ slots, uint64_t n,
                                 unsigned long long *out) {
    unsigned long long c = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        c += slots[i] != ~0ull;
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

// (document blocks, bands) grid for n documents.
static dim3 band_grid(uint64_t n, uint32_t bands, int threads = kBloomThreads) {
    const uint64_t bx = (n + threads - 1) / threads;
    return dim3((unsigned)(bx ? bx : 1), bands, 1);
}

cudaError_t launch_popcount(const uint32_t *words, uint64_t n, unsigned long long *out,
                            cudaStream_t s) {
    k_popcount<<<grid_for(n, 256), 256, 0, s>>>(words, n, out); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_count_occupied(const uint64_t *slots, uint64_t n, unsigned long long *out,
                                  cudaStream_t s) {
    k_count_occupied<<<grid_for(n, 256), 256, 0, s>>>(slots, n, out); count_launch();
    return cudaGetLastError();
}

// Insert passes over the filters: one slice of at most kSliceBytes per pass
// when the batch has enough bits to set per slice to reuse it and a filter
// takes at most kMaxSlices slices (every pass recomputes every key's
// positions: the 3 GB filters of a billion-document index would take 47
// passes, measured 2.7x slower than one).  Standard layout only: a blocked
// filter's inserts set k bits in one sector per key and ran faster in one
// pass (8M Pareto batch: 73.0M vs 70.8M docs/s), and the exact key tables
// are not bit arrays.
constexpr uint64_t kMaxSlices = 4;

static uint32_t filter_passes(const BloomArgs &a, uint64_t dcap) {
    if (a.layout != 0 || dcap < (1ull << 15)) return 1;
    const uint64_t p = (a.words_per_filter * 4 + kSliceBytes - 1) / kSliceBytes;
    return (uint32_t)(p < 1 || p > kMaxSlices ? 1 : p);
}

static BloomArgs pass_args(BloomArgs a, uint32_t p, uint32_t np) {
    const uint64_t per = (a.words_per_filter + np - 1) / np;
    a.word_lo = per * p;
    a.word_hi = p + 1 == np ? ~0ull : per * (p + 1);
    a.first_pass = p == 0;
    a.last_pass = p + 1 == np;
    return a;
}

cudaError_t launch_probe(const BloomArgs &a, uint64_t dcap, cudaStream_t s) {
    k_probe<<<band_grid(dcap, a.bands, kProbeThreads), kProbeThreads, 0, s>>>(pass_args(a, 0, 1));
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_classify(const BloomArgs &a, uint64_t dcap, uint32_t *block_counts,
                            uint32_t *total, uint32_t *ulist, cudaStream_t s) {
    k_classify<<<band_grid(dcap, a.bands), kBloomThreads, 0, s>>>(a); count_launch();
    const uint32_t nb = (uint32_t)((dcap + kStatusThreads - 1) / kStatusThreads);
    k_status<<<nb ? nb : 1, kStatusThreads, 0, s>>>(a, block_counts); count_launch();
    k_scan_counts<<<1, kStatusThreads, 0, s>>>(block_counts, nb ? nb : 1, total); count_launch();
    k_compact<<<nb ? nb : 1, kStatusThreads, 0, s>>>(a, block_counts, ulist); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_count_keys(const BloomArgs &a, const uint32_t *ulist, uint32_t nu,
                              unsigned long long *band_counts, cudaStream_t s) {
    k_count_keys<<<band_grid(nu, a.bands), kBloomThreads, 0, s>>>(a, ulist, nu, band_counts);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_resolve_setup(const BloomArgs &a, const uint32_t *ulist, uint32_t nu,
                                 const ResolveTable &t, int insert_all, cudaStream_t s) {
    k_rk_insert<<<band_grid(nu, a.bands), kBloomThreads, 0, s>>>(a, ulist, nu, t); count_launch();
    k_fixed_setters<<<band_grid(a.D, a.bands), kBloomThreads, 0, s>>>(a, t, insert_all);
    count_launch();
    k_cache_slots<<<band_grid(nu, a.bands), kBloomThreads, 0, s>>>(a, ulist, nu, t); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_resolve_sweep(const BloomArgs &a, const uint32_t *ulist, uint32_t nu,
                                 const ResolveTable &t, uint64_t table_slots, int insert_all,
                                 cudaStream_t s) {
    k_sweep_begin<<<1, 1, 0, s>>>(t); count_launch();
    k_iter_reset<<<grid_for(table_slots, 256), 256, 0, s>>>(t, table_slots, 0); count_launch();
    if (!insert_all) {
        k_iter_setters<<<band_grid(nu, a.bands), kBloomThreads, 0, s>>>(a, ulist, nu, t, 0);
        count_launch();
    }
    k_iter_eval<<<grid_for(nu, 256), 256, 0, s>>>(a, ulist, nu, t, insert_all); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_resolve_in_order(const BloomArgs &a, const uint32_t *ulist, uint32_t nu,
                                    const ResolveTable &t, uint64_t table_slots,
                                    uint32_t settled, cudaStream_t s) {
    k_iter_reset<<<grid_for(table_slots, 256), 256, 0, s>>>(t, table_slots, 1); count_launch();
    if (settled > 0) {
        k_iter_setters<<<band_grid(settled, a.bands), kBloomThreads, 0, s>>>(a, ulist, settled, t, 1);
        count_launch();
    }
    k_in_order<<<1, 32, 0, s>>>(a, ulist, nu, t, settled); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_finalize_insert(const BloomArgs &a, const uint32_t *ulist, uint32_t nu,
                                   const ResolveTable &t, int insert_all, uint8_t *flags,
                                   uint8_t *insd, unsigned long long *dup_count, cudaStream_t s) {
    k_finalize<<<grid_for(a.D, 256), 256, 0, s>>>(a, ulist, nu, t, insert_all, flags, insd,
                                                   dup_count); count_launch();
    const uint32_t np = filter_passes(a, a.D);
    for (uint32_t p = 0; p < np; ++p) {
        k_insert<<<band_grid(a.D, a.bands), kBloomThreads, 0, s>>>(pass_args(a, p, np), insd);
        count_launch();
    }
    return cudaGetLastError();
}

}  // namespace lshb
