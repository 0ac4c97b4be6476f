// C ABI of the LSHBloom library: handles, sizing, scratch, chunked batches,
// the stage pipeline, persistence.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/lshbloom.h"
#include "bloom_kernels.cuh"
#include "lshb_internal.h"
#include "runtime_internal.h"

using namespace lshb;

// ---- errors -------------------------------------------------------------------

static thread_local std::string g_last_error;

lshb_status lshb::fail(lshb_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

lshb_status lshb::cuda_fail(cudaError_t e, const char *what) {
    return fail(LSHB_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call)                                                            \
    do {                                                                    \
        cudaError_t e_ = (call);                                            \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);                 \
    } while (0)

extern "C" const char *lshbloom_last_error(void) { return g_last_error.c_str(); }

static std::atomic<uint64_t> g_launches{0};
void lshb::count_launch(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
uint64_t lshb::launches_total() { return g_launches.load(std::memory_order_relaxed); }

// ---- sizing and coefficients (host) ----------------------------------------------

// Bits per filter (Sec. 4.5: m = -n ln p / (ln 2)^2, natural log), rounded up
// to whole bits and then to a multiple of 256 bits; k = round(m/n ln 2).
static void size_filter(uint64_t n, double p, uint64_t *m, uint32_t *k) {
    const double ln2 = std::log(2.0);
    const double bits = -(double)n * std::log(p) / (ln2 * ln2);
    uint64_t mm = (uint64_t)std::ceil(bits);
    mm = ((mm + 255) / 256) * 256;
    if (mm == 0) mm = 256;
    long kk = std::lround((double)mm / (double)n * ln2);
    *m = mm;
    *k = (uint32_t)(kk < 1 ? 1 : kk);
}

// Blocked layout (not in the paper): a key's k positions are uniform draws,
// with replacement, inside one 256-bit block.  With i keys in a block its
// set-bit count Z has the occupancy law of i*k draws over 256 cells, and a
// query's k draws all land on set bits with probability E[(Z/256)^k];
// block loads are Poisson with mean 256 n / m.
namespace {
struct BlockedFpModel {
    uint32_t k;
    std::vector<double> occ = std::vector<double>(257, 0.0);  // law of Z after g.size() keys
    std::vector<double> pw = std::vector<double>(257, 0.0);   // (z/256)^k
    std::vector<double> g;                                    // g[i] = E[(Z/256)^k | i keys]
    explicit BlockedFpModel(uint32_t k_) : k(k_) {
        occ[0] = 1.0;
        for (int z = 0; z <= 256; ++z) pw[z] = std::pow(z / 256.0, (double)k);
    }
    double hit(uint32_t i) {
        while (g.size() <= i) {
            double s = 0.0;
            for (int z = 0; z <= 256; ++z) s += occ[z] * pw[z];
            g.push_back(s);
            for (uint32_t u = 0; u < k; ++u) {  // one more draw: z -> z or z+1
                for (int z = 256; z >= 1; --z) occ[z] = occ[z] * (z / 256.0) + occ[z - 1] * ((257 - z) / 256.0);
                occ[0] = 0.0;
            }
        }
        return g[i];
    }
    double fp(uint64_t n, uint64_t m) {
        if (n == 0) return 0.0;
        const double lam = 256.0 * (double)n / (double)m;
        const double half = 12.0 * std::sqrt(lam) + 30.0;
        const uint32_t i0 = lam - half > 0.0 ? (uint32_t)std::floor(lam - half) : 0u;
        const uint32_t i1 = (uint32_t)std::ceil(lam + half);
        double s = 0.0;
        for (uint32_t i = i0; i <= i1; ++i)
            s += std::exp(-lam + i * std::log(lam) - std::lgamma(i + 1.0)) * hit(i);
        return s;
    }
};
}  // namespace

// Bits and k of a blocked filter meeting rate p at n keys: for each k up to
// the standard k + 8 (at most 64), the fewest blocks whose model rate is <= p
// (the rate falls as blocks are added: bracket from half the standard
// layout's blocks, then bisect); the fewest blocks over all k win, ties to
// the smaller k.
static void size_filter_blocked(uint64_t n, double p, uint64_t *m, uint32_t *k) {
    uint64_t m_std;
    uint32_t k_std;
    size_filter(n, p, &m_std, &k_std);
    const uint64_t B0 = std::max<uint64_t>(m_std / 256, 1);
    const uint32_t kmax = std::min<uint32_t>(k_std + 8, kMaxK);
    uint64_t best = ~0ull;
    uint32_t best_k = k_std;
    for (uint32_t kk = 1; kk <= kmax; ++kk) {
        BlockedFpModel M(kk);
        auto ok = [&](uint64_t blocks) { return M.fp(n, 256 * blocks) <= p; };
        uint64_t lo = std::max<uint64_t>(B0 / 2, 1), hi = B0;
        bool found = true;
        while (!ok(hi)) {
            lo = hi;
            hi *= 2;
            if (hi > (B0 << 24)) {
                found = false;
                break;
            }
        }
        if (!found) continue;
        while (lo > 1 && ok(lo)) {
            hi = lo;
            lo /= 2;
        }
        if (ok(lo)) hi = lo;
        while (hi - lo > 1) {
            const uint64_t mid = lo + (hi - lo) / 2;
            (ok(mid) ? hi : lo) = mid;
        }
        if (hi < best) {
            best = hi;
            best_k = kk;
        }
    }
    *m = 256 * best;
    *k = best_k;
}

extern "C" lshb_status lshbloom_filter_sizing(uint64_t n_expected, double fp_rate, uint32_t layout,
                                              uint64_t *m_bits, uint32_t *k) {
    if (!m_bits || !k || n_expected < 1 || !(fp_rate > 0.0 && fp_rate < 1.0) ||
        layout > LSHB_EXACT_KEYS)
        return fail(LSHB_ERR_ARG, "bad argument");
    if (layout == LSHB_BLOOM_BLOCKED) size_filter_blocked(n_expected, fp_rate, m_bits, k);
    else size_filter(n_expected, fp_rate, m_bits, k);
    return LSHB_OK;
}

// SplitMix64 stream (Steele, Lea, Flood 2014) of `seed`: a_i, b_i alternately.
static void draw_coefficients(uint64_t seed, uint32_t P, uint64_t *a, uint64_t *b) {
    uint64_t state = seed;
    auto next = [&state]() {
        state += kGolden;
        return mix64(state);
    };
    for (uint32_t i = 0; i < P; ++i) {
        a[i] = 1 + next() % (kP61 - 1);
        b[i] = next() % kP61;
    }
}

// ---- handle ---------------------------------------------------------------------

extern "C" void lshbloom_config_default(lshb_config *cfg) {
    if (!cfg) return;
    memset(cfg, 0, sizeof *cfg);
    cfg->num_perm = 121;
    cfg->bands = 11;
    cfg->rows = 11;
    cfg->ngram = 5;
    cfg->n_expected = 10000;
    cfg->fp_rate = 1e-5;
    cfg->seed = 1;
    cfg->insert_mode = LSHB_INSERT_NONDUP;
    cfg->exec_mode = LSHB_EXEC_BATCHED;
    cfg->device = -1;
}

lshbloom::~lshbloom() {
    if (device >= 0) cudaSetDevice(device);
    for (auto &b : bufs) b.release();
    if (filters) cudaFree(filters);
    for (int i = 0; i < 2; ++i) {
        if (ev_stage_free[i]) cudaEventDestroy(ev_stage_free[i]);
        if (ev_stage_ready[i]) cudaEventDestroy(ev_stage_ready[i]);
        for (int j = 0; j < 2; ++j)
            if (ev_h2d[i][j]) cudaEventDestroy(ev_h2d[i][j]);
    }
    for (int i = 0; i < 3; ++i)
        if (ev_t[i]) cudaEventDestroy(ev_t[i]);
    for (int i = 0; i < 2; ++i)
        if (ev_p[i]) cudaEventDestroy(ev_p[i]);
    if (ev_order) cudaEventDestroy(ev_order);
    if (counters) cudaFree(counters);
    if (host_counters) cudaFreeHost(host_counters);
    if (stream) cudaStreamDestroy(stream);
    if (copy_stream) cudaStreamDestroy(copy_stream);
    destroy_batched_state(this);
}

void DevBuf::release() {
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
}

lshb_status DevBuf::reserve(size_t want) {
    if (want <= bytes) return LSHB_OK;
    release();
    size_t nb = std::max(want, (size_t)256);
    cudaError_t e = cudaMalloc(&ptr, nb);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ptr = nullptr;
        return fail(LSHB_ERR_OOM, "device allocation of %zu bytes failed", nb);
    }
    bytes = nb;
    return LSHB_OK;
}

static lshb_status validate_config(const lshb_config *c) {
    if (c->num_perm < 1 || c->num_perm > 1024) return fail(LSHB_ERR_ARG, "num_perm must be 1..1024");
    if (c->bands < 1 || c->bands > (uint32_t)kMaxBands) return fail(LSHB_ERR_ARG, "bands must be 1..64");
    if (c->rows < 1) return fail(LSHB_ERR_ARG, "rows must be >= 1");
    if ((uint64_t)c->bands * c->rows > c->num_perm)
        return fail(LSHB_ERR_ARG, "bands*rows (%u) exceeds num_perm (%u)", c->bands * c->rows,
                    c->num_perm);
    if (c->ngram < 1 || c->ngram > 64) return fail(LSHB_ERR_ARG, "ngram must be 1..64");
    if (c->band_key > LSHB_BAND_WEIGHTED) return fail(LSHB_ERR_ARG, "band_key must be 0 or 1");
    if (c->n_expected < 1) return fail(LSHB_ERR_ARG, "n_expected must be >= 1");
    if (!(c->fp_rate > 0.0 && c->fp_rate < 1.0)) return fail(LSHB_ERR_ARG, "fp_rate must be in (0,1)");
    if (c->insert_mode > 1) return fail(LSHB_ERR_ARG, "bad insert_mode");
    if (c->exec_mode > 1) return fail(LSHB_ERR_ARG, "bad exec_mode");
    if (c->bloom_layout > 2) return fail(LSHB_ERR_ARG, "bad bloom_layout");
    if (c->item_shingles != 0 && (c->item_shingles < 64 || c->item_shingles > (1u << 20)))
        return fail(LSHB_ERR_ARG, "item_shingles must be 0 (autotuned) or 64..2^20");
    if ((c->perm_a == nullptr) != (c->perm_b == nullptr))
        return fail(LSHB_ERR_ARG, "perm_a and perm_b must be given together");
    if (c->perm_a) {
        for (uint32_t i = 0; i < c->num_perm; ++i) {
            if (c->perm_a[i] < 1 || c->perm_a[i] > kP61 - 1)
                return fail(LSHB_ERR_ARG, "perm_a[%u] outside [1, 2^61-2]", i);
            if (c->perm_b[i] > kP61 - 1) return fail(LSHB_ERR_ARG, "perm_b[%u] outside [0, 2^61-2]", i);
        }
    }
    return LSHB_OK;
}

// Passes of the signature stage: each pass covers up to 32*PPL permutations
// (PPL in {1, 2, 4, 8} per lane); P <= 256 takes a single pass.
static void plan_passes(lshbloom *h) {
    h->passes.clear();
    uint32_t p0 = 0;
    while (p0 < h->P) {
        const uint32_t rem = h->P - p0;
        int ppl = 8;
        if (rem <= 32) ppl = 1;
        else if (rem <= 64) ppl = 2;
        else if (rem <= 128) ppl = 4;
        const uint32_t npc = std::min<uint32_t>(rem, 32u * ppl);
        SigPass ps;
        ps.p0 = p0;
        ps.ppl = ppl;
        ps.npc = npc;
        memset(&ps.c, 0, sizeof ps.c);
        for (uint32_t i = 0; i < npc; ++i) {
            const uint64_t a = h->a[p0 + i], b = h->b[p0 + i];
            ps.c.a0[i] = (uint32_t)a;
            ps.c.a1[i] = (uint32_t)(a >> 32);
            ps.c.b0[i] = (uint32_t)b;
            ps.c.b1[i] = (uint32_t)(b >> 32);
        }
        h->passes.push_back(ps);
        p0 += npc;
    }
}

lshb_status lshb::init_handle(lshbloom *h, const lshb_config *cfg) {
    lshb_status st = validate_config(cfg);
    if (st != LSHB_OK) return st;
    h->cfg = *cfg;
    h->cfg.perm_a = nullptr;
    h->cfg.perm_b = nullptr;
    h->P = cfg->num_perm;
    h->bands = cfg->bands;
    h->rows = cfg->rows;
    h->ngram = cfg->ngram;
    h->insert_all = cfg->insert_mode == LSHB_INSERT_ALL;
    h->layout = cfg->bloom_layout;
    h->p = cfg->fp_is_effective ? 1.0 - std::pow(1.0 - cfg->fp_rate, 1.0 / (double)cfg->bands)
                                : cfg->fp_rate;
    if (!(h->p > 0.0 && h->p < 1.0)) return fail(LSHB_ERR_ARG, "per-filter rate out of range");
    if (h->layout == LSHB_BLOOM_BLOCKED) size_filter_blocked(cfg->n_expected, h->p, &h->m, &h->k);
    else size_filter(cfg->n_expected, h->p, &h->m, &h->k);
    if (h->k > (uint32_t)kMaxK) return fail(LSHB_ERR_ARG, "k = %u exceeds 64; raise fp_rate", h->k);
    h->words_per_filter = ((h->m / 32) + 31) / 32 * 32;  // 128-byte aligned filters
    if (h->layout == LSHB_EXACT_KEYS) {
        // One table of uint64 keys per band, at most half full at n_expected;
        // the key itself is the one "position".  Slot `cap` records the key
        // 2^64 - 1 (the empty marker of the others); the table is padded to
        // a multiple of 128 bytes like the filters.
        uint64_t cap = 1024;
        while (cap < 2 * cfg->n_expected) cap <<= 1;
        h->k = 1;
        h->m = 1ull << 58;
        h->exact_cap = cap;
        h->words_per_filter = ((cap + 1) * 2 + 31) / 32 * 32;
    }
    h->a.resize(h->P);
    h->b.resize(h->P);
    if (cfg->perm_a) {
        memcpy(h->a.data(), cfg->perm_a, sizeof(uint64_t) * h->P);
        memcpy(h->b.data(), cfg->perm_b, sizeof(uint64_t) * h->P);
    } else {
        draw_coefficients(cfg->seed, h->P, h->a.data(), h->b.data());
    }
    plan_passes(h);
    h->max_docs = cfg->max_batch_docs ? cfg->max_batch_docs : (1ull << 18);
    h->max_docs = std::min<uint64_t>(h->max_docs, 1ull << 22);
    h->max_tokens = cfg->max_batch_tokens ? cfg->max_batch_tokens : (1ull << 28);
    // The batched form keeps no per-token scratch: larger chunks, fewer tails.
    h->max_docs_batched = cfg->max_batch_docs ? h->max_docs : (1ull << 20);
    h->max_tokens_batched = cfg->max_batch_tokens ? h->max_tokens : (1ull << 31);

    int dev = cfg->device;
    if (dev < 0) CK(cudaGetDevice(&dev));
    h->device = dev;
    CK(cudaSetDevice(dev));
    h->pageable_access = device_reads_pageable(dev);
    CK(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
    for (int i = 0; i < 2; ++i) {
        CK(cudaEventCreateWithFlags(&h->ev_stage_free[i], cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&h->ev_stage_ready[i], cudaEventDisableTiming));
        CK(cudaEventCreate(&h->ev_h2d[i][0]));
        CK(cudaEventCreate(&h->ev_h2d[i][1]));
    }
    for (int i = 0; i < 3; ++i) CK(cudaEventCreate(&h->ev_t[i]));
    for (int i = 0; i < 2; ++i) CK(cudaEventCreate(&h->ev_p[i]));
    CK(cudaEventCreateWithFlags(&h->ev_order, cudaEventDisableTiming));
    const size_t fbytes = (size_t)h->bands * h->words_per_filter * 4;
    cudaError_t e = cudaMalloc(&h->filters, fbytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        h->filters = nullptr;
        return fail(LSHB_ERR_OOM, "filters: %zu bytes", fbytes);
    }
    CK(cudaMemsetAsync(h->filters, h->layout == LSHB_EXACT_KEYS ? 0xff : 0, fbytes, h->stream));
    CK(cudaMalloc(&h->counters, kCounterBytes));
    CK(cudaMemsetAsync(h->counters, 0, kCounterBytes, h->stream));
    CK(cudaMallocHost(&h->host_counters, kCounterBytes));
    CK(cudaStreamSynchronize(h->stream));
    return LSHB_OK;
}

extern "C" lshb_status lshbloom_create_ex(const lshb_config *cfg, lshbloom_t **out) {
    if (!cfg || !out) return fail(LSHB_ERR_ARG, "NULL argument");
    *out = nullptr;
    lshbloom *h = new (std::nothrow) lshbloom();
    if (!h) return fail(LSHB_ERR_OOM, "host allocation failed");
    lshb_status st = init_handle(h, cfg);
    if (st != LSHB_OK) {
        std::string msg = g_last_error;
        delete h;
        g_last_error = msg;
        return st;
    }
    *out = h;
    return LSHB_OK;
}

extern "C" lshb_status lshbloom_create(uint32_t P, uint32_t b, uint32_t r, uint64_t n_expected,
                                       double fp_rate, lshbloom_t **out) {
    lshb_config c;
    lshbloom_config_default(&c);
    c.num_perm = P;
    c.bands = b;
    c.rows = r;
    c.n_expected = n_expected;
    c.fp_rate = fp_rate;
    return lshbloom_create_ex(&c, out);
}

extern "C" lshb_status lshbloom_create_threshold(double T, uint32_t P, uint64_t n_expected,
                                                 double p_eff, lshbloom_t **out) {
    if (!out) return fail(LSHB_ERR_ARG, "NULL out");
    uint32_t b = 0, r = 0;
    lshb_status st = lshbloom_optimal_br(T, P, &b, &r);
    if (st != LSHB_OK) return st;
    lshb_config c;
    lshbloom_config_default(&c);
    c.num_perm = P;
    c.bands = b;
    c.rows = r;
    c.n_expected = n_expected;
    c.fp_rate = p_eff;
    c.fp_is_effective = 1;
    return lshbloom_create_ex(&c, out);
}

extern "C" void lshbloom_destroy(lshbloom_t *h) { delete h; }

// ---- pointers and chunk planning ---------------------------------------------------

// Device address of a page-locked host buffer the GPU can read in place (over
// NVLink-C2C on Grace hosts, or PCIe), or nullptr for pageable memory.
const void *lshb::mapped_host_pointer(const void *p) {
    if (!p) return nullptr;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

const void *lshb::host_read_pointer(bool pageable_access, const void *p) {
    if (const void *m = mapped_host_pointer(p)) return m;
    return pageable_access ? p : nullptr;
}

bool lshb::device_reads_pageable(int device) {
    int pma = 0, host_tables = 0;
    if (cudaDeviceGetAttribute(&pma, cudaDevAttrPageableMemoryAccess, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&host_tables, cudaDevAttrPageableMemoryAccessUsesHostPageTables,
                               device) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return pma && host_tables;
}

bool lshb::is_device_pointer(const void *p) {
    if (!p) return false;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Host copy of the batch offsets (validated: non-decreasing); device offsets
// are read on stream s, after the work already enqueued there.
lshb_status lshb::host_offsets(lshbloom *h, const uint64_t *offsets, uint64_t D, bool dev,
                               std::vector<uint64_t> &out, cudaStream_t s) {
    (void)h;
    out.resize(D + 1);
    if (dev) {
        CK(cudaMemcpyAsync(out.data(), offsets, (D + 1) * 8, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    } else {
        memcpy(out.data(), offsets, (D + 1) * 8);
    }
    for (uint64_t i = 0; i < D; ++i)
        if (out[i + 1] < out[i]) return fail(LSHB_ERR_CSR, "offsets decrease at %llu", (unsigned long long)i);
    return LSHB_OK;
}

// Chunks [lo, hi) of at most max_docs documents and, when tokens are staged or
// the plain path stores shingle hashes, at most max_tokens tokens (a longer
// single document is a chunk of its own).
// With first_tokens > 0 the token bound ramps up: first_tokens for the first
// chunk, four times more for each next one, up to max_tokens (staged host
// inputs: the first copy, which nothing hides, stays short, and each later
// copy fits under the compute of the chunk before it).
void lshb::plan_chunks(const lshbloom *h, const std::vector<uint64_t> &off, bool bound_tokens,
                       std::vector<std::pair<uint64_t, uint64_t>> &chunks, uint64_t first_tokens) {
    chunks.clear();
    const uint64_t D = off.size() - 1;
    uint64_t lo = 0;
    uint64_t ramp = first_tokens;
    while (lo < D) {
        uint64_t hi = std::min(D, lo + h->max_docs);
        if (bound_tokens) {
            const uint64_t cap = ramp ? std::min(ramp, h->max_tokens) : h->max_tokens;
            if (ramp && ramp < h->max_tokens) ramp *= 4;
            const uint64_t lim = off[lo] + cap;
            // largest hi with off[hi] <= lim, at least lo + 1
            uint64_t a = lo + 1, b = hi;
            if (off[a] > lim) {
                hi = a;
            } else {
                while (a < b) {
                    const uint64_t mid = (a + b + 1) / 2;
                    if (off[mid] <= lim) a = mid; else b = mid - 1;
                }
                hi = a;
            }
        }
        chunks.emplace_back(lo, hi);
        lo = hi;
    }
}

// ---- scratch ----------------------------------------------------------------------

lshb_status lshb::ensure_chunk_scratch(lshbloom *h, uint64_t Dc, uint64_t Tc, bool plain_hashes,
                                       bool need_sig) {
    lshb_status st;
    const uint64_t b = h->bands;
    if ((st = h->buf(B_KEYS).reserve(Dc * b * 8)) != LSHB_OK) return st;
    if ((st = h->buf(B_MISS).reserve(Dc * b * 8)) != LSHB_OK) return st;
    if ((st = h->buf(B_CAND).reserve(Dc * 8)) != LSHB_OK) return st;
    if ((st = h->buf(B_STATUS).reserve(Dc)) != LSHB_OK) return st;
    if ((st = h->buf(B_PREHIT).reserve(Dc)) != LSHB_OK) return st;
    if ((st = h->buf(B_FLAGS).reserve(Dc)) != LSHB_OK) return st;
    if ((st = h->buf(B_INSD).reserve(Dc)) != LSHB_OK) return st;
    if ((st = h->buf(B_ULIST).reserve(Dc * 4)) != LSHB_OK) return st;
    if ((st = h->buf(B_BLOCKCNT).reserve(((Dc + kStatusThreads - 1) / kStatusThreads + 1) * 4)) !=
        LSHB_OK)
        return st;
    if ((st = h->buf(B_OFFSTAGE).reserve((Dc + 1) * 8)) != LSHB_OK) return st;
    if (need_sig || h->passes.size() > 1 || h->cfg.exec_mode == LSHB_EXEC_PLAIN)
        if ((st = h->buf(B_SIG).reserve(Dc * h->P * 4)) != LSHB_OK) return st;
    if (plain_hashes)
        if ((st = h->buf(B_HASHES).reserve(std::max<uint64_t>(Tc, 1) * 4)) != LSHB_OK) return st;
    // sketch: one region of 2-bit cells per band
    const uint64_t sbytes = (uint64_t)h->bands * (sketch_cells_for(h, Dc) / 16) * 4;
    if ((st = h->buf(B_SKETCH).reserve(sbytes)) != LSHB_OK) return st;
    return LSHB_OK;
}

lshb_status lshb::ensure_stage(lshbloom *h, uint64_t Tc) {
    for (int i = 0; i < 2; ++i) {
        lshb_status st = h->stage_tok[i].reserve(std::max<uint64_t>(Tc, 1) * 4);
        if (st != LSHB_OK) return st;
    }
    return LSHB_OK;
}

// Account the completed staging copy of buffer sb (its events bracket the
// copy on the copy stream; it has finished once the chunk that read it has).
lshb_status lshb::stage_copy_done(lshbloom *h, int sb) {
    if (!h->h2d_pending[sb]) return LSHB_OK;
    CK(cudaEventSynchronize(h->ev_h2d[sb][1]));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h->ev_h2d[sb][0], h->ev_h2d[sb][1]));
    h->t_h2d_ms += ms;
    h->h2d_bytes += h->h2d_pending[sb];
    h->h2d_pending[sb] = 0;
    return LSHB_OK;
}

// Copy ntok host tokens into staging buffer sb on the copy stream once the
// buffer is free; ev_stage_ready[sb] marks the end.
lshb_status lshb::stage_copy(lshbloom *h, int sb, const uint32_t *src, uint64_t ntok) {
    lshb_status st = stage_copy_done(h, sb);
    if (st != LSHB_OK) return st;
    CK(cudaStreamWaitEvent(h->copy_stream, h->ev_stage_free[sb], 0));
    if (ntok) {
        CK(cudaEventRecord(h->ev_h2d[sb][0], h->copy_stream));
        CK(cudaMemcpyAsync(h->stage_tok[sb].ptr, src, ntok * 4, cudaMemcpyHostToDevice,
                           h->copy_stream));
        CK(cudaEventRecord(h->ev_h2d[sb][1], h->copy_stream));
        h->h2d_pending[sb] = ntok * 4;
    }
    CK(cudaEventRecord(h->ev_stage_ready[sb], h->copy_stream));
    return LSHB_OK;
}

// ---- the stage pipeline on one chunk (device-resident inputs) --------------------

// Signature stage: band keys into B_KEYS (and signatures into sig_out if given).
lshb_status lshb::run_signatures(lshbloom *h, const ChunkIn &in, uint32_t *sig_out,
                                 uint32_t *hash_out, bool want_keys, cudaStream_t s) {
    const int ngt = ngram_template(h->ngram);
    SigArgs a;
    memset(&a, 0, sizeof a);
    a.band_key = h->cfg.band_key;
    a.offsets = in.offsets;
    a.tokens = in.tokens;
    a.tok_base = in.tok_base;
    a.D = in.D;
    a.ngram = h->ngram;
    a.P = h->P;
    a.bands = h->bands;
    a.rows = h->rows;
    uint64_t *keys = (uint64_t *)h->buf(B_KEYS).ptr;
    const bool plain = h->cfg.exec_mode == LSHB_EXEC_PLAIN;
    if (hash_out || plain) {
        a.hash_out = hash_out ? hash_out : (uint32_t *)h->buf(B_HASHES).ptr;
        CK(launch_shingle_hash(ngt, a, s));
        if (hash_out) return LSHB_OK;
    }
    uint32_t *sig = sig_out ? sig_out : (uint32_t *)h->buf(B_SIG).ptr;
    const bool single = h->passes.size() == 1;
    for (const SigPass &ps : h->passes) {
        a.p0 = ps.p0;
        a.npc = ps.npc;
        a.c = ps.c;
        a.sig_out = (single && !sig_out && !plain) ? nullptr : sig;
        a.keys_out = (single && want_keys && !plain) ? keys : nullptr;
        if (plain) {
            a.hashes = (const uint32_t *)h->buf(B_HASHES).ptr;
            CK(launch_minhash_hashes(ps.ppl, a, s));
        } else {
            cudaError_t e;
            if (ngt == 5) e = launch_sig_ng5(ps.ppl, a, s);
            else if (ngt == 1) e = launch_sig_ng1(ps.ppl, a, s);
            else e = launch_sig_ng0(ps.ppl, a, s);
            CK(e);
        }
    }
    if (want_keys && (!single || plain))
        CK(launch_band_keys(sig, h->P, h->bands, h->rows, h->cfg.band_key, in.D, keys, s));
    return LSHB_OK;
}

// Two cells per possible mark (k per document and band): a missing bit of
// one document is then marked by another unrelated one with probability
// 1 - e^(-1/2), and all k = 17 missing bits of a band (a false candidate)
// with probability about 1e-7.  With k <= 2 (the exact key sets: one
// "position" per band) that rate would make nearly every document uncertain,
// so those take 64 cells per document and band (a false candidate per band
// with probability about 1/64).
uint64_t lshb::sketch_cells_for(const lshbloom *h, uint64_t dcap) {
    const uint64_t per_doc = h->k <= 2 ? 64 : 2 * (uint64_t)h->k;
    const uint64_t cells = std::max<uint64_t>(per_doc * std::max<uint64_t>(dcap, 1), 1024);
    return (cells + 15) / 16 * 16;
}

uint64_t lshb::probe_sectors_per_key(const lshbloom *h) {
    return h->layout == LSHB_BLOOM_STANDARD ? h->k : 1u;
}

BloomArgs lshb::bloom_args(lshbloom *h, uint64_t D, uint64_t dcap) {
    BloomArgs b;
    memset(&b, 0, sizeof b);
    b.D = D;
    b.bands = h->bands;
    b.k = h->k;
    b.layout = h->layout;
    b.m_bits = h->m;
    b.words_per_filter = h->words_per_filter;
    b.exact_cap = h->exact_cap;
    b.filters = h->filters;
    b.keys = (const uint64_t *)h->buf(B_KEYS).ptr;
    b.key_sd = h->bands;  // row-major; the batched form switches to band-major
    b.key_sj = 1;
    b.miss = (uint64_t *)h->buf(B_MISS).ptr;
    b.mstride = dcap;
    b.sketch = (uint32_t *)h->buf(B_SKETCH).ptr;
    b.sketch_cells = sketch_cells_for(h, dcap);
    b.status = (uint8_t *)h->buf(B_STATUS).ptr;
    b.cand = (uint64_t *)h->buf(B_CAND).ptr;
    b.prehit = (uint8_t *)h->buf(B_PREHIT).ptr;
    b.error = h->counters + C_ERROR;
    b.word_lo = 0;
    b.word_hi = ~0ull;
    b.first_pass = b.last_pass = 1;
    return b;
}

// Bloom stage: probe, classify, resolve the uncertain documents, insert.
// Band keys are in B_KEYS; writes flags into `flags_dev` (device, D bytes).
lshb_status lshb::run_bloom(lshbloom *h, uint64_t D, uint8_t *flags_dev, cudaStream_t s) {
    BloomArgs A = bloom_args(h, D, D);
    CK(cudaMemsetAsync(A.sketch, 0, (uint64_t)h->bands * (A.sketch_cells / 16) * 4, s));
    CK(cudaMemsetAsync(A.cand, 0, D * 8, s));
    CK(cudaMemsetAsync(A.prehit, 0, D, s));
    CK(cudaMemsetAsync(h->counters, 0, kChunkCounterBytes, s));
    CK(cudaEventRecord(h->ev_p[0], s));
    CK(launch_probe(A, D, s));
    CK(cudaEventRecord(h->ev_p[1], s));
    h->probe_sectors += D * h->bands * probe_sectors_per_key(h);
    uint32_t *ulist = (uint32_t *)h->buf(B_ULIST).ptr;
    CK(launch_classify(A, D, (uint32_t *)h->buf(B_BLOCKCNT).ptr, h->counters + C_NU, ulist, s));
    CK(cudaMemcpyAsync(h->host_counters, h->counters, kChunkCounterBytes, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    float ms_probe = 0.f;
    CK(cudaEventElapsedTime(&ms_probe, h->ev_p[0], h->ev_p[1]));
    h->t_probe_ms += ms_probe;
    return resolve_and_insert(h, A, flags_dev, s);
}

// Second half of the Bloom stage, once probes and the classification are in
// place and the counters have been read back: resolve the uncertain
// documents in stream order, write the flags, insert.
lshb_status lshb::resolve_and_insert(lshbloom *h, const BloomArgs &A, uint8_t *flags_dev,
                                     cudaStream_t s) {
    uint32_t *ulist = (uint32_t *)h->buf(B_ULIST).ptr;
    const uint32_t nu = h->host_counters[C_NU];
    ResolveTable T;
    memset(&T, 0, sizeof T);
    if (nu > 0) {
        h->uncertain_docs += nu;
        // candidate bits per band size the table's segments
        unsigned long long *bc = (unsigned long long *)(h->counters + C_BANDCOUNT);
        CK(cudaMemsetAsync(bc, 0, 8 * kMaxBands, s));
        CK(launch_count_keys(A, ulist, nu, bc, s));
        CK(cudaMemcpyAsync(h->host_counters + C_BANDCOUNT, bc, 8 * kMaxBands,
                           cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        const unsigned long long *hbc = (const unsigned long long *)(h->host_counters + C_BANDCOUNT);
        uint64_t slots = 0;
        for (uint32_t j = 0; j < h->bands; ++j) {
            uint64_t cap = 64;
            while (cap < 2 * hbc[j] + 16) cap <<= 1;
            T.seg_base[j] = slots;
            T.seg_mask[j] = (uint32_t)(cap - 1);
            slots += cap + 1;  // + the slot of the position 2^64 - 1
        }
        if (slots > (1ull << 31)) return fail(LSHB_ERR_OOM, "resolution table too large");
        lshb_status st;
        if ((st = h->buf(B_HT_KEYS).reserve(slots * 8)) != LSHB_OK) return st;
        if ((st = h->buf(B_HT_FIXED).reserve(slots * 4)) != LSHB_OK) return st;
        if ((st = h->buf(B_HT_FIRST).reserve(slots * 4)) != LSHB_OK) return st;
        if ((st = h->buf(B_HT_SLOTS).reserve((uint64_t)nu * h->bands * h->k * 4)) != LSHB_OK) return st;
        if ((st = h->buf(B_HT_INS).reserve(nu)) != LSHB_OK) return st;
        if ((st = h->buf(B_HT_UDUP).reserve(nu)) != LSHB_OK) return st;
        T.keys = (uint64_t *)h->buf(B_HT_KEYS).ptr;
        T.first_fixed = (uint32_t *)h->buf(B_HT_FIXED).ptr;
        T.first = (uint32_t *)h->buf(B_HT_FIRST).ptr;
        T.slots = (uint32_t *)h->buf(B_HT_SLOTS).ptr;
        T.ins = (uint8_t *)h->buf(B_HT_INS).ptr;
        T.udup = (uint8_t *)h->buf(B_HT_UDUP).ptr;
        T.ctl = h->counters + C_SWEEPCTL;
        CK(cudaMemsetAsync(T.keys, 0xff, slots * 8, s));
        CK(cudaMemsetAsync(T.first_fixed, 0xff, slots * 4, s));
        CK(cudaMemsetAsync(T.ins, 1, nu, s));
        CK(cudaMemsetAsync(T.udup, 0, nu, s));
        CK(cudaMemsetAsync(T.ctl, 0, 16, s));
        CK(launch_resolve_setup(A, ulist, nu, T, h->insert_all, s));
        // Jacobi sweeps, enqueued in growing groups; a sweep after the one
        // that changed nothing returns at once, and the host looks once per
        // group.  One sweep decides everything when every document inserts.
        const uint32_t max_sweeps = h->insert_all ? 1 : 64;
        uint32_t queued = 0, group = 2, run = 0;
        bool done = false;
        while (!done && queued < max_sweeps) {
            const uint32_t g = std::min(group, max_sweeps - queued);
            for (uint32_t i = 0; i < g; ++i)
                CK(launch_resolve_sweep(A, ulist, nu, T, slots, h->insert_all, s));
            queued += g;
            group = std::min<uint32_t>(group * 2, 16);
            CK(cudaMemcpyAsync(h->host_counters + C_SWEEPCTL, T.ctl, 16, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            done = h->host_counters[C_SWEEPCTL + 1] != 0;
            run = h->host_counters[C_SWEEPCTL + 2];
        }
        h->resolve_rounds += run;
        if (!done && !h->insert_all) {
            // Not settled after max_sweeps: the first `run` uncertain
            // documents are final; finish the rest in order.
            CK(launch_resolve_in_order(A, ulist, nu, T, slots, std::min(run, nu), s));
            h->resolve_rounds++;
        }
    }
    unsigned long long *dupc = (unsigned long long *)(h->counters + C_DUPCOUNT);
    CK(launch_finalize_insert(A, ulist, nu, T, h->insert_all, flags_dev,
                              (uint8_t *)h->buf(B_INSD).ptr, dupc, s));
    CK(cudaMemcpyAsync(h->host_counters, h->counters, kChunkCounterBytes, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (h->host_counters[C_ERROR] != 0)
        return fail(LSHB_ERR_CUDA, "device error word 0x%x", h->host_counters[C_ERROR]);
    h->dups_seen += *(unsigned long long *)(h->host_counters + C_DUPCOUNT);
    return LSHB_OK;
}

// ---- batch driver ---------------------------------------------------------------

enum class Job { Dedup, Signatures, Keys, Hashes };

static lshb_status run_batch(lshbloom *h, const uint64_t *offsets, const uint32_t *tokens,
                             uint64_t D, void *out, Job job, cudaStream_t user_stream,
                             bool require_device, uint64_t *keys_out = nullptr) {
    if (D == 0) return LSHB_OK;
    if (!offsets || !tokens || !out) return fail(LSHB_ERR_ARG, "NULL pointer with D > 0");
    std::lock_guard<std::mutex> lock(h->mu);
    CK(cudaSetDevice(h->device));
    const bool off_dev = is_device_pointer(offsets);
    bool tok_dev = is_device_pointer(tokens);
    const bool out_dev = is_device_pointer(out);
    const bool keys_dev = keys_out && is_device_pointer(keys_out);
    if (require_device && (!off_dev || !tok_dev || !out_dev))
        return fail(LSHB_ERR_ARG, "lshbloom_dedup_async takes device pointers only");
    // Host tokens the GPU can read are read in place by the kernels: measured
    // on a GB300, the copy engine staging a batch ran at 40-100 GB/s while the
    // signature kernel was running (211 GB/s alone), whereas the kernel's own
    // reads over the host link cost it 1% of its time.  Others are staged.
    bool tok_in_place = false;
    if (!tok_dev && !h->cfg.stage_host_inputs) {
        if (const void *m = host_read_pointer(h->pageable_access, tokens)) {
            tokens = (const uint32_t *)m;
            tok_dev = tok_in_place = true;
        }
    }
    cudaStream_t s = user_stream ? user_stream : h->stream;
    // A synchronous call runs on the handle's own (non-blocking) stream: order
    // it after everything already enqueued on the legacy default stream, where
    // a caller's device inputs are usually produced.
    if (!user_stream && (off_dev || tok_dev || out_dev)) {
        CK(cudaEventRecord(h->ev_order, cudaStreamLegacy));
        CK(cudaStreamWaitEvent(s, h->ev_order, 0));
    }
    std::vector<uint64_t> off;
    lshb_status st = host_offsets(h, offsets, D, off_dev, off, s);
    if (st != LSHB_OK) return st;
    if (tok_in_place && job == Job::Dedup) h->host_read_bytes += (off[D] - off[0]) * 4;
    if (job == Job::Dedup && h->cfg.exec_mode == LSHB_EXEC_BATCHED && h->passes.size() == 1) {
        return run_batched(h, offsets, tokens, D, (uint8_t *)out, off, off_dev, tok_dev, out_dev, s,
                           keys_out, keys_dev);
    }
    const bool plain = h->cfg.exec_mode == LSHB_EXEC_PLAIN;
    const bool need_hash_buf = plain && job != Job::Hashes;
    std::vector<std::pair<uint64_t, uint64_t>> chunks;
    plan_chunks(h, off, need_hash_buf || !tok_dev || job == Job::Hashes, chunks);
    uint64_t Dc = 0, Tc = 0;
    for (auto &c : chunks) {
        Dc = std::max(Dc, c.second - c.first);
        Tc = std::max(Tc, off[c.second] - off[c.first]);
    }
    if ((st = ensure_chunk_scratch(h, Dc, Tc, need_hash_buf, job == Job::Signatures)) != LSHB_OK)
        return st;
    if (!tok_dev && (st = ensure_stage(h, Tc)) != LSHB_OK) return st;
    DevBuf &hashbuf = h->buf(B_HASHOUT);
    if (job == Job::Hashes && !out_dev && (st = hashbuf.reserve(std::max<uint64_t>(Tc, 1) * 4)) != LSHB_OK)
        return st;
    DevBuf &outbuf = h->buf(B_OUTSTAGE);
    size_t out_row = job == Job::Signatures ? (size_t)h->P * 4
                     : job == Job::Keys     ? (size_t)h->bands * 8
                                            : 1;
    if (job != Job::Hashes && !out_dev && (st = outbuf.reserve(Dc * out_row)) != LSHB_OK) return st;

    uint64_t *d_off_stage = (uint64_t *)h->buf(B_OFFSTAGE).ptr;
    // Host tokens: chunk c+1 is copied on the copy stream into the other
    // staging buffer while chunk c computes.
    auto issue_copy = [&](size_t ci) -> lshb_status {
        const uint64_t t0 = off[chunks[ci].first], nt = off[chunks[ci].second] - t0;
        return stage_copy(h, (int)(ci & 1), tokens + t0, nt);
    };
    if (!tok_dev && !chunks.empty() && (st = issue_copy(0)) != LSHB_OK) return st;
    // The next chunk's copy is issued once this chunk's first kernels are
    // queued, so a copy call that blocks the host never leaves the GPU idle.
    auto prefetch_next = [&](size_t ci) -> lshb_status {
        if (tok_dev || ci + 1 >= chunks.size()) return LSHB_OK;
        return issue_copy(ci + 1);
    };
    for (size_t ci = 0; ci < chunks.size(); ++ci) {
        const uint64_t lo = chunks[ci].first, hi = chunks[ci].second, Dn = hi - lo;
        ChunkIn in;
        in.D = Dn;
        if (off_dev) {
            in.offsets = offsets + lo;
        } else {
            CK(cudaMemcpyAsync(d_off_stage, offsets + lo, (Dn + 1) * 8, cudaMemcpyHostToDevice, s));
            in.offsets = d_off_stage;
        }
        if (tok_dev) {
            in.tokens = tokens + off[lo];
            in.tok_base = off[lo];
        } else {
            const int sb = (int)(ci & 1);
            CK(cudaStreamWaitEvent(s, h->ev_stage_ready[sb], 0));
            in.tokens = (const uint32_t *)h->stage_tok[sb].ptr;
            in.tok_base = off[lo];
        }
        if (job == Job::Dedup) {
            CK(cudaEventRecord(h->ev_t[0], s));
            if ((st = run_signatures(h, in, nullptr, nullptr, true, s)) != LSHB_OK) return st;
            CK(cudaEventRecord(h->ev_t[1], s));
            if ((st = prefetch_next(ci)) != LSHB_OK) return st;
            uint8_t *fl = out_dev ? (uint8_t *)out + lo : (uint8_t *)outbuf.ptr;
            if (keys_out)
                CK(cudaMemcpyAsync(keys_out + lo * h->bands, h->buf(B_KEYS).ptr, Dn * h->bands * 8,
                                   keys_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
            if ((st = run_bloom(h, Dn, fl, s)) != LSHB_OK) return st;
            CK(cudaEventRecord(h->ev_t[2], s));
            CK(cudaEventSynchronize(h->ev_t[2]));
            if (!tok_dev && (st = stage_copy_done(h, (int)(ci & 1))) != LSHB_OK) return st;
            float ms_sig = 0.f, ms_bloom = 0.f;
            CK(cudaEventElapsedTime(&ms_sig, h->ev_t[0], h->ev_t[1]));
            CK(cudaEventElapsedTime(&ms_bloom, h->ev_t[1], h->ev_t[2]));
            h->t_sig_ms += ms_sig;
            h->t_bloom_ms += ms_bloom;
            h->sig_chunks += 1;
            if (!out_dev) CK(cudaMemcpyAsync((uint8_t *)out + lo, fl, Dn, cudaMemcpyDeviceToHost, s));
            h->docs_seen += Dn;
        } else if (job == Job::Signatures) {
            uint32_t *so = out_dev ? (uint32_t *)out + lo * h->P : (uint32_t *)outbuf.ptr;
            if ((st = run_signatures(h, in, so, nullptr, false, s)) != LSHB_OK) return st;
            if (!out_dev)
                CK(cudaMemcpyAsync((uint32_t *)out + lo * h->P, so, Dn * h->P * 4,
                                   cudaMemcpyDeviceToHost, s));
        } else if (job == Job::Keys) {
            if ((st = run_signatures(h, in, nullptr, nullptr, true, s)) != LSHB_OK) return st;
            uint64_t *ko = (uint64_t *)h->buf(B_KEYS).ptr;
            CK(cudaMemcpyAsync((uint64_t *)out + lo * h->bands, ko, Dn * h->bands * 8,
                               out_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
        } else {
            const uint64_t t0 = off[lo] - off[0], nt = off[hi] - off[lo];
            uint32_t *ho = out_dev ? (uint32_t *)out + t0 : (uint32_t *)hashbuf.ptr;
            if ((st = run_signatures(h, in, nullptr, ho, false, s)) != LSHB_OK) return st;
            if (!out_dev && nt)
                CK(cudaMemcpyAsync((uint32_t *)out + t0, ho, nt * 4, cudaMemcpyDeviceToHost, s));
        }
        if (job != Job::Dedup && (st = prefetch_next(ci)) != LSHB_OK) return st;
        if (!tok_dev) CK(cudaEventRecord(h->ev_stage_free[ci & 1], s));
    }
    if (!require_device) CK(cudaStreamSynchronize(s));
    if (!tok_dev)
        for (int sb = 0; sb < 2; ++sb)
            if ((st = stage_copy_done(h, sb)) != LSHB_OK) return st;
    return LSHB_OK;
}

// Dedup calls add their host wall-clock time to the handle's call_ms.
static lshb_status run_batch_timed(lshbloom *h, const uint64_t *offsets, const uint32_t *tokens,
                                   uint64_t D, void *out, Job job, cudaStream_t user_stream,
                                   bool require_device, uint64_t *keys_out = nullptr) {
    const auto t0 = std::chrono::steady_clock::now();
    const lshb_status st =
        run_batch(h, offsets, tokens, D, out, job, user_stream, require_device, keys_out);
    if (h && job == Job::Dedup) {
        std::lock_guard<std::mutex> lock(h->mu);
        h->t_call_ms +=
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    return st;
}

extern "C" lshb_status lshbloom_dedup(lshbloom_t *h, const uint64_t *offsets,
                                      const uint32_t *tokens, uint64_t D, uint8_t *flags_out) {
    if (!h) return fail(LSHB_ERR_ARG, "NULL handle");
    return run_batch_timed(h, offsets, tokens, D, flags_out, Job::Dedup, nullptr, false);
}

extern "C" lshb_status lshbloom_dedup_keys(lshbloom_t *h, const uint64_t *offsets,
                                           const uint32_t *tokens, uint64_t D, uint8_t *flags_out,
                                           uint64_t *keys_out) {
    if (!h) return fail(LSHB_ERR_ARG, "NULL handle");
    if (D > 0 && !keys_out) return fail(LSHB_ERR_ARG, "NULL keys_out");
    return run_batch_timed(h, offsets, tokens, D, flags_out, Job::Dedup, nullptr, false, keys_out);
}

extern "C" lshb_status lshbloom_dedup_from_keys(lshbloom_t *h, const uint64_t *keys, uint64_t D,
                                                uint8_t *flags_out) {
    if (!h) return fail(LSHB_ERR_ARG, "NULL handle");
    if (D == 0) return LSHB_OK;
    if (!keys || !flags_out) return fail(LSHB_ERR_ARG, "NULL pointer with D > 0");
    const auto t0 = std::chrono::steady_clock::now();
    std::lock_guard<std::mutex> lock(h->mu);
    CK(cudaSetDevice(h->device));
    const bool keys_dev = is_device_pointer(keys), out_dev = is_device_pointer(flags_out);
    cudaStream_t s = h->stream;
    if (keys_dev || out_dev) {
        CK(cudaEventRecord(h->ev_order, cudaStreamLegacy));
        CK(cudaStreamWaitEvent(s, h->ev_order, 0));
    }
    const uint64_t dcap = std::min<uint64_t>(D, h->max_docs_batched);
    lshb_status st;
    if ((st = ensure_chunk_scratch(h, dcap, 0, false, false)) != LSHB_OK) return st;
    DevBuf &outbuf = h->buf(B_OUTSTAGE);
    if (!out_dev && (st = outbuf.reserve(dcap)) != LSHB_OK) return st;
    for (uint64_t lo = 0; lo < D; lo += dcap) {
        const uint64_t Dn = std::min(dcap, D - lo);
        CK(cudaEventRecord(h->ev_t[1], s));
        CK(cudaMemcpyAsync(h->buf(B_KEYS).ptr, keys + lo * h->bands, Dn * h->bands * 8,
                           keys_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
        uint8_t *fl = out_dev ? flags_out + lo : (uint8_t *)outbuf.ptr;
        if ((st = run_bloom(h, Dn, fl, s)) != LSHB_OK) return st;
        CK(cudaEventRecord(h->ev_t[2], s));
        if (!out_dev) CK(cudaMemcpyAsync(flags_out + lo, fl, Dn, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, h->ev_t[1], h->ev_t[2]));
        h->t_bloom_ms += ms;
        h->docs_seen += Dn;
    }
    h->t_call_ms +=
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return LSHB_OK;
}

extern "C" lshb_status lshbloom_dedup_async(lshbloom_t *h, const uint64_t *offsets,
                                            const uint32_t *tokens, uint64_t D, uint8_t *flags_out,
                                            void *stream) {
    if (!h) return fail(LSHB_ERR_ARG, "NULL handle");
    return run_batch_timed(h, offsets, tokens, D, flags_out, Job::Dedup, (cudaStream_t)stream, true);
}

extern "C" lshb_status lshbloom_signatures(lshbloom_t *h, const uint64_t *offsets,
                                           const uint32_t *tokens, uint64_t D, uint32_t *sig_out) {
    if (!h) return fail(LSHB_ERR_ARG, "NULL handle");
    return run_batch(h, offsets, tokens, D, sig_out, Job::Signatures, nullptr, false);
}

extern "C" lshb_status lshbloom_band_keys(lshbloom_t *h, const uint64_t *offsets,
                                          const uint32_t *tokens, uint64_t D, uint64_t *keys_out) {
    if (!h) return fail(LSHB_ERR_ARG, "NULL handle");
    return run_batch(h, offsets, tokens, D, keys_out, Job::Keys, nullptr, false);
}

extern "C" lshb_status lshbloom_shingle_hashes(lshbloom_t *h, const uint64_t *offsets,
                                               const uint32_t *tokens, uint64_t D, uint32_t *h_out) {
    if (!h) return fail(LSHB_ERR_ARG, "NULL handle");
    return run_batch(h, offsets, tokens, D, h_out, Job::Hashes, nullptr, false);
}

// ---- inspection, reset, persistence --------------------------------------------

extern "C" lshb_status lshbloom_coefficients(const lshbloom_t *h, uint64_t *a_out, uint64_t *b_out) {
    if (!h || !a_out || !b_out) return fail(LSHB_ERR_ARG, "NULL argument");
    memcpy(a_out, h->a.data(), sizeof(uint64_t) * h->P);
    memcpy(b_out, h->b.data(), sizeof(uint64_t) * h->P);
    return LSHB_OK;
}

extern "C" lshb_status lshbloom_filter_bytes(lshbloom_t *h, uint32_t band, uint8_t *host_out) {
    if (!h || !host_out) return fail(LSHB_ERR_ARG, "NULL argument");
    if (band >= h->bands) return fail(LSHB_ERR_ARG, "band %u out of range", band);
    std::lock_guard<std::mutex> lock(h->mu);
    CK(cudaSetDevice(h->device));
    const uint8_t *src = (const uint8_t *)(h->filters + (uint64_t)band * h->words_per_filter);
    const size_t nbytes =
        h->layout == LSHB_EXACT_KEYS ? (size_t)h->words_per_filter * 4 : (size_t)(h->m + 7) / 8;
    CK(cudaMemcpyAsync(host_out, src, nbytes, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return LSHB_OK;
}

extern "C" lshb_status lshbloom_reset(lshbloom_t *h) {
    if (!h) return fail(LSHB_ERR_ARG, "NULL handle");
    std::lock_guard<std::mutex> lock(h->mu);
    CK(cudaSetDevice(h->device));
    CK(cudaMemsetAsync(h->filters, h->layout == LSHB_EXACT_KEYS ? 0xff : 0,
                       (size_t)h->bands * h->words_per_filter * 4, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->docs_seen = h->dups_seen = h->resolve_rounds = h->uncertain_docs = 0;
    return LSHB_OK;
}

extern "C" lshb_status lshbloom_stats(lshbloom_t *h, lshb_stats *out) {
    if (!h || !out) return fail(LSHB_ERR_ARG, "NULL argument");
    std::lock_guard<std::mutex> lock(h->mu);
    CK(cudaSetDevice(h->device));
    memset(out, 0, sizeof *out);
    out->num_perm = h->P;
    out->bands = h->bands;
    out->rows = h->rows;
    out->ngram = h->ngram;
    out->k = h->k;
    out->insert_mode = h->cfg.insert_mode;
    out->exec_mode = h->cfg.exec_mode;
    out->item_shingles = h->item_shingles;
    out->m_bits = h->m;
    out->filter_bytes = h->layout == LSHB_EXACT_KEYS ? h->words_per_filter * 4 : h->m / 8;
    out->docs_seen = h->docs_seen;
    out->dups_seen = h->dups_seen;
    out->fp_rate = h->p;
    out->resolve_rounds = h->resolve_rounds;
    out->uncertain_docs = h->uncertain_docs;
    out->kernel_launches = launches_total();
    out->sig_ms = h->t_sig_ms;
    out->bloom_ms = h->t_bloom_ms;
    out->sig_chunks = h->sig_chunks;
    out->probe_ms = h->t_probe_ms;
    out->probe_sectors = h->probe_sectors;
    out->h2d_ms = h->t_h2d_ms;
    out->h2d_bytes = h->h2d_bytes;
    out->call_ms = h->t_call_ms;
    out->host_read_bytes = h->host_read_bytes;
    out->chunk_docs = h->max_docs_batched;
    out->pipelined_chunks = h->pipelined_chunks;
    unsigned long long *cnt = (unsigned long long *)(h->counters + C_POPCOUNT);
    const bool exact = h->layout == LSHB_EXACT_KEYS;
    for (uint32_t j = 0; j < h->bands; ++j) {
        CK(cudaMemsetAsync(cnt, 0, 8, h->stream));
        const uint32_t *f = h->filters + (uint64_t)j * h->words_per_filter;
        if (exact)
            CK(launch_count_occupied((const uint64_t *)f, h->words_per_filter / 2, cnt, h->stream));
        else
            CK(launch_popcount(f, h->words_per_filter, cnt, h->stream));
        CK(cudaMemcpyAsync(h->host_counters, h->counters, kChunkCounterBytes,
                           cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        // set bits per bit, or stored keys per key slot for the exact-key tables
        out->fill[j] = (double)*(unsigned long long *)(h->host_counters + C_POPCOUNT) /
                       (exact ? (double)h->exact_cap : (double)h->m);
    }
    return LSHB_OK;
}

namespace {
struct FileHeader {
    char magic[8];            // "LSHBLOOM"
    uint32_t version, P, bands, rows, ngram, k, insert_mode, bloom_layout;
    uint64_t n_expected, seed, m_bits, words_per_filter, docs_seen, dups_seen;
    double fp_rate_cfg, p;
    int32_t fp_is_effective, band_key;
};
}  // namespace

extern "C" lshb_status lshbloom_save(lshbloom_t *h, const char *path) {
    if (!h || !path) return fail(LSHB_ERR_ARG, "NULL argument");
    std::lock_guard<std::mutex> lock(h->mu);
    CK(cudaSetDevice(h->device));
    FileHeader hd;
    memset(&hd, 0, sizeof hd);
    memcpy(hd.magic, "LSHBLOOM", 8);
    hd.version = 1;
    hd.P = h->P; hd.bands = h->bands; hd.rows = h->rows; hd.ngram = h->ngram; hd.k = h->k;
    hd.insert_mode = h->cfg.insert_mode;
    hd.bloom_layout = h->cfg.bloom_layout;
    hd.n_expected = h->cfg.n_expected; hd.seed = h->cfg.seed; hd.m_bits = h->m;
    hd.words_per_filter = h->words_per_filter; hd.docs_seen = h->docs_seen;
    hd.dups_seen = h->dups_seen; hd.fp_rate_cfg = h->cfg.fp_rate; hd.p = h->p;
    hd.fp_is_effective = h->cfg.fp_is_effective;
    hd.band_key = (int32_t)h->cfg.band_key;
    FILE *f = fopen(path, "wb");
    if (!f) return fail(LSHB_ERR_IO, "cannot open %s for writing", path);
    bool ok = fwrite(&hd, sizeof hd, 1, f) == 1;
    ok = ok && fwrite(h->a.data(), 8, h->P, f) == h->P && fwrite(h->b.data(), 8, h->P, f) == h->P;
    const size_t fbytes = (size_t)h->words_per_filter * 4;
    std::vector<uint8_t> tmp(fbytes);
    for (uint32_t j = 0; ok && j < h->bands; ++j) {
        cudaError_t e = cudaMemcpy(tmp.data(), h->filters + (uint64_t)j * h->words_per_filter, fbytes,
                                   cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            fclose(f);
            return cuda_fail(e, "filter download");
        }
        ok = fwrite(tmp.data(), 1, fbytes, f) == fbytes;
    }
    ok = (fclose(f) == 0) && ok;
    if (!ok) return fail(LSHB_ERR_IO, "write to %s failed", path);
    return LSHB_OK;
}

extern "C" lshb_status lshbloom_load(const char *path, int32_t device, lshbloom_t **out) {
    if (!path || !out) return fail(LSHB_ERR_ARG, "NULL argument");
    *out = nullptr;
    FILE *f = fopen(path, "rb");
    if (!f) return fail(LSHB_ERR_IO, "cannot open %s", path);
    FileHeader hd;
    if (fread(&hd, sizeof hd, 1, f) != 1 || memcmp(hd.magic, "LSHBLOOM", 8) != 0 || hd.version != 1) {
        fclose(f);
        return fail(LSHB_ERR_IO, "%s is not an LSHBloom index", path);
    }
    std::vector<uint64_t> a(hd.P), b(hd.P);
    if (hd.P == 0 || hd.P > 1024 || fread(a.data(), 8, hd.P, f) != hd.P ||
        fread(b.data(), 8, hd.P, f) != hd.P) {
        fclose(f);
        return fail(LSHB_ERR_IO, "%s: truncated header", path);
    }
    lshb_config c;
    lshbloom_config_default(&c);
    c.num_perm = hd.P; c.bands = hd.bands; c.rows = hd.rows; c.ngram = hd.ngram;
    c.n_expected = hd.n_expected; c.fp_rate = hd.fp_rate_cfg; c.fp_is_effective = hd.fp_is_effective;
    c.insert_mode = hd.insert_mode; c.seed = hd.seed; c.perm_a = a.data(); c.perm_b = b.data();
    c.bloom_layout = hd.bloom_layout;
    c.band_key = (uint32_t)hd.band_key;
    c.device = device;
    lshbloom_t *h = nullptr;
    lshb_status st = lshbloom_create_ex(&c, &h);
    if (st != LSHB_OK) {
        fclose(f);
        return st;
    }
    if (h->m != hd.m_bits || h->words_per_filter != hd.words_per_filter || h->k != hd.k) {
        fclose(f);
        lshbloom_destroy(h);
        return fail(LSHB_ERR_IO, "%s: sizing does not match this build", path);
    }
    const size_t fbytes = (size_t)h->words_per_filter * 4;
    std::vector<uint8_t> tmp(fbytes);
    for (uint32_t j = 0; j < h->bands; ++j) {
        if (fread(tmp.data(), 1, fbytes, f) != fbytes) {
            fclose(f);
            lshbloom_destroy(h);
            return fail(LSHB_ERR_IO, "%s: truncated filters", path);
        }
        cudaError_t e = cudaMemcpy(h->filters + (uint64_t)j * h->words_per_filter, tmp.data(), fbytes,
                                   cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            fclose(f);
            lshbloom_destroy(h);
            return cuda_fail(e, "filter upload");
        }
    }
    fclose(f);
    h->docs_seen = hd.docs_seen;
    h->dups_seen = hd.dups_seen;
    *out = h;
    return LSHB_OK;
}

// ---- (b, r) tuning (Eqs. 1-2) -------------------------------------------------------

// Gauss-Legendre quadrature (16 nodes) on 64 equal panels.
static double gl_integral(double lo, double hi, uint32_t b, uint32_t r, bool fp) {
    static const double xs[8] = {0.0950125098376374, 0.2816035507792589, 0.4580167776572274,
                                 0.6178762444026438, 0.7554044083550030, 0.8656312023878318,
                                 0.9445750230732326, 0.9894009349916499};
    static const double ws[8] = {0.1894506104550685, 0.1826034150449236, 0.1691565193950025,
                                 0.1495959888165767, 0.1246289712555339, 0.0951585116824928,
                                 0.0622535239386479, 0.0271524594117541};
    const int panels = 64;
    const double hw = (hi - lo) / panels;
    double acc = 0.0;
    for (int p = 0; p < panels; ++p) {
        const double c = lo + (p + 0.5) * hw, half = 0.5 * hw;
        for (int i = 0; i < 8; ++i) {
            for (int sgn = -1; sgn <= 1; sgn += 2) {
                const double t = c + sgn * half * xs[i];
                const double miss = std::pow(1.0 - std::pow(t, (double)r), (double)b);
                acc += ws[i] * half * (fp ? 1.0 - miss : miss);
            }
        }
    }
    return acc;
}

extern "C" lshb_status lshbloom_optimal_br(double T, uint32_t P, uint32_t *b_out, uint32_t *r_out) {
    if (!b_out || !r_out || P < 1 || !(T > 0.0 && T < 1.0)) return fail(LSHB_ERR_ARG, "bad argument");
    double best = 1e300;
    uint32_t bb = 1, rr = 1;
    for (uint32_t b = 1; b <= P; ++b)
        for (uint32_t r = 1; (uint64_t)b * r <= P; ++r) {
            const double err = 0.5 * gl_integral(0.0, T, b, r, true) + 0.5 * gl_integral(T, 1.0, b, r, false);
            if (err < best) {
                best = err;
                bb = b;
                rr = r;
            }
        }
    *b_out = bb;
    *r_out = rr;
    return LSHB_OK;
}
