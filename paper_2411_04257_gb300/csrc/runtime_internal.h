// Host-side state of a handle and the runtime's internal entry points.
#pragma once

#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <mutex>
#include <utility>
#include <vector>

#include "../../include/lshbloom.h"
#include "bloom_kernels.cuh"
#include "lshb_internal.h"

namespace lshb {

struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
    lshb_status reserve(size_t want);  // grow-only; contents are not kept
    void release();
};

enum BufId {
    B_KEYS, B_MISS, B_CAND, B_STATUS, B_PREHIT, B_FLAGS, B_INSD, B_ULIST, B_BLOCKCNT, B_OFFSTAGE,
    B_SIG, B_HASHES, B_SKETCH, B_HT_KEYS, B_HT_FIXED, B_HT_FIRST, B_HT_SLOTS,
    B_HT_INS, B_HT_UDUP, B_HASHOUT, B_OUTSTAGE, B_KEYSTAGE, B_NBUF
};

// Slots of the device counter block (uint32 units; kCounterBytes in all).
enum CounterId {
    C_NU = 0,         // uncertain documents of the chunk
    C_ERROR = 2,      // device error bits
    C_DUPCOUNT = 6,   // (u64) duplicates of the chunk
    C_POPCOUNT = 8,   // (u64) popcount scratch
    C_QUEUE = 10,     // (u64) batched work-queue head
    C_SWEEPCTL = 12,  // 4 words: sweep changed, sweeps done, sweeps run, scratch
    C_BANDCOUNT = 64  // (u64 x 64) candidate bits of uncertain documents per band
};
constexpr size_t kCounterBytes = 1024;
constexpr size_t kChunkCounterBytes = 64;  // C_NU .. C_SWEEPCTL: cleared per chunk

struct SigPass {
    uint32_t p0, npc;
    int ppl;  // permutations per lane of the kernel instantiation
    PermSlice c;
};

struct ChunkIn {
    const uint64_t *offsets = nullptr;  // device, D+1
    const uint32_t *tokens = nullptr;   // device; document d starts at offsets[d] - tok_base
    uint64_t tok_base = 0;
    uint64_t D = 0;
};

struct BatchedState;

}  // namespace lshb

struct lshbloom {
    std::mutex mu;
    lshb_config cfg{};
    int device = -1;
    uint32_t P = 0, bands = 0, rows = 0, ngram = 0, k = 0;
    bool insert_all = false;
    uint32_t layout = 0;   // 0 standard, 1 blocked, 2 exact key sets
    double p = 0.0;
    uint64_t m = 0, words_per_filter = 0;
    uint64_t exact_cap = 0;  // exact layout: key slots per band table (power of two)
    std::vector<uint64_t> a, b;
    std::vector<lshb::SigPass> passes;
    uint32_t *filters = nullptr;
    cudaStream_t stream = nullptr, copy_stream = nullptr;
    cudaEvent_t ev_stage_free[2] = {nullptr, nullptr};
    cudaEvent_t ev_stage_ready[2] = {nullptr, nullptr};
    cudaEvent_t ev_h2d[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // bracket each staging copy
    uint64_t h2d_pending[2] = {0, 0};                                    // bytes of the copy in flight
    double t_h2d_ms = 0.0, t_call_ms = 0.0;
    uint64_t h2d_bytes = 0, host_read_bytes = 0;
    bool pageable_access = false;  // the device reads pageable host memory via host page tables
    lshb::DevBuf stage_tok[2];
    uint32_t *counters = nullptr;       // device, kCounterBytes
    uint32_t *host_counters = nullptr;  // pinned mirror
    lshb::DevBuf bufs[lshb::B_NBUF];
    uint64_t max_docs = 0, max_tokens = 0;
    uint64_t max_docs_batched = 0, max_tokens_batched = 0;
    // batched-form chunk autotuner (max_batch_docs = 0): candidate being
    // tried, wall time per document of each tried candidate, and the choice
    uint32_t chunk_trial = 0;
    double chunk_ms_per_doc[4] = {0, 0, 0, 0};
    bool chunk_warm = false, chunk_tuned = false;
    uint32_t item_shingles = 0;
    lshb::BatchedState *batched = nullptr;
    uint64_t docs_seen = 0, dups_seen = 0, resolve_rounds = 0, uncertain_docs = 0;
    cudaEvent_t ev_t[3] = {nullptr, nullptr, nullptr};  // stage timers
    double t_sig_ms = 0.0, t_bloom_ms = 0.0;
    uint64_t sig_chunks = 0;
    uint64_t pipelined_chunks = 0;  // batched form: Bloom stages overlapped with the next signatures
    cudaEvent_t ev_p[2] = {nullptr, nullptr};  // bracket the probe kernel (one-kernel-per-stage form)
    cudaEvent_t ev_order = nullptr;  // orders a synchronous call after the legacy default stream
    double t_probe_ms = 0.0;
    uint64_t probe_sectors = 0;                // band-key probes issued by that kernel
    bool probe_pending = false;

    lshb::DevBuf &buf(lshb::BufId id) { return bufs[id]; }
    ~lshbloom();
};

namespace lshb {

// Staging copies of host tokens into stage_tok[sb] on the copy stream, and
// the accounting of the one that completed.
lshb_status stage_copy(lshbloom *h, int sb, const uint32_t *src, uint64_t ntok);
lshb_status stage_copy_done(lshbloom *h, int sb);

lshb_status fail(lshb_status st, const char *fmt, ...);
lshb_status cuda_fail(cudaError_t e, const char *what);
lshb_status init_handle(lshbloom *h, const lshb_config *cfg);
bool is_device_pointer(const void *p);
const void *mapped_host_pointer(const void *p);
// Address the kernels can read host buffer p through, or nullptr when it must
// be staged: its device mapping when pinned, p itself when the device reads
// pageable memory in place.
const void *host_read_pointer(bool pageable_access, const void *p);
bool device_reads_pageable(int device);
lshb_status host_offsets(lshbloom *h, const uint64_t *offsets, uint64_t D, bool dev,
                         std::vector<uint64_t> &out, cudaStream_t s);
void plan_chunks(const lshbloom *h, const std::vector<uint64_t> &off, bool bound_tokens,
                 std::vector<std::pair<uint64_t, uint64_t>> &chunks,
                 uint64_t first_tokens = 0);
lshb_status ensure_chunk_scratch(lshbloom *h, uint64_t Dc, uint64_t Tc, bool plain_hashes,
                                 bool need_sig);
lshb_status ensure_stage(lshbloom *h, uint64_t Tc);
lshb_status run_signatures(lshbloom *h, const ChunkIn &in, uint32_t *sig_out, uint32_t *hash_out,
                           bool want_keys, cudaStream_t s);
// Sketch cells per band for batches of up to dcap documents.
uint64_t sketch_cells_for(const lshbloom *h, uint64_t dcap);
// Bloom-stage arguments for a batch of D documents in scratch sized for dcap.
BloomArgs bloom_args(lshbloom *h, uint64_t D, uint64_t dcap);
// Probe sectors one band key addresses (k, or one block / one key).
uint64_t probe_sectors_per_key(const lshbloom *h);
lshb_status run_bloom(lshbloom *h, uint64_t D, uint8_t *flags_dev, cudaStream_t s);
lshb_status resolve_and_insert(lshbloom *h, const BloomArgs &A, uint8_t *flags_dev,
                               cudaStream_t s);

// Several CSR batches in one launch of the persistent kernel (batched.cu):
// their band keys, written to each batch's keys_out.  The state keeps the
// launch's scratch; the caller starts a launch only once the previous launch
// of the same state has completed on the GPU.
struct Segment;  // segment.h
struct SegmentState;
constexpr uint32_t kMaxSegments = 256;
SegmentState *segment_state_create();
void segment_state_destroy(SegmentState *st);
// The launch's device error word as copied back at its end (valid once the
// launch has completed); nonzero = work-queue inconsistency.
uint32_t segment_state_error(const SegmentState *st);
lshb_status launch_keys_segments(lshbloom *h, SegmentState *st, const Segment *segs,
                                 uint32_t nseg, uint64_t D, uint64_t T, cudaStream_t s);

// Batched (persistent, graph-launched) form.
lshb_status run_batched(lshbloom *h, const uint64_t *offsets, const uint32_t *tokens, uint64_t D,
                        uint8_t *flags, const std::vector<uint64_t> &off, bool off_dev,
                        bool tok_dev, bool out_dev, cudaStream_t s, uint64_t *keys_out,
                        bool keys_dev);
void destroy_batched_state(lshbloom *h);

}  // namespace lshb
