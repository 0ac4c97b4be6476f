// Batched form of the path: one persistent fused kernel over a work queue of
// (document, shingle range) items, launched through a captured CUDA graph.
//
// Per chunk the graph runs: per-document item counts, a scan, the item ->
// document map and the persistent kernel (SHA-1 + MinHash for its item; a
// document split over several items merges its minima with atomicMin and the
// last item to finish forms the band keys).  The per-chunk pointers and sizes
// are copied into a device-side parameter block at the start of the graph, so
// one instantiated graph per signature slot serves every chunk of a handle.
//
// Chunks of short documents are pipelined over two streams: the signature
// graphs run on a private stream up to two chunks ahead while the Bloom stage
// of a chunk (probes, classification, in-batch order resolution, insert:
// stream-ordered, driven from the host) runs on the caller's stream behind an
// event.  The chunks take three signature slots (parameter block, work-queue
// counter, band keys) in turn; the Bloom stages stay in chunk order on one
// stream, so the flags are those of one sequential stream.  While pipelined,
// some of the persistent kernel's blocks return at once, leaving block slots
// on every SM to the Bloom stage; when the Bloom stage is a small share of a
// chunk (long documents) the chunks run one after the other with every block.
//
// Long documents no longer serialise on one warp and heavy-tailed length
// mixes balance across the GPU; the item size is picked by a short timing
// sweep on the first chunk.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>

#include "batched_kernels.cuh"
#include "runtime_internal.h"

namespace lshb {

// ---- host side ---------------------------------------------------------------------

// The signature slots the chunks take in turn: the signature stream runs up
// to kSigSlots - 1 chunks ahead of the Bloom stage.
constexpr int kSigSlots = 3;

struct SigSlot {
    DynParams *dyn = nullptr;           // device parameter block
    DynParams *dyn_host = nullptr;      // pinned source of the graph's first copy
    unsigned long long *ctr = nullptr;  // device: [0] work-queue head, [1] error word
    uint32_t *err_host = nullptr;       // pinned copy of the error word
    DevBuf keys;                        // bands x dcap, band-major
    DevBuf off_stage;                   // the chunk's offsets when the caller's are on the host
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // bracket the persistent kernel
    cudaEvent_t done = nullptr;                // everything of the slot's launch is complete

    void drop_graph() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
    }
    ~SigSlot() {
        drop_graph();
        keys.release();
        off_stage.release();
        if (dyn) cudaFree(dyn);
        if (ctr) cudaFree(ctr);
        if (dyn_host) cudaFreeHost(dyn_host);
        if (err_host) cudaFreeHost(err_host);
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
        if (done) cudaEventDestroy(done);
    }
};

struct BatchedState {
    uint64_t dcap = 0, item_cap = 0;
    uint32_t item = 0;
    int grid = 0;                               // occupancy x SMs
    int sms = 0, occupancy = 0;                 // persistent-kernel blocks per SM
    int reserve = 0;                            // block slots per SM left to the Bloom stage
    SigSlot slot[kSigSlots];
    DevBuf item_count, item_start, block_sums, item_doc, pending, sig_partial;
    cudaStream_t sig_stream = nullptr;          // the signature graphs
    cudaStream_t cap_stream = nullptr;          // private stream for graph capture
    cudaEvent_t ev_start = nullptr;             // orders the signature stream after the caller's
    uint64_t graph_kernels = 0;                 // kernels one launch of a graph runs
    // stage times of the chunks run one after the other: pick `reserve`
    double sig_ms = 0.0, bloom_ms = 0.0;
    uint32_t measured_chunks = 0;
    bool reserve_decided = false;

    void drop_graphs() {
        for (SigSlot &sl : slot) sl.drop_graph();
    }
    ~BatchedState() {
        drop_graphs();
        item_count.release(); item_start.release(); block_sums.release();
        item_doc.release(); pending.release(); sig_partial.release();
        if (ev_start) cudaEventDestroy(ev_start);
        if (sig_stream) cudaStreamDestroy(sig_stream);
        if (cap_stream) cudaStreamDestroy(cap_stream);
    }
};

void destroy_batched_state(lshbloom *h) {
    delete h->batched;
    h->batched = nullptr;
}

#define BCK(call)                                                           \
    do {                                                                    \
        cudaError_t e_ = (call);                                            \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);                 \
    } while (0)

template <int NG, int PPL>
static cudaError_t go_batched(const BatchArgs &a, int grid, cudaStream_t s) {
    k_batched<NG, PPL><<<grid, kBatchThreads, 0, s>>>(a);
    count_launch();
    return cudaGetLastError();
}

template <int NG>
static cudaError_t dispatch_ppl(int ppl, const BatchArgs &a, int grid, cudaStream_t s) {
    switch (ppl) {
        case 1: return go_batched<NG, 1>(a, grid, s);
        case 2: return go_batched<NG, 2>(a, grid, s);
        case 4: return go_batched<NG, 4>(a, grid, s);
        case 8: return go_batched<NG, 8>(a, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

static cudaError_t launch_k_batched(int ngt, int ppl, const BatchArgs &a, int grid, cudaStream_t s) {
    if (ngt == 5) return dispatch_ppl<5>(ppl, a, grid, s);
    if (ngt == 1) return dispatch_ppl<1>(ppl, a, grid, s);
    return dispatch_ppl<0>(ppl, a, grid, s);
}

template <int NG, int PPL>
static int occ_batched() {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batched<NG, PPL>, kBatchThreads, 0);
    return nb > 0 ? nb : 1;
}

// Resident blocks of the persistent kernel per SM.
static int batched_occupancy(int ngt, int ppl) {
    int nb = 1;
#define LSHB_OCC(NGV)                                                    \
    switch (ppl) {                                                        \
        case 1: nb = occ_batched<NGV, 1>(); break;                        \
        case 2: nb = occ_batched<NGV, 2>(); break;                        \
        case 4: nb = occ_batched<NGV, 4>(); break;                        \
        default: nb = occ_batched<NGV, 8>(); break;                       \
    }
    if (ngt == 5) { LSHB_OCC(5) } else if (ngt == 1) { LSHB_OCC(1) } else { LSHB_OCC(0) }
#undef LSHB_OCC
    return nb;
}

// Blocks of the persistent kernel: its occupancy on every SM.
static int batched_grid(int ngt, int ppl) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return batched_occupancy(ngt, ppl) * (sms > 0 ? sms : 1);
}

static BatchArgs make_args(lshbloom *h, BatchedState *b, int p) {
    BatchArgs a;
    memset(&a, 0, sizeof a);
    const SigPass &ps = h->passes[0];
    SigSlot &sl = b->slot[p];
    a.dyn = sl.dyn;
    a.item_shingles = b->item;
    a.ngram = h->ngram;
    a.P = h->P;
    a.npc = ps.npc;
    a.bands = h->bands;
    a.rows = h->rows;
    a.band_key = h->cfg.band_key;
    a.item_count = (uint32_t *)b->item_count.ptr;
    a.item_start = (uint64_t *)b->item_start.ptr;
    a.block_sums = (uint64_t *)b->block_sums.ptr;
    a.item_doc = (uint32_t *)b->item_doc.ptr;
    a.item_cap = b->item_cap;
    a.pending = (uint32_t *)b->pending.ptr;
    a.sig_partial = (uint32_t *)b->sig_partial.ptr;
    a.queue = sl.ctr;
    a.keys = (uint64_t *)sl.keys.ptr;
    a.key_rows = b->dcap;
    a.cand = nullptr;    // the Bloom stage clears its own
    a.prehit = nullptr;
    a.error = reinterpret_cast<uint32_t *>(sl.ctr + 1);
    a.c = ps.c;
    return a;
}

// Per-document item counts, their scan and the item -> document map for a
// launch of up to dcap documents described by a.dyn.
static cudaError_t enqueue_items(const BatchArgs &a, uint64_t dcap, cudaStream_t s) {
    const unsigned nb = (unsigned)((dcap + kScanBlock - 1) / kScanBlock);
    unsigned pg = (unsigned)std::min<uint64_t>((dcap + 255) / 256, 16384);
    k_batch_prepare<<<pg ? pg : 1, 256, 0, s>>>(a);
    count_launch();
    k_scan_reduce<<<nb ? nb : 1, kScanBlock, 0, s>>>(a);
    count_launch();
    k_scan_top<<<1, kScanBlock, 0, s>>>(a, nb ? nb : 1);
    count_launch();
    k_scan_down<<<nb ? nb : 1, kScanBlock, 0, s>>>(a);
    count_launch();
    k_expand<<<pg ? pg : 1, 256, 0, s>>>(a);
    count_launch();
    return cudaGetLastError();
}

// The signature work of one chunk in slot p, for the chunk described by the
// slot's pinned parameter block (enqueued on s; also what a graph captures).
static lshb_status enqueue_sig(lshbloom *h, BatchedState *b, int p, cudaStream_t s,
                               bool time_kernel) {
    SigSlot &sl = b->slot[p];
    const BatchArgs a = make_args(h, b, p);
    BCK(cudaMemcpyAsync(sl.dyn, sl.dyn_host, sizeof(DynParams), cudaMemcpyHostToDevice, s));
    BCK(cudaMemsetAsync(sl.ctr, 0, 2 * sizeof(unsigned long long), s));
    BCK(enqueue_items(a, b->dcap, s));
    // Under capture the records must be external to become event-record nodes
    // of the graph (then every replay times the persistent kernel).
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    BCK(cudaStreamIsCapturing(s, &cap));
    const unsigned rec_flags = cap == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : 0u;
    if (time_kernel) BCK(cudaEventRecordWithFlags(sl.ev0, s, rec_flags));
    BCK(launch_k_batched(ngram_template(h->ngram), h->passes[0].ppl, a, b->grid, s));
    if (time_kernel) BCK(cudaEventRecordWithFlags(sl.ev1, s, rec_flags));
    return LSHB_OK;
}

// Block slots per SM left to the Bloom stage.  A handle's first call runs its
// chunks one after the other and measures both stages.  From the next call
// on, when the Bloom stage took at least kPipelineShare of a chunk's time,
// the chunks are pipelined and the persistent kernel leaves
// kReserveFactor x that share of each SM's block slots (rounded down, at
// least one, at most half) to the Bloom stage.  Measured on the 8M-document
// Pareto batch (Bloom stage 43% of a serial chunk, 10 slots per SM): 125.8 ms
// per call one after the other; pipelined with 1 to 6 slots left 123.5,
// 121.9, 117.6, 117.1, 124.2, 136.0 ms.  With longer documents the Bloom
// stage is a few per cent of a chunk and the chunks stay serial: leaving two
// slots on the billion-document stream (16%) measured 1.8% slower.
constexpr double kPipelineShare = 0.3;
constexpr double kReserveFactor = 0.75;

static int pick_reserve(BatchedState *b) {
    if (b->reserve_decided || b->measured_chunks == 0) return b->reserve;
    b->reserve_decided = true;
    const double share = b->bloom_ms / std::max(1e-9, b->sig_ms + b->bloom_ms);
    if (share < kPipelineShare) return 0;
    const int r = (int)(kReserveFactor * share * b->occupancy);
    return std::max(1, std::min(b->occupancy / 2, r));
}

static lshb_status ensure_state(lshbloom *h, uint64_t dcap, uint64_t tcap) {
    BatchedState *b = h->batched;
    if (!b) {
        b = h->batched = new BatchedState();
        for (SigSlot &sl : b->slot) {
            BCK(cudaMalloc(&sl.dyn, sizeof(DynParams)));
            BCK(cudaMallocHost(&sl.dyn_host, sizeof(DynParams)));
            BCK(cudaMalloc(&sl.ctr, 2 * sizeof(unsigned long long)));
            BCK(cudaMallocHost(&sl.err_host, sizeof(uint32_t)));
            BCK(cudaEventCreate(&sl.ev0));
            BCK(cudaEventCreate(&sl.ev1));
            BCK(cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming));
        }
        BCK(cudaEventCreateWithFlags(&b->ev_start, cudaEventDisableTiming));
        BCK(cudaStreamCreateWithFlags(&b->sig_stream, cudaStreamNonBlocking));
        BCK(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
    }
    // the graph's grids follow the largest chunk of the call
    if (dcap != b->dcap) {
        b->drop_graphs();
        b->dcap = dcap;
    }
    lshb_status st;
    // item_doc capacity: every item but a document's last holds a full
    // item of the smallest candidate size.
    const uint64_t icap = tcap / kItemCandidates[0] + b->dcap + 1;
    if (icap > b->item_cap) {
        b->drop_graphs();
        b->item_cap = icap;
    }
    if ((st = b->item_count.reserve(b->dcap * 4)) != LSHB_OK) return st;
    if ((st = b->item_start.reserve((b->dcap + 1) * 8)) != LSHB_OK) return st;
    if ((st = b->block_sums.reserve(((b->dcap + kScanBlock - 1) / kScanBlock + 1) * 8)) != LSHB_OK)
        return st;
    if ((st = b->item_doc.reserve(b->item_cap * 4)) != LSHB_OK) return st;
    if ((st = b->pending.reserve(b->dcap * 4)) != LSHB_OK) return st;
    if ((st = b->sig_partial.reserve(b->dcap * h->P * 4)) != LSHB_OK) return st;
    for (SigSlot &sl : b->slot) {
        if ((st = sl.keys.reserve(b->dcap * h->bands * 8)) != LSHB_OK) return st;
        if ((st = sl.off_stage.reserve((b->dcap + 1) * 8)) != LSHB_OK) return st;
    }
    if ((st = ensure_chunk_scratch(h, b->dcap, 0, false, false)) != LSHB_OK) return st;
    if (!b->grid) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
        b->sms = std::max(1, b->sms);
        b->occupancy = batched_occupancy(ngram_template(h->ngram), h->passes[0].ppl);
        b->grid = b->occupancy * b->sms;
    }
    b->reserve = pick_reserve(b);
    return LSHB_OK;
}

// Time the persistent kernel alone for each item size on (a prefix of) the
// first chunk and keep the fastest (slot 0, on the signature stream).
static lshb_status autotune(lshbloom *h, const DynParams &chunk) {
    BatchedState *b = h->batched;
    cudaStream_t s = b->sig_stream;
    DynParams sample = chunk;
    sample.D = std::min<uint64_t>(chunk.D, 1ull << 16);
    float best = 1e30f;
    uint32_t best_item = 256;
    for (uint32_t item : kItemCandidates) {
        b->item = item;
        BCK(cudaStreamSynchronize(s));  // the pinned parameter block is free
        *b->slot[0].dyn_host = sample;
        lshb_status st = enqueue_sig(h, b, 0, s, true);
        if (st != LSHB_OK) return st;
        BCK(cudaStreamSynchronize(s));
        float ms = 0.f;
        BCK(cudaEventElapsedTime(&ms, b->slot[0].ev0, b->slot[0].ev1));
        if (ms < best) {
            best = ms;
            best_item = item;
        }
    }
    b->item = best_item;
    h->item_shingles = best_item;
    b->drop_graphs();
    return LSHB_OK;
}

static lshb_status ensure_graphs(lshbloom *h) {
    BatchedState *b = h->batched;
    for (int p = 0; p < kSigSlots; ++p) {
        SigSlot &sl = b->slot[p];
        if (sl.exec) continue;
        cudaStream_t cs = b->cap_stream;
        const uint64_t counted = launches_total();
        BCK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        lshb_status st = enqueue_sig(h, b, p, cs, true);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(cs, &g);
        // capture enqueues nothing: take back what the launch wrappers
        // counted, and count it per graph launch instead
        b->graph_kernels = launches_total() - counted;
        count_launch(counted - launches_total());
        if (st != LSHB_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        sl.graph = g;
        BCK(cudaGraphInstantiate(&sl.exec, g, 0));
    }
    return LSHB_OK;
}

// Chunk sizes the batched form's autotuner tries, in documents, on calls of at
// least kChunkTuneMinDocs documents (smaller calls cannot tell them apart).
constexpr uint64_t kChunkCandidates[4] = {1ull << 18, 1ull << 19, 1ull << 20, 1ull << 21};
constexpr uint64_t kChunkTuneMinDocs = 1ull << 22;

static lshb_status run_batched_chunks(lshbloom *h, const uint64_t *offsets,
                                      const uint32_t *tokens, uint64_t D, uint8_t *flags,
                                      const std::vector<uint64_t> &off, bool off_dev,
                                      bool tok_dev, bool out_dev, cudaStream_t s,
                                      uint64_t *keys_out, bool keys_dev);

// Chunk size: max_batch_docs when set; otherwise, among calls of at least
// kChunkTuneMinDocs documents, the first runs with the largest candidate (it
// pays for allocations and the item-size tuning), the next four try each
// candidate once, timing the whole call per document (chunking never changes
// a result), and later calls keep the fastest.
lshb_status run_batched(lshbloom *h, const uint64_t *offsets, const uint32_t *tokens, uint64_t D,
                        uint8_t *flags, const std::vector<uint64_t> &off, bool off_dev,
                        bool tok_dev, bool out_dev, cudaStream_t s, uint64_t *keys_out,
                        bool keys_dev) {
    const bool tune = !h->cfg.max_batch_docs && !h->chunk_tuned && D >= kChunkTuneMinDocs;
    const bool trial = tune && h->chunk_warm;
    if (tune) h->max_docs_batched = kChunkCandidates[trial ? h->chunk_trial : 3];
    if (tune && !trial) {
        h->chunk_warm = true;
        return run_batched_chunks(h, offsets, tokens, D, flags, off, off_dev, tok_dev, out_dev, s,
                                  keys_out, keys_dev);
    }
    const auto t0 = std::chrono::steady_clock::now();
    lshb_status st = run_batched_chunks(h, offsets, tokens, D, flags, off, off_dev, tok_dev,
                                        out_dev, s, keys_out, keys_dev);
    if (st != LSHB_OK || !trial) return st;
    h->chunk_ms_per_doc[h->chunk_trial] =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count() /
        (double)D;
    if (++h->chunk_trial == 4) {
        uint32_t best = 0;
        for (uint32_t c = 1; c < 4; ++c)
            if (h->chunk_ms_per_doc[c] < h->chunk_ms_per_doc[best]) best = c;
        h->max_docs_batched = kChunkCandidates[best];
        h->chunk_tuned = true;
    }
    return LSHB_OK;
}

static lshb_status pipeline_chunks(lshbloom *h, const uint64_t *offsets, const uint32_t *tokens,
                                   uint8_t *flags, const std::vector<uint64_t> &off,
                                   const std::vector<std::pair<uint64_t, uint64_t>> &chunks,
                                   bool off_dev, bool tok_dev, bool out_dev, cudaStream_t s,
                                   uint64_t *keys_out, bool keys_dev);

static lshb_status run_batched_chunks(lshbloom *h, const uint64_t *offsets,
                                      const uint32_t *tokens, uint64_t D, uint8_t *flags,
                                      const std::vector<uint64_t> &off, bool off_dev,
                                      bool tok_dev, bool out_dev, cudaStream_t s,
                                      uint64_t *keys_out, bool keys_dev) {
    if (off.size() != D + 1) return fail(LSHB_ERR_ARG, "offsets of %llu documents expected",
                                         (unsigned long long)D);
    // chunks: documents and (for staged or very large inputs) tokens bounded
    const uint64_t dmax = h->max_docs_batched;
    std::vector<std::pair<uint64_t, uint64_t>> chunks;
    {
        // Staged host inputs take the same large chunks as resident ones, so a
        // batch costs a few host round trips, ramped from 2^28 tokens so that
        // the first, unhidden copy stays short.
        const uint64_t save_docs = h->max_docs, save_tok = h->max_tokens;
        h->max_docs = dmax;
        h->max_tokens = h->max_tokens_batched;
        plan_chunks(h, off, true, chunks,
                    tok_dev ? 0 : std::min<uint64_t>(1ull << 28, h->max_tokens_batched));
        h->max_docs = save_docs;
        h->max_tokens = save_tok;
    }
    uint64_t dcap = 0, tcap = 0;
    for (auto &c : chunks) {
        dcap = std::max(dcap, c.second - c.first);
        tcap = std::max(tcap, off[c.second] - off[c.first]);
    }
    lshb_status st;
    if ((st = ensure_state(h, dcap, tcap)) != LSHB_OK) return st;
    if (!tok_dev && (st = ensure_stage(h, tcap)) != LSHB_OK) return st;
    BatchedState *b = h->batched;
    if (!out_dev && (st = h->buf(B_OUTSTAGE).reserve(b->dcap)) != LSHB_OK) return st;
    // row-major keys on their way to host keys_out
    if (keys_out && !keys_dev && (st = h->buf(B_KEYSTAGE).reserve(b->dcap * h->bands * 8)) != LSHB_OK)
        return st;
    st = pipeline_chunks(h, offsets, tokens, flags, off, chunks, off_dev, tok_dev, out_dev, s,
                         keys_out, keys_dev);
    // on every exit nothing of the call is left running on the signature stream
    cudaError_t e1 = cudaStreamSynchronize(b->sig_stream);
    cudaError_t e2 = cudaStreamSynchronize(s);
    if (st != LSHB_OK) return st;
    if (e1 != cudaSuccess) return cuda_fail(e1, "cudaStreamSynchronize(signature stream)");
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamSynchronize");
    return LSHB_OK;
}

// The chunk loop.  Chunk c uses signature slot c mod kSigSlots.  On the
// host, when pipelined: launch the signature graphs up to chunk
// c + kSigSlots - 1 (signature stream), then run the Bloom stage of chunk c
// (caller's stream); otherwise launch chunk c's signatures and run its Bloom
// stage.  A slot is reused kSigSlots chunks later, after the Bloom stage that
// read its keys has completed on the host, so its parameter block, keys and
// offsets are free by then.
static lshb_status pipeline_chunks(lshbloom *h, const uint64_t *offsets, const uint32_t *tokens,
                                   uint8_t *flags, const std::vector<uint64_t> &off,
                                   const std::vector<std::pair<uint64_t, uint64_t>> &chunks,
                                   bool off_dev, bool tok_dev, bool out_dev, cudaStream_t s,
                                   uint64_t *keys_out, bool keys_dev) {
    BatchedState *b = h->batched;
    cudaStream_t ss = b->sig_stream;
    const bool pipelined = b->reserve > 0 && chunks.size() > 1;
    lshb_status st;
    // the signature stream starts after everything already enqueued on s
    BCK(cudaEventRecord(b->ev_start, s));
    BCK(cudaStreamWaitEvent(ss, b->ev_start, 0));

    auto issue_copy = [&](size_t ci) -> lshb_status {
        const uint64_t t0 = off[chunks[ci].first], nt = off[chunks[ci].second] - t0;
        return stage_copy(h, (int)(ci & 1), tokens + t0, nt);
    };

    // Signatures of chunk ci into its slot, on the signature stream (token
    // staging buffer ci & 1 when the caller's tokens are staged).
    auto launch_sig = [&](size_t ci) -> lshb_status {
        const int p = (int)(ci % kSigSlots), sb = (int)(ci & 1);
        SigSlot &sl = b->slot[p];
        const uint64_t lo = chunks[ci].first, hi = chunks[ci].second, Dn = hi - lo;
        DynParams dp;
        memset(&dp, 0, sizeof dp);
        dp.D = Dn;
        if (pipelined) dp.active_blocks = (uint32_t)((b->occupancy - b->reserve) * b->sms);
        if (off_dev) {
            dp.offsets = offsets + lo;
        } else {
            BCK(cudaMemcpyAsync(sl.off_stage.ptr, offsets + lo, (Dn + 1) * 8, cudaMemcpyHostToDevice,
                                ss));
            dp.offsets = (const uint64_t *)sl.off_stage.ptr;
        }
        dp.tok_base = off[lo];
        if (tok_dev) {
            dp.tokens = tokens + off[lo];
        } else {
            if (ci == 0 && (st = issue_copy(0)) != LSHB_OK) return st;
            BCK(cudaStreamWaitEvent(ss, h->ev_stage_ready[sb], 0));
            dp.tokens = (const uint32_t *)h->stage_tok[sb].ptr;
        }
        if (b->item == 0) {
            if (h->cfg.item_shingles) {
                b->item = h->cfg.item_shingles;
                h->item_shingles = b->item;
            } else if ((st = autotune(h, dp)) != LSHB_OK) {
                return st;
            }
        }
        if ((st = ensure_graphs(h)) != LSHB_OK) return st;
        *sl.dyn_host = dp;  // read by the graph's first node
        BCK(cudaGraphLaunch(sl.exec, ss));
        count_launch(b->graph_kernels);  // prepare, scan, expand, persistent kernel
        BCK(cudaEventRecord(sl.done, ss));
        if (!tok_dev) BCK(cudaEventRecord(h->ev_stage_free[sb], ss));
        // Prefetch the next chunk's tokens only now, while this chunk computes:
        // a copy call that blocks the host then no longer idles the GPU.
        if (!tok_dev && ci + 1 < chunks.size() && (st = issue_copy(ci + 1)) != LSHB_OK) return st;
        return LSHB_OK;
    };

    // Bloom stage of chunk ci, on s, after its slot's signatures.
    auto finish = [&](size_t ci) -> lshb_status {
        const int p = (int)(ci % kSigSlots);
        SigSlot &sl = b->slot[p];
        const uint64_t lo = chunks[ci].first, Dn = chunks[ci].second - lo;
        BCK(cudaStreamWaitEvent(s, sl.done, 0));
        BCK(cudaEventRecord(h->ev_t[0], s));
        BloomArgs A = bloom_args(h, Dn, b->dcap);
        A.keys = (const uint64_t *)sl.keys.ptr;  // band-major
        A.key_sd = 1;
        A.key_sj = b->dcap;
        BCK(cudaMemsetAsync(h->counters, 0, kChunkCounterBytes, s));
        BCK(cudaMemsetAsync(A.sketch, 0, (uint64_t)h->bands * (A.sketch_cells / 16) * 4, s));
        BCK(cudaMemsetAsync(A.cand, 0, Dn * 8, s));
        BCK(cudaMemsetAsync(A.prehit, 0, Dn, s));
        BCK(cudaMemcpyAsync(sl.err_host, sl.ctr + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        BCK(cudaEventRecord(h->ev_p[0], s));
        BCK(launch_probe(A, Dn, s));
        BCK(cudaEventRecord(h->ev_p[1], s));
        h->probe_sectors += Dn * h->bands * probe_sectors_per_key(h);
        BCK(launch_classify(A, Dn, (uint32_t *)h->buf(B_BLOCKCNT).ptr, h->counters + C_NU,
                            (uint32_t *)h->buf(B_ULIST).ptr, s));
        BCK(cudaMemcpyAsync(h->host_counters, h->counters, kChunkCounterBytes,
                            cudaMemcpyDeviceToHost, s));
        BCK(cudaStreamSynchronize(s));
        if (*sl.err_host != 0)
            return fail(LSHB_ERR_CUDA, "device error word 0x%x (signature stage)", *sl.err_host);
        float ms_k7 = 0.f, ms_probe = 0.f;
        BCK(cudaEventElapsedTime(&ms_k7, sl.ev0, sl.ev1));
        BCK(cudaEventElapsedTime(&ms_probe, h->ev_p[0], h->ev_p[1]));
        h->t_probe_ms += ms_probe;
        if (keys_out) {
            // the keys, band-major in the slot, leave row-major
            uint64_t *dst = keys_dev ? keys_out + lo * h->bands : (uint64_t *)h->buf(B_KEYSTAGE).ptr;
            const uint64_t n = Dn * h->bands;
            k_keys_row_major<<<(unsigned)std::min<uint64_t>((n + 255) / 256, 8192), 256, 0, s>>>(
                (const uint64_t *)sl.keys.ptr, b->dcap, Dn, h->bands, dst);
            count_launch();
            BCK(cudaGetLastError());
            if (!keys_dev)
                BCK(cudaMemcpyAsync(keys_out + lo * h->bands, dst, n * 8, cudaMemcpyDeviceToHost, s));
        }
        uint8_t *fl = out_dev ? flags + lo : (uint8_t *)h->buf(B_OUTSTAGE).ptr;
        if ((st = resolve_and_insert(h, A, fl, s)) != LSHB_OK) return st;
        BCK(cudaEventRecord(h->ev_t[2], s));
        if (!out_dev) BCK(cudaMemcpyAsync(flags + lo, fl, Dn, cudaMemcpyDeviceToHost, s));
        BCK(cudaEventSynchronize(h->ev_t[2]));
        float ms_bloom = 0.f;
        BCK(cudaEventElapsedTime(&ms_bloom, h->ev_t[0], h->ev_t[2]));
        h->t_sig_ms += ms_k7;       // the persistent kernel
        h->t_bloom_ms += ms_bloom;  // the Bloom stage on its stream
        h->sig_chunks += 1;
        h->docs_seen += Dn;
        if (!pipelined) {
            b->sig_ms += ms_k7;
            b->bloom_ms += ms_bloom;
            b->measured_chunks += 1;
        }
        return LSHB_OK;
    };

    const size_t n = chunks.size();
    size_t launched = 0;
    for (size_t ci = 0; ci < n; ++ci) {
        // pipelined: chunks up to ci + kSigSlots - 1 are launched; each one's
        // slot was last read by a Bloom stage already finished
        const size_t ahead = pipelined ? std::min(n, ci + kSigSlots) : ci + 1;
        for (; launched < ahead; ++launched)
            if ((st = launch_sig(launched)) != LSHB_OK) return st;
        if ((st = finish(ci)) != LSHB_OK) return st;
        if (pipelined && ci + 1 < n) h->pipelined_chunks += 1;
    }
    // account the staging copies still pending (each buffer's last one)
    if (!tok_dev)
        for (int sb = 0; sb < 2; ++sb)
            if ((st = stage_copy_done(h, sb)) != LSHB_OK) return st;
    return LSHB_OK;
}

// ---- several CSR batches in one launch (the server's signature stage) ---------------

struct SegmentState {
    uint64_t dcap = 0, item_cap = 0;
    int grid = 0;
    DynParams *dyn = nullptr, *dyn_host = nullptr;       // device / pinned
    Segment *segs = nullptr, *segs_host = nullptr;       // device / pinned, kMaxSegments
    unsigned long long *queue = nullptr;                 // device work-queue head
    uint32_t *error = nullptr, *error_host = nullptr;    // device / pinned error word
    DevBuf item_count, item_start, block_sums, item_doc, pending, sig_partial;

    ~SegmentState() {
        item_count.release(); item_start.release(); block_sums.release();
        item_doc.release(); pending.release(); sig_partial.release();
        if (dyn) cudaFree(dyn);
        if (segs) cudaFree(segs);
        if (queue) cudaFree(queue);
        if (error) cudaFree(error);
        if (dyn_host) cudaFreeHost(dyn_host);
        if (segs_host) cudaFreeHost(segs_host);
        if (error_host) cudaFreeHost(error_host);
    }
};

SegmentState *segment_state_create() { return new (std::nothrow) SegmentState(); }
void segment_state_destroy(SegmentState *st) { delete st; }
uint32_t segment_state_error(const SegmentState *st) { return st->error_host ? *st->error_host : 0u; }

lshb_status launch_keys_segments(lshbloom *h, SegmentState *st, const Segment *segs,
                                 uint32_t nseg, uint64_t D, uint64_t T, cudaStream_t s) {
    if (nseg == 0 || nseg > kMaxSegments || D == 0)
        return fail(LSHB_ERR_ARG, "segment launch of %u batches, %llu documents", nseg,
                    (unsigned long long)D);
    if (!st->dyn) {
        BCK(cudaMalloc(&st->dyn, sizeof(DynParams)));
        BCK(cudaMalloc(&st->segs, sizeof(Segment) * kMaxSegments));
        BCK(cudaMalloc(&st->queue, 8));
        BCK(cudaMalloc(&st->error, 4));
        BCK(cudaMemset(st->error, 0, 4));
        BCK(cudaMallocHost(&st->dyn_host, sizeof(DynParams)));
        BCK(cudaMallocHost(&st->segs_host, sizeof(Segment) * kMaxSegments));
        BCK(cudaMallocHost(&st->error_host, 4));
        *st->error_host = 0;
    }
    const uint32_t item = h->cfg.item_shingles ? h->cfg.item_shingles : 512u;
    st->dcap = std::max(st->dcap, D);
    st->item_cap = std::max(st->item_cap, T / kItemCandidates[0] + D + 1);
    lshb_status r;
    if ((r = st->item_count.reserve(st->dcap * 4)) != LSHB_OK) return r;
    if ((r = st->item_start.reserve((st->dcap + 1) * 8)) != LSHB_OK) return r;
    if ((r = st->block_sums.reserve(((st->dcap + kScanBlock - 1) / kScanBlock + 1) * 8)) != LSHB_OK)
        return r;
    if ((r = st->item_doc.reserve(st->item_cap * 4)) != LSHB_OK) return r;
    if ((r = st->pending.reserve(st->dcap * 4)) != LSHB_OK) return r;
    if ((r = st->sig_partial.reserve(st->dcap * h->P * 4)) != LSHB_OK) return r;
    if (!st->grid) st->grid = batched_grid(ngram_template(h->ngram), h->passes[0].ppl);
    // the pinned blocks are free: the previous launch of this state is complete
    memcpy(st->segs_host, segs, sizeof(Segment) * nseg);
    memset(st->dyn_host, 0, sizeof(DynParams));
    st->dyn_host->D = D;
    st->dyn_host->segs = st->segs;
    st->dyn_host->nseg = nseg;
    BatchArgs a;
    memset(&a, 0, sizeof a);
    const SigPass &ps = h->passes[0];
    a.dyn = st->dyn;
    a.item_shingles = item;
    a.ngram = h->ngram;
    a.P = h->P;
    a.npc = ps.npc;
    a.bands = h->bands;
    a.rows = h->rows;
    a.band_key = h->cfg.band_key;
    a.item_count = (uint32_t *)st->item_count.ptr;
    a.item_start = (uint64_t *)st->item_start.ptr;
    a.block_sums = (uint64_t *)st->block_sums.ptr;
    a.item_doc = (uint32_t *)st->item_doc.ptr;
    a.item_cap = st->item_cap;
    a.pending = (uint32_t *)st->pending.ptr;
    a.sig_partial = (uint32_t *)st->sig_partial.ptr;
    a.queue = st->queue;
    a.error = st->error;
    a.c = ps.c;
    BCK(cudaMemcpyAsync(st->segs, st->segs_host, sizeof(Segment) * nseg, cudaMemcpyHostToDevice, s));
    BCK(cudaMemcpyAsync(st->dyn, st->dyn_host, sizeof(DynParams), cudaMemcpyHostToDevice, s));
    BCK(cudaMemsetAsync(st->queue, 0, 8, s));
    BCK(enqueue_items(a, D, s));
    BCK(launch_k_batched(ngram_template(h->ngram), ps.ppl, a, st->grid, s));
    BCK(cudaMemcpyAsync(st->error_host, st->error, 4, cudaMemcpyDeviceToHost, s));
    return LSHB_OK;
}

}  // namespace lshb
