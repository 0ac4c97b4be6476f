/*
 * lshbloom.h -- C ABI of the GB300 LSHBloom deduplication library.
 *
 * LSHBloom (arxiv 2411.04257) decides, for each document of a stream, whether
 * it is a near-duplicate of an earlier one.  A document is a set of word
 * n-grams (Sec. 2.2); its MinHash signature holds, for each of P universal
 * hash permutations, the minimum permuted shingle hash (Sec. 2.2, Sec. 4.1);
 * the signature's first b*r rows form b bands of r rows, each reduced to one
 * integer key by summation (Sec. 4.1); each band key is queried in, and then
 * inserted into, that band's Bloom filter (Sec. 4.1, Sec. 4.2).  A document is
 * a duplicate when any band's key is found (Sec. 4.2).  Documents are judged
 * in stream order against every earlier document (Sec. 2.1, Sec. 4.4.2).
 *
 * Conventions fixed by this library where the paper names none (the CPU
 * reference implements the same conventions independently):
 *   - shingle hash: SHA-1 (FIPS 180-4) of the n tokens as little-endian
 *     uint32 bytes, first four digest bytes as a little-endian uint32
 *     (Sec. 4.1 names SHA1; Sec. 4.3 32-bit hash values);
 *   - a document of 0 < L < n tokens has one shingle of all L tokens; an
 *     empty document has none and keeps the all-(2^32-1) signature;
 *   - permutation i: ((a_i h + b_i) mod (2^61 - 1)) mod 2^32, exact on the
 *     93-bit product; (a_i, b_i) drawn from a SplitMix64 stream of `seed` in
 *     the order a_0, b_0, a_1, ...: a = 1 + x mod (2^61 - 2), b = x mod (2^61 - 1);
 *   - band key j: sum of rows j*r .. j*r+r-1, modulo 2^64 (a weighted sum
 *     when lshb_config.band_key = LSHB_BAND_WEIGHTED, see lshb_band_key);
 *   - probes: x = mix64(key ^ j*0x9e3779b97f4a7c15), y = mix64(x ^
 *     0x6a09e667f3bcc909) | 1, q_u = high64((x + u*y) * m), u < k
 *     (Kirsch-Mitzenmacher double hashing; mix64 is the SplitMix64 finaliser);
 *   - filter size m = ceil(-n ln p / (ln 2)^2) rounded up to a multiple of 256
 *     bits (Sec. 4.5), k = max(1, round(m/n ln 2)) (the blocked layout has
 *     its own rule, see lshbloom_filter_sizing); p_eff splits as
 *     p = 1 - (1 - p_eff)^(1/b) (Sec. 4.3);
 *   - insert rule: by default only documents judged not duplicate are
 *     inserted (Sec. 4.4.2); LSHB_INSERT_ALL inserts every document.
 *
 * Threading: calls on one handle are serialised by the handle.  Different
 * handles are independent.  All functions return an lshb_status; on failure
 * lshbloom_last_error() gives a message for the calling thread.  A call that
 * fails argument or CSR validation changes no state.
 *
 * Memory: pointers marked "host or device" may point to host memory (pageable
 * or pinned) or to device memory of the handle's GPU; the library finds out
 * which with cudaPointerGetAttributes and copies as needed.  Host tokens are
 * not copied where the GPU can read them: page-locked (pinned) buffers through
 * their device mapping, and, on devices that report pageable-memory access
 * through the host's page tables (a GB300 on a Grace host, over NVLink-C2C),
 * pageable buffers too; the kernels then read them in place, so they must
 * stay unchanged until the call returns.  Other host tokens, and all of them
 * when lshb_config.stage_host_inputs is set, are staged through device
 * buffers.  The caller owns all buffers it passes; the handle owns its
 * filters and scratch.
 *
 * Ordering of device buffers: the synchronous calls (lshbloom_dedup,
 * lshbloom_dedup_keys, lshbloom_signatures, lshbloom_band_keys,
 * lshbloom_shingle_hashes) run on the handle's own stream after all work
 * enqueued before the call on the legacy default stream; device inputs
 * written on another stream must be complete before the call (or pass that
 * stream to lshbloom_dedup_async).
 *
 * CSR batches: document d of a batch of D documents is
 * tokens[offsets[d] .. offsets[d+1]-1]; offsets has D+1 non-decreasing
 * entries (offsets[0] need not be 0); tokens holds uint32 word hashes.
 */
#ifndef LSHBLOOM_H
#define LSHBLOOM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LSHB_API __attribute__((visibility("default")))
#else
#define LSHB_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lshbloom lshbloom_t;

typedef enum {
    LSHB_OK = 0,
    LSHB_ERR_ARG = -1,     /* bad argument or parameter combination */
    LSHB_ERR_CSR = -2,     /* offsets not non-decreasing */
    LSHB_ERR_OOM = -3,     /* device or host allocation failed */
    LSHB_ERR_CUDA = -4,    /* a CUDA call failed */
    LSHB_ERR_TIMEOUT = -5, /* a bounded device wait ran out */
    LSHB_ERR_IO = -6,      /* file read/write failed or bad file */
    LSHB_ERR_BUSY = -7     /* no admission slot / memory (serving) */
} lshb_status;

typedef enum { LSHB_INSERT_NONDUP = 0, LSHB_INSERT_ALL = 1 } lshb_insert_mode;

/* Filter layout.  STANDARD is the paper's filter (Sec. 2.4): k positions over
 * all m bits.  BLOCKED is a variant beyond the paper (after Putze, Sanders and
 * Singler 2007): all k positions of a key inside one 256-bit block, each an
 * independent byte of a SplitMix64 word of y (y as for the standard layout),
 * block = high64(x * m/256); one 32-byte sector per probed key instead of k,
 * at a higher false-positive rate for the same m and k.  A BLOCKED index is
 * therefore sized by its own rule (lshbloom_filter_sizing): the fewest
 * 256-bit blocks, over k, whose modelled rate meets the per-filter p. */
/* EXACT_KEYS replaces the filters by exact sets of band keys (one
 * open-addressing table of uint64 per band, 2^ceil(log2(2 n_expected)) slots,
 * empty = 2^64-1): the bucket rule of MinHashLSH (Sec. 2.3) on the same band
 * keys, i.e. the index without Bloom false positives (Eq. 3 with p_eff = 0),
 * at several times the memory.  It is the same-device baseline for what the
 * filters save; filter_bytes then returns the band's table. */
typedef enum {
    LSHB_BLOOM_STANDARD = 0,
    LSHB_BLOOM_BLOCKED = 1,
    LSHB_EXACT_KEYS = 2
} lshb_bloom_layout;

/* Band key of b bands of r signature rows x_0 .. x_{r-1} (band j).  SUM is
 * the paper's reduction, (sum_t x_t) mod 2^64 (Sec. 4.1, the Carter-Wegman
 * form with the signature values as the per-row hashes).  WEIGHTED is a
 * variant beyond the paper: (sum_t c_{j,t} x_t) mod 2^64 with fixed odd
 * weights c_{j,t} = SplitMix64-finaliser(0x9e3779b97f4a7c15 * ((j << 10) + t
 * + 1)) | 1.  Minima of many shingles cluster near 0, so plain sums of
 * unrelated documents collide far more often than 2^-32; the weights restore
 * a bound of about 2^-32 for distinct bands. */
typedef enum { LSHB_BAND_SUM = 0, LSHB_BAND_WEIGHTED = 1 } lshb_band_key;

typedef enum {
    LSHB_EXEC_PLAIN = 0,   /* one kernel per stage */
    LSHB_EXEC_BATCHED = 1  /* persistent fused kernel over a work queue, graph-launched */
} lshb_exec_mode;

typedef struct {
    uint32_t num_perm;        /* P, >= 1, <= 1024 */
    uint32_t bands;           /* b, >= 1, <= 64 */
    uint32_t rows;            /* r, >= 1, b*r <= P */
    uint32_t ngram;           /* n, word n-gram size, 1..64 (default 5) */
    uint64_t n_expected;      /* documents the filters are sized for, >= 1 */
    double fp_rate;           /* per-filter p in (0,1), or p_eff if fp_is_effective */
    int32_t fp_is_effective;  /* nonzero: fp_rate is p_eff over all b filters */
    uint32_t insert_mode;     /* lshb_insert_mode */
    uint64_t seed;            /* permutation coefficient seed (default 1) */
    const uint64_t *perm_a;   /* optional host array[P] of a_i in [1, 2^61-2] */
    const uint64_t *perm_b;   /* optional host array[P] of b_i in [0, 2^61-2] */
    uint32_t exec_mode;       /* lshb_exec_mode (default BATCHED) */
    int32_t device;           /* CUDA device ordinal, -1 = current */
    uint64_t max_batch_docs;  /* docs per internal chunk, 0 = default: 262144 in the
                                 plain form; in the batched form autotuned over calls
                                 of at least 2^22 documents (the first four such
                                 calls try 2^18, 2^19, 2^20 and 2^21 documents per
                                 chunk, later ones keep the fastest per document),
                                 2^20 until then */
    uint64_t max_batch_tokens;/* tokens per internal chunk, 0 = default (2^28 in the plain
                                 form; 2^31 in the batched form, where host inputs
                                 are staged through two device buffers of that size,
                                 the first chunk of a call ramped up from 2^28) */
    uint32_t item_shingles;   /* batched mode: shingles per work item, 0 = autotuned */
    uint32_t bloom_layout;    /* lshb_bloom_layout (default STANDARD) */
    uint32_t stage_host_inputs; /* nonzero: always copy host tokens to the device through
                                   staging buffers instead of letting the kernels read them
                                   in place (see "Memory" above) */
    uint32_t band_key;        /* lshb_band_key (default SUM, the paper's) */
    uint32_t reserved[4];
} lshb_config;

typedef struct {
    uint32_t num_perm, bands, rows, ngram, k, insert_mode, exec_mode, item_shingles;
    uint64_t m_bits;          /* bits per filter */
    uint64_t filter_bytes;    /* bytes per filter as stored (m_bits / 8) */
    uint64_t docs_seen;       /* documents judged so far */
    uint64_t dups_seen;       /* of which duplicates */
    double fp_rate;           /* per-filter p actually used */
    double fill[64];          /* fraction of set bits per filter (first `bands`) */
    uint64_t resolve_rounds;  /* in-batch order-resolution iterations so far */
    uint64_t uncertain_docs;  /* documents that needed in-batch resolution */
    uint64_t kernel_launches; /* kernels this library has launched in this process */
    double sig_ms;            /* device time in the signature stage (CUDA events; the
                                 persistent kernel alone in the batched form) */
    double bloom_ms;          /* device time in the Bloom stage (CUDA events; in the
                                 batched form from the chunk's signatures to its flags,
                                 overlapping the next chunk's signatures when pipelined) */
    uint64_t sig_chunks;      /* signature-stage launches timed in sig_ms */
    double probe_ms;          /* device time of the Bloom probe kernel (both forms) */
    uint64_t probe_sectors;   /* 32-byte sectors that kernel's probes address (k per band key,
                                 one per band key in the blocked and exact layouts) */
    double h2d_ms;            /* copy-stream time of the token copies of host inputs (CUDA events) */
    uint64_t h2d_bytes;       /* bytes those copies moved */
    double call_ms;           /* host wall-clock time spent inside dedup calls */
    uint64_t host_read_bytes; /* host token bytes the kernels read in place (no copy) */
    uint64_t chunk_docs;      /* batched form: documents per internal chunk now in use
                                 (max_batch_docs, or the autotuner's current choice) */
    uint64_t pipelined_chunks; /* batched form: chunks whose Bloom stage ran while the next
                                 chunk's signatures were being computed */
} lshb_stats;

/* Fill *cfg with defaults: P=121, b=11, r=11, n=5, n_expected=10000,
 * fp_rate=1e-5 (per filter), seed=1, INSERT_NONDUP, BATCHED, device -1. */
LSHB_API void lshbloom_config_default(lshb_config *cfg);

/* Create an index of b Bloom filters sized for n_expected documents at
 * per-filter false-positive rate fp_rate (Sec. 4.5 sizing; Sec. 4.1: one
 * filter per band).  Other settings take lshbloom_config_default values.
 * *out receives the handle.  Errors: ERR_ARG (b*r > P, fp not in (0,1),
 * n_expected = 0, out NULL), ERR_OOM, ERR_CUDA. */
LSHB_API lshb_status lshbloom_create(uint32_t P, uint32_t b, uint32_t r, uint64_t n_expected,
                            double fp_rate, lshbloom_t **out);

/* Create from a full configuration (see lshb_config).  Errors as above. */
LSHB_API lshb_status lshbloom_create_ex(const lshb_config *cfg, lshbloom_t **out);

/* Create the index the way the paper parameterises it: a Jaccard threshold T
 * in (0, 1) and P permutations give (b, r) by lshbloom_optimal_br (Eqs. 1-2,
 * Sec. 4.3); an effective false-positive rate p_eff over all b filters gives
 * the per-filter rate p = 1 - (1 - p_eff)^(1/b) (Sec. 4.3) and the sizing of
 * Sec. 4.5.  Other settings take lshbloom_config_default values. */
LSHB_API lshb_status lshbloom_create_threshold(double T, uint32_t P, uint64_t n_expected,
                                               double p_eff, lshbloom_t **out);

/* Judge D documents in stream order against all earlier documents of this
 * handle (Sec. 2.1, Sec. 4.2) and insert them (Sec. 4.1, Sec. 4.4.2).
 * offsets: host or device uint64[D+1]; tokens: host or device uint32, indexed
 * by offsets; flags_out: host or device uint8[D], 1 = duplicate.  Returns
 * when flags_out is written.  D = 0 is a no-op.  Errors: ERR_ARG (NULL
 * pointer with D > 0), ERR_CSR (offsets decreasing; no state changed),
 * ERR_OOM, ERR_CUDA, ERR_TIMEOUT. */
LSHB_API lshb_status lshbloom_dedup(lshbloom_t *h, const uint64_t *offsets, const uint32_t *tokens,
                           uint64_t D, uint8_t *flags_out);

/* As lshbloom_dedup with device pointers only, ordered on `stream` (a
 * cudaStream_t; NULL = the legacy default stream).  The host may block while
 * it plans chunks and when a batch needs in-batch order resolution; flags_out
 * is complete when the stream reaches the end of the enqueued work.  The
 * batched form may compute the signatures of later chunks on a private
 * stream of the handle, started after the work enqueued on `stream` before
 * the call; each chunk's Bloom stage runs on `stream` after them. */
LSHB_API lshb_status lshbloom_dedup_async(lshbloom_t *h, const uint64_t *offsets, const uint32_t *tokens,
                                 uint64_t D, uint8_t *flags_out, void *stream);

/* As lshbloom_dedup, and also write the band keys (Sec. 4.1) the judgement
 * used: keys_out is host or device uint64[D][b], row-major. */
LSHB_API lshb_status lshbloom_dedup_keys(lshbloom_t *h, const uint64_t *offsets,
                                         const uint32_t *tokens, uint64_t D, uint8_t *flags_out,
                                         uint64_t *keys_out);

/* The Bloom-index half of lshbloom_dedup (Sec. 4.1, Sec. 4.2, Sec. 4.4.2) on
 * band keys computed elsewhere: documents 0 .. D-1 with band keys
 * keys[d*b .. d*b + b-1] (host or device uint64[D][b], row-major; any 64-bit
 * values) are judged in order against all earlier documents of this handle
 * and inserted by the insert rule, exactly as lshbloom_dedup judges the keys
 * it computes.  flags_out: host or device uint8[D], 1 = duplicate.  D = 0 is
 * a no-op.  Errors: ERR_ARG (NULL pointer with D > 0), ERR_OOM, ERR_CUDA. */
LSHB_API lshb_status lshbloom_dedup_from_keys(lshbloom_t *h, const uint64_t *keys, uint64_t D,
                                              uint8_t *flags_out);

/* MinHash signatures of D documents (Sec. 2.2, Sec. 4.1), without touching the
 * filters.  sig_out: host or device uint32[D][P], row-major.  Errors as for
 * lshbloom_dedup. */
LSHB_API lshb_status lshbloom_signatures(lshbloom_t *h, const uint64_t *offsets, const uint32_t *tokens,
                                uint64_t D, uint32_t *sig_out);

/* Band keys of D documents (Sec. 4.1), without touching the filters.
 * keys_out: host or device uint64[D][b], row-major. */
LSHB_API lshb_status lshbloom_band_keys(lshbloom_t *h, const uint64_t *offsets, const uint32_t *tokens,
                               uint64_t D, uint64_t *keys_out);

/* Band keys like lshbloom_band_keys, for callers that cannot let the library
 * allocate device memory (applications whose GPU memory all belongs to their
 * own fixed-budget pool, or latency-critical loops where cudaMalloc's
 * device-wide synchronisation would stall other streams).  The paper has no
 * counterpart: this is a deployment variant of the same computation.
 * With P <= 256 (one signature pass) the signature kernel writes the keys
 * directly and no intermediate matrix exists.  With P > 256 the signature
 * matrix lives in a 16 MiB array compiled into the library, which every GPU
 * that loads the library holds until the process exits; D * P * 4 bytes must
 * fit in it (D <= 8192 at P = 512, D <= 4096 at P = 1024), and
 * larger batches get LSHB_ERR_ARG with the limit in the message.
 * offsets, tokens, keys_out: device pointers (as lshbloom_band_keys;
 * keys_out is uint64[D][b]); work is ordered on `stream` (a cudaStream_t,
 * NULL = legacy default stream) and the call waits for it once, after
 * checking that the offsets do not decrease (LSHB_ERR_CSR otherwise).
 * The first call on each device looks up the array's device address; make
 * that first call before any stream capture.  All calls share the one array
 * (each call rewrites every row it reads, nothing needs clearing): calls
 * that overlap on the GPU, from two threads or two streams, race.
 * A successful call allocates no memory; a failed one records its message
 * for lshbloom_last_error. */
LSHB_API lshb_status lshbloom_band_keys_static(lshbloom_t *h, const uint64_t *offsets,
                                               const uint32_t *tokens, uint64_t D,
                                               uint64_t *keys_out, void *stream);

/* Shingle hashes (Sec. 4.1 base hash) of D documents: for document d,
 * h_out[offsets[d] - offsets[0] + s] is the hash of shingle s for
 * s < shingles(d); the other n-1 entries of each document are 0.
 * h_out: host or device uint32[offsets[D] - offsets[0]]. */
LSHB_API lshb_status lshbloom_shingle_hashes(lshbloom_t *h, const uint64_t *offsets,
                                    const uint32_t *tokens, uint64_t D, uint32_t *h_out);

/* Copy the permutation coefficients (host uint64[P] each). */
LSHB_API lshb_status lshbloom_coefficients(const lshbloom_t *h, uint64_t *a_out, uint64_t *b_out);

/* Copy filter `band` to host memory: ceil(m/8) bytes, bit q of the filter at
 * byte q/8, bit q%8 (least significant first).  EXACT_KEYS: the band's table
 * as uint64 slots (stats filter_bytes bytes): cap key slots (cap a power of
 * two, 2^64-1 = empty), then one slot that is 0 when the key 2^64-1 is in the
 * set (2^64-1 otherwise), then 15 empty padding slots. */
LSHB_API lshb_status lshbloom_filter_bytes(lshbloom_t *h, uint32_t band, uint8_t *host_out);

/* Clear every filter and the document counters. */
LSHB_API lshb_status lshbloom_reset(lshbloom_t *h);

/* Sizes, counters and per-filter fill. */
LSHB_API lshb_status lshbloom_stats(lshbloom_t *h, lshb_stats *out);

/* Write the index (a header with every parameter and counter, then the b
 * filters) to `path`; load it back into a new handle on the current (or
 * `device` >= 0) GPU.  A loaded index continues the stream exactly. */
LSHB_API lshb_status lshbloom_save(lshbloom_t *h, const char *path);
LSHB_API lshb_status lshbloom_load(const char *path, int32_t device, lshbloom_t **out);

/* (b, r) with b*r <= P minimising the equal-weight sum of the LSH false
 * positive and false negative integrals at threshold T (Eqs. 1-2, Sec. 4.3). */
LSHB_API lshb_status lshbloom_optimal_br(double T, uint32_t P, uint32_t *b_out, uint32_t *r_out);

/* Bits m and probe count k of one filter for n_expected keys at per-filter
 * false-positive rate fp_rate, as lshbloom_create_ex sizes them.  STANDARD
 * (and EXACT_KEYS' nominal figure): m = -n ln p / (ln 2)^2 (Sec. 4.5),
 * rounded up to whole bits and a multiple of 256, k = max(1, round(m/n ln 2)).
 * BLOCKED (beyond the paper): the smallest m, in 256-bit blocks, and its k
 * (1 .. min(64, standard k + 8)) whose rate under the blocked model is at
 * most p; the model takes Poisson(256 n / m) keys per block and, given i
 * keys, the chance E[(Z/256)^k] that a query's k uniform positions all land
 * on the Z bits that i*k uniform positions set.  Host only: no GPU needed.
 * m_bits, k: caller-owned outputs.  LSHB_ERR_ARG for n_expected < 1, p
 * outside (0, 1), an unknown layout or a NULL output. */
LSHB_API lshb_status lshbloom_filter_sizing(uint64_t n_expected, double fp_rate, uint32_t layout,
                                            uint64_t *m_bits, uint32_t *k);

/* ---- Serving: continuous batching over resident indexes ----------------------
 *
 * A server owns a device-memory budget and a worker thread.  Requests (CSR
 * batches for one of its indexes) are admitted in arrival order as soon as an
 * in-flight slot and enough of the budget are free.  Each index has a stream
 * for signatures: whenever its previous launch is done, all its admitted
 * requests not yet started go into one launch of the persistent signature
 * kernel (one work queue over their documents, long documents split), so
 * requests that arrive while others are on the GPU join the next launch, and
 * the indexes' launches overlap.  The Bloom stage of each index runs in
 * arrival order, over the run of its oldest requests whose keys are ready,
 * as one batch, so every request is judged against exactly the documents
 * submitted before it to the same index (Sec. 2.1): its flags equal those of
 * lshbloom_dedup calls made one after the other in submission order.  The
 * filters stay resident across requests. */
typedef struct lshbloom_server lshbloom_server_t;

/* indexes: n handles (same device; P <= 256) that the server uses exclusively
 * until destroyed.  mem_budget_bytes: device memory for in-flight requests
 * (the keys of each, and the offsets and tokens the GPU cannot read in place),
 * allocated once here; each index's signature launches also keep scratch of
 * their own (work-item lists and merged signature rows of split documents,
 * grown to the largest launch, at most 2^18 documents).  max_inflight: at most
 * this many admitted requests (1..256).  Errors: ERR_ARG, ERR_OOM, ERR_CUDA. */
LSHB_API lshb_status lshbloom_server_create(lshbloom_t *const *indexes, uint32_t n,
                                            uint64_t mem_budget_bytes, uint32_t max_inflight,
                                            lshbloom_server_t **out);

/* Queue D documents (host offsets[D+1], host tokens) for index `index`; the
 * flags land in host flags_out[D].  The three buffers must stay valid until
 * the request completes.  Offsets and tokens the GPU can read in place (see
 * "Memory" above; none when an index of the server sets stage_host_inputs)
 * are read by the kernels directly and take no budget; others are copied
 * into the budget.  *ticket identifies the request.  ERR_BUSY when the
 * request alone needs more than the memory budget; ERR_CSR for decreasing
 * offsets. */
LSHB_API lshb_status lshbloom_server_submit(lshbloom_server_t *s, uint32_t index,
                                            const uint64_t *offsets, const uint32_t *tokens,
                                            uint64_t D, uint8_t *flags_out, uint64_t *ticket);

/* Wait up to timeout_ms (< 0: forever) for a request.  Returns LSHB_OK when
 * it completed (its own status otherwise), ERR_TIMEOUT when still running.
 * latency_us (optional) receives submit-to-completion time in microseconds.
 * A completed ticket can be waited on once. */
LSHB_API lshb_status lshbloom_server_wait(lshbloom_server_t *s, uint64_t ticket, double timeout_ms,
                                          double *latency_us);

/* Finish every queued request, stop the worker, release the budget.  The
 * indexes stay valid (and hold every request's insertions). NULL is a no-op. */
LSHB_API void lshbloom_server_destroy(lshbloom_server_t *s);

/* Message of the last failed call on this thread ("" if none). */
LSHB_API const char *lshbloom_last_error(void);

/* Release the handle and everything it owns.  NULL is a no-op. */
LSHB_API void lshbloom_destroy(lshbloom_t *h);

#ifdef __cplusplus
}
#endif

#endif /* LSHBLOOM_H */
