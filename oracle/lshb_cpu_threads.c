/*
 * Multi-threaded driver over the LSHBloom CPU oracle -- TEST AND BASELINE
 * INFRASTRUCTURE ONLY.
 *
 * The paper's own system parallelises MinHash over worker processes and
 * keeps the index writes sequential, so that each document is checked
 * against the documents before it when it is inserted (Sec. 4.4.2).  This
 * file does the same with threads over the unchanged single-threaded oracle
 * functions of lshb_oracle.c:
 *   - band keys (shingling, SHA-1, MinHash, band sums: Sec. 2.2, Sec. 4.1)
 *     depend on one document only; worker threads take blocks of documents
 *     from a shared counter and call or_batch_band_keys on them;
 *   - the stream decision (Sec. 2.1, Sec. 4.2) runs on one thread, in
 *     document order, through or_index_dedup_keys.
 * The result is bit-identical to or_index_dedup on the same documents (a CPU
 * test checks it).  It serves two purposes: the parity tests verify every
 * document's band keys at the workloads' full sizes in reasonable time, and
 * the benchmark reports it as the multi-core CPU baseline.  Nothing in the
 * GPU product path loads it.
 */
#include <pthread.h>
#include <stdatomic.h>
#include <stdint.h>
#include <stdlib.h>

#define ORT_API __attribute__((visibility("default")))

/* Defined in lshb_oracle.c (same shared library). */
void or_batch_band_keys(const uint64_t *offsets, const uint32_t *tokens, uint64_t D, uint32_t n,
                        uint32_t P, const uint64_t *a, const uint64_t *b, uint32_t bands,
                        uint32_t rows, uint32_t mode, uint64_t *keys_out);
void or_index_dedup_keys(void *ix, const uint64_t *keys, uint64_t D, uint8_t *flags);

typedef struct {
    const uint64_t *off;
    const uint32_t *tok;
    uint64_t D, grain;
    uint32_t n, P, bands, rows, mode;
    const uint64_t *a, *b;
    uint64_t *keys;
    _Atomic uint64_t next;
} ort_job;

static void *ort_worker(void *arg) {
    ort_job *J = (ort_job *)arg;
    for (;;) {
        const uint64_t lo = atomic_fetch_add(&J->next, J->grain);
        if (lo >= J->D) break;
        const uint64_t hi = lo + J->grain < J->D ? lo + J->grain : J->D;
        or_batch_band_keys(J->off + lo, J->tok, hi - lo, J->n, J->P, J->a, J->b, J->bands,
                           J->rows, J->mode, J->keys + lo * J->bands);
    }
    return NULL;
}

/* Band keys of D documents (keys_out: D x bands) on up to `threads` threads,
 * the calling thread included.  Returns the number of threads that ran. */
ORT_API uint32_t ort_batch_band_keys(const uint64_t *offsets, const uint32_t *tokens, uint64_t D,
                                     uint32_t n, uint32_t P, const uint64_t *a, const uint64_t *b,
                                     uint32_t bands, uint32_t rows, uint32_t mode,
                                     uint64_t *keys_out, uint32_t threads) {
    ort_job J;
    J.off = offsets; J.tok = tokens; J.D = D; J.grain = 16;
    J.n = n; J.P = P; J.bands = bands; J.rows = rows; J.mode = mode;
    J.a = a; J.b = b; J.keys = keys_out;
    atomic_init(&J.next, 0);
    if (threads < 1) threads = 1;
    pthread_t *tid = (pthread_t *)malloc(sizeof(pthread_t) * threads);
    uint32_t started = 0;
    for (uint32_t t = 1; t < threads; ++t)
        if (pthread_create(&tid[started], NULL, ort_worker, &J) == 0) started++;
    ort_worker(&J);
    for (uint32_t t = 0; t < started; ++t) pthread_join(tid[t], NULL);
    free(tid);
    return started + 1;
}

/* The paper's CPU design on the oracle: blocks of `block_docs` documents;
 * each block's band keys in parallel, then its stream decisions in order.
 * `ix` is an or_index of lshb_oracle.c created with the same P, bands, rows,
 * n-gram size, coefficients and band-key mode.  Returns the threads used. */
ORT_API uint32_t ort_index_dedup(void *ix, const uint64_t *offsets, const uint32_t *tokens,
                                 uint64_t D, uint8_t *flags, uint32_t n, uint32_t P,
                                 const uint64_t *a, const uint64_t *b, uint32_t bands,
                                 uint32_t rows, uint32_t mode, uint32_t threads,
                                 uint64_t block_docs) {
    if (block_docs == 0) block_docs = 65536;
    const uint64_t cap = block_docs < D ? block_docs : D;
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (cap ? cap : 1) * bands);
    uint32_t used = 1;
    for (uint64_t lo = 0; lo < D; lo += block_docs) {
        const uint64_t hi = lo + block_docs < D ? lo + block_docs : D;
        used = ort_batch_band_keys(offsets + lo, tokens, hi - lo, n, P, a, b, bands, rows, mode,
                                   keys, threads);
        or_index_dedup_keys(ix, keys, hi - lo, flags + lo);
    }
    free(keys);
    return used;
}
