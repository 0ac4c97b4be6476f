// Serving: a request server with continuous batching over resident indexes.
//
// Requests wait in one FIFO.  A worker thread admits the head of the FIFO as
// soon as an in-flight slot and enough of the device-memory budget are free.
// Each index has a signature stream: whenever its previous launch is done,
// every admitted request of that index not yet started goes into one launch
// of the persistent kernel (one work queue of (document, shingle range) items
// over all of them, long documents split), after the copy-in of whatever the
// GPU cannot read in place; the indexes' launches run at the same time, and
// requests that arrive while a launch computes join the next one.  The Bloom
// stage of an index then runs, in arrival order, over the longest run of that
// index's oldest requests whose signatures are done: their band keys are laid
// end to end and judged as one batch, which is the same as judging the
// requests one after the other (Sec. 2.1, Sec. 4.4.2), so each request is
// judged against exactly the requests submitted before it to the same index,
// while the Bloom stage's fixed costs (a few kernel launches and host round
// trips) are paid once per group instead of once per request.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "runtime_internal.h"
#include "segment.h"

using namespace lshb;

namespace {

using Clock = std::chrono::steady_clock;

enum class RState { Pending, Running, Done };

struct Request {
    uint64_t ticket = 0;
    uint32_t index = 0;
    uint64_t D = 0, T = 0, tok0 = 0;
    const uint64_t *h_off = nullptr;
    const uint32_t *h_tok = nullptr;
    const uint64_t *in_off = nullptr;  // offsets / tokens the kernels read in place (or nullptr:
    const uint32_t *in_tok = nullptr;  // copied into the budget)
    uint8_t *h_flags = nullptr;
    uint64_t bytes = 0, pool_off = 0;
    uint64_t *d_off = nullptr;
    uint32_t *d_tok = nullptr;
    uint64_t *d_keys = nullptr;
    int slot = -1;
    bool keyed = false;  // the signature stage is over (band keys in d_keys, or a failure)
    RState state = RState::Pending;
    lshb_status status = LSHB_OK;
    Clock::time_point t_submit, t_done;
};

// First-fit allocator over the budget (offsets, 256-byte granules).
struct Pool {
    uint8_t *base = nullptr;
    uint64_t size = 0;
    std::map<uint64_t, uint64_t> free_;  // offset -> length

    void init(uint8_t *b, uint64_t n) {
        base = b;
        size = n;
        free_.clear();
        free_[0] = n;
    }
    bool alloc(uint64_t n, uint64_t *off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                *off = it->first;
                const uint64_t rest = it->second - n;
                const uint64_t at = it->first + n;
                free_.erase(it);
                if (rest) free_[at] = rest;
                return true;
            }
        }
        return false;
    }
    void release(uint64_t off, uint64_t n) {
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

uint64_t align256(uint64_t x) { return (x + 255) & ~255ull; }

}  // namespace

struct lshbloom_server {
    std::vector<lshbloom *> idx;
    int device = 0;
    uint32_t bands = 0;
    bool pageable_access = false;  // the device reads pageable host memory in place
    bool stage_inputs = false;     // an index asked for staged host inputs
    Pool pool;
    void *pool_mem = nullptr;
    std::vector<int> free_slots;
    std::deque<Request *> fifo;
    std::vector<std::deque<Request *>> running;  // per index, arrival order
    // per index: the signature stream, its launch state, the admitted
    // requests not yet launched and those of the launch in flight
    std::vector<cudaStream_t> sig_stream;
    std::vector<cudaEvent_t> sig_event;
    std::vector<SegmentState *> seg;
    std::vector<std::deque<Request *>> sig_wait;
    std::vector<std::vector<Request *>> sig_flight;
    std::unordered_map<uint64_t, Request *> reqs;
    std::mutex mu;
    // cv_work: submissions and freed memory (the signature thread);
    // cv_bloom: requests whose signature stage ended (the Bloom threads);
    // cv_done: finished requests (callers of lshbloom_server_wait)
    std::condition_variable cv_work, cv_bloom, cv_done;
    std::thread worker;                    // admission and signature launches
    std::vector<std::thread> bloom_workers;  // one per index: its Bloom stages
    bool stop = false;
    uint64_t next_ticket = 1;

    void loop();
    void bloom_loop(uint32_t i);
    std::vector<Request *> launch(uint32_t i);
    lshb_status bloom(const std::vector<Request *> &group);
};

// Documents and batches of one signature launch at most.
constexpr uint64_t kMaxLaunchDocs = 1ull << 18;

// Documents of one grouped Bloom stage at most (a group always takes at least
// its first request).
constexpr uint64_t kMaxGroupDocs = 1ull << 20;

// Budget of a request: its keys, and the offsets and tokens that are copied
// rather than read in place.
static uint64_t request_bytes(uint64_t D, uint64_t T, uint32_t bands, bool copy_off, bool copy_tok) {
    return (copy_off ? align256((D + 1) * 8) : 0) + (copy_tok ? align256(T * 4) : 0) +
           align256(D * bands * 8);
}

// One signature launch for index i: the oldest admitted requests not yet
// started, up to kMaxLaunchDocs documents and kMaxSegments requests (the
// signature thread only; index i has no launch in flight).  Returns the
// requests that failed before or at the launch, their status set, for the
// caller to hand on under the lock.
std::vector<Request *> lshbloom_server::launch(uint32_t i) {
    std::vector<Request *> failed;
    lshbloom *h = idx[i];
    cudaStream_t s = sig_stream[i];
    std::vector<Segment> segs;
    std::vector<Request *> batch;
    uint64_t D = 0, T = 0;
    while (!sig_wait[i].empty() && segs.size() < kMaxSegments) {
        Request *r = sig_wait[i].front();
        if (!batch.empty() && D + r->D > kMaxLaunchDocs) break;
        sig_wait[i].pop_front();
        uint8_t *p = pool.base + r->pool_off;
        cudaError_t e = cudaSuccess;
        if (!r->in_off) {
            r->d_off = (uint64_t *)p;
            p += align256((r->D + 1) * 8);
            e = cudaMemcpyAsync(r->d_off, r->h_off, (r->D + 1) * 8, cudaMemcpyHostToDevice, s);
        }
        if (e == cudaSuccess && !r->in_tok) {
            r->d_tok = (uint32_t *)p;
            p += align256(r->T * 4);
            if (r->T)
                e = cudaMemcpyAsync(r->d_tok, r->h_tok + r->tok0, r->T * 4, cudaMemcpyHostToDevice, s);
        }
        r->d_keys = (uint64_t *)p;
        if (e != cudaSuccess) {
            r->status = cuda_fail(e, "request copy-in");
            failed.push_back(r);
            continue;
        }
        Segment sg;
        sg.offsets = r->in_off ? r->in_off : r->d_off;
        sg.tokens = r->in_tok ? r->in_tok : r->d_tok;
        sg.tok_base = r->in_tok ? 0 : r->tok0;
        sg.doc0 = D;
        sg.keys_out = r->d_keys;
        segs.push_back(sg);
        batch.push_back(r);
        D += r->D;
        T += r->T;
    }
    if (batch.empty()) return failed;
    lshb_status st = launch_keys_segments(h, seg[i], segs.data(), (uint32_t)segs.size(), D, T, s);
    cudaError_t e = cudaSuccess;
    if (st == LSHB_OK && (e = cudaEventRecord(sig_event[i], s)) != cudaSuccess)
        st = cuda_fail(e, "event");
    if (st != LSHB_OK) {
        cudaStreamSynchronize(s);
        for (Request *r : batch) r->status = st;
        failed.insert(failed.end(), batch.begin(), batch.end());
        return failed;
    }
    sig_flight[i] = batch;
    return failed;
}

// Bloom stage of a group of requests of one index, in arrival order, as one
// batch (the worker thread only).
lshb_status lshbloom_server::bloom(const std::vector<Request *> &group) {
    lshbloom *h = idx[group.front()->index];
    std::lock_guard<std::mutex> lock(h->mu);
    uint64_t D = 0;
    for (Request *r : group) D += r->D;
    lshb_status st = ensure_chunk_scratch(h, D, 0, false, false);
    if (st != LSHB_OK) return st;
    cudaError_t e;
    uint64_t *keys = (uint64_t *)h->buf(B_KEYS).ptr;
    uint64_t at = 0;
    for (Request *r : group) {
        if ((e = cudaMemcpyAsync(keys + at * h->bands, r->d_keys, r->D * h->bands * 8,
                                 cudaMemcpyDeviceToDevice, h->stream)) != cudaSuccess)
            return cuda_fail(e, "keys");
        at += r->D;
    }
    uint8_t *flags = (uint8_t *)h->buf(B_FLAGS).ptr;
    if ((st = run_bloom(h, D, flags, h->stream)) != LSHB_OK) return st;
    at = 0;
    for (Request *r : group) {
        if ((e = cudaMemcpyAsync(r->h_flags, flags + at, r->D, cudaMemcpyDeviceToHost, h->stream)) !=
            cudaSuccess)
            return cuda_fail(e, "flags");
        at += r->D;
    }
    if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return cuda_fail(e, "sync");
    h->docs_seen += D;
    return LSHB_OK;
}

// The signature thread: admission, signature launches, their completion.
void lshbloom_server::loop() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        // admission: FIFO head while a slot and enough memory are free
        bool moved = false;
        while (!fifo.empty() && !free_slots.empty()) {
            Request *r = fifo.front();
            uint64_t off = 0;
            if (!pool.alloc(r->bytes, &off)) break;
            r->pool_off = off;
            r->slot = free_slots.back();
            free_slots.pop_back();
            r->state = RState::Running;
            fifo.pop_front();
            running[r->index].push_back(r);
            sig_wait[r->index].push_back(r);
            moved = true;
        }
        bool any_running = false;
        for (auto &q : running) any_running |= !q.empty();
        if (stop && fifo.empty() && !any_running) break;
        lk.unlock();
        // a finished launch hands its requests to the Bloom threads; an idle
        // index starts its waiting requests
        std::vector<Request *> ended;
        std::vector<lshb_status> ended_status;
        for (uint32_t i = 0; i < idx.size(); ++i) {
            if (!sig_flight[i].empty()) {
                const cudaError_t q = cudaEventQuery(sig_event[i]);
                if (q == cudaErrorNotReady) continue;
                lshb_status st = LSHB_OK;
                if (q != cudaSuccess) st = cuda_fail(q, "signature stage");
                else if (segment_state_error(seg[i]) != 0)
                    st = fail(LSHB_ERR_CUDA, "signature stage: device error word 0x%x",
                              segment_state_error(seg[i]));
                for (Request *r : sig_flight[i]) {
                    ended.push_back(r);
                    ended_status.push_back(st);
                }
                sig_flight[i].clear();
                moved = true;
            }
            if (!sig_wait[i].empty()) {
                for (Request *r : launch(i)) {
                    ended.push_back(r);
                    ended_status.push_back(r->status);
                }
                moved = true;
            }
        }
        lk.lock();
        for (size_t k = 0; k < ended.size(); ++k) {
            if (ended_status[k] != LSHB_OK) ended[k]->status = ended_status[k];
            ended[k]->keyed = true;
        }
        if (!ended.empty()) cv_bloom.notify_all();
        if (!moved) {
            // nothing moved: wait for a submission or freed memory, or poll
            // the GPU again soon
            cv_work.wait_for(lk, std::chrono::microseconds(50));
        }
    }
}

// The Bloom thread of index i: the oldest requests of the index whose
// signature stage has ended, as one group, in arrival order.
void lshbloom_server::bloom_loop(uint32_t i) {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        cv_bloom.wait(lk, [&] {
            return (!running[i].empty() && running[i].front()->keyed) ||
                   (stop && fifo.empty() && running[i].empty());
        });
        if (running[i].empty()) break;  // stopping, nothing left for this index
        std::vector<Request *> group;
        uint64_t docs = 0;
        for (Request *r : running[i]) {
            if (!r->keyed) break;
            if (r->status != LSHB_OK) {
                if (group.empty()) group.push_back(r);  // a failed request finishes alone
                break;
            }
            if (!group.empty() && docs + r->D > kMaxGroupDocs) break;
            group.push_back(r);
            docs += r->D;
        }
        lk.unlock();
        if (group.front()->status == LSHB_OK) {
            const lshb_status st = bloom(group);
            for (Request *r : group) r->status = st;
        }
        lk.lock();
        for (size_t k = 0; k < group.size(); ++k) running[i].pop_front();
        for (Request *r : group) {
            r->t_done = Clock::now();
            r->state = RState::Done;
            pool.release(r->pool_off, r->bytes);
            free_slots.push_back(r->slot);
        }
        cv_done.notify_all();
        cv_work.notify_one();
    }
}

extern "C" lshb_status lshbloom_server_create(lshbloom_t *const *indexes, uint32_t n,
                                              uint64_t mem_budget_bytes, uint32_t max_inflight,
                                              lshbloom_server_t **out) {
    if (!indexes || n == 0 || !out || max_inflight == 0 || max_inflight > 256 ||
        mem_budget_bytes < 4096)
        return fail(LSHB_ERR_ARG, "bad server arguments");
    *out = nullptr;
    for (uint32_t i = 0; i < n; ++i) {
        if (!indexes[i]) return fail(LSHB_ERR_ARG, "NULL index %u", i);
        if (indexes[i]->device != indexes[0]->device)
            return fail(LSHB_ERR_ARG, "indexes must share one device");
        if (indexes[i]->passes.size() != 1) return fail(LSHB_ERR_ARG, "serving needs P <= 256");
    }
    lshbloom_server *s = new (std::nothrow) lshbloom_server();
    if (!s) return fail(LSHB_ERR_OOM, "host allocation");
    s->idx.assign(indexes, indexes + n);
    s->device = indexes[0]->device;
    s->bands = 0;
    for (auto *h : s->idx) {
        s->bands = std::max(s->bands, h->bands);
        s->stage_inputs = s->stage_inputs || h->cfg.stage_host_inputs;
    }
    s->pageable_access = device_reads_pageable(s->device);
    cudaSetDevice(s->device);
    cudaError_t e = cudaMalloc(&s->pool_mem, mem_budget_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return fail(LSHB_ERR_OOM, "server budget of %llu bytes", (unsigned long long)mem_budget_bytes);
    }
    s->pool.init((uint8_t *)s->pool_mem, mem_budget_bytes & ~255ull);
    for (uint32_t i = 0; i < max_inflight; ++i) s->free_slots.push_back((int)(max_inflight - 1 - i));
    s->running.resize(n);
    s->sig_wait.resize(n);
    s->sig_flight.resize(n);
    s->sig_stream.assign(n, nullptr);
    s->sig_event.assign(n, nullptr);
    s->seg.assign(n, nullptr);
    for (uint32_t i = 0; i < n; ++i) {
        cudaStreamCreateWithFlags(&s->sig_stream[i], cudaStreamNonBlocking);
        cudaEventCreateWithFlags(&s->sig_event[i], cudaEventDisableTiming);
        s->seg[i] = segment_state_create();
        if (!s->seg[i]) {
            lshbloom_server_destroy(s);
            return fail(LSHB_ERR_OOM, "host allocation");
        }
    }
    s->worker = std::thread([s] { s->loop(); });
    for (uint32_t i = 0; i < n; ++i) s->bloom_workers.emplace_back([s, i] { s->bloom_loop(i); });
    *out = s;
    return LSHB_OK;
}

extern "C" lshb_status lshbloom_server_submit(lshbloom_server_t *s, uint32_t index,
                                              const uint64_t *offsets, const uint32_t *tokens,
                                              uint64_t D, uint8_t *flags_out, uint64_t *ticket) {
    if (!s || !ticket || index >= s->idx.size()) return fail(LSHB_ERR_ARG, "bad submit arguments");
    if (D > 0 && (!offsets || !tokens || !flags_out)) return fail(LSHB_ERR_ARG, "NULL pointer with D > 0");
    for (uint64_t i = 0; i < D; ++i)
        if (offsets[i + 1] < offsets[i]) return fail(LSHB_ERR_CSR, "offsets decrease at %llu", (unsigned long long)i);
    Request *r = new (std::nothrow) Request();
    if (!r) return fail(LSHB_ERR_OOM, "host allocation");
    r->index = index;
    r->D = D;
    r->tok0 = D ? offsets[0] : 0;
    r->T = D ? offsets[D] - offsets[0] : 0;
    r->h_off = offsets;
    r->h_tok = tokens;
    r->h_flags = flags_out;
    if (D && !s->stage_inputs) {
        r->in_off = (const uint64_t *)host_read_pointer(s->pageable_access, offsets);
        r->in_tok = (const uint32_t *)host_read_pointer(s->pageable_access, tokens);
    }
    r->bytes = request_bytes(D, r->T, s->bands, !r->in_off, !r->in_tok);
    if (r->bytes > s->pool.size) {
        const uint64_t need = r->bytes;
        delete r;
        return fail(LSHB_ERR_BUSY, "request needs %llu bytes, the server budget is %llu",
                    (unsigned long long)need, (unsigned long long)s->pool.size);
    }
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> g(s->mu);
        r->ticket = s->next_ticket++;
        s->reqs[r->ticket] = r;
        if (D == 0) {
            r->state = RState::Done;
            r->t_done = r->t_submit;
        } else {
            s->fifo.push_back(r);
        }
        *ticket = r->ticket;
    }
    s->cv_work.notify_one();
    return LSHB_OK;
}

extern "C" lshb_status lshbloom_server_wait(lshbloom_server_t *s, uint64_t ticket, double timeout_ms,
                                            double *latency_us) {
    if (!s) return fail(LSHB_ERR_ARG, "NULL server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(LSHB_ERR_ARG, "unknown ticket %llu", (unsigned long long)ticket);
    Request *r = it->second;
    auto done = [r] { return r->state == RState::Done; };
    if (timeout_ms < 0) {
        s->cv_done.wait(lk, done);
    } else if (!s->cv_done.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms), done)) {
        return fail(LSHB_ERR_TIMEOUT, "request %llu still running", (unsigned long long)ticket);
    }
    if (latency_us)
        *latency_us = std::chrono::duration<double, std::micro>(r->t_done - r->t_submit).count();
    const lshb_status st = r->status;
    s->reqs.erase(it);
    delete r;
    if (st != LSHB_OK) return fail(st, "request %llu failed", (unsigned long long)ticket);
    return LSHB_OK;
}

extern "C" void lshbloom_server_destroy(lshbloom_server_t *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    s->cv_bloom.notify_all();
    if (s->worker.joinable()) s->worker.join();
    {
        // the signature thread is gone: every admitted request has ended its
        // signature stage; wake the Bloom threads to drain and stop
        std::lock_guard<std::mutex> g(s->mu);
    }
    s->cv_bloom.notify_all();
    for (auto &t : s->bloom_workers)
        if (t.joinable()) t.join();
    cudaSetDevice(s->device);
    for (auto &kv : s->reqs) delete kv.second;
    for (auto st : s->sig_stream)
        if (st) cudaStreamDestroy(st);
    for (auto ev : s->sig_event)
        if (ev) cudaEventDestroy(ev);
    for (auto *st : s->seg) segment_state_destroy(st);
    if (s->pool_mem) cudaFree(s->pool_mem);
    delete s;
}
