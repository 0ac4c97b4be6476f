// lshbloom_band_keys_static: band keys without any allocation by the call.
//
// Some callers cannot let a library allocate device memory: applications
// that hand all GPU memory to their own pool with a fixed budget, and
// latency-critical loops where cudaMalloc's implicit synchronisation of the
// whole device would stall unrelated streams.  This entry point computes the
// same band keys as lshbloom_band_keys without allocating: with more than 256
// permutations (several signature passes) the intermediate signature matrix
// lives in a fixed array compiled into the library; with one pass the
// signature kernel writes the keys directly.  The caller still provides the
// input and output buffers.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "runtime_internal.h"

namespace lshb {

// 16 MiB of signature rows (P uint32 per document), held by every GPU that
// loads this library until the process exits.
constexpr size_t kStaticSigBytes = 16u << 20;
static __device__ __align__(256) uint32_t g_static_sig[kStaticSigBytes / 4];
// 0 when the offsets handed to the last call were non-decreasing.
static __device__ __align__(256) uint32_t g_static_bad_offsets;

__global__ void k_check_offsets(const uint64_t *__restrict__ off, uint64_t D) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < D;
         i += (uint64_t)gridDim.x * blockDim.x)
        if (off[i + 1] < off[i]) g_static_bad_offsets = 1u;
}

// Device address of g_static_sig, looked up once per device with that device
// current (the host-side name of the array is only a stand-in).
static uint32_t *static_sig_address(int dev, cudaError_t *err) {
    static std::mutex mu;
    static uint32_t *addr[64] = {nullptr};
    if (dev < 0 || dev >= 64) {
        *err = cudaErrorInvalidDevice;
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        *err = cudaGetSymbolAddress(&p, g_static_sig);
        if (*err != cudaSuccess) return nullptr;
        addr[dev] = (uint32_t *)p;
    }
    *err = cudaSuccess;
    return addr[dev];
}

}  // namespace lshb

using namespace lshb;

extern "C" LSHB_API lshb_status lshbloom_band_keys_static(lshbloom_t *h, const uint64_t *offsets,
                                                           const uint32_t *tokens, uint64_t D,
                                                           uint64_t *keys_out, void *stream) {
    if (!h) return fail(LSHB_ERR_ARG, "NULL handle");
    if (D == 0) return LSHB_OK;
    if (!offsets || !tokens || !keys_out) return fail(LSHB_ERR_ARG, "NULL pointer with D > 0");
    // More than one signature pass (P > 256) keeps the signature matrix in the
    // fixed array.  Compared by division: D * P * 4 can wrap around 2^64.
    const bool single = h->passes.size() == 1;
    const uint64_t max_docs = kStaticSigBytes / (4ull * h->P);
    if (!single && D > max_docs)
        return fail(LSHB_ERR_ARG,
                    "lshbloom_band_keys_static: %llu documents x %u permutations need more "
                    "signature scratch than the fixed array holds (%zu bytes, at most %llu "
                    "documents)",
                    (unsigned long long)D, h->P, kStaticSigBytes, (unsigned long long)max_docs);
    if (!is_device_pointer(offsets) || !is_device_pointer(tokens) || !is_device_pointer(keys_out))
        return fail(LSHB_ERR_ARG, "lshbloom_band_keys_static takes device pointers only");
    std::lock_guard<std::mutex> lock(h->mu);
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    uint32_t *sig = static_sig_address(h->device, &e);
    if (!sig) return cuda_fail(e, "cudaGetSymbolAddress(g_static_sig)");
    cudaStream_t s = (cudaStream_t)stream;

    // Reject decreasing offsets before any kernel reads tokens through them.
    const uint32_t zero = 0;
    uint32_t bad = 0;
    if ((e = cudaMemcpyToSymbolAsync(g_static_bad_offsets, &zero, 4, 0, cudaMemcpyHostToDevice, s)) !=
        cudaSuccess)
        return cuda_fail(e, "clear offsets flag");
    uint64_t blocks = (D + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_check_offsets<<<(unsigned)blocks, 256, 0, s>>>(offsets, D);
    count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "k_check_offsets");
    if ((e = cudaMemcpyFromSymbolAsync(&bad, g_static_bad_offsets, 4, 0, cudaMemcpyDeviceToHost, s)) !=
        cudaSuccess)
        return cuda_fail(e, "read offsets flag");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    if (bad) return fail(LSHB_ERR_CSR, "offsets decrease");

    SigArgs a;
    memset(&a, 0, sizeof a);
    a.band_key = h->cfg.band_key;
    a.offsets = offsets;
    a.tokens = tokens;
    a.tok_base = 0;
    a.D = D;
    a.ngram = h->ngram;
    a.P = h->P;
    a.bands = h->bands;
    a.rows = h->rows;
    // One pass: the kernel's epilogue writes the band keys itself, with no
    // signature matrix in between.
    a.sig_out = single ? nullptr : sig;
    a.keys_out = single ? keys_out : nullptr;
    const int ngt = ngram_template(h->ngram);
    for (const SigPass &ps : h->passes) {
        a.p0 = ps.p0;
        a.npc = ps.npc;
        a.c = ps.c;
        if (ngt == 5) e = launch_sig_ng5(ps.ppl, a, s);
        else if (ngt == 1) e = launch_sig_ng1(ps.ppl, a, s);
        else e = launch_sig_ng0(ps.ppl, a, s);
        if (e != cudaSuccess) return cuda_fail(e, "signature kernel");
    }
    if (!single &&
        (e = launch_band_keys(sig, h->P, h->bands, h->rows, h->cfg.band_key, D, keys_out, s)) !=
            cudaSuccess)
        return cuda_fail(e, "band-key kernel");
    return LSHB_OK;
}
