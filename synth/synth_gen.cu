// Device twin of synth/corpus.py: the same counter-based draws and the same
// host-built tables, so a corpus generated here is byte-identical to the one
// numpy generates.  Holds none of the deduplication method's arithmetic.
#include <cuda_runtime.h>

#include <cstdint>

#define SYN_API extern "C" __attribute__((visibility("default")))

namespace {

constexpr uint64_t kGold = 0x9e3779b97f4a7c15ull;
constexpr int kMaxChain = 64;
enum { F_LEN = 1, F_DUP, F_SRC, F_MUT, F_MUTPOS, F_TOK, F_VOCAB };

struct SynthParams {
    const uint64_t *zipf_cdf;   // V
    const uint32_t *word_hash;  // V
    const uint32_t *length;     // 2^16
    const uint64_t *mut_thr;    // 2^10
    uint64_t vocab;
    uint64_t dup_thr;
    uint64_t window;
    uint64_t fkey[8];           // per-field keys, index = field
};

__device__ __forceinline__ uint64_t smix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t draw(const SynthParams &p, int field, uint64_t i, uint64_t j) {
    return smix(p.fkey[field] + smix(i * kGold + j));
}

__device__ __forceinline__ bool is_dup(const SynthParams &p, uint64_t d) {
    return d > 0 && draw(p, F_DUP, d, 0) < p.dup_thr;
}

__device__ __forceinline__ uint64_t source(const SynthParams &p, uint64_t d) {
    uint64_t span = d > 0 ? d : 1;
    if (p.window > 0 && span > p.window) span = p.window;
    return d - 1 - draw(p, F_SRC, d, 0) % span;
}

__device__ __forceinline__ uint32_t own_length(const SynthParams &p, uint64_t d) {
    return p.length[draw(p, F_LEN, d, 0) >> 48];
}

__device__ __forceinline__ uint64_t mut_threshold(const SynthParams &p, uint64_t d) {
    return p.mut_thr[draw(p, F_MUT, d, 0) >> 54];
}

__device__ __forceinline__ uint32_t fresh(const SynthParams &p, uint64_t c, uint64_t pos) {
    const uint64_t r = draw(p, F_TOK, c, pos);
    // first index with cdf[idx] > r
    uint64_t lo = 0, hi = p.vocab;
    while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        if (p.zipf_cdf[mid] > r) hi = mid; else lo = mid + 1;
    }
    if (lo >= p.vocab) lo = p.vocab - 1;
    return p.word_hash[lo];
}

__global__ void k_lengths(const __grid_constant__ SynthParams p, uint64_t d0, uint64_t D,
                          uint64_t *lens) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < D;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t cur = d0 + i;
        for (int t = 0; t < kMaxChain; ++t) {
            if (!is_dup(p, cur)) break;
            cur = source(p, cur);
        }
        lens[i] = own_length(p, cur);
    }
}

__global__ void k_tokens(const __grid_constant__ SynthParams p, uint64_t d0, uint64_t D,
                         const uint64_t *offsets, uint32_t *tokens) {
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const int lane = threadIdx.x & 31;
    for (uint64_t i = warp; i < D; i += nw) {
        const uint64_t d = d0 + i;
        const uint64_t o0 = offsets[i] - offsets[0], L = offsets[i + 1] - offsets[i];
        for (uint64_t pos = lane; pos < L; pos += 32) {
            uint64_t cur = d;
            for (int t = 0; t < kMaxChain; ++t) {
                if (!is_dup(p, cur)) break;
                if (draw(p, F_MUTPOS, cur, pos) < mut_threshold(p, cur)) break;
                cur = source(p, cur);
            }
            tokens[o0 + pos] = fresh(p, cur, pos);
        }
    }
}

}  // namespace

SYN_API int synth_doc_lengths(const SynthParams *p, uint64_t d0, uint64_t D, uint64_t *lens,
                              void *stream) {
    if (!p || (!lens && D)) return 1;
    if (D == 0) return 0;
    uint64_t blocks = (D + 255) / 256;
    if (blocks > 65536) blocks = 65536;
    k_lengths<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(*p, d0, D, lens);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

SYN_API int synth_tokens(const SynthParams *p, uint64_t d0, uint64_t D, const uint64_t *offsets,
                         uint32_t *tokens, void *stream) {
    if (!p || (D && (!offsets || !tokens))) return 1;
    if (D == 0) return 0;
    uint64_t blocks = (D * 32 + 255) / 256;
    if (blocks > 65536) blocks = 65536;
    k_tokens<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(*p, d0, D, offsets, tokens);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}
