// Plain (one kernel per stage) signature path: shingle hashes to memory, then
// MinHash minima from them (the signature kernel reading stored hashes), then
// band keys from the signature matrix.
#include "sig_kernels.cuh"

namespace lshb {

int ngram_template(uint32_t ngram) {
    if (ngram == 1) return 1;
    if (ngram == 5) return 5;
    return 0;
}

template <typename K>
static int occupancy_grid(K kernel, int threads) {
    int dev = 0, nb = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, 0);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return (nb > 0 ? nb : 1) * (sms > 0 ? sms : 1);
}

static int clamp_grid(int g, uint64_t D) {
    const uint64_t need = (D + kSigThreads / 32 - 1) / (kSigThreads / 32);
    return (int)(need < (uint64_t)g ? (need > 0 ? need : 1) : (uint64_t)g);
}

template <int NG>
static cudaError_t hash_go(const SigArgs &a, cudaStream_t s) {
    static int g[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (!g[dev & 63]) g[dev & 63] = occupancy_grid(k_shingle_hash<NG>, kSigThreads);
    k_shingle_hash<NG><<<clamp_grid(g[dev & 63], a.D), kSigThreads, 0, s>>>(a); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_shingle_hash(int ngram_tmpl, const SigArgs &a, cudaStream_t s) {
    switch (ngram_tmpl) {
        case 1: return hash_go<1>(a, s);
        case 5: return hash_go<5>(a, s);
        default: return hash_go<0>(a, s);
    }
}

// Stage 2 of the plain form: the generic signature kernel with `a.hashes` set.
cudaError_t launch_minhash_hashes(int ppl, const SigArgs &a, cudaStream_t s) {
    return launch_sig_ng0(ppl, a, s);
}

// Band key j of document d from signature rows j*r .. j*r+r-1 (mod 2^64).
__global__ void k_band_keys(const uint32_t *__restrict__ sig, uint32_t P, uint32_t bands,
                            uint32_t rows, uint32_t band_key, uint64_t D,
                            uint64_t *__restrict__ keys) {
    const uint64_t n = D * bands;
    for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t d = idx / bands;
        const uint32_t j = (uint32_t)(idx % bands);
        keys[idx] = band_key_of(sig + d * P + (uint64_t)j * rows, rows, j, band_key);
    }
}

cudaError_t launch_band_keys(const uint32_t *sig, uint32_t P, uint32_t bands, uint32_t rows,
                             uint32_t band_key, uint64_t D, uint64_t *keys, cudaStream_t s) {
    const uint64_t n = D * bands;
    uint64_t blocks = (n + 255) / 256;
    if (blocks == 0) blocks = 1;
    if (blocks > 65535ull * 16) blocks = 65535ull * 16;
    k_band_keys<<<(unsigned)blocks, 256, 0, s>>>(sig, P, bands, rows, band_key, D, keys);
    count_launch();
    return cudaGetLastError();
}

}  // namespace lshb
