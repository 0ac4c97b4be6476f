// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace lshb {

constexpr int kMaxPC = 256;       // permutations handled by one signature pass (8 per lane)
constexpr int kSigThreads = 64;   // threads per signature block (2 warps)
constexpr int kMaxBands = 64;
constexpr int kMaxK = 64;

// One pass worth of permutation coefficients, split into 32-bit halves so the
// kernels can read them as constant-bank operands.
struct PermSlice {
    uint32_t a0[kMaxPC], a1[kMaxPC], b0[kMaxPC], b1[kMaxPC];
};

// Arguments of the signature-stage kernels (passed as a __grid_constant__
// parameter: everything, coefficients included, lives in the constant bank).
struct SigArgs {
    const uint64_t *offsets;  // D+1 entries; document d is tokens[offsets[d]-tok_base ...]
    const uint32_t *tokens;
    uint64_t tok_base;
    uint64_t D;
    uint32_t ngram;
    uint32_t P;               // row stride of sig_out
    uint32_t p0;              // first permutation of this pass
    uint32_t npc;             // permutations in this pass (<= the kernel's PC)
    uint32_t bands, rows;     // band-key epilogue (used when keys_out != nullptr)
    uint32_t band_key;        // lshb_band_key
    uint32_t *sig_out;        // D x P, or nullptr
    uint64_t *keys_out;       // D x bands, or nullptr
    const uint32_t *hashes;   // minhash-from-hashes input, indexed like tokens
    uint32_t *hash_out;       // shingle-hash output, indexed like tokens
    PermSlice c;
};

// Process-wide count of kernels this library has launched.
void count_launch(uint64_t n = 1);
uint64_t launches_total();

// Signature stage (sig_*.cu).
int ngram_template(uint32_t ngram);  // 1, 5, or 0 (runtime n)
cudaError_t launch_sig_ng0(int ppl, const SigArgs &a, cudaStream_t s);
cudaError_t launch_sig_ng1(int ppl, const SigArgs &a, cudaStream_t s);
cudaError_t launch_sig_ng5(int ppl, const SigArgs &a, cudaStream_t s);
cudaError_t launch_shingle_hash(int ngram_tmpl, const SigArgs &a, cudaStream_t s);
cudaError_t launch_minhash_hashes(int ppl, const SigArgs &a, cudaStream_t s);
cudaError_t launch_band_keys(const uint32_t *sig, uint32_t P, uint32_t bands, uint32_t rows,
                             uint32_t band_key, uint64_t D, uint64_t *keys, cudaStream_t s);

}  // namespace lshb
