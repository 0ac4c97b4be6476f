// Instantiates the signature kernel for one compile-time n-gram size (LSHB_NG)
// and every lane width PPL, plus a dispatcher.  Included by one translation
// unit per n-gram size so the instantiations compile in parallel.
#pragma once

#include "sig_kernels.cuh"

#define LSHB_CAT2(a, b) a##b
#define LSHB_CAT(a, b) LSHB_CAT2(a, b)

namespace lshb {

template <int PPL>
static cudaError_t LSHB_CAT(sig_go_ng, LSHB_NG)(const SigArgs &a, cudaStream_t s) {
    static int grid_for_dev[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    int &g = grid_for_dev[dev & 63];
    if (g == 0) {
        int nb = 0, sms = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sig<LSHB_NG, PPL>, kSigThreads, 0);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        g = (nb > 0 ? nb : 1) * (sms > 0 ? sms : 1);
    }
    const uint64_t need = (a.D + kSigThreads / 32 - 1) / (kSigThreads / 32);
    const int grid = (int)(need < (uint64_t)g ? (need > 0 ? need : 1) : (uint64_t)g);
    k_sig<LSHB_NG, PPL><<<grid, kSigThreads, 0, s>>>(a); count_launch();
    return cudaGetLastError();
}

cudaError_t LSHB_CAT(launch_sig_ng, LSHB_NG)(int ppl, const SigArgs &a, cudaStream_t s) {
    switch (ppl) {
        case 1: return LSHB_CAT(sig_go_ng, LSHB_NG)<1>(a, s);
        case 2: return LSHB_CAT(sig_go_ng, LSHB_NG)<2>(a, s);
        case 4: return LSHB_CAT(sig_go_ng, LSHB_NG)<4>(a, s);
        case 8: return LSHB_CAT(sig_go_ng, LSHB_NG)<8>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace lshb
