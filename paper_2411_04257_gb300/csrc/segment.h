// One CSR batch of a multi-batch launch of the persistent signature kernel
// (the server's requests): its documents are documents doc0 .. doc0 + D - 1
// of the launch; document d's tokens are tokens[offsets[d - doc0] - tok_base]
// and its band keys go to keys_out[(d - doc0) * bands ...].
#pragma once

#include <cstdint>

namespace lshb {

struct Segment {
    const uint64_t *offsets;
    const uint32_t *tokens;
    uint64_t tok_base;
    uint64_t doc0;
    uint64_t *keys_out;
};

}  // namespace lshb
