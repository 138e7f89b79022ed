// The coarsening hierarchy behind the opaque gosh_hierarchy handle.
#pragma once

#include <memory>
#include <vector>

#include "common.cuh"

// Level 0 aliases the caller's CSR; levels >= 1 and every map are device
// buffers from the stream-ordered allocator, held in `owned` (shared: the
// hierarchies coarsened together as one union of graphs point into common
// buffers, freed with the last of them, after a device sync since the handle
// carries no stream).
struct gosh_hierarchy {
    std::vector<int64_t> n, nnz;
    std::vector<int64_t *> rowptr;
    std::vector<int32_t *> col;
    std::vector<int32_t *> map;  // map[i]: G_i -> G_{i+1}
    std::vector<std::shared_ptr<void>> owned;
    ~gosh_hierarchy() {
        if (!owned.empty()) cudaDeviceSynchronize();
    }
};

// A device buffer from dev_alloc as a shared owner (returned to its
// allocator on the legacy stream when the last owner goes).
inline std::shared_ptr<void> device_owner(void *p) {
    return std::shared_ptr<void>(p, [](void *q) {
        if (q) gosh::dev_free(q, 0);
    });
}
