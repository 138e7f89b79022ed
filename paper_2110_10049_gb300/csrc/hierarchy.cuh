// The coarsening hierarchy behind the opaque gosh_hierarchy handle.
#pragma once

#include <vector>

#include "common.cuh"

// Level 0 aliases the caller's CSR; levels >= 1 and every map are owned and
// come from the stream-ordered allocator (released after a device sync, since
// the handle carries no stream).
struct gosh_hierarchy {
    std::vector<int64_t> n, nnz;
    std::vector<int64_t *> rowptr;
    std::vector<int32_t *> col;
    std::vector<int32_t *> map;  // map[i]: G_i -> G_{i+1}
    ~gosh_hierarchy() {
        if (rowptr.size() > 1 || !map.empty()) cudaDeviceSynchronize();
        for (size_t i = 1; i < rowptr.size(); ++i) {
            cudaFreeAsync(rowptr[i], 0);
            cudaFreeAsync(col[i], 0);
        }
        for (int32_t *m : map) cudaFreeAsync(m, 0);
    }
};
