// Pinned host memory kept across calls (grow-only: pinning costs far more
// than filling).  A call that finds its arena in use by another call takes a
// private region instead.
#pragma once

#include <mutex>

#include "common.cuh"

namespace gosh {

struct PinnedArena {
    std::mutex mu;
    char *ptr = nullptr;
    size_t cap = 0;
    bool busy = false;
    // Frees the region unless a call holds it; returns the bytes freed.
    size_t release() {
        std::lock_guard<std::mutex> lock(mu);
        if (busy || !ptr) return 0;
        cudaFreeHost(ptr);
        const size_t freed = cap;
        ptr = nullptr;
        cap = 0;
        return freed;
    }
};

struct PinnedLease {
    PinnedArena &arena;
    char *ptr = nullptr;
    bool shared = false;
    explicit PinnedLease(PinnedArena &a) : arena(a) {}
    PinnedLease(const PinnedLease &) = delete;
    PinnedLease &operator=(const PinnedLease &) = delete;
    gosh_status acquire(size_t bytes, const char *what) {
        if (bytes == 0) bytes = 256;
        {
            std::lock_guard<std::mutex> lock(arena.mu);
            if (!arena.busy) {
                if (arena.cap < bytes) {
                    if (arena.ptr) cudaFreeHost(arena.ptr);
                    arena.ptr = nullptr;
                    arena.cap = 0;
                    if (cudaMallocHost(&arena.ptr, bytes) != cudaSuccess) {
                        arena.ptr = nullptr;
                        cudaGetLastError();
                        set_error("pinned allocation of %zu bytes of %s failed", bytes, what);
                        return GOSH_ERR_OOM;
                    }
                    arena.cap = bytes;
                }
                arena.busy = true;
                shared = true;
                ptr = arena.ptr;
                return GOSH_OK;
            }
        }
        if (cudaMallocHost(&ptr, bytes) != cudaSuccess) {
            ptr = nullptr;
            cudaGetLastError();
            set_error("pinned allocation of %zu bytes of %s failed", bytes, what);
            return GOSH_ERR_OOM;
        }
        return GOSH_OK;
    }
    ~PinnedLease() {
        if (shared) {
            std::lock_guard<std::mutex> lock(arena.mu);
            arena.busy = false;
        } else if (ptr) {
            cudaFreeHost(ptr);
        }
    }
};

}  // namespace gosh
