// Device primitives of libgosh: exclusive prefix sums and a stable LSD radix
// sort.  Both are deterministic (no atomics decide any output position), which
// the bit-exact coarsening and the fixed-order reduction of the deterministic
// training mode rely on.
#include <algorithm>
#include <unordered_map>

#include "common.cuh"

namespace gosh {
namespace {

// Block-wide exclusive scan of one int64 per thread; returns the block total.
__device__ __forceinline__ int64_t block_exclusive_scan(int64_t x, int64_t *smem_warp, int64_t &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) smem_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        int64_t w = lane < nw ? smem_warp[lane] : 0;
        int64_t winc = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, winc, o);
            if (lane >= o) winc += y;
        }
        if (lane < nw) smem_warp[lane] = winc - w;
        if (lane == 31) smem_warp[32] = winc;
    }
    __syncthreads();
    const int64_t excl = smem_warp[warp] + inc - x;
    total = smem_warp[32];
    return excl;
}

// ---------------------------------------------------------------------------
// Single-pass exclusive scan with decoupled look-back: each block claims the
// next tile from an atomic counter (so every tile it waits for belongs to a
// block that is already running), publishes its tile sum, then walks back
// over the published words of earlier tiles until it meets an inclusive
// prefix, and publishes its own.  A status word packs (epoch, flag, value):
// the epoch of the call, so words left by earlier calls in the per-stream
// workspace never look ready and no reset is needed; flag 1 = tile sum,
// 2 = inclusive prefix.  The wait is bounded: after kLookbackPolls fruitless
// polls the block raises the error word and stops waiting (the output is then
// wrong, which the error word reports).  Inputs are counts: non-negative,
// with a total below 2^38.
// ---------------------------------------------------------------------------
constexpr int kLbThreads = 256;
constexpr int kLbItems = 16;
constexpr int kLbTile = kLbThreads * kLbItems;
constexpr uint32_t kLookbackPolls = 1u << 22;
constexpr int kEpochShift = 40, kFlagShift = 38;
constexpr uint64_t kValueMask = (uint64_t(1) << kFlagShift) - 1;

__device__ __forceinline__ uint64_t lb_word(uint64_t epoch, uint64_t flag, int64_t value) {
    return (epoch << kEpochShift) | (flag << kFlagShift) | ((uint64_t)value & kValueMask);
}

template <typename In>
__global__ void __launch_bounds__(kLbThreads) scan_lookback(const In *__restrict__ in, int64_t *__restrict__ out,
                                                            int64_t n, int64_t *__restrict__ total,
                                                            unsigned long long *status,
                                                            unsigned long long *counter, unsigned long long base,
                                                            uint64_t epoch, int *err) {
    GOSH_DEP_WAIT();
    __shared__ int64_t sw[33];
    __shared__ int64_t s_tile, s_prefix;
    if (threadIdx.x == 0) s_tile = (int64_t)(atomicAdd(counter, 1ull) - base);
    __syncthreads();
    const int64_t tile = s_tile;
    const int64_t i0 = tile * kLbTile + (int64_t)threadIdx.x * kLbItems;
    int64_t v[kLbItems];
    int64_t sum = 0;
#pragma unroll
    for (int j = 0; j < kLbItems; ++j) {
        v[j] = i0 + j < n ? (int64_t)in[i0 + j] : 0;
        sum += v[j];
    }
    int64_t agg;
    int64_t run = block_exclusive_scan(sum, sw, agg);
    if (threadIdx.x == 0) {
        int64_t prefix = 0;
        if (tile == 0) {
            atomicExch(status, lb_word(epoch, 2, agg));
        } else {
            atomicExch(status + tile, lb_word(epoch, 1, agg));
            uint32_t polls = 0;
            for (int64_t j = tile - 1; j >= 0;) {
                const uint64_t w = *reinterpret_cast<volatile unsigned long long *>(status + j);
                if ((w >> kEpochShift) != epoch) {
                    if (++polls > kLookbackPolls) {
                        atomicExch(err, 1);
                        break;
                    }
                    continue;
                }
                prefix += (int64_t)(w & kValueMask);
                if (((w >> kFlagShift) & 3) == 2) break;
                --j;
            }
            atomicExch(status + tile, lb_word(epoch, 2, prefix + agg));
        }
        s_prefix = prefix;
    }
    __syncthreads();
    run += s_prefix;
#pragma unroll
    for (int j = 0; j < kLbItems; ++j) {
        if (i0 + j < n) out[i0 + j] = run;
        run += v[j];
    }
    if (total && (tile + 1) * kLbTile >= n && threadIdx.x == 0) *total = s_prefix + agg;
}

// Per host thread and stream: the tile status words (zeroed once, then only
// ever overwritten with later epochs) and the tile counter (monotonic: a call
// claims tiles base .. base + ntiles - 1).  An event orders a workspace's use
// after its previous use even if the stream handle was recycled.
struct LookbackWork {
    unsigned long long *status = nullptr;
    unsigned long long *counter = nullptr;
    int64_t cap = 0;
    uint64_t epoch = 0;
    unsigned long long base = 0;
    cudaEvent_t last = nullptr;
};

gosh_status lookback_work(cudaStream_t s, int64_t ntiles, LookbackWork **out) {
    static thread_local std::unordered_map<cudaStream_t, LookbackWork> works;
    LookbackWork &w = works[s];
    if (w.last) GOSH_TRY_CUDA(cudaStreamWaitEvent(s, w.last, 0));
    else GOSH_TRY_CUDA(cudaEventCreateWithFlags(&w.last, cudaEventDisableTiming));
    if (!w.counter) {
        GOSH_TRY_CUDA(cudaMallocAsync(&w.counter, sizeof(unsigned long long), s));
        GOSH_TRY_CUDA(cudaMemsetAsync(w.counter, 0, sizeof(unsigned long long), s));
        w.base = 0;
    }
    const uint64_t kMaxEpoch = (uint64_t(1) << (64 - kEpochShift)) - 1;
    if (w.cap < ntiles || w.epoch >= kMaxEpoch) {
        if (w.status) GOSH_TRY_CUDA(cudaFreeAsync(w.status, s));
        const int64_t cap = std::max<int64_t>(ntiles, std::max<int64_t>(256, 2 * w.cap));
        GOSH_TRY_CUDA(cudaMallocAsync(&w.status, sizeof(unsigned long long) * cap, s));
        GOSH_TRY_CUDA(cudaMemsetAsync(w.status, 0, sizeof(unsigned long long) * cap, s));
        w.cap = cap;
        w.epoch = 0;
    }
    ++w.epoch;
    *out = &w;
    return GOSH_OK;
}

template <typename In>
gosh_status scan_exclusive(const In *in, int64_t *out, int64_t n, int64_t *total, cudaStream_t s) {
    if (n <= 0) {
        if (total) GOSH_TRY_CUDA(cudaMemsetAsync(total, 0, sizeof(int64_t), s));
        return GOSH_OK;
    }
    const int64_t tiles = ceil_div(n, kLbTile);
    LookbackWork *w = nullptr;
    GOSH_TRY(lookback_work(s, tiles, &w));
    launch_dep(scan_lookback<In>, (unsigned)tiles, kLbThreads, 0, s, in, out, n, total, w->status, w->counter, w->base, w->epoch, device_error_word());
    w->base += (unsigned long long)tiles;
    GOSH_TRY_CUDA(cudaGetLastError());
    GOSH_TRY_CUDA(cudaEventRecord(w->last, s));
    return GOSH_OK;
}

// ---------------------------------------------------------------------------
// Radix sort: 8-bit digits, 256 threads x 8 keys per tile.  Warp w of a tile
// owns keys [w*256, w*256+256) of the tile, taken 32 at a time in index order,
// so (warp, step, lane) order is index order and the scatter is stable.
// ---------------------------------------------------------------------------
constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kSortWarps = kSortThreads / 32;

// Digit histogram of one pass over the current arrangement of the keys:
// counts[digit * nblocks + block] (each pass needs its own: a block's counts
// depend on which keys the previous pass placed in it).
template <typename K>
__global__ void __launch_bounds__(kSortThreads) radix_hist(const K *__restrict__ keys, int64_t n, int shift,
                                                           int64_t *__restrict__ counts, int64_t nblocks) {
    GOSH_DEP_WAIT();
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * kSortTile + warp * 256 + lane;
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
        const int64_t idx = base + i * 32;
        if (idx < n) atomicAdd(&h[(uint32_t)(keys[idx] >> shift) & 255u], 1u);
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

template <typename K, bool kVals>
__global__ void __launch_bounds__(kSortThreads) radix_scatter(
    const K *__restrict__ kin, const uint32_t *__restrict__ vin, K *__restrict__ kout,
    uint32_t *__restrict__ vout, int64_t n, int shift, const int64_t *__restrict__ offsets,
    int64_t nblocks) {
    GOSH_DEP_WAIT();
    __shared__ uint32_t wcnt[kSortWarps][256];
    __shared__ int64_t gbase[256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) wcnt[w][threadIdx.x] = 0;
    gbase[threadIdx.x] = offsets[(int64_t)threadIdx.x * nblocks + blockIdx.x];
    __syncthreads();
    const uint32_t lt_mask = (1u << lane) - 1u;
    const int64_t base = (int64_t)blockIdx.x * kSortTile + warp * 256 + lane;
    K key[kSortItems];
    uint32_t val[kSortItems];
    uint32_t rank[kSortItems];
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
        const int64_t idx = base + i * 32;
        const bool ok = idx < n;
        key[i] = ok ? kin[idx] : K(0);
        if (kVals) val[i] = ok ? vin[idx] : 0u;
        const uint32_t digit = ok ? ((uint32_t)(key[i] >> shift) & 255u) : 256u;
        const uint32_t peers = __match_any_sync(0xffffffffu, digit);
        uint32_t pre = 0;
        if (ok) pre = wcnt[warp][digit];
        __syncwarp();
        if (ok && (peers & lt_mask) == 0) wcnt[warp][digit] = pre + __popc(peers);
        __syncwarp();
        rank[i] = pre + __popc(peers & lt_mask);
    }
    __syncthreads();
    {
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) {
            const uint32_t c = wcnt[w][threadIdx.x];
            wcnt[w][threadIdx.x] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
        const int64_t idx = base + i * 32;
        if (idx < n) {
            const uint32_t digit = (uint32_t)(key[i] >> shift) & 255u;
            const int64_t pos = gbase[digit] + wcnt[warp][digit] + rank[i];
            kout[pos] = key[i];
            if (kVals) vout[pos] = val[i];
        }
    }
}

// LSD radix sort over the given digit shifts, ping-ponging between (keys,
// vals) and (kalt, valt): per pass a histogram of the current arrangement,
// one scan, one stable scatter.  Returns in *in_alt whether the result ended
// in the alternate buffers (an odd pass count).
template <typename K>
gosh_status radix_sort_pp(K *keys, uint32_t *vals, K *kalt, uint32_t *valt, int64_t n, const int *shifts,
                          int ndigits, cudaStream_t s, bool *in_alt) {
    *in_alt = false;
    if (n <= 1 || ndigits == 0) return GOSH_OK;
    const int64_t nblocks = ceil_div(n, kSortTile);
    Scratch counts, offs;
    GOSH_TRY(counts.alloc(sizeof(int64_t) * 256 * nblocks, s));
    GOSH_TRY(offs.alloc(sizeof(int64_t) * 256 * nblocks, s));
    K *ka = keys, *kb = kalt;
    uint32_t *va = vals, *vb = valt;
    for (int d = 0; d < ndigits; ++d) {
        launch_dep(radix_hist<K>, (unsigned)nblocks, kSortThreads, 0, s, ka, n, shifts[d], counts.as<int64_t>(), nblocks);
        GOSH_TRY(scan_exclusive<int64_t>(counts.as<int64_t>(), offs.as<int64_t>(), 256 * nblocks, nullptr, s));
        if (vals)
            launch_dep(radix_scatter<K, true>, (unsigned)nblocks, kSortThreads, 0, s, ka, va, kb, vb, n, shifts[d], offs.as<int64_t>(), nblocks);
        else
            launch_dep(radix_scatter<K, false>, (unsigned)nblocks, kSortThreads, 0, s, ka, nullptr, kb, nullptr, n, shifts[d], offs.as<int64_t>(), nblocks);
        GOSH_TRY_CUDA(cudaGetLastError());
        K *kt = ka; ka = kb; kb = kt;
        uint32_t *vt = va; va = vb; vb = vt;
    }
    *in_alt = ka != keys;
    return GOSH_OK;
}

template <typename K>
gosh_status radix_sort(K *keys, uint32_t *vals, int64_t n, const int *shifts, int ndigits, cudaStream_t s) {
    if (n <= 1 || ndigits == 0) return GOSH_OK;
    Scratch kalt, valt;
    GOSH_TRY(kalt.alloc(sizeof(K) * n, s));
    if (vals) GOSH_TRY(valt.alloc(sizeof(uint32_t) * n, s));
    bool in_alt = false;
    GOSH_TRY(radix_sort_pp<K>(keys, vals, kalt.as<K>(), valt.as<uint32_t>(), n, shifts, ndigits, s, &in_alt));
    if (in_alt) {
        GOSH_TRY_CUDA(cudaMemcpyAsync(keys, kalt.as<K>(), sizeof(K) * n, cudaMemcpyDeviceToDevice, s));
        if (vals)
            GOSH_TRY_CUDA(cudaMemcpyAsync(vals, valt.as<uint32_t>(), sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
    }
    return GOSH_OK;
}

}  // namespace

gosh_status scan_exclusive_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *total,
                               cudaStream_t s) {
    return scan_exclusive<int64_t>(in, out, n, total, s);
}
gosh_status scan_exclusive_u8_to_i64(const uint8_t *in, int64_t *out, int64_t n, int64_t *total,
                                     cudaStream_t s) {
    return scan_exclusive<uint8_t>(in, out, n, total, s);
}
gosh_status scan_exclusive_i32_to_i64(const int32_t *in, int64_t *out, int64_t n, int64_t *total,
                                      cudaStream_t s) {
    return scan_exclusive<int32_t>(in, out, n, total, s);
}

gosh_status radix_sort_u32(uint32_t *keys, uint32_t *vals, int64_t n, int begin_bit, int end_bit,
                           cudaStream_t s) {
    int shifts[4];
    int nd = 0;
    for (int b = begin_bit; b < end_bit && nd < 4; b += 8) shifts[nd++] = b;
    return radix_sort<uint32_t>(keys, vals, n, shifts, nd, s);
}

gosh_status radix_sort_u32_pp(uint32_t *keys, uint32_t *vals, uint32_t *kalt, uint32_t *valt, int64_t n, int begin_bit,
                              int end_bit, cudaStream_t s, bool *in_alt) {
    int shifts[4];
    int nd = 0;
    for (int b = begin_bit; b < end_bit && nd < 4; b += 8) shifts[nd++] = b;
    return radix_sort_pp<uint32_t>(keys, vals, kalt, valt, n, shifts, nd, s, in_alt);
}

gosh_status radix_sort_u64(uint64_t *keys, uint32_t *vals, int64_t n, const int *shifts,
                           int ndigits, cudaStream_t s) {
    return radix_sort<uint64_t>(keys, vals, n, shifts, ndigits, s);
}

}  // namespace gosh
