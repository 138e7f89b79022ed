// The C ABI of libgosh (include/gosh.h): argument checks, the small kernels
// around the training step (initialisation, copy projection, CSR validation,
// pair scores and AUC) and the end-to-end driver of Alg. 2.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <mutex>
#include <unordered_map>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <type_traits>
#include <vector>

#include "hierarchy.cuh"

namespace gosh {

static thread_local char g_error[1024] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_error, sizeof(g_error), fmt, ap);
    va_end(ap);
}
void clear_error() { g_error[0] = 0; }

static std::atomic<unsigned long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

namespace {
std::mutex g_alloc_mu;
gosh_alloc_fn g_alloc = nullptr;
gosh_free_fn g_free = nullptr;
void *g_alloc_ctx = nullptr;
struct CallerBlock {
    size_t bytes;
    gosh_free_fn free;
    void *ctx;
};
std::unordered_map<void *, CallerBlock> g_caller_blocks;  // blocks lent by a caller's allocator
}  // namespace

cudaError_t dev_alloc(void **p, size_t bytes, cudaStream_t s) {
    gosh_alloc_fn fa;
    gosh_free_fn ff;
    void *ctx;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        fa = g_alloc;
        ff = g_free;
        ctx = g_alloc_ctx;
    }
    if (!fa) {
        keep_pool_memory();
        return cudaMallocAsync(p, bytes, s);
    }
    void *q = fa(bytes, (void *)s, ctx);
    if (!q) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    if (((uintptr_t)q & 255u) != 0) {  // not the promised alignment: give it back
        ff(q, bytes, (void *)s, ctx);
        *p = nullptr;
        return cudaErrorInvalidValue;
    }
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        g_caller_blocks[q] = {bytes, ff, ctx};
    }
    *p = q;
    return cudaSuccess;
}

void dev_free(void *p, cudaStream_t s) {
    if (!p) return;
    CallerBlock b{0, nullptr, nullptr};
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        auto it = g_caller_blocks.find(p);
        if (it != g_caller_blocks.end()) {
            b = it->second;
            g_caller_blocks.erase(it);
        }
    }
    if (b.free) b.free(p, b.bytes, (void *)s, b.ctx);
    else cudaFreeAsync(p, s);
}

void keep_pool_memory() {
    static std::atomic<unsigned long long> done_mask{0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
    const unsigned long long bit = 1ull << dev;
    if (done_mask.load(std::memory_order_relaxed) & bit) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t threshold = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &threshold);
    }
    cudaGetLastError();
    done_mask.fetch_or(bit);
}

int *device_error_word() {
    static std::mutex mu;
    static int *words[64] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!words[dev]) {
        if (cudaMalloc(&words[dev], sizeof(int)) != cudaSuccess || cudaMemset(words[dev], 0, sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            words[dev] = nullptr;
        }
    }
    return words[dev];
}

gosh_status train_level_impl(const gosh_csr *g, void *M, int level, int epochs, const gosh_params *p,
                             cudaStream_t s, double *loss_per_epoch, unsigned long long *n_updates);
gosh_status coarsen_impl(const gosh_csr *g0, int threshold, double shrink, int max_levels, cudaStream_t s,
                         gosh_hierarchy **out);
gosh_status coarsen_batch_impl(const gosh_csr *graphs, int G, int threshold, double shrink, int max_levels,
                               cudaStream_t s, std::vector<gosh_hierarchy *> &out);
gosh_status persistent_levels(gosh_hierarchy *h, const std::vector<void *> &bufs, int lowest, const gosh_params &p,
                              unsigned long long *n_updates, cudaStream_t s);
gosh_status mlp_train(gosh_mlp *m, const gosh_csr *g, const int32_t *map, const void *Mc, const void *Mf,
                      gosh_dtype dt, int epochs, double lr, int batch, int64_t max_rows, cudaStream_t s,
                      double *final_loss, bool use_kept);
gosh_status mlp_project(gosh_mlp *m, const void *Mc, const int32_t *map, const gosh_csr *g, void *Mf, gosh_dtype dt,
                        cudaStream_t s, int64_t keep_rows_of);

namespace {

int grid_for(int64_t work, int threads = 256) {
    const int64_t cap = (int64_t)num_sms() * 16;
    const int64_t g = ceil_div(work > 0 ? work : 1, threads);
    return (int)(g < cap ? g : cap);
}

bool dim_ok(int d) { return d == 8 || d == 16 || d == 32 || d == 64 || d == 128; }
bool dtype_ok(gosh_dtype t) { return t == GOSH_F32 || t == GOSH_BF16 || t == GOSH_F16; }
bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// ---------------------------------------------------------------- validation
enum : unsigned { kBadRowptr = 1, kBadRange = 2, kUnsorted = 4, kSelfLoop = 8, kAsym = 16 };

__global__ void validate_kernel(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col, int64_t n,
                                unsigned *__restrict__ flags, unsigned long long *__restrict__ first_bad) {
    GOSH_DEP_WAIT();
    const int64_t nnz = rowptr[n];
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = rowptr[v], e = rowptr[v + 1];
        unsigned bad = 0;
        if (b > e || b < 0 || e > nnz || (v == 0 && b != 0)) bad |= kBadRowptr;
        else {
            for (int64_t p = b; p < e; ++p) {
                const int32_t u = col[p];
                if (u < 0 || u >= n) { bad |= kBadRange; break; }
                if (u == v) bad |= kSelfLoop;
                if (p > b && col[p - 1] >= u) bad |= kUnsorted;
                // symmetric: v must appear in row u (binary search)
                int64_t lo = rowptr[u], hi = rowptr[u + 1];
                if (lo < 0 || hi > nnz || lo > hi) { bad |= kBadRowptr; break; }
                while (lo < hi) {
                    const int64_t mid = (lo + hi) >> 1;
                    if (col[mid] < v) lo = mid + 1; else hi = mid;
                }
                if (lo >= rowptr[u + 1] || col[lo] != v) bad |= kAsym;
            }
        }
        if (bad) {
            atomicOr(flags, bad);
            atomicMin(first_bad, (unsigned long long)v);
        }
    }
}

// ---------------------------------------------------------------- init
template <typename T>
__device__ __forceinline__ T from_float(float x);
template <> __device__ __forceinline__ float from_float<float>(float x) { return x; }
template <> __device__ __forceinline__ __nv_bfloat16 from_float<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
template <> __device__ __forceinline__ __half from_float<__half>(float x) { return __float2half_rn(x); }

template <typename T>
__global__ void init_kernel(T *__restrict__ M, int64_t n, int d, uint32_t level, uint64_t seed, uint64_t graph) {
    GOSH_DEP_WAIT();
    const int nq = (d + 3) / 4;
    const int64_t total = n * nq;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = i / nq;
        const int q = (int)(i % nq);
        const Philox4 w = philox4x64_10((uint64_t)v, (uint64_t)q, (uint64_t)level, kTagInit, seed, graph);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = 4 * q + j;
            if (c < d) {
                const double unit = (double)(w.w[j] >> 11) * 0x1.0p-53;
                const double x = (unit - 0.5) / (double)d;
                M[v * d + c] = from_float<T>((float)x);
            }
        }
    }
}

// ---------------------------------------------------------------- projection
__global__ void project_copy_kernel(const uint4 *__restrict__ Mc, const int32_t *__restrict__ map, uint4 *__restrict__ Mf,
                                    int64_t n_fine, int vecs) {
    GOSH_DEP_WAIT();
    const int64_t total = n_fine * vecs;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = i / vecs;
        const int q = (int)(i % vecs);
        Mf[i] = __ldg(Mc + (int64_t)__ldg(map + v) * vecs + q);
    }
}

// ---------------------------------------------------------------- scores / AUC
template <typename T, int L>
__global__ void pair_scores_kernel(const T *__restrict__ M, int d, const int32_t *__restrict__ pairs, int64_t np,
                                   float *__restrict__ out) {
    GOSH_DEP_WAIT();
    constexpr int PV = Store<T>::kPerVec;
    constexpr int G = 32 / L;
    const int lane = threadIdx.x & 31, gl = lane % L;
    const int64_t warp_id = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int vecs = d / PV;
    for (int64_t base = warp_id * G; base < np; base += nwarps * G) {
        const int64_t i = base + lane / L;
        float part = 0.0f;
        if (i < np) {
            const int64_t u = pairs[2 * i], v = pairs[2 * i + 1];
            const uint4 *pu = reinterpret_cast<const uint4 *>(M + u * d);
            const uint4 *pv = reinterpret_cast<const uint4 *>(M + v * d);
            for (int q = gl; q < vecs; q += L) {
                float a[PV], b[PV];
                Store<T>::unpack(pu[q], a);
                Store<T>::unpack(pv[q], b);
#pragma unroll
                for (int e = 0; e < PV; ++e) part = fmaf(a[e], b[e], part);
            }
        }
#pragma unroll
        for (int o = L / 2; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (i < np && gl == 0) out[i] = part;
    }
}

template <typename T>
void launch_pair_scores(const void *M, int d, const int32_t *pairs, int64_t np, float *out, cudaStream_t s) {
    constexpr int L = 8;
    const int64_t groups = np;
    const int64_t cap = (int64_t)num_sms() * 16;
    int64_t g = ceil_div(groups * L, 256);
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    launch_dep(pair_scores_kernel<T, L>, (int)g, 256, 0, s, static_cast<const T *>(M), d, pairs, np, out);
}

__global__ void score_keys(const float *__restrict__ score, int64_t n, uint32_t *__restrict__ key,
                           uint32_t *__restrict__ idx) {
    GOSH_DEP_WAIT();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float f = score[i];
        if (f == 0.0f) f = 0.0f;  // -0 and +0 tie
        const uint32_t u = __float_as_uint(f);
        key[i] = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
        idx[i] = (uint32_t)i;
    }
}

__global__ void neg_flags(const uint32_t *__restrict__ idx, int64_t n, int64_t npos, uint8_t *__restrict__ f) {
    GOSH_DEP_WAIT();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        f[i] = idx[i] >= (uint64_t)npos ? 1 : 0;
}

__global__ void auc_partials(const uint32_t *__restrict__ key, const uint32_t *__restrict__ idx,
                             const int64_t *__restrict__ neg_before, int64_t n, int64_t npos,
                             double *__restrict__ parts) {
    GOSH_DEP_WAIT();
    __shared__ double s[256];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (idx[i] >= (uint64_t)npos) continue;
        const uint32_t k = key[i];
        int64_t lo = 0, hi = i;  // first position with key >= k
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (key[mid] < k) lo = mid + 1; else hi = mid;
        }
        int64_t lo2 = i + 1, hi2 = n;  // first position with key > k
        while (lo2 < hi2) {
            const int64_t mid = (lo2 + hi2) >> 1;
            if (key[mid] <= k) lo2 = mid + 1; else hi2 = mid;
        }
        const int64_t below = neg_before[lo];
        const int64_t tied = neg_before[lo2] - below;
        acc += (double)below + 0.5 * (double)tied;
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) parts[blockIdx.x] = s[0];
}

__global__ void sum_partials(const double *__restrict__ parts, int n, double *__restrict__ out) {
    GOSH_DEP_WAIT();
    __shared__ double s[256];
    double t = 0.0;
    for (int i = threadIdx.x; i < n; i += 256) t += parts[i];
    s[threadIdx.x] = t;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s[0];
}

gosh_status check_csr(const gosh_csr *g) {
    GOSH_CHECK_ARG(g != nullptr, "csr is NULL");
    GOSH_CHECK_ARG(g->n >= 1 && g->n < (int64_t(1) << 31), "n must be in [1, 2^31) (got %lld)", (long long)g->n);
    GOSH_CHECK_ARG(g->rowptr != nullptr && g->col != nullptr, "csr pointers are NULL");
    return GOSH_OK;
}

template <typename F>
gosh_status by_dtype(gosh_dtype t, F &&f) {
    switch (t) {
    case GOSH_F32: f((float *)nullptr); return GOSH_OK;
    case GOSH_BF16: f((__nv_bfloat16 *)nullptr); return GOSH_OK;
    case GOSH_F16: f((__half *)nullptr); return GOSH_OK;
    }
    set_error("unknown dtype");
    return GOSH_ERR_INVALID_ARG;
}

struct EventTimer {
    cudaEvent_t a = nullptr, b = nullptr;
    cudaStream_t s;
    explicit EventTimer(cudaStream_t st) : s(st) {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        cudaEventRecord(a, s);
    }
    float stop() {
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        return ms;
    }
    ~EventTimer() {
        cudaEventDestroy(a);
        cudaEventDestroy(b);
    }
};

// A fixed set of events recorded on a stream and read after a synchronize.
struct EventList {
    std::vector<cudaEvent_t> e;
    std::vector<bool> rec;
    explicit EventList(int n) : e(n, nullptr), rec(n, false) {
        for (auto &x : e) cudaEventCreate(&x);
    }
    void record(int i, cudaStream_t s) {
        if (i < (int)e.size() && cudaEventRecord(e[i], s) == cudaSuccess) rec[i] = true;
    }
    // 0 unless both events were recorded
    double elapsed(int a, int b) const {
        float ms = 0.f;
        if (a < (int)e.size() && b < (int)e.size() && rec[a] && rec[b] &&
            cudaEventElapsedTime(&ms, e[a], e[b]) != cudaSuccess) {
            cudaGetLastError();
            ms = 0.f;
        }
        return ms;
    }
    ~EventList() {
        for (auto &x : e) cudaEventDestroy(x);
    }
};

bool is_device_ptr(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

// Epoch schedule of Sec. 3 (see gosh_level_epochs): with the |E| unit of
// Sec. 6 the total e is first converted to passes over V by the input
// graph's density nnz_0 / n_0 (rounded half up in integers); then a fraction
// p of it goes uniformly to the D levels and the rest geometrically (level i
// twice level i-1), levels >= 1 floored and level 0 the remainder.
gosh_status level_epochs(int e, double p, int D, int unit, const int64_t *n, const int64_t *nnz, int *out) {
    GOSH_CHECK_ARG(D >= 1 && out != nullptr, "need D >= 1 and an output array");
    GOSH_CHECK_ARG(e >= 0 && p >= 0 && p <= 1, "epochs must be >= 0 and p in [0, 1]");
    GOSH_CHECK_ARG(unit == 0 || unit == 1, "epoch_unit must be 0 (passes over V) or 1 (|E| draws)");
    if (unit == 1 && e > 0) {
        GOSH_CHECK_ARG(n != nullptr && nnz != nullptr, "epoch_unit 1 needs the size of G_0");
        GOSH_CHECK_ARG(n[0] >= 1 && nnz[0] >= 0, "bad size of G_0");
        // floor((2 e nnz + n) / (2 n)) without overflow: e < 2^31, nnz < 2^62
        const unsigned __int128 num = (unsigned __int128)2 * (unsigned)e * (uint64_t)nnz[0] + (uint64_t)n[0];
        const unsigned __int128 q = num / ((unsigned __int128)2 * (uint64_t)n[0]);
        GOSH_CHECK_ARG(q <= (unsigned __int128)INT32_MAX, "the pass count overflows");
        e = q < 1 ? 1 : (int)q;
    }
    if (D == 1) {
        out[0] = e;
        return GOSH_OK;
    }
    const double denom = std::pow(2.0, D) - 1.0;
    int rest = 0;
    for (int i = 1; i < D; ++i) {
        out[i] = (int)std::floor(p * e / D + (1.0 - p) * e * std::pow(2.0, i) / denom);
        rest += out[i];
    }
    out[0] = e - rest;
    return GOSH_OK;
}

gosh_status check_params(const gosh_params *p) {
    GOSH_CHECK_ARG(p != nullptr, "params is NULL");
    GOSH_CHECK_ARG(dtype_ok(p->dtype), "unknown dtype %d", (int)p->dtype);
    GOSH_CHECK_ARG(dim_ok(p->d), "d must be 8, 16, 32, 64 or 128 (got %d)", p->d);
    GOSH_CHECK_ARG(p->k >= 0 && p->k <= 15, "k must be in 0..15 (got %d)", p->k);
    GOSH_CHECK_ARG(p->lr > 0 && std::isfinite(p->lr), "lr must be positive");
    GOSH_CHECK_ARG(p->lr_floor >= 0 && p->lr_floor <= 1, "lr_floor must be in [0, 1]");
    GOSH_CHECK_ARG(p->mode == GOSH_HOGWILD || p->mode == GOSH_DETERMINISTIC, "unknown mode %d", (int)p->mode);
    GOSH_CHECK_ARG(p->epochs >= 0, "epochs must be >= 0");
    GOSH_CHECK_ARG(p->p >= 0 && p->p <= 1, "p must be in [0, 1]");
    GOSH_CHECK_ARG(p->shrink > 0 && p->shrink <= 1, "shrink must be in (0, 1]");
    GOSH_CHECK_ARG(p->epoch_overlap >= 0 && p->epoch_overlap <= 8, "epoch_overlap must be in 0..8 (got %d)",
                   p->epoch_overlap);
    GOSH_CHECK_ARG(p->overlap_min_vertices >= 0, "overlap_min_vertices must be >= 0");
    GOSH_CHECK_ARG(p->epoch_unit == 0 || p->epoch_unit == 1, "epoch_unit must be 0 or 1 (got %d)", p->epoch_unit);
    GOSH_CHECK_ARG(p->cooperative_epochs == 0 || p->cooperative_epochs == 1, "cooperative_epochs must be 0 or 1 (got %d)",
                   p->cooperative_epochs);
    return GOSH_OK;
}

gosh_status check_host_csr(const int64_t *rowptr, const int32_t *col, int64_t n, bool symmetric) {
    GOSH_CHECK_ARG(rowptr != nullptr && col != nullptr && n >= 1, "csr pointers are NULL or n < 1");
    GOSH_CHECK_ARG(rowptr[0] == 0, "rowptr[0] must be 0");
    for (int64_t v = 0; v < n; ++v)
        GOSH_CHECK_ARG(rowptr[v + 1] >= rowptr[v], "rowptr decreases at row %lld", (long long)v);
    for (int64_t v = 0; v < n; ++v) {
        const int64_t b = rowptr[v], e = rowptr[v + 1];
        for (int64_t q = b; q < e; ++q) {
            const int32_t u = col[q];
            GOSH_CHECK_ARG(u >= 0 && u < n, "row %lld: column %d out of range", (long long)v, (int)u);
            GOSH_CHECK_ARG(u != v, "row %lld: self-loop", (long long)v);
            GOSH_CHECK_ARG(q == b || col[q - 1] < u, "row %lld: columns not strictly ascending", (long long)v);
            if (symmetric)
                GOSH_CHECK_ARG(std::binary_search(col + rowptr[u], col + rowptr[u + 1], (int32_t)v),
                               "row %lld: entry %d has no reverse entry", (long long)v, (int)u);
        }
    }
    return GOSH_OK;
}

}  // namespace gosh

using namespace gosh;

extern "C" {

gosh_status gosh_set_allocator(gosh_alloc_fn alloc, gosh_free_fn free, void *ctx) {
    clear_error();
    GOSH_CHECK_ARG((alloc == nullptr) == (free == nullptr), "give both allocator functions or neither");
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc = alloc;
    g_free = free;
    g_alloc_ctx = alloc ? ctx : nullptr;
    return GOSH_OK;
}

gosh_status gosh_level_epochs(int epochs, double p, int D, int epoch_unit, const int64_t *n, const int64_t *nnz,
                              int *out) {
    clear_error();
    return level_epochs(epochs, p, D, epoch_unit, n, nnz, out);
}

gosh_status gosh_params_default(gosh_params *p) {
    if (!p) return GOSH_ERR_INVALID_ARG;
    memset(p, 0, sizeof(*p));
    p->d = 128;
    p->k = 3;
    p->lr = 0.035;
    p->lr_floor = 1e-4;
    p->epochs = 200;
    p->p = 0.3;
    p->threshold = 100;
    p->shrink = 0.8;
    p->max_levels = GOSH_MAX_LEVELS;
    p->dtype = GOSH_F32;
    p->mode = GOSH_HOGWILD;
    p->det_batch = 4096;
    p->seed = 20211020;
    p->validate = 0;
    p->projection = 0;
    p->mlp_hidden = 256;
    p->mlp_epochs = 1;
    p->mlp_lr = 1e-3;
    p->mlp_batch = 8192;
    p->mlp_max_rows = 32768;
    p->p_gpu = 3;
    p->s_gpu = 2;
    p->B = 5;
    p->large_parts = 0;
    p->persistent_small_levels = 0;
    p->vertices_per_warp = 0;
    p->walk_length = 8;
    p->walk_window = 3;
    p->large_serial = 0;
    p->large_evict = 0;
    p->overlap_min_vertices = 65536;
    p->epoch_overlap = 1;
    p->cooperative_epochs = 0;
    return GOSH_OK;
}

const char *gosh_last_error(void) { return g_error; }

unsigned long long gosh_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

unsigned long long gosh_release_host_buffers(void) {
    return (unsigned long long)(large_release_pinned() + walks_release_pinned());
}

gosh_status gosh_device_check(void *stream) {
    clear_error();
    cudaStream_t s = (cudaStream_t)stream;
    GOSH_TRY_CUDA(cudaStreamSynchronize(s));
    int raised = 0;
    GOSH_TRY(noalloc_take_error(&raised));
    if (raised) {
        set_error("a bounded device-side wait timed out in an earlier gosh_train_level_noalloc call");
        return GOSH_ERR_TIMEOUT;
    }
    int *w = device_error_word();
    if (!w) return GOSH_OK;
    int h = 0;
    GOSH_TRY_CUDA(cudaMemcpy(&h, w, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) {
        GOSH_TRY_CUDA(cudaMemset(w, 0, sizeof(int)));
        set_error("a bounded device-side wait timed out in an earlier asynchronous call");
        return GOSH_ERR_TIMEOUT;
    }
    return GOSH_OK;
}

gosh_status gosh_validate_csr(const gosh_csr *g, void *stream) {
    clear_error();
    GOSH_TRY(check_csr(g));
    GOSH_CHECK_ARG(g->on_device, "gosh_validate_csr needs a device CSR");
    cudaStream_t s = (cudaStream_t)stream;
    Scratch buf;
    GOSH_TRY(buf.alloc(16, s));
    unsigned *flags = buf.as<unsigned>();
    unsigned long long *first = reinterpret_cast<unsigned long long *>(buf.as<char>() + 8);
    GOSH_TRY_CUDA(cudaMemsetAsync(flags, 0, 4, s));
    GOSH_TRY_CUDA(cudaMemsetAsync(first, 0xff, 8, s));
    (validate_kernel<<<grid_for(g->n), 256, 0, s>>>(g->rowptr, g->col, g->n, flags, first), note_launch());
    unsigned hf = 0;
    unsigned long long hv = 0;
    GOSH_TRY_CUDA(cudaMemcpyAsync(&hf, flags, 4, cudaMemcpyDeviceToHost, s));
    GOSH_TRY_CUDA(cudaMemcpyAsync(&hv, first, 8, cudaMemcpyDeviceToHost, s));
    GOSH_TRY_CUDA(cudaStreamSynchronize(s));
    if (hf) {
        set_error("invalid CSR (first bad row %llu):%s%s%s%s%s", hv, hf & kBadRowptr ? " row pointer" : "",
                  hf & kBadRange ? " id out of range" : "", hf & kUnsorted ? " row not strictly ascending" : "",
                  hf & kSelfLoop ? " self-loop" : "", hf & kAsym ? " not symmetric" : "");
        return GOSH_ERR_INVALID_ARG;
    }
    return GOSH_OK;
}

gosh_status gosh_coarsen(const gosh_csr *g0, int threshold, double shrink, int max_levels, void *stream,
                         gosh_hierarchy **out) {
    clear_error();
    GOSH_TRY(check_csr(g0));
    GOSH_CHECK_ARG(out != nullptr, "out is NULL");
    GOSH_CHECK_ARG(g0->on_device, "gosh_coarsen needs a device CSR");
    GOSH_CHECK_ARG(shrink > 0 && shrink <= 1, "shrink must be in (0, 1]");
    return coarsen_impl(g0, threshold, shrink, max_levels, (cudaStream_t)stream, out);
}

gosh_status gosh_coarsen_batch(const gosh_csr *graphs, int n_graphs, int threshold, double shrink, int max_levels,
                               void *stream, gosh_hierarchy **out) {
    clear_error();
    GOSH_CHECK_ARG(out != nullptr && graphs != nullptr && n_graphs >= 1, "bad graphs / n_graphs / out");
    for (int g = 0; g < n_graphs; ++g) {
        out[g] = nullptr;
        GOSH_TRY(check_csr(&graphs[g]));
        GOSH_CHECK_ARG(graphs[g].on_device && graphs[g].n >= 1, "graph %d: needs a device CSR with n >= 1", g);
    }
    GOSH_CHECK_ARG(shrink > 0 && shrink <= 1, "shrink must be in (0, 1]");
    std::vector<gosh_hierarchy *> hs;
    GOSH_TRY(coarsen_batch_impl(graphs, n_graphs, threshold, shrink, max_levels, (cudaStream_t)stream, hs));
    for (int g = 0; g < n_graphs; ++g) out[g] = hs[g];
    return GOSH_OK;
}

int gosh_hierarchy_levels(const gosh_hierarchy *h) { return h ? (int)h->n.size() : 0; }

gosh_status gosh_hierarchy_level(const gosh_hierarchy *h, int i, gosh_csr *g_i, const int32_t **map_i) {
    clear_error();
    GOSH_CHECK_ARG(h != nullptr && i >= 0 && i < (int)h->n.size(), "level %d out of range", i);
    if (g_i) {
        g_i->n = h->n[i];
        g_i->rowptr = h->rowptr[i];
        g_i->col = h->col[i];
        g_i->on_device = 1;
    }
    if (map_i) *map_i = i < (int)h->map.size() ? h->map[i] : nullptr;
    return GOSH_OK;
}

gosh_status gosh_hierarchy_sizes(const gosh_hierarchy *h, int i, int64_t *n, int64_t *nnz) {
    clear_error();
    GOSH_CHECK_ARG(h != nullptr && i >= 0 && i < (int)h->n.size(), "level %d out of range", i);
    if (n) *n = h->n[i];
    if (nnz) *nnz = h->nnz[i];
    return GOSH_OK;
}

gosh_status gosh_hierarchy_copy_level(const gosh_hierarchy *h, int i, int64_t *rowptr, int32_t *col, int32_t *map,
                                      void *stream) {
    clear_error();
    GOSH_CHECK_ARG(h != nullptr && i >= 0 && i < (int)h->n.size(), "level %d out of range", i);
    cudaStream_t s = (cudaStream_t)stream;
    if (rowptr)
        GOSH_TRY_CUDA(cudaMemcpyAsync(rowptr, h->rowptr[i], sizeof(int64_t) * (h->n[i] + 1), cudaMemcpyDeviceToHost, s));
    if (col && h->nnz[i] > 0)
        GOSH_TRY_CUDA(cudaMemcpyAsync(col, h->col[i], sizeof(int32_t) * h->nnz[i], cudaMemcpyDeviceToHost, s));
    if (map && i < (int)h->map.size())
        GOSH_TRY_CUDA(cudaMemcpyAsync(map, h->map[i], sizeof(int32_t) * h->n[i], cudaMemcpyDeviceToHost, s));
    GOSH_TRY_CUDA(cudaStreamSynchronize(s));
    return GOSH_OK;
}

void gosh_hierarchy_free(gosh_hierarchy *h) { delete h; }

gosh_status gosh_init_embedding(void *M, int64_t n, int d, gosh_dtype dtype, int level, uint64_t seed,
                                uint64_t graph_id, void *stream) {
    clear_error();
    GOSH_CHECK_ARG(M != nullptr && n >= 0, "bad M / n");
    GOSH_CHECK_ARG(dtype_ok(dtype) && dim_ok(d), "bad d / dtype");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t work = n * ((d + 3) / 4);
    GOSH_TRY(by_dtype(dtype, [&](auto *tp) {
        using T = std::remove_pointer_t<decltype(tp)>;
        launch_dep(init_kernel<T>, grid_for(work), 256, 0, s, static_cast<T *>(M), n, d, (uint32_t)level, seed, graph_id);
    }));
    GOSH_TRY_CUDA(cudaGetLastError());
    return GOSH_OK;
}

gosh_status gosh_train_level(const gosh_csr *g, void *M, int level, int epochs, const gosh_params *params,
                             void *stream, double *loss_per_epoch, unsigned long long *n_updates) {
    clear_error();
    GOSH_TRY(check_csr(g));
    GOSH_TRY(check_params(params));
    GOSH_CHECK_ARG(g->on_device, "gosh_train_level needs a device CSR");
    GOSH_CHECK_ARG(M != nullptr && aligned16(M), "M must be a 16-byte aligned device pointer");
    GOSH_CHECK_ARG(epochs >= 0 && level >= 0, "bad epochs / level");
    return train_level_impl(g, M, level, epochs, params, (cudaStream_t)stream, loss_per_epoch, n_updates);
}

}  // extern "C"

namespace gosh {
namespace {
// Element i takes the half (i & 1) of the 32-bit hash of pair i / 2, the
// assignment Store<T>::pack uses for a row's 16-byte vectors.
__global__ void round_sr_kernel(const float *__restrict__ x, uint16_t *__restrict__ out, int64_t n, uint32_t seed,
                                int half) {
    GOSH_DEP_WAIT();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t r = sr_pair_bits(seed + (uint32_t)(i >> 1));
        const uint32_t r16 = (i & 1) ? (r >> 16) : (r & 0xffffu);
        out[i] = (uint16_t)(half ? f16_sr_bits(x[i], r16) : bf16_sr_bits(x[i], r16));
    }
}
}  // namespace
}  // namespace gosh

extern "C" {

gosh_status gosh_round_stochastic(const float *x, void *out, int64_t n, gosh_dtype dtype, uint64_t seed,
                                  void *stream) {
    clear_error();
    GOSH_CHECK_ARG(x && out && n >= 0, "NULL pointer or negative n");
    GOSH_CHECK_ARG(dtype == GOSH_BF16 || dtype == GOSH_F16, "dtype must be GOSH_BF16 or GOSH_F16");
    if (n == 0) return GOSH_OK;
    const uint32_t s32 = (uint32_t)seed ^ mix32((uint32_t)(seed >> 32));
    launch_dep(round_sr_kernel, grid_for(n), 256, 0, (cudaStream_t)stream, x, static_cast<uint16_t *>(out), n, s32,
                                                                    dtype == GOSH_F16 ? 1 : 0);
    GOSH_TRY_CUDA(cudaGetLastError());
    return GOSH_OK;
}

gosh_status gosh_project(const void *M_coarse, int64_t n_coarse, const int32_t *map, void *M_fine, int64_t n_fine,
                         int d, gosh_dtype dtype, void *stream) {
    clear_error();
    GOSH_CHECK_ARG(M_coarse && M_fine && map, "NULL pointer");
    GOSH_CHECK_ARG(aligned16(M_coarse) && aligned16(M_fine), "M must be 16-byte aligned");
    GOSH_CHECK_ARG(n_coarse >= 1 && n_fine >= 0, "bad sizes");
    GOSH_CHECK_ARG(dtype_ok(dtype) && dim_ok(d), "bad d / dtype");
    cudaStream_t s = (cudaStream_t)stream;
    const int vecs = (int)(d * dtype_size(dtype) / 16);
    launch_dep(project_copy_kernel, grid_for(n_fine * vecs), 256, 0, s, static_cast<const uint4 *>(M_coarse), map,
                                                                static_cast<uint4 *>(M_fine), n_fine, vecs);
    GOSH_TRY_CUDA(cudaGetLastError());
    return GOSH_OK;
}

gosh_status gosh_pair_scores(const void *M, int d, gosh_dtype dtype, const int32_t *pairs, int64_t npairs, float *out,
                             void *stream) {
    clear_error();
    GOSH_CHECK_ARG(M && pairs && out && npairs >= 0, "bad arguments");
    GOSH_CHECK_ARG(dtype_ok(dtype) && dim_ok(d), "bad d / dtype");
    cudaStream_t s = (cudaStream_t)stream;
    if (npairs == 0) return GOSH_OK;
    GOSH_TRY(by_dtype(dtype, [&](auto *tp) {
        using T = std::remove_pointer_t<decltype(tp)>;
        launch_pair_scores<T>(M, d, pairs, npairs, out, s);
    }));
    GOSH_TRY_CUDA(cudaGetLastError());
    return GOSH_OK;
}

gosh_status gosh_link_auc(const void *M, int d, gosh_dtype dtype, const int32_t *pos, int64_t npos,
                          const int32_t *neg, int64_t nneg, void *stream, double *auc) {
    clear_error();
    GOSH_CHECK_ARG(auc != nullptr, "auc is NULL");
    GOSH_CHECK_ARG(npos > 0 && nneg > 0, "need positive and negative pairs");
    GOSH_CHECK_ARG(npos + nneg < (int64_t(1) << 32), "too many pairs");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = npos + nneg;
    Scratch score, key, idx, flag, before, parts, out;
    GOSH_TRY(score.alloc(sizeof(float) * n, s));
    GOSH_TRY(key.alloc(sizeof(uint32_t) * n, s));
    GOSH_TRY(idx.alloc(sizeof(uint32_t) * n, s));
    GOSH_TRY(flag.alloc(n, s));
    GOSH_TRY(before.alloc(sizeof(int64_t) * (n + 1), s));
    const int grid = grid_for(n);
    GOSH_TRY(parts.alloc(sizeof(double) * grid, s));
    GOSH_TRY(out.alloc(sizeof(double), s));
    GOSH_TRY(gosh_pair_scores(M, d, dtype, pos, npos, score.as<float>(), stream));
    GOSH_TRY(gosh_pair_scores(M, d, dtype, neg, nneg, score.as<float>() + npos, stream));
    launch_dep(score_keys, grid, 256, 0, s, score.as<float>(), n, key.as<uint32_t>(), idx.as<uint32_t>());
    GOSH_TRY(radix_sort_u32(key.as<uint32_t>(), idx.as<uint32_t>(), n, 0, 32, s));
    launch_dep(neg_flags, grid, 256, 0, s, idx.as<uint32_t>(), n, npos, flag.as<uint8_t>());
    GOSH_TRY(scan_exclusive_u8_to_i64(flag.as<uint8_t>(), before.as<int64_t>(), n, before.as<int64_t>() + n, s));
    launch_dep(auc_partials, grid, 256, 0, s, key.as<uint32_t>(), idx.as<uint32_t>(), before.as<int64_t>(), n, npos,
                                      parts.as<double>());
    launch_dep(sum_partials, 1, 256, 0, s, parts.as<double>(), grid, out.as<double>());
    double U = 0.0;
    GOSH_TRY_CUDA(cudaMemcpyAsync(&U, out.ptr, sizeof(double), cudaMemcpyDeviceToHost, s));
    GOSH_TRY_CUDA(cudaStreamSynchronize(s));
    *auc = U / ((double)npos * (double)nneg);
    return GOSH_OK;
}

gosh_status gosh_embed(const gosh_csr *g0, const gosh_params *params, void *M0_out, void *stream, gosh_stats *stats) {
    clear_error();
    const auto t_start = std::chrono::steady_clock::now();
    GOSH_TRY(check_csr(g0));
    GOSH_TRY(check_params(params));
    GOSH_CHECK_ARG(M0_out != nullptr, "M0_out is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const gosh_params &p = *params;
    const size_t row_bytes = (size_t)p.d * dtype_size(p.dtype);

    // inputs on the device
    gosh_csr g = *g0;
    Scratch rp_dev, col_dev;
    if (!g0->on_device) {
        int64_t nnz = g0->rowptr[g0->n];
        GOSH_CHECK_ARG(nnz >= 0, "rowptr[n] < 0");
        GOSH_TRY(rp_dev.alloc(sizeof(int64_t) * (g0->n + 1), s));
        GOSH_TRY(col_dev.alloc(sizeof(int32_t) * (nnz > 0 ? nnz : 1), s));
        GOSH_TRY_CUDA(cudaMemcpyAsync(rp_dev.ptr, g0->rowptr, sizeof(int64_t) * (g0->n + 1), cudaMemcpyHostToDevice, s));
        if (nnz > 0)
            GOSH_TRY_CUDA(cudaMemcpyAsync(col_dev.ptr, g0->col, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, s));
        g.rowptr = rp_dev.as<int64_t>();
        g.col = col_dev.as<int32_t>();
        g.on_device = 1;
    }
    if (p.validate) GOSH_TRY(gosh_validate_csr(&g, stream));

    // Alg. 4
    gosh_hierarchy *h = nullptr;
    double coarsen_ms = 0.0;
    if (p.max_levels == 1) {
        h = new gosh_hierarchy();
        int64_t nnz = 0;
        GOSH_TRY_CUDA(cudaMemcpyAsync(&nnz, g.rowptr + g.n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        GOSH_TRY_CUDA(cudaStreamSynchronize(s));
        h->n.push_back(g.n);
        h->nnz.push_back(nnz);
        h->rowptr.push_back(const_cast<int64_t *>(g.rowptr));
        h->col.push_back(const_cast<int32_t *>(g.col));
    } else {
        EventTimer t(s);
        GOSH_TRY(coarsen_impl(&g, p.threshold, p.shrink, p.max_levels, s, &h));
        coarsen_ms = t.stop();
    }
    struct Guard {
        gosh_hierarchy *h;
        ~Guard() { delete h; }
    } guard{h};
    const int D = (int)h->n.size();
    std::vector<int> ep(D);
    GOSH_TRY(level_epochs(p.epochs, p.p, D, p.epoch_unit, h->n.data(), h->nnz.data(), ep.data()));

    // embedding buffers: even levels in the output (or a device copy of it), odd levels in tmp
    const bool out_dev = is_device_ptr(M0_out);
    Scratch out_buf, tmp_buf, counter;
    void *even = M0_out;
    if (!out_dev) {
        GOSH_TRY(out_buf.alloc(row_bytes * g.n, s));
        even = out_buf.ptr;
    } else {
        GOSH_CHECK_ARG(aligned16(M0_out), "M0_out must be 16-byte aligned");
    }
    if (D > 1) GOSH_TRY(tmp_buf.alloc(row_bytes * h->n[1], s));
    auto buf = [&](int i) { return (i % 2 == 0) ? even : tmp_buf.ptr; };
    GOSH_TRY(counter.alloc(sizeof(unsigned long long), s));
    GOSH_TRY_CUDA(cudaMemsetAsync(counter.ptr, 0, sizeof(unsigned long long), s));

    // per-level events, read once at the end so that no level waits for the host
    EventList ev(stats ? 2 * D + 1 : 0);
    // On request (persistent_small_levels), the small levels (|V_i| <= 2^17)
    // of a lock-free, copy-projection run go through one persistent launch;
    // the large levels keep one launch per epoch with the best kernel.
    int top = D - 1;  // highest level still to train below
    const bool persist = p.persistent_small_levels && p.mode == GOSH_HOGWILD && p.projection == 0 && D > 1 &&
                         (p.dtype == GOSH_F32 || p.dtype == GOSH_BF16) && p.lanes_per_row == 0 &&
                         p.samples_per_pass == 0;
    int lowest = D;
    if (persist)
        while (lowest > 1 && h->n[lowest - 1] <= (int64_t(1) << 17)) --lowest;
    if (persist && lowest <= D - 1) {
        std::vector<void *> bufs(D);
        for (int i = 0; i < D; ++i) bufs[i] = buf(i);
        ev.record(2 * (D - 1) + 1, s);
        GOSH_TRY(persistent_levels(h, bufs, lowest, p, counter.as<unsigned long long>(), s));
        ev.record(2 * lowest, s);
        GOSH_TRY(gosh_project(buf(lowest), h->n[lowest], h->map[lowest - 1], buf(lowest - 1), h->n[lowest - 1], p.d,
                              p.dtype, stream));
        top = lowest - 1;
    } else {
        GOSH_TRY(gosh_init_embedding(buf(D - 1), h->n[D - 1], p.d, p.dtype, D - 1, p.seed, p.graph_id, stream));
    }
    // learned projection: one network for the whole run, trained after each
    // level i < D-1 on (features from M_{i+1}, trained M_i) before M_{i+1}'s
    // buffer is reused for M_{i-1}
    struct MlpGuard {
        gosh_mlp *m = nullptr;
        ~MlpGuard() { gosh_mlp_free(m); }
    } mlp;
    if (p.projection == 1 && D > 1)
        GOSH_TRY(gosh_mlp_create(p.d, p.mlp_hidden > 0 ? p.mlp_hidden : 256, p.seed ^ 0x6d6c70ull, &mlp.m));
    for (int i = top; i >= 0; --i) {
        gosh_csr gi{h->n[i], h->rowptr[i], h->col[i], 1};
        ev.record(2 * i + 1, s);
        GOSH_TRY(train_level_impl(&gi, buf(i), i, ep[i], &p, s, nullptr, counter.as<unsigned long long>()));
        ev.record(2 * i, s);
        if (mlp.m && i <= D - 2 && i > 0)
            GOSH_TRY(mlp_train(mlp.m, &gi, h->map[i], buf(i + 1), buf(i), p.dtype, p.mlp_epochs > 0 ? p.mlp_epochs : 1,
                               p.mlp_lr > 0 ? p.mlp_lr : 1e-3, p.mlp_batch > 0 ? p.mlp_batch : 8192, p.mlp_max_rows,
                               s, nullptr, true));
        if (i > 0) {
            gosh_csr gf{h->n[i - 1], h->rowptr[i - 1], h->col[i - 1], 1};
            // the projection keeps the feature rows level i-1's training will use
            // (same table M_i, still unchanged then)
            if (mlp.m && i <= D - 2)
                GOSH_TRY(mlp_project(mlp.m, buf(i), h->map[i - 1], &gf, buf(i - 1), p.dtype, s,
                                     i - 1 > 0 ? (p.mlp_max_rows > 0 ? p.mlp_max_rows : -1) : 0));
            else
                GOSH_TRY(gosh_project(buf(i), h->n[i], h->map[i - 1], buf(i - 1), h->n[i - 1], p.d, p.dtype, stream));
        }
    }
    std::vector<double> train_ms(D, 0.0);
    double project_ms = 0.0;
    if (!out_dev)
        GOSH_TRY_CUDA(cudaMemcpyAsync(M0_out, even, row_bytes * g.n, cudaMemcpyDeviceToHost, s));
    unsigned long long updates = 0;
    GOSH_TRY_CUDA(cudaMemcpyAsync(&updates, counter.ptr, sizeof(updates), cudaMemcpyDeviceToHost, s));
    GOSH_TRY_CUDA(cudaStreamSynchronize(s));
    GOSH_TRY(gosh_device_check(stream));
    if (stats) {
        for (int i = 0; i < D; ++i) {
            train_ms[i] = ev.elapsed(2 * i + 1, 2 * i);
            if (i > 0) project_ms += ev.elapsed(2 * i, 2 * i - 1);
        }
        memset(stats, 0, sizeof(*stats));
        stats->levels = D;
        for (int i = 0; i < D && i < GOSH_MAX_LEVELS; ++i) {
            stats->n[i] = h->n[i];
            stats->nnz[i] = h->nnz[i];
            stats->epochs[i] = ep[i];
            stats->train_ms[i] = train_ms[i];
        }
        stats->coarsen_ms = coarsen_ms;
        stats->project_ms = project_ms;
        stats->updates = updates;
        stats->total_ms =
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    }
    return GOSH_OK;
}

}  // extern "C"
