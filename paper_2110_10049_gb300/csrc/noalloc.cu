// gosh_train_level_noalloc: the lock-free training step with its per-epoch
// loss monitor, for callers that cannot allocate device memory.
//
// gosh_train_level takes its scratch (one FP64 partial loss sum per thread
// block) from cudaMallocAsync.  Some callers cannot allow that: code running
// inside a host framework that owns every byte of device memory through its
// own arena, services that run under a fixed memory budget, or callers that
// must never let the library touch the allocator (cudaMalloc and cudaFree can
// synchronise the device).  This variant keeps that scratch in a file-scope
// device array instead, so it allocates nothing; the caller still passes M,
// the loss and the counter buffers.
#include <mutex>

#include "train.cuh"

namespace gosh {

gosh_status pick_train_kernel(gosh_dtype dtype, int d, int k, int mode, int lanes, int pass, int64_t n,
                              const TrainKernel **out);
int train_mode(const gosh_params *p);
int tile_vertices(const gosh_params *p, int64_t n, int lanes, int pass);

namespace {

// At most this many thread blocks may contribute a partial loss sum (32 KB).
// A launch uses at most (SMs x resident blocks per SM) of the chosen kernel:
// 152 x 8 = 1216 for the 256-thread register kernels on a GB300, and at most
// 152 x 16 = 2432 for the 128-thread TMA-staged ones (2048 threads per SM);
// the entry point checks the grid against this size before any launch.
constexpr int kNoAllocMaxPartials = 4096;
static_assert(kNoAllocMaxPartials >= 152 * (2048 / 128), "static scratch below the GB300 worst case");

// Shared by every call on a device and never cleared: each launch writes the
// slots [0, grid) before the finalising kernel reads them.
static __device__ __align__(256) double g_noalloc_partials[kNoAllocMaxPartials];

// Raised (set to 1) by a training kernel whose bounded wait gave up; read and
// cleared by gosh_device_check through noalloc_take_error.
static __device__ __align__(256) int g_noalloc_err;

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_partials_ptr[kMaxDevices] = {nullptr};
int *g_err_ptr[kMaxDevices] = {nullptr};

// Device addresses of g_noalloc_partials and g_noalloc_err on the current
// device.  In host code the symbol names are only host-side stand-ins, so the
// addresses are looked up once per device with cudaGetSymbolAddress (this
// first lookup may load the library's device code, so make the first call on
// a device before any stream capture begins).
gosh_status scratch_on_current_device(double **partials, int **err) {
    int dev = 0;
    GOSH_TRY_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("device %d out of range for the static scratch table", dev);
        return GOSH_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_partials_ptr[dev]) {
        void *p = nullptr, *q = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e == cudaSuccess) e = cudaGetSymbolAddress(&q, g_noalloc_err);
        if (e != cudaSuccess || p == nullptr || q == nullptr) {
            set_error("cudaGetSymbolAddress(static scratch) on device %d: %s", dev, cudaGetErrorString(e));
            return GOSH_ERR_CUDA;
        }
        g_err_ptr[dev] = static_cast<int *>(q);
        g_partials_ptr[dev] = static_cast<double *>(p);
    }
    *partials = g_partials_ptr[dev];
    *err = g_err_ptr[dev];
    return GOSH_OK;
}

// Sum of the grid's partials into out (fixed order, one block).
__global__ void noalloc_loss_finalize(const double *__restrict__ parts, int nparts, double *__restrict__ out) {
    GOSH_DEP_WAIT();
    __shared__ double s[256];
    double t = 0.0;
    for (int i = threadIdx.x; i < nparts; i += 256) t += parts[i];
    s[threadIdx.x] = t;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s[0];
}

}  // namespace

// Reads and clears the static error word of the current device (only if an
// allocation-free call has run there; no allocation either way).  *raised is
// set to 1 if a bounded wait of such a call gave up since the last read.
gosh_status noalloc_take_error(int *raised) {
    *raised = 0;
    int dev = 0;
    GOSH_TRY_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return GOSH_OK;
    int *w = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        w = g_err_ptr[dev];
    }
    if (!w) return GOSH_OK;
    int h = 0;
    GOSH_TRY_CUDA(cudaMemcpy(&h, w, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) {
        GOSH_TRY_CUDA(cudaMemset(w, 0, sizeof(int)));
        *raised = 1;
    }
    return GOSH_OK;
}

}  // namespace gosh

using namespace gosh;

extern "C" gosh_status gosh_train_level_noalloc(const gosh_csr *g, void *M, int level, int epochs,
                                                const gosh_params *p, void *stream, double *loss_per_epoch,
                                                unsigned long long *n_updates) {
    clear_error();
    GOSH_CHECK_ARG(g != nullptr && p != nullptr, "NULL graph or params");
    GOSH_CHECK_ARG(g->on_device && g->n >= 1 && g->rowptr && g->col, "needs a device CSR with n >= 1");
    GOSH_CHECK_ARG(M != nullptr && ((uintptr_t)M & 15u) == 0, "M must be a 16-byte aligned device pointer");
    GOSH_CHECK_ARG(epochs >= 0 && level >= 0, "bad epochs / level");
    GOSH_CHECK_ARG(p->d == 8 || p->d == 16 || p->d == 32 || p->d == 64 || p->d == 128,
                   "d must be 8, 16, 32, 64 or 128 (got %d)", p->d);
    GOSH_CHECK_ARG(p->k >= 0 && p->k <= kMaxK, "k must be in 0..%d (got %d)", kMaxK, p->k);
    GOSH_CHECK_ARG(p->dtype == GOSH_F32 || p->dtype == GOSH_BF16 || p->dtype == GOSH_F16, "unknown dtype");
    if (p->mode != GOSH_HOGWILD) {
        set_error("gosh_train_level_noalloc serves GOSH_HOGWILD only: the deterministic mode needs scratch "
                  "proportional to det_batch; use gosh_train_level");
        return GOSH_ERR_UNSUPPORTED;
    }
    const TrainKernel *kern = nullptr;
    GOSH_TRY(pick_train_kernel(p->dtype, p->d, p->k, train_mode(p), p->lanes_per_row, p->samples_per_pass, g->n,
                               &kern));
    if (epochs == 0) return GOSH_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = g->n;
    const int cap_blocks = num_sms() * kern->blocks_per_sm;
    const int64_t want = ceil_div(ceil_div(n, tile_vertices(p, n, kern->lanes, kern->pass)), kern->warps);
    const int grid = (int)(want < cap_blocks ? (want > 0 ? want : 1) : cap_blocks);
    if (loss_per_epoch && grid > kNoAllocMaxPartials) {
        set_error("gosh_train_level_noalloc: %d thread blocks exceed the static scratch of %d partial loss sums",
                  grid, kNoAllocMaxPartials);
        return GOSH_ERR_INVALID_ARG;
    }
    double *partials = nullptr;
    int *err = nullptr;
    GOSH_TRY(scratch_on_current_device(&partials, &err));
    if (!loss_per_epoch) partials = nullptr;
    TrainArgs a{};
    a.rowptr = g->rowptr;
    a.col = g->col;
    a.M = M;
    a.n = n;
    a.k = p->k;
    a.seed = p->seed;
    a.graph = p->graph_id;
    a.level = (uint32_t)level;
    a.n_updates = n_updates;
    a.loss_partials = partials;
    a.err = err;
    a.src_begin = 0;
    a.src_end = n;
    a.tile = tile_vertices(p, n, kern->lanes, kern->pass);
    for (int j = 0; j < epochs; ++j) {
        const double f = 1.0 - (double)j / (double)epochs;
        a.lr = (float)(p->lr * (f > p->lr_floor ? f : p->lr_floor));
        a.epoch = (uint32_t)j;
        kern->launch(a, grid, s);
        if (loss_per_epoch) launch_dep(noalloc_loss_finalize, 1, 256, 0, s, partials, grid, loss_per_epoch + j);
    }
    GOSH_TRY_CUDA(cudaGetLastError());
    return GOSH_OK;
}
