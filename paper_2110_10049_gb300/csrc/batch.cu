// Many graphs (and all their coarse levels) trained in one persistent launch.
//
// Every graph's schedule is a list of phases: initialise its coarsest
// embedding, then for each level i = D-1..0 one phase per epoch (Alg. 3) and,
// for i > 0, one copy-projection phase (Alg. 2).  Phases of one graph run in
// order (epochs are serialised, Sec. 3.1); phases of different graphs run
// concurrently.  Work items are chunks of 32 * tiles sources (or rows).
//
// Scheduling, per graph, in device memory:
//   word = (phase << 40) | items taken   (one atomicAdd grabs an item and names its phase)
//   done = items of the current phase completed
// The warp that completes the last item of a phase resets `done`, then
// publishes the next phase by exchanging `word`; writes of the finished
// phase are ordered before that by __threadfence (release), and a warp that
// grabs an item of the next phase fences before reading (acquire).  Idle
// warps move to other graphs; a warp that finds no work for kIdleNs
// nanoseconds sets the error flag and leaves (bounded wait).
//
// The launch (counter resets + kernel) is captured once in a CUDA graph and
// replayed.  An autotuner times the compiled (lanes per row, samples per
// pass, sources per work item) variants on the batch and keeps the fastest.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "hierarchy.cuh"
#include "train_kernels.cuh"

namespace gosh {

gosh_status coarsen_impl(const gosh_csr *g0, int threshold, double shrink, int max_levels, cudaStream_t s,
                         gosh_hierarchy **out);
gosh_status coarsen_batch_impl(const gosh_csr *graphs, int G, int threshold, double shrink, int max_levels,
                               cudaStream_t s, std::vector<gosh_hierarchy *> &out);

namespace {

enum : int { kPhaseInit = 0, kPhaseTrain = 1, kPhaseProject = 2 };
constexpr unsigned long long kTakenMask = (1ull << 40) - 1;
constexpr unsigned long long kIdleNs = 4000000000ull;  // 4 s without finding work

struct Phase {
    int type;
    int level;
    uint32_t epoch;
    float lr;
    int64_t n;      // sources (train) or rows (init, project)
    int64_t items;  // work items
    const int64_t *rowptr;
    const int32_t *col;
    void *M;            // trained / written matrix
    const void *Msrc;   // projection source (coarse level)
    const int32_t *map; // projection map
};

struct GraphCtl {
    unsigned long long word;
    unsigned long long done;
};

struct BatchArgs {
    const Phase *phases;
    const int *first;
    const int *count;
    GraphCtl *ctl;
    int G;
    int k;
    int d;
    uint64_t seed, graph_base;
    int rows_per_item;
    unsigned long long *graphs_done;
    int *err;
    unsigned long long *n_updates;
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

template <typename T>
__device__ __forceinline__ T cvt_store(float x);
template <> __device__ __forceinline__ float cvt_store<float>(float x) { return x; }
template <> __device__ __forceinline__ __nv_bfloat16 cvt_store<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }

template <typename T, int D>
__device__ void init_rows(const Phase &ph, int64_t r0, int64_t r1, uint64_t seed, uint64_t graph, int lane) {
    T *M = static_cast<T *>(ph.M);
    constexpr int NQ = D / 4;
    for (int64_t i = r0 * NQ + lane; i < r1 * NQ; i += 32) {
        const int64_t v = i / NQ;
        const int q = (int)(i % NQ);
        const Philox4 w = philox4x64_10((uint64_t)v, (uint64_t)q, (uint64_t)ph.level, kTagInit, seed, graph);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const double unit = (double)(w.w[j] >> 11) * 0x1.0p-53;
            M[v * D + 4 * q + j] = cvt_store<T>((float)((unit - 0.5) / (double)D));
        }
    }
}

template <typename T, int D>
__device__ void project_rows(const Phase &ph, int64_t r0, int64_t r1, int lane) {
    constexpr int V = D * (int)sizeof(T) / 16;
    const uint4 *src = static_cast<const uint4 *>(ph.Msrc);
    uint4 *dst = static_cast<uint4 *>(ph.M);
    for (int64_t i = r0 * V + lane; i < r1 * V; i += 32) {
        const int64_t v = i / V;
        const int q = (int)(i % V);
        dst[i] = __ldcg(src + (int64_t)__ldg(ph.map + v) * V + q);
    }
}

template <typename T, int D, int L, int P>
__global__ void __launch_bounds__(kTrainWarps * 32) batch_kernel(BatchArgs b) {
    GOSH_DEP_WAIT();
    constexpr int MODE = kModeRed;  // atomic row changes (16-bit: stochastically rounded)
    __shared__ int32_t s_u[kTrainWarps][32 * kSlotStride];
    __shared__ uint32_t s_sr[kTrainWarps][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int g = (int)(((int64_t)blockIdx.x * kTrainWarps + warp) % b.G);
    int misses = 0;
    unsigned backoff = 32;
    unsigned long long idle_since = 0;
    double loss = 0.0;
    unsigned long long applied = 0;
    volatile unsigned long long *vdone = b.graphs_done;
    while (*vdone < (unsigned long long)b.G) {
        GraphCtl *c = &b.ctl[g];
        const int first = b.first[g], count = b.count[g];
        unsigned long long got = ~0ull;
        if (lane == 0) {
            const unsigned long long w = *reinterpret_cast<volatile unsigned long long *>(&c->word);
            const int ph = (int)(w >> 40);
            if (ph < count && (w & kTakenMask) < (unsigned long long)b.phases[first + ph].items)
                got = atomicAdd(&c->word, 1ull);
        }
        got = __shfl_sync(0xffffffffu, got, 0);
        bool worked = false;
        if (got != ~0ull) {
            const int ph = (int)(got >> 40);
            const int64_t item = (int64_t)(got & kTakenMask);
            if (ph < count && item < b.phases[first + ph].items) {
                __threadfence();  // acquire: the previous phase's writes are visible
                const Phase &P_ = b.phases[first + ph];
                const int64_t r0 = item * b.rows_per_item;
                const int64_t r1 = r0 + b.rows_per_item < P_.n ? r0 + b.rows_per_item : P_.n;
                const uint64_t gid = b.graph_base + (uint64_t)g;
                if (P_.type == kPhaseTrain) {
                    TrainArgs a{};
                    a.rowptr = P_.rowptr;
                    a.col = P_.col;
                    a.M = P_.M;
                    a.n = P_.n;
                    a.k = b.k;
                    a.seed = b.seed;
                    a.graph = gid;
                    a.level = (uint32_t)P_.level;
                    a.epoch = P_.epoch;
                    a.lr = P_.lr;
                    a.src_begin = r0;
                    a.src_end = r1;
                    a.tile = 32;
                    for (int64_t v0 = r0; v0 < r1; v0 += 32)
                        train_tile<T, D, L, P, MODE>(a, v0, s_u[warp], s_sr[warp], loss, applied);
                } else if (P_.type == kPhaseInit) {
                    init_rows<T, D>(P_, r0, r1, b.seed, gid, lane);
                } else {
                    project_rows<T, D>(P_, r0, r1, lane);
                }
                __syncwarp();
                if (lane == 0) {
                    __threadfence();  // release this item's writes
                    const unsigned long long d = atomicAdd(&c->done, 1ull);
                    if (d + 1 == (unsigned long long)P_.items) {
                        c->done = 0;
                        __threadfence();
                        atomicExch(&c->word, (unsigned long long)(ph + 1) << 40);
                        if (ph + 1 == count) atomicAdd(b.graphs_done, 1ull);
                    }
                }
                __syncwarp();
                worked = true;
            }
        }
        if (worked) {
            misses = 0;
            idle_since = 0;
            backoff = 32;
            continue;
        }
        g = g + 1 == b.G ? 0 : g + 1;
        if (++misses >= b.G) {  // a full sweep found nothing: back off (exponentially), bounded
            misses = 0;
            const unsigned long long now = global_ns();
            if (idle_since == 0) idle_since = now;
            else if (now - idle_since > kIdleNs) {
                if (lane == 0) atomicExch(b.err, 1);
                break;
            }
            __nanosleep(backoff);
            backoff = backoff < 2048 ? backoff * 2 : 2048;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) applied += __shfl_xor_sync(0xffffffffu, applied, o);
    if (lane == 0 && applied && b.n_updates) atomicAdd(b.n_updates, applied);
}

struct BatchKernel {
    void (*launch)(const BatchArgs &, int grid, cudaStream_t);
    int blocks_per_sm;
    int lanes, pass;
};

template <typename T, int D, int L, int P>
void launch_batch(const BatchArgs &b, int grid, cudaStream_t s) {
    launch_dep(batch_kernel<T, D, L, P>, grid, kTrainWarps * 32, 0, s, b);
}

template <typename T, int D, int L, int P>
BatchKernel make_batch() {
    BatchKernel k;
    k.launch = &launch_batch<T, D, L, P>;
    k.blocks_per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k.blocks_per_sm, batch_kernel<T, D, L, P>, kTrainWarps * 32, 0);
    if (k.blocks_per_sm < 1) k.blocks_per_sm = 1;
    k.lanes = L;
    k.pass = P;
    return k;
}

struct BatchEntry {
    gosh_dtype dtype;
    int d, lanes, pass;
    BatchKernel (*make)();
};

#define GOSH_BV(TY, CODE, D, L, P) {CODE, D, L, P, &make_batch<TY, D, L, P>}
#define GOSH_BVD(TY, CODE, D)                                                                                  \
    GOSH_BV(TY, CODE, D, (D * (int)sizeof(TY) / 16), 2), GOSH_BV(TY, CODE, D, (D * (int)sizeof(TY) / 16), 4), \
        GOSH_BV(TY, CODE, D, (D * (int)sizeof(TY) / 32), 2), GOSH_BV(TY, CODE, D, (D * (int)sizeof(TY) / 32), 4)
const BatchEntry kBatchEntries[] = {
    GOSH_BVD(float, GOSH_F32, 32),         GOSH_BVD(float, GOSH_F32, 64),         GOSH_BVD(float, GOSH_F32, 128),
    GOSH_BVD(__nv_bfloat16, GOSH_BF16, 32), GOSH_BVD(__nv_bfloat16, GOSH_BF16, 64), GOSH_BVD(__nv_bfloat16, GOSH_BF16, 128),
};
#undef GOSH_BVD
#undef GOSH_BV

std::mutex g_batch_mu;
std::map<int, BatchKernel> g_batch_made;
// autotuned (lanes, pass, rows per item) per (dtype, d, k)
std::map<std::tuple<int, int, int>, std::tuple<int, int, int>> g_tuned;

const BatchKernel *find_batch(gosh_dtype dtype, int d, int lanes, int pass) {
    std::lock_guard<std::mutex> lock(g_batch_mu);
    for (int i = 0; i < (int)(sizeof(kBatchEntries) / sizeof(kBatchEntries[0])); ++i) {
        const BatchEntry &e = kBatchEntries[i];
        if (e.dtype == dtype && e.d == d && e.lanes == lanes && e.pass == pass) {
            auto it = g_batch_made.find(i);
            if (it == g_batch_made.end()) it = g_batch_made.emplace(i, e.make()).first;
            return &it->second;
        }
    }
    return nullptr;
}

// Device-resident schedule of the whole batch.
struct Plan {
    std::vector<Phase> phases;
    std::vector<int> first, count;
    Scratch d_phases, d_first, d_count, d_ctl, d_done, d_err;
};

// Phases of levels D-1 .. lowest of every graph (projections between them).
gosh_status build_plan(const std::vector<gosh_hierarchy *> &hs, const std::vector<std::vector<void *>> &bufs,
                       const gosh_params &p, int epochs, int rows_per_item, Plan &plan, cudaStream_t s,
                       int lowest = 0) {
    plan.phases.clear();
    plan.first.clear();
    plan.count.clear();
    for (size_t gi = 0; gi < hs.size(); ++gi) {
        const gosh_hierarchy *h = hs[gi];
        const int D = (int)h->n.size();
        std::vector<int> ep(D);
        GOSH_TRY(level_epochs(epochs, p.p, D, p.epoch_unit, h->n.data(), h->nnz.data(), ep.data()));
        plan.first.push_back((int)plan.phases.size());
        auto items = [&](int64_t n) { return (n + rows_per_item - 1) / rows_per_item; };
        Phase init{};
        init.type = kPhaseInit;
        init.level = D - 1;
        init.n = h->n[D - 1];
        init.items = items(init.n);
        init.M = bufs[gi][D - 1];
        plan.phases.push_back(init);
        for (int i = D - 1; i >= lowest; --i) {
            for (int j = 0; j < ep[i]; ++j) {
                Phase t{};
                t.type = kPhaseTrain;
                t.level = i;
                t.epoch = (uint32_t)j;
                const double f = 1.0 - (double)j / (double)ep[i];
                t.lr = (float)(p.lr * (f > p.lr_floor ? f : p.lr_floor));
                t.n = h->n[i];
                t.items = items(t.n);
                t.rowptr = h->rowptr[i];
                t.col = h->col[i];
                t.M = bufs[gi][i];
                plan.phases.push_back(t);
            }
            if (i > lowest) {
                Phase pr{};
                pr.type = kPhaseProject;
                pr.level = i - 1;
                pr.n = h->n[i - 1];
                pr.items = items(pr.n);
                pr.M = bufs[gi][i - 1];
                pr.Msrc = bufs[gi][i];
                pr.map = h->map[i - 1];
                plan.phases.push_back(pr);
            }
        }
        plan.count.push_back((int)plan.phases.size() - plan.first.back());
    }
    const int G = (int)hs.size();
    GOSH_TRY(plan.d_phases.alloc(sizeof(Phase) * plan.phases.size(), s));
    GOSH_TRY(plan.d_first.alloc(sizeof(int) * G, s));
    GOSH_TRY(plan.d_count.alloc(sizeof(int) * G, s));
    GOSH_TRY(plan.d_ctl.alloc(sizeof(GraphCtl) * G, s));
    GOSH_TRY(plan.d_done.alloc(sizeof(unsigned long long), s));
    GOSH_TRY(plan.d_err.alloc(sizeof(int), s));
    GOSH_TRY_CUDA(cudaMemcpyAsync(plan.d_phases.ptr, plan.phases.data(), sizeof(Phase) * plan.phases.size(),
                                  cudaMemcpyHostToDevice, s));
    GOSH_TRY_CUDA(cudaMemcpyAsync(plan.d_first.ptr, plan.first.data(), sizeof(int) * G, cudaMemcpyHostToDevice, s));
    GOSH_TRY_CUDA(cudaMemcpyAsync(plan.d_count.ptr, plan.count.data(), sizeof(int) * G, cudaMemcpyHostToDevice, s));
    GOSH_TRY_CUDA(cudaStreamSynchronize(s));
    return GOSH_OK;
}

// Runs the plan once as a captured CUDA graph (counter resets + persistent kernel).
gosh_status run_plan(Plan &plan, const BatchKernel *kern, const gosh_params &p, int rows_per_item,
                     unsigned long long *n_updates, cudaStream_t s, float *ms_out) {
    const int G = (int)plan.first.size();
    BatchArgs b{};
    b.phases = plan.d_phases.as<Phase>();
    b.first = plan.d_first.as<int>();
    b.count = plan.d_count.as<int>();
    b.ctl = plan.d_ctl.as<GraphCtl>();
    b.G = G;
    b.k = p.k;
    b.d = p.d;
    b.seed = p.seed;
    b.graph_base = p.graph_id;
    b.rows_per_item = rows_per_item;
    b.graphs_done = plan.d_done.as<unsigned long long>();
    b.err = plan.d_err.as<int>();
    b.n_updates = n_updates;
    // no more warps than the widest moment of the schedule can use: with G
    // graphs at most G phases run at once, each with at most max-items items
    int64_t max_items = 1;
    for (const Phase &ph : plan.phases) max_items = std::max<int64_t>(max_items, ph.items);
    const int64_t useful = std::max<int64_t>(1, ceil_div(max_items * G, kTrainWarps));
    const int grid = (int)std::min<int64_t>((int64_t)num_sms() * kern->blocks_per_sm, useful);

    cudaStream_t cs;
    GOSH_TRY_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaMemsetAsync(b.ctl, 0, sizeof(GraphCtl) * G, cs);
        cudaMemsetAsync(b.graphs_done, 0, sizeof(unsigned long long), cs);
        cudaMemsetAsync(b.err, 0, sizeof(int), cs);
        kern->launch(b, grid, cs);
        e = cudaStreamEndCapture(cs, &graph);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = cudaGraphLaunch(exec, s);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, b.err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    float ms = 0.f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        set_error("batched launch: %s", cudaGetErrorString(e));
        return GOSH_ERR_CUDA;
    }
    if (herr) {
        set_error("batched launch: a warp found no work for 4 s (schedule stalled)");
        return GOSH_ERR_TIMEOUT;
    }
    if (ms_out) *ms_out = ms;
    return GOSH_OK;
}

}  // namespace

// Trains levels D-1 .. lowest of one hierarchy in one persistent launch: the
// initialisation of M_{D-1}, every epoch of those levels and the copy
// projections between them, with no host round trip between epochs (the
// small levels of a hierarchy are otherwise bound by launch latency).
// bufs[i] holds M_i.  Same Philox streams as the per-epoch launches.
gosh_status persistent_levels(gosh_hierarchy *h, const std::vector<void *> &bufs, int lowest, const gosh_params &p,
                              unsigned long long *n_updates, cudaStream_t s) {
    const int L0 = p.d * (int)dtype_size(p.dtype) / 16;
    int lanes = p.dtype == GOSH_F32 ? L0 : L0 / 2, pass = 2, rpi = 64;
    {
        std::lock_guard<std::mutex> lock(g_batch_mu);
        auto it = g_tuned.find(std::make_tuple((int)p.dtype, p.d, p.k));
        if (it != g_tuned.end()) std::tie(lanes, pass, rpi) = it->second;
    }
    const BatchKernel *kern = find_batch(p.dtype, p.d, lanes, pass);
    if (!kern) {
        set_error("no persistent kernel for dtype %d, d %d", (int)p.dtype, p.d);
        return GOSH_ERR_UNSUPPORTED;
    }
    std::vector<gosh_hierarchy *> hs{h};
    std::vector<std::vector<void *>> bv{bufs};
    Plan plan;
    GOSH_TRY(build_plan(hs, bv, p, p.epochs, rpi, plan, s, lowest));
    return run_plan(plan, kern, p, rpi, n_updates, s, nullptr);
}

}  // namespace gosh

using namespace gosh;

extern "C" gosh_status gosh_embed_batch(int n_graphs, const gosh_csr *graphs, const gosh_params *params,
                                        void *const *M_out, void *stream, gosh_batch_stats *stats) {
    clear_error();
    GOSH_CHECK_ARG(n_graphs >= 1 && graphs && params && M_out, "bad arguments");
    const gosh_params &p = *params;
    GOSH_CHECK_ARG(p.dtype == GOSH_F32 || p.dtype == GOSH_BF16, "batched training serves FP32 and BF16 tables");
    GOSH_CHECK_ARG(p.d == 32 || p.d == 64 || p.d == 128, "d must be 32, 64 or 128");
    GOSH_CHECK_ARG(p.k >= 0 && p.k <= kMaxK, "k must be in 0..%d", kMaxK);
    GOSH_CHECK_ARG(p.mode == GOSH_HOGWILD, "batched training is lock-free (GOSH_HOGWILD)");
    GOSH_CHECK_ARG(p.epochs >= 0 && p.lr > 0, "bad epochs / lr");
    cudaStream_t s = (cudaStream_t)stream;
    const auto t0 = std::chrono::steady_clock::now();
    const size_t row = (size_t)p.d * dtype_size(p.dtype);

    for (int gi = 0; gi < n_graphs; ++gi) {
        GOSH_CHECK_ARG(graphs[gi].on_device && graphs[gi].n >= 1, "graph %d: needs a device CSR with n >= 1", gi);
        GOSH_CHECK_ARG(((uintptr_t)M_out[gi] & 15) == 0, "graph %d: M_out must be 16-byte aligned", gi);
    }
    // coarsen every graph: one union of the graphs still coarsening per level
    std::vector<gosh_hierarchy *> hs(n_graphs, nullptr);
    struct Free {
        std::vector<gosh_hierarchy *> &v;
        ~Free() {
            for (auto *h : v) delete h;
        }
    } free_hs{hs};
    GOSH_TRY(coarsen_batch_impl(graphs, n_graphs, p.threshold, p.shrink, p.max_levels > 0 ? p.max_levels : 64, s, hs));
    const double coarsen_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();

    // embedding buffers: level 0 is the caller's, coarser levels one arena
    int64_t arena_rows = 0;
    for (auto *h : hs)
        for (size_t i = 1; i < h->n.size(); ++i) arena_rows += h->n[i];
    Scratch arena, counter;
    GOSH_TRY(arena.alloc(row * (arena_rows > 0 ? arena_rows : 1), s));
    GOSH_TRY(counter.alloc(sizeof(unsigned long long), s));
    std::vector<std::vector<void *>> bufs(hs.size());
    int64_t off = 0;
    for (size_t gi = 0; gi < hs.size(); ++gi) {
        bufs[gi].push_back(M_out[gi]);
        for (size_t i = 1; i < hs[gi]->n.size(); ++i) {
            bufs[gi].push_back(arena.as<char>() + off * row);
            off += hs[gi]->n[i];
        }
    }

    // autotune (lanes per row, samples per pass, sources per work item) once per (dtype, d, k)
    int lanes = p.lanes_per_row, pass = p.samples_per_pass, rpi = 64;
    bool tuned_now = false;
    if (lanes <= 0 || pass <= 0) {
        const auto key = std::make_tuple((int)p.dtype, p.d, p.k);
        bool have = false;
        {
            std::lock_guard<std::mutex> lock(g_batch_mu);
            auto it = g_tuned.find(key);
            if (it != g_tuned.end()) {
                std::tie(lanes, pass, rpi) = it->second;
                have = true;
            }
        }
        if (!have) {
            const int L0 = p.d * (int)dtype_size(p.dtype) / 16;
            float best = 1e30f;
            const int tune_epochs = std::max(4, std::min(p.epochs, 16));
            for (int L : {L0, L0 / 2})
                for (int P : {2, 4})
                    for (int r : {32, 64, 128}) {
                        const BatchKernel *k = find_batch(p.dtype, p.d, L, P);
                        if (!k) continue;
                        Plan plan;
                        GOSH_TRY(build_plan(hs, bufs, p, tune_epochs, r, plan, s));
                        float ms = 0.f;
                        GOSH_TRY(run_plan(plan, k, p, r, nullptr, s, &ms));
                        if (ms < best) {
                            best = ms;
                            lanes = L;
                            pass = P;
                            rpi = r;
                        }
                    }
            std::lock_guard<std::mutex> lock(g_batch_mu);
            g_tuned[key] = std::make_tuple(lanes, pass, rpi);
            tuned_now = true;
        }
    }
    const BatchKernel *kern = find_batch(p.dtype, p.d, lanes, pass);
    if (!kern) {
        set_error("no batched kernel for lanes_per_row %d, samples_per_pass %d", lanes, pass);
        return GOSH_ERR_UNSUPPORTED;
    }
    Plan plan;
    GOSH_TRY(build_plan(hs, bufs, p, p.epochs, rpi, plan, s));
    GOSH_TRY_CUDA(cudaMemsetAsync(counter.ptr, 0, sizeof(unsigned long long), s));
    float ms = 0.f;
    GOSH_TRY(run_plan(plan, kern, p, rpi, counter.as<unsigned long long>(), s, &ms));
    unsigned long long updates = 0;
    GOSH_TRY_CUDA(cudaMemcpyAsync(&updates, counter.ptr, sizeof(updates), cudaMemcpyDeviceToHost, s));
    GOSH_TRY_CUDA(cudaStreamSynchronize(s));
    if (stats) {
        stats->graphs = n_graphs;
        stats->phases = (int64_t)plan.phases.size();
        stats->lanes_per_row = lanes;
        stats->samples_per_pass = pass;
        stats->sources_per_item = rpi;
        stats->autotuned = tuned_now ? 1 : 0;
        stats->coarsen_ms = coarsen_ms;
        stats->train_ms = ms;
        stats->updates = updates;
        int64_t v0 = 0;
        for (auto *h : hs) v0 += h->n[0];
        stats->level0_vertices = v0;
        stats->total_ms =
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    return GOSH_OK;
}
