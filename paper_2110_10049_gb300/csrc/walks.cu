// Random-walk positives (GOSH Sec. 3.2, the variant the paper calls GOSHW):
// the host draws the walks and their pairs, the GPU applies Alg. 1 to each
// pair with k uniform negatives.
//
// Per epoch j of a level: one walk of l vertices from every vertex v (step t
// moves to a uniform neighbour: Philox block (v, t/4, level<<32 | j,
// kTagWalk), word t%4; a vertex without neighbours ends the walk), and every
// pair (w_i, w_j) with 0 < j - i <= g is a positive with source w_i.  The
// pairs of the walk from v sit at positions v*W .. v*W + W - 1 (W = pairs of
// a full walk, ranked i ascending, then j ascending); positions past a
// shorter walk and pairs whose ends coincide are holes.  The epoch visits the
// positions in a pseudo-random order (walk_position: a Feistel permutation),
// which is the shuffle the paper applies to the samples.
//
// Pipeline: host threads fill the pinned pair table of epoch j+1 while the
// table of epoch j is copied to the device (a copy stream) and trained (the
// caller's stream); two pinned and two device tables alternate.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <thread>
#include <vector>

#include "pinned.cuh"
#include "train_kernels.cuh"

namespace gosh {
namespace {

template <typename T, int D, int L, int P>
__global__ void __launch_bounds__(kTrainWarps * 32, train_min_blocks<T>(D / L, kModeRed)) train_pairs_kernel(TrainArgs a) {
    __shared__ int32_t s_u[kTrainWarps][32 * kSlotStride];
    __shared__ uint32_t s_sr[kTrainWarps][32];
    __shared__ int32_t s_src[kTrainWarps][32];
    GOSH_DEP_WAIT();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t ntiles = (a.src_end - a.src_begin + a.tile - 1) / a.tile;
    const int64_t wstride = (int64_t)gridDim.x * kTrainWarps;
    double loss_acc = 0.0;
    unsigned long long applied = 0;
    for (int64_t tile = (int64_t)blockIdx.x * kTrainWarps + warp; tile < ntiles; tile += wstride)
        train_tile<T, D, L, P, kModeRed, kTileDraws | kTileRounds, true>(a, a.src_begin + tile * a.tile, s_u[warp],
                                                                         s_sr[warp], loss_acc, applied, s_src[warp]);
    if (a.n_updates) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) applied += __shfl_xor_sync(0xffffffffu, applied, o);
        if (lane == 0 && applied) atomicAdd(a.n_updates, applied);
    }
}

struct PairsKernel {
    void (*launch)(const TrainArgs &, int grid, cudaStream_t);
    int blocks_per_sm;
    int lanes;
};

template <typename T, int D, int L, int P>
void launch_pairs(const TrainArgs &a, int grid, cudaStream_t s) {
    launch_dep(train_pairs_kernel<T, D, L, P>, grid, kTrainWarps * 32, 0, s, a);
}

template <typename T, int D, int L, int P>
PairsKernel make_pairs() {
    PairsKernel k;
    k.launch = &launch_pairs<T, D, L, P>;
    k.blocks_per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k.blocks_per_sm, train_pairs_kernel<T, D, L, P>, kTrainWarps * 32,
                                                  0);
    if (k.blocks_per_sm < 1) k.blocks_per_sm = 1;
    k.lanes = L;
    return k;
}

// Variants: natural lanes (one 16-byte vector per lane) with all samples of
// k <= 3 in one pass, and (16-bit tables) half the lanes with two per pass,
// the level-0 choice of the vertex-sampled step.
const PairsKernel *pick_pairs(gosh_dtype dt, int d, int lanes) {
    static std::once_flag once;
    static PairsKernel f32[3][2], b16[3][2];
    std::call_once(once, [] {
        f32[0][0] = make_pairs<float, 32, 8, 4>();
        f32[0][1] = make_pairs<float, 32, 4, 2>();
        f32[1][0] = make_pairs<float, 64, 16, 4>();
        f32[1][1] = make_pairs<float, 64, 8, 2>();
        f32[2][0] = make_pairs<float, 128, 32, 4>();
        f32[2][1] = make_pairs<float, 128, 16, 2>();
        b16[0][0] = make_pairs<__nv_bfloat16, 32, 4, 4>();
        b16[0][1] = make_pairs<__nv_bfloat16, 32, 2, 2>();
        b16[1][0] = make_pairs<__nv_bfloat16, 64, 8, 4>();
        b16[1][1] = make_pairs<__nv_bfloat16, 64, 4, 2>();
        b16[2][0] = make_pairs<__nv_bfloat16, 128, 16, 4>();
        b16[2][1] = make_pairs<__nv_bfloat16, 128, 8, 2>();
    });
    const int di = d == 32 ? 0 : d == 64 ? 1 : d == 128 ? 2 : -1;
    if (di < 0) return nullptr;
    PairsKernel *tab = dt == GOSH_F32 ? f32[di] : dt == GOSH_BF16 ? b16[di] : nullptr;
    if (!tab) return nullptr;
    if (lanes <= 0) return dt == GOSH_F32 ? &tab[0] : &tab[1];
    for (int i = 0; i < 2; ++i)
        if (tab[i].lanes == lanes) return &tab[i];
    return nullptr;
}

// Permutation key of an epoch (the rounds use mix32(key + r)).
uint32_t walk_key(uint64_t seed, uint64_t graph, int level, int epoch) {
    uint32_t k = mix32((uint32_t)seed ^ ((uint32_t)level << 24));
    k = mix32(k ^ (uint32_t)(seed >> 32) ^ (uint32_t)epoch);
    return mix32(k ^ mix32((uint32_t)graph ^ (uint32_t)(graph >> 32)));
}

int walk_bits(uint64_t P) {
    int h = 1;
    while ((uint64_t(1) << (2 * h)) < P) ++h;
    return h;
}

// The pair positions of the walks from v0 .. v1-1 of one epoch into out
// (2 int32 per position, rows v*W ..).  kGroup walks advance in lockstep:
// their neighbour reads are independent, so the host cores overlap the cache
// misses of a step.
void walk_fill(const int64_t *rowptr, const int32_t *col, int64_t v0, int64_t v1, int l, int gw, int64_t W,
               int level, int epoch, uint64_t seed, uint64_t graph, int32_t *out) {
    constexpr int kGroup = 128;
    std::vector<int32_t> w((size_t)kGroup * l);
    int len[kGroup];
    int64_t at[kGroup];
    Philox4 words[kGroup];
    const uint64_t ctr2 = ((uint64_t)(uint32_t)level << 32) | (uint32_t)epoch;
    for (int64_t gs = v0; gs < v1; gs += kGroup) {
        const int cnt = (int)std::min<int64_t>(kGroup, v1 - gs);
        for (int b = 0; b < cnt; ++b) {
            w[(size_t)b * l] = (int32_t)(gs + b);
            len[b] = 1;
            __builtin_prefetch(rowptr + gs + b);
        }
        for (int t = 0; t + 1 < l; ++t) {
            // pass 1: the entry each live walk moves through (row pointers,
            // prefetched one step earlier), and a prefetch of that entry;
            // pass 2: the neighbour reads, all independent, then a prefetch
            // of the next step's row pointers
            for (int b = 0; b < cnt; ++b) {
                at[b] = -1;
                if (len[b] != t + 1) continue;  // this walk has ended
                if ((t & 3) == 0)
                    words[b] = philox4x64_10((uint64_t)(gs + b), (uint64_t)(t >> 2), ctr2, kTagWalk, seed, graph);
                const int64_t cur = w[(size_t)b * l + t];
                const int64_t off = rowptr[cur], deg = rowptr[cur + 1] - off;
                if (deg > 0) {
                    at[b] = off + (int64_t)uniform_index(words[b].w[t & 3], (uint64_t)deg);
                    __builtin_prefetch(col + at[b]);
                }
            }
            for (int b = 0; b < cnt; ++b) {
                if (at[b] < 0) continue;
                const int32_t nx = col[at[b]];
                w[(size_t)b * l + t + 1] = nx;
                len[b] = t + 2;
                __builtin_prefetch(rowptr + nx);
            }
        }
        for (int b = 0; b < cnt; ++b) {
            const int32_t *wb = w.data() + (size_t)b * l;
            int32_t *pp = out + 2 * (gs + b) * W;
            for (int i = 0; i + 1 < l; ++i)
                for (int j = i + 1; j < l && j - i <= gw; ++j, pp += 2) {
                    const bool ok = j < len[b] && wb[i] != wb[j];
                    pp[0] = ok ? wb[i] : -1;
                    pp[1] = ok ? wb[j] : -1;
                }
        }
    }
}

int64_t walk_positions_per_walk(int l, int gw) {
    int64_t W = 0;
    for (int i = 0; i + 1 < l; ++i) W += std::min(gw, l - 1 - i);
    return W;
}

PinnedArena g_walk_pinned;

}  // namespace

size_t walks_release_pinned() { return g_walk_pinned.release(); }
}  // namespace gosh

using namespace gosh;

extern "C" {

gosh_status gosh_train_level_walks(const gosh_csr *g, void *M, int level, int epochs, const gosh_params *p,
                                   void *stream, unsigned long long *n_updates, gosh_walk_stats *stats) {
    clear_error();
    GOSH_CHECK_ARG(g && p && M, "NULL argument");
    GOSH_TRY(check_params(p));
    GOSH_CHECK_ARG(g->n >= 1 && g->n < (int64_t(1) << 31), "bad n");
    GOSH_CHECK_ARG(((uintptr_t)M & 15) == 0, "M must be a 16-byte aligned device pointer");
    GOSH_CHECK_ARG(p->mode == GOSH_HOGWILD, "walk sampling is lock-free (GOSH_HOGWILD)");
    GOSH_CHECK_ARG(p->dtype == GOSH_F32 || p->dtype == GOSH_BF16, "walk sampling serves FP32 and BF16 tables");
    GOSH_CHECK_ARG(p->k >= 0 && p->k <= 3, "walk sampling serves k <= 3 (got %d)", p->k);
    const int l = p->walk_length, gw = p->walk_window;
    GOSH_CHECK_ARG(l >= 2 && l <= 256 && gw >= 1, "need 2 <= walk_length <= 256 and walk_window >= 1");
    const PairsKernel *kern = pick_pairs(p->dtype, p->d, p->lanes_per_row);
    GOSH_CHECK_ARG(kern != nullptr, "no walk kernel for dtype %d, d %d, lanes_per_row %d", (int)p->dtype, p->d,
                   p->lanes_per_row);
    if (epochs <= 0) return GOSH_OK;
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = g->n;

    // the walks read a host CSR (copied back once if the caller's is on the device)
    std::vector<int64_t> hrp;
    std::vector<int32_t> hcol;
    const int64_t *rowptr = g->rowptr;
    const int32_t *col = g->col;
    if (g->on_device) {
        hrp.resize(n + 1);
        GOSH_TRY_CUDA(cudaMemcpyAsync(hrp.data(), g->rowptr, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, s));
        GOSH_TRY_CUDA(cudaStreamSynchronize(s));
        hcol.resize(hrp[n] > 0 ? hrp[n] : 1);
        if (hrp[n] > 0)
            GOSH_TRY_CUDA(cudaMemcpyAsync(hcol.data(), g->col, sizeof(int32_t) * hrp[n], cudaMemcpyDeviceToHost, s));
        GOSH_TRY_CUDA(cudaStreamSynchronize(s));
        rowptr = hrp.data();
        col = hcol.data();
    }
    if (p->validate) GOSH_TRY(check_host_csr(rowptr, col, n, false));

    const int64_t W = walk_positions_per_walk(l, gw);
    const int64_t P = n * W;  // positions per epoch
    const size_t bytes = sizeof(int32_t) * 2 * (size_t)P;
    PinnedLease lease(g_walk_pinned);
    GOSH_TRY(lease.acquire(2 * bytes, "walk pairs"));
    int32_t *hb[2] = {reinterpret_cast<int32_t *>(lease.ptr), reinterpret_cast<int32_t *>(lease.ptr + bytes)};
    Scratch db[2];
    for (auto &b : db) GOSH_TRY(b.alloc(bytes, s));

    // ---- host: the pair table of one epoch, walks spread over threads ----
    const int nt = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    double gen_ms = 0.0, wait_ms = 0.0;
    auto generate = [&](int epoch, int32_t *out) {
        const auto tg = std::chrono::steady_clock::now();
        constexpr int64_t kWalksPerItem = 4096;
        std::atomic<int64_t> next{0};
        auto work = [&]() {
            for (int64_t v0 = next.fetch_add(kWalksPerItem); v0 < n; v0 = next.fetch_add(kWalksPerItem))
                walk_fill(rowptr, col, v0, std::min(v0 + kWalksPerItem, n), l, gw, W, level, epoch, p->seed,
                          p->graph_id, out);
        };
        std::vector<std::thread> th;
        for (int t = 1; t < nt; ++t) th.emplace_back(work);
        work();
        for (auto &x : th) x.join();
        gen_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tg).count();
    };

    cudaStream_t cs = nullptr;
    GOSH_TRY_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaEvent_t h2d_done[2] = {nullptr, nullptr}, kern_done[2] = {nullptr, nullptr};
    struct Cleanup {
        cudaStream_t &cs;
        cudaEvent_t *a, *b;
        ~Cleanup() {
            if (cs) {
                cudaStreamSynchronize(cs);
                cudaStreamDestroy(cs);
            }
            for (int i = 0; i < 2; ++i) {
                if (a[i]) cudaEventDestroy(a[i]);
                if (b[i]) cudaEventDestroy(b[i]);
            }
        }
    } cleanup{cs, h2d_done, kern_done};
    for (int i = 0; i < 2; ++i) {
        GOSH_TRY_CUDA(cudaEventCreateWithFlags(&h2d_done[i], cudaEventDisableTiming));
        GOSH_TRY_CUDA(cudaEventCreateWithFlags(&kern_done[i], cudaEventDisableTiming));
    }
    // the tables of the first two epochs may only be overwritten once the
    // stream has reached this call (the caller's earlier work may use them)
    GOSH_TRY_CUDA(cudaEventRecord(kern_done[0], s));
    GOSH_TRY_CUDA(cudaEventRecord(kern_done[1], s));

    TrainArgs a{};
    a.M = M;
    a.n = n;
    a.k = p->k;
    a.seed = p->seed;
    a.graph = p->graph_id;
    a.level = (uint32_t)level;
    a.n_updates = n_updates;
    a.err = device_error_word();
    a.src_begin = 0;
    a.src_end = P;
    a.walk_h = walk_bits((uint64_t)P);
    const int G = 32 / kern->lanes;
    int tile = p->vertices_per_warp > 0 ? p->vertices_per_warp : 32;
    tile = std::max(G, std::min(32, tile)) / G * G;
    a.tile = tile;
    const int64_t want = ceil_div(ceil_div(P, tile), kTrainWarps);
    const int64_t cap = (int64_t)num_sms() * kern->blocks_per_sm;
    const int grid = (int)std::max<int64_t>(1, std::min(want, cap));

    generate(0, hb[0]);
    for (int j = 0; j < epochs; ++j) {
        const int b = j & 1;
        GOSH_TRY_CUDA(cudaStreamWaitEvent(cs, kern_done[b], 0));  // device table b is free
        GOSH_TRY_CUDA(cudaMemcpyAsync(db[b].ptr, hb[b], bytes, cudaMemcpyHostToDevice, cs));
        GOSH_TRY_CUDA(cudaEventRecord(h2d_done[b], cs));
        GOSH_TRY_CUDA(cudaStreamWaitEvent(s, h2d_done[b], 0));
        const double f = 1.0 - (double)j / (double)epochs;
        a.lr = (float)(p->lr * (f > p->lr_floor ? f : p->lr_floor));
        a.epoch = (uint32_t)j;
        a.pairs = db[b].as<int32_t>();
        a.walk_key = walk_key(p->seed, p->graph_id, level, j);
        kern->launch(a, grid, s);
        GOSH_TRY_CUDA(cudaGetLastError());
        GOSH_TRY_CUDA(cudaEventRecord(kern_done[b], s));
        if (j + 1 < epochs) {
            // host table b^1 is free once epoch j-1's copy from it is done
            const auto tw = std::chrono::steady_clock::now();
            GOSH_TRY_CUDA(cudaEventSynchronize(h2d_done[b ^ 1]));
            wait_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tw).count();
            generate(j + 1, hb[b ^ 1]);
        }
    }
    GOSH_TRY_CUDA(cudaStreamSynchronize(s));
    if (stats) {
        stats->positions = P;
        stats->epochs = epochs;
        stats->host_ms = gen_ms;
        stats->total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        stats->h2d_bytes = (int64_t)bytes * epochs;
    }
    (void)wait_ms;
    return GOSH_OK;
}

gosh_status gosh_walk_pairs(const gosh_csr *g, int walk_length, int walk_window, int level, int epoch,
                            uint64_t seed, uint64_t graph_id, int32_t *pairs) {
    clear_error();
    GOSH_CHECK_ARG(g && pairs && !g->on_device, "needs a host CSR and a host output");
    GOSH_CHECK_ARG(g->n >= 1 && g->n < (int64_t(1) << 31), "bad n");
    GOSH_CHECK_ARG(walk_length >= 2 && walk_length <= 256 && walk_window >= 1,
                   "need 2 <= walk_length <= 256 and walk_window >= 1");
    GOSH_TRY(check_host_csr(g->rowptr, g->col, g->n, false));
    walk_fill(g->rowptr, g->col, 0, g->n, walk_length, walk_window, walk_positions_per_walk(walk_length, walk_window),
              level, epoch, seed, graph_id, pairs);
    return GOSH_OK;
}

gosh_status gosh_walk_order(int64_t positions, int level, int epoch, uint64_t seed, uint64_t graph_id,
                            int64_t *order) {
    clear_error();
    GOSH_CHECK_ARG(order && positions >= 1, "bad positions / order");
    const uint32_t key = walk_key(seed, graph_id, level, epoch);
    const int h = walk_bits((uint64_t)positions);
    for (int64_t i = 0; i < positions; ++i) order[i] = (int64_t)walk_position((uint64_t)i, (uint64_t)positions, key, h);
    return GOSH_OK;
}

}  // extern "C"
