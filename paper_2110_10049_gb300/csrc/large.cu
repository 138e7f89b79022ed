// LargeGraphGPU (Sec. 5): training a level whose embedding and graph exceed
// the device budget.  V is split into K contiguous parts V^0..V^{K-1} (M into
// the matching submatrices); a round visits every part pair (a, b), a >= b, in
// inside-out order (0,0),(1,0),(1,1),(2,0),... and runs kernel K_{a,b}: every
// u in V^a with neighbours in V^b draws B positives uniformly from
// Gamma(u) & V^b, each followed by k negatives uniform over V^b, and
// symmetrically for u in V^b when a != b.  r = ceil(e/B) rounds; a global
// atomic counter stops positives at e*|V|.
//
// GB300 realisation: the host keeps M and the CSR in pinned memory.  The
// device holds P_GPU part bins and S_GPU edge-block bins.  Edge block (a, b)
// = for each u in V^a the sub-range of its sorted row that falls in V^b
// (parts are id ranges, so it is found by binary search), stored with local
// ids; blocks are built once on host threads and streamed every round.  A
// single host thread issues the DAG of the paper's three task kinds
// asynchronously: submatrix swaps (MST: D2H of the evicted part, H2D of the
// needed one) on the bin's stream, edge-block copies (SCT) on the edge bin's
// stream, kernels (KT) alternating over two streams; cudaEvents carry every
// dependency (a kernel waits for its parts and block; a swap waits for every
// kernel that used the bin and for the host copy of the incoming part to be
// fresh; an edge bin is refilled after its last kernel).  Victims are chosen
// by the known future order (farthest next use).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <cmath>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "pinned.cuh"
#include "train_kernels.cuh"

namespace gosh {
namespace {

constexpr int kMaxSlots = 32;  // B * (k+1) sample ids per source kept in shared memory
constexpr uint64_t kTagLarge = 3;

struct PairArgs {
    void *Ma, *Mb;                    // bins of parts a and b (local rows)
    int64_t na, nb;                   // part sizes
    int64_t start_a, start_b;         // first global id of each part
    const int64_t *rp_ab;             // [na+1] block (a,b): rows of V^a, local column ids in V^b
    const int32_t *col_ab;
    const int64_t *rp_ba;             // [nb+1] block (b,a) (a != b)
    const int32_t *col_ba;
    const int32_t *pool;              // host sample pool (or null: positives from the edge block):
                                      // B positives per source (V^a, then V^b), local ids, -1 = none
    int same;                         // a == b
    int B, k;
    int epochs_total;                 // e of this level
    int round;
    float lr, lr_floor;
    uint64_t seed, graph, tag;        // Philox key and stream tag
    uint32_t level;
    unsigned long long *positives;    // global counter
    unsigned long long cap;           // e * |V|
    unsigned long long *n_updates;
};

// One tile of 32 sources (side A: V^a, side B: V^b).  Lane j draws source j's
// B positives and k negatives each (shared memory), then L-lane groups apply
// the B*(k+1) updates of their source with the source row in registers.
template <typename T, int D, int L, int P, int MODE>
__device__ void pair_tile(const PairArgs &a, int64_t s0, int64_t nsrc, int32_t *su, float *slr,
                          unsigned long long &applied) {
    constexpr bool RED = MODE == kModeRed;
    constexpr bool RED16 = RED && !std::is_same<T, float>::value;
    constexpr int E = D / L;
    constexpr int G = 32 / L;
    const int lane = threadIdx.x & 31, grp = lane / L, gl = lane % L;
    const int ns = a.B * (a.k + 1);
    // ---- draws ----
    int npos = 0;
    {
        const int64_t s = s0 + lane;
        if (s < nsrc) {
            const bool sideA = s < a.na;
            const int64_t u = sideA ? s : s - a.na;
            const int64_t *rp = sideA ? a.rp_ab : a.rp_ba;
            const int32_t *cl = sideA ? a.col_ab : a.col_ba;
            const int64_t nopp = sideA ? a.nb : a.na;
            const int64_t ug = (sideA ? a.start_a : a.start_b) + u;
            const int32_t *pp = a.pool ? a.pool + s * a.B : nullptr;
            const int64_t lo = pp ? 0 : rp[u];
            const int64_t cnt = pp ? (__ldg(pp) >= 0 ? 1 : 0) : rp[u + 1] - lo;
            for (int j = 0; j < a.B; ++j) {
                const uint32_t t = (uint32_t)(a.round * a.B + j);
                const int ks = j * (a.k + 1);
                for (int blk = 0; blk * 4 < a.k + 1; ++blk) {
                    const Philox4 w = philox4x64_10((uint64_t)ug, (uint64_t)blk, ((uint64_t)a.level << 32) | t, a.tag,
                                                    a.seed, a.graph);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int m = blk * 4 + q;
                        if (m <= a.k) {
                            int32_t id;
                            if (m == 0) {
                                if (pp) id = __ldg(pp + j);
                                else id = cnt > 0 ? __ldg(cl + lo + (int64_t)uniform_index(w.w[0], (uint64_t)cnt)) : -1;
                            } else {
                                const int64_t x = (int64_t)uniform_index(w.w[q], (uint64_t)nopp);
                                id = (a.same && x == u) ? -1 : (int32_t)x;
                            }
                            su[lane * kMaxSlots + ks + m] = id;
                        }
                    }
                }
                const double f = 1.0 - (double)t / (double)a.epochs_total;
                slr[lane * 8 + j] = a.lr * (float)(f > a.lr_floor ? f : a.lr_floor);
            }
            npos = cnt > 0 ? a.B : 0;
        }
    }
    // ---- cap on positives (global counter) ----
    int before = npos;  // inclusive prefix over lanes
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, before, o);
        if (lane >= o) before += y;
    }
    // The tile takes its positives from the global count in one addition; in
    // source order, slot group jj of a source is dropped once the count before
    // it (old + positives of earlier sources + jj if the source has positives)
    // reaches the cap: exactly the sequential per-positive count when tiles
    // claim in order.  A tile without positives still reads the count (adds 0),
    // since its sources' negatives stop with the budget as well.
    const int tile_pos = __shfl_sync(0xffffffffu, before, 31);
    unsigned long long old = 0;
    if (lane == 0) old = atomicAdd(a.positives, (unsigned long long)tile_pos);
    old = __shfl_sync(0xffffffffu, old, 0);
    const long long allowed = old >= a.cap ? 0 : (long long)(a.cap - old);
    const int my_first = before - npos;  // positives of this lane's source start here
    __syncwarp();
    // ---- updates ----
#pragma unroll 1
    for (int q = 0; q < L; ++q) {
        const int j = q * G + grp;
        const int64_t s = s0 + j;
        const bool active = s < nsrc;
        const bool sideA = s < a.na;
        const int64_t u = active ? (sideA ? s : s - a.na) : 0;
        T *Mown = static_cast<T *>(sideA ? a.Ma : a.Mb);
        T *Mopp = static_cast<T *>(sideA ? a.Mb : a.Ma);
        const int first = __shfl_sync(0xffffffffu, my_first, j);
        const bool has_pos = __shfl_sync(0xffffffffu, npos, j) > 0;
        const uint32_t sr = std::is_same<T, float>::value
                                ? 0u
                                : sr_source_seed(a.seed, a.graph ^ a.tag, a.level, (uint32_t)a.round, (sideA ? a.start_a : a.start_b) + u);
        float r[E];
        if (active) load_row<T, E, L>(Mown + u * D, gl, r);
        else {
#pragma unroll
            for (int e = 0; e < E; ++e) r[e] = 0.0f;
        }
        float r0[RED ? E : 1];
        if (RED) {
#pragma unroll
            for (int e = 0; e < E; ++e) r0[e] = r[e];
        }
#pragma unroll 1
        for (int p0 = 0; p0 < ns; p0 += P) {
            int32_t us[P];
            float row[P][E];
#pragma unroll
            for (int x = 0; x < P; ++x) {
                const int t = p0 + x;
                int32_t id = (active && t < ns) ? su[j * kMaxSlots + t] : -1;
                const int jj = t / (a.k + 1);  // positive group of this slot
                if (id >= 0 && first + (has_pos ? jj : 0) >= allowed) id = -1;  // over the global cap
                us[x] = id;
            }
#pragma unroll
            for (int x = 0; x < P; ++x) {
                if (us[x] >= 0) load_row<T, E, L>(Mopp + (int64_t)us[x] * D, gl, row[x]);
                else {
#pragma unroll
                    for (int e = 0; e < E; ++e) row[x][e] = 0.0f;
                }
            }
#pragma unroll
            for (int x = 0; x < P; ++x) {
                const int t = p0 + x;
                const bool ok = us[x] >= 0;
                float part = 0.0f;
#pragma unroll
                for (int e = 0; e < E; ++e) part = fmaf(r[e], row[x][e], part);
                const float xx = group_sum<L>(part);
                const int jj = t / (a.k + 1);
                const float b = (t % (a.k + 1)) == 0 ? 1.0f : 0.0f;
                const float lr = (active && t < ns) ? slr[j * 8 + jj] : 0.0f;
                const float score = ok ? (b - sigmoid_f(xx)) * lr : 0.0f;
#pragma unroll
                for (int e = 0; e < E; ++e) r[e] = fmaf(row[x][e], score, r[e]);
                float old16[RED16 ? E : 1];
                if (RED16) {
#pragma unroll
                    for (int e = 0; e < E; ++e) old16[e] = row[x][e];
                }
#pragma unroll
                for (int e = 0; e < E; ++e) row[x][e] = fmaf(r[e], score, row[x][e]);
                if (ok) {
                    if constexpr (RED16) {
                        red_row16<T, D, E, L>(Mopp + (int64_t)us[x] * D, row[x], old16, sr, t, gl);
                    } else if (RED) {
                        float c[E];
#pragma unroll
                        for (int e = 0; e < E; ++e) c[e] = r[e] * score;
                        red_row<E, L>(reinterpret_cast<float *>(Mopp) + (int64_t)us[x] * D, c, gl);
                    } else {
                        store_row<T, D, E, L>(Mopp + (int64_t)us[x] * D, row[x], sr, t, gl);
                    }
                    if (gl == 0) ++applied;
                }
#pragma unroll
                for (int x2 = x + 1; x2 < P; ++x2)
                    if (ok && us[x2] == us[x]) {
#pragma unroll
                        for (int e = 0; e < E; ++e) row[x2][e] = row[x][e];
                    }
            }
        }
        if (active) {
            if constexpr (RED16) {
                red_row16<T, D, E, L>(Mown + u * D, r, r0, sr, ns, gl);
            } else if (RED) {
                float dr[E];
#pragma unroll
                for (int e = 0; e < E; ++e) dr[e] = r[e] - r0[RED ? e : 0];
                red_row<E, L>(reinterpret_cast<float *>(Mown) + u * D, dr, gl);
            } else {
                store_row<T, D, E, L>(Mown + u * D, r, sr, ns, gl);
            }
        }
    }
    __syncwarp();
}

template <typename T, int D, int L, int P>
__global__ void __launch_bounds__(kTrainWarps * 32) pair_kernel(PairArgs a) {
    GOSH_DEP_WAIT();
    constexpr int MODE = kModeRed;  // atomic row changes (16-bit: stochastically rounded)
    __shared__ int32_t su[kTrainWarps][32 * kMaxSlots];
    __shared__ float slr[kTrainWarps][32 * 8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t nsrc = a.na + (a.same ? 0 : a.nb);
    const int64_t tiles = (nsrc + 31) / 32;
    unsigned long long applied = 0;
    for (int64_t t = (int64_t)blockIdx.x * kTrainWarps + warp; t < tiles; t += (int64_t)gridDim.x * kTrainWarps)
        pair_tile<T, D, L, P, MODE>(a, t * 32, nsrc, su[warp], slr[warp], applied);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) applied += __shfl_xor_sync(0xffffffffu, applied, o);
    if (lane == 0 && applied && a.n_updates) atomicAdd(a.n_updates, applied);
}

typedef void (*PairLaunch)(const PairArgs &, int, cudaStream_t);

template <typename T, int D, int L, int P>
void launch_pair(const PairArgs &a, int grid, cudaStream_t s) {
    launch_dep(pair_kernel<T, D, L, P>, grid, kTrainWarps * 32, 0, s, a);
}

PairLaunch pick_pair_kernel(gosh_dtype dt, int d) {
    // two 16-byte vectors per lane for BF16, one for FP32; two sample rows per pass
    if (dt == GOSH_F32) {
        if (d == 32) return &launch_pair<float, 32, 8, 2>;
        if (d == 64) return &launch_pair<float, 64, 16, 2>;
        if (d == 128) return &launch_pair<float, 128, 32, 2>;
    } else if (dt == GOSH_BF16) {
        if (d == 32) return &launch_pair<__nv_bfloat16, 32, 2, 2>;
        if (d == 64) return &launch_pair<__nv_bfloat16, 64, 4, 2>;
        if (d == 128) return &launch_pair<__nv_bfloat16, 128, 8, 2>;
    }
    return nullptr;
}

// Pinned host memory for edge blocks and for the sample-pool ring, kept across calls.
PinnedArena g_pinned, g_pinned_pools;

// Edge block (a, b) of one pair, built once on the host in pinned memory.
struct Block {
    int64_t *rp_ab = nullptr, *rp_ba = nullptr;
    int32_t *col_ab = nullptr, *col_ba = nullptr;
    int64_t m_ab = 0, m_ba = 0;
    size_t bytes = 0;
    char *base = nullptr;  // inside the pinned region: rp_ab | col_ab | rp_ba | col_ba
};

}  // namespace

size_t large_release_pinned() { return g_pinned.release() + g_pinned_pools.release(); }

// Inside-out order of one round: (0,0),(1,0),(1,1),(2,0),(2,1),(2,2),...
void large_pair_order(int K, std::vector<std::pair<int, int>> &order) {
    order.clear();
    for (int a = 0; a < K; ++a)
        for (int b = 0; b <= a; ++b) order.push_back({a, b});
}

// The edge blocks of one LargeGraphGPU call, all in one host region: block i
// holds pair (a, b) = order[i] as rp_ab | col_ab | rp_ba | col_ba (row
// pointers from 0, entries as local ids of the opposite part; no ba side
// when a == b), each array 256-byte aligned.  A block side (u in V^a,
// entries in V^b) is built in row chunks (items) spread over host threads.
// plan() only counts the entries of each chunk (one walk per row splits it
// at every part boundary by binary searches of its sorted row) and lays the
// blocks out; place() puts them in a region; fill(k) writes item k.
struct EdgeBlocks {
    struct Side {
        int blk;
        bool ab;
        int pa, pb;  // parts of the rows and of the entries
        int64_t a0, a1, b0, b1;
        int64_t entries;
    };
    struct Item {
        int side;
        int64_t r0;   // first row offset in the side
        int64_t off;  // entries of the side before this chunk
    };
    static constexpr int64_t kChunkRows = 32768;
    const int64_t *rowptr = nullptr;
    const int32_t *col = nullptr;
    int K = 0;
    std::vector<int64_t> start;
    std::vector<std::pair<int, int>> order;
    std::vector<Block> blocks;
    std::vector<Side> sides;
    std::vector<Item> items;
    size_t total_bytes = 0, max_block = 0;

    static size_t al(size_t x) { return (x + 255) / 256 * 256; }

    void row_range(const Side &sd, int64_t r, const int32_t **lo, const int32_t **hi) const {
        const int64_t u = sd.a0 + r;
        const int32_t *row = col + rowptr[u], *end = col + rowptr[u + 1];
        *lo = std::lower_bound(row, end, (int32_t)sd.b0);
        *hi = std::lower_bound(*lo, end, (int32_t)sd.b1);
    }

    void plan(const int64_t *rp, const int32_t *cl, int parts, const std::vector<int64_t> &st, int nt) {
        rowptr = rp;
        col = cl;
        K = parts;
        start = st;
        large_pair_order(K, order);
        blocks.assign(order.size(), Block{});
        sides.clear();
        items.clear();
        for (size_t i = 0; i < order.size(); ++i) {
            const int a = order[i].first, b = order[i].second;
            sides.push_back({(int)i, true, a, b, start[a], start[a + 1], start[b], start[b + 1], 0});
            if (a != b) sides.push_back({(int)i, false, b, a, start[b], start[b + 1], start[a], start[a + 1], 0});
        }
        for (size_t j = 0; j < sides.size(); ++j)
            for (int64_t r = 0; r < sides[j].a1 - sides[j].a0; r += kChunkRows) items.push_back({(int)j, r, 0});
        // counts of every (row part, entry part) pair from one walk of each row
        // chunk: K - 1 binary searches per row split it at every part boundary
        std::vector<int64_t> part_chunk(K + 1, 0);  // first row chunk of each part
        for (int a = 0; a < K; ++a) part_chunk[a + 1] = part_chunk[a] + ceil_div(start[a + 1] - start[a], kChunkRows);
        std::vector<int64_t> pcount((size_t)part_chunk[K] * K, 0);  // [row chunk][entry part]
        {
            std::vector<std::pair<int, int64_t>> rchunks;  // (part, first row offset)
            for (int a = 0; a < K; ++a)
                for (int64_t r = 0; r < start[a + 1] - start[a]; r += kChunkRows) rchunks.push_back({a, r});
            std::atomic<size_t> next{0};
            auto work = [&]() {
                std::vector<int64_t> c(K);
                for (size_t k = next.fetch_add(1); k < rchunks.size(); k = next.fetch_add(1)) {
                    const int a = rchunks[k].first;
                    const int64_t r0 = rchunks[k].second, r1 = std::min(r0 + kChunkRows, start[a + 1] - start[a]);
                    std::fill(c.begin(), c.end(), 0);
                    for (int64_t r = r0; r < r1; ++r) {
                        const int64_t u = start[a] + r;
                        const int32_t *row = col + rowptr[u], *end = col + rowptr[u + 1];
                        const int32_t *prev = row;
                        for (int b = 0; b < K; ++b) {
                            const int32_t *nx = b + 1 < K ? std::lower_bound(prev, end, (int32_t)start[b + 1]) : end;
                            c[b] += nx - prev;
                            prev = nx;
                        }
                    }
                    for (int b = 0; b < K; ++b) pcount[(size_t)k * K + b] = c[b];
                }
            };
            std::vector<std::thread> th;
            for (int t = 1; t < nt; ++t) th.emplace_back(work);
            work();
            for (auto &x : th) x.join();
        }
        for (size_t k = 0; k < items.size(); ++k) {  // items are grouped by side, in row order
            Side &sd = sides[items[k].side];
            const int64_t rc = part_chunk[sd.pa] + items[k].r0 / kChunkRows;
            items[k].off = sd.entries;
            sd.entries += pcount[(size_t)rc * K + sd.pb];
        }
        total_bytes = 0;
        max_block = 0;
        for (size_t i = 0; i < blocks.size(); ++i) {
            Block &B = blocks[i];
            const int a = order[i].first, b = order[i].second;
            const int64_t na = start[a + 1] - start[a], nb = start[b + 1] - start[b];
            for (const Side &sd : sides)
                if (sd.blk == (int)i) (sd.ab ? B.m_ab : B.m_ba) = sd.entries;
            B.bytes = al(sizeof(int64_t) * (na + 1)) + al(sizeof(int32_t) * B.m_ab) +
                      al(a != b ? sizeof(int64_t) * (nb + 1) : 0) + al(sizeof(int32_t) * B.m_ba);
            max_block = std::max(max_block, B.bytes);
            total_bytes += B.bytes;
        }
    }

    void place(char *base) {
        size_t off = 0;
        for (size_t i = 0; i < blocks.size(); ++i) {
            Block &B = blocks[i];
            const int a = order[i].first, b = order[i].second;
            const int64_t na = start[a + 1] - start[a], nb = start[b + 1] - start[b];
            B.base = base + off;
            off += B.bytes;
            B.rp_ab = reinterpret_cast<int64_t *>(B.base);
            B.col_ab = reinterpret_cast<int32_t *>(B.base + al(sizeof(int64_t) * (na + 1)));
            B.rp_ba = reinterpret_cast<int64_t *>(reinterpret_cast<char *>(B.col_ab) + al(sizeof(int32_t) * B.m_ab));
            B.col_ba = reinterpret_cast<int32_t *>(reinterpret_cast<char *>(B.rp_ba) +
                                                   al(a != b ? sizeof(int64_t) * (nb + 1) : 0));
        }
    }

    void fill(size_t k) const {
        const Item &it = items[k];
        const Side &sd = sides[it.side];
        const Block &B = blocks[sd.blk];
        int32_t *out = sd.ab ? B.col_ab : B.col_ba;
        int64_t *rp = sd.ab ? B.rp_ab : B.rp_ba;
        const int64_t r1 = std::min(it.r0 + kChunkRows, sd.a1 - sd.a0);
        const int32_t b0 = (int32_t)sd.b0;
        int64_t at = it.off;
        for (int64_t r = it.r0; r < r1; ++r) {
            const int32_t *lo, *hi;
            row_range(sd, r, &lo, &hi);
            rp[r] = at;
            for (const int32_t *q = lo; q < hi; ++q) out[at++] = *q - b0;
        }
        if (r1 == sd.a1 - sd.a0) rp[r1] = at;  // the side's last chunk closes its row pointer
    }
};

// Host sample pools (Sec. 5: host threads draw each kernel's positives and
// ship them to the device just in time; negatives stay device-drawn).  The pool of kernel K_{a,b} in round r holds, for every source
// of the pair (V^a, then V^b when a != b), its B positives as local ids of
// the opposite part, or -1 when it has no neighbour there.  A positive is
// drawn exactly as the device draws it from an edge block (Philox word 0 of
// block (u, 0, level << 32 | r*B + j, tag), a uniform neighbour in the
// opposite part's id range), so both streaming forms train on the same samples.
struct PoolDraw {
    const int64_t *rowptr = nullptr;
    const int32_t *col = nullptr;
    std::vector<int64_t> start;
    int K = 1, B = 1;
    uint32_t level = 0;
    uint64_t seed = 0, graph = 0;

    int64_t sources(int a, int b) const {
        return (start[a + 1] - start[a]) + (a != b ? start[b + 1] - start[b] : 0);
    }
    // sources [s0, s1) of pair (a, b) in round r -> out[(s - s0) * B + j]
    void fill(int a, int b, int r, int64_t s0, int64_t s1, int32_t *out) const {
        const int64_t na = start[a + 1] - start[a];
        const uint64_t tag = K == 1 ? kTagSample : (kTagLarge | ((uint64_t)(a * K + b) << 8));
        for (int64_t s = s0; s < s1; ++s) {
            const bool sideA = s < na;
            const int own = sideA ? a : b, opp = sideA ? b : a;
            const int64_t ug = start[own] + (sideA ? s : s - na);
            const int32_t *row = col + rowptr[ug], *end = col + rowptr[ug + 1];
            const int32_t *lo = std::lower_bound(row, end, (int32_t)start[opp]);
            const int32_t *hi = std::lower_bound(lo, end, (int32_t)start[opp + 1]);
            const uint64_t cnt = (uint64_t)(hi - lo);
            int32_t *o = out + (s - s0) * B;
            for (int j = 0; j < B; ++j) {
                if (cnt == 0) {
                    o[j] = -1;
                    continue;
                }
                const uint32_t t = (uint32_t)(r * B + j);
                const Philox4 w = philox4x64_10((uint64_t)ug, 0, ((uint64_t)level << 32) | t, tag, seed, graph);
                o[j] = lo[uniform_index(w.w[0], cnt)] - (int32_t)start[opp];
            }
        }
    }
};

// The bin that holds part x for kernel i of seq: the bin already holding it
// (*load = false), else (*load = true) an empty bin, else the bin whose part
// is next used farthest ahead in seq.  A bin holding a part of kernel i is
// never chosen, so two bins always suffice.  With spare_prev, bins holding a
// part of kernel i-1 are passed over while another candidate exists: the
// copy then need not wait for that kernel, which may still run (the overlap
// Sec. 5.2 describes: with M^0, M^1, M^5 resident, M^2 replaces M^0 while
// K_{5,1} runs), at the cost of more copies than the farthest-next-use rule.
int large_bin_for(const std::vector<int> &bin_part, const std::vector<std::pair<int, int>> &seq, size_t i, int x,
                  bool spare_prev, bool *load) {
    const int nb = (int)bin_part.size();
    for (int bi = 0; bi < nb; ++bi)
        if (bin_part[bi] == x) {
            *load = false;
            return bi;
        }
    *load = true;
    const int keep0 = seq[i].first, keep1 = seq[i].second;
    const int prev0 = i > 0 ? seq[i - 1].first : -1, prev1 = i > 0 ? seq[i - 1].second : -1;
    for (int pass = spare_prev ? 0 : 1; pass < 2; ++pass) {
        int victim = -1;
        size_t far = 0;
        for (int bi = 0; bi < nb; ++bi) {
            const int part = bin_part[bi];
            if (part == keep0 || part == keep1) continue;
            if (part < 0) return bi;
            if (pass == 0 && (part == prev0 || part == prev1)) continue;
            size_t nxt = seq.size() + 1;
            for (size_t j = i + 1; j < seq.size(); ++j)
                if (seq[j].first == part || seq[j].second == part) {
                    nxt = j;
                    break;
                }
            if (victim < 0 || nxt > far) {
                victim = bi;
                far = nxt;
            }
        }
        if (victim >= 0) return victim;
    }
    return -1;
}

}  // namespace gosh

using namespace gosh;

extern "C" {

/* See include/gosh.h. */
int gosh_large_plan(int64_t n, int K, int p_gpu, int rounds, int evict, int *pairs_out, int *loads_out,
                    int cap_tasks) {
    // Host-only simulation of the submatrix-bin schedule: for each kernel of
    // `rounds` rounds, the pair (a, b) and the part loaded into a bin before
    // it (or -1 entries), with the bin choice of gosh_train_level_large
    // (large_bin_for: farthest next use).
    if (K < 1 || p_gpu < 2 || p_gpu > 999 || rounds < 0 || (evict != 0 && evict != 1) || cap_tasks < 0 ||
        (cap_tasks > 0 && (!pairs_out || !loads_out)))
        return -2;
    if ((int64_t)rounds * K * (K + 1) / 2 > cap_tasks) return -1;
    std::vector<std::pair<int, int>> order;
    large_pair_order(K, order);
    std::vector<std::pair<int, int>> seq;
    for (int r = 0; r < rounds; ++r)
        for (auto &pr : order) seq.push_back(pr);
    std::vector<int> bin(p_gpu, -1);
    for (size_t i = 0; i < seq.size(); ++i) {
        const int need[2] = {seq[i].first, seq[i].second};
        int loads[2] = {-1, -1};
        for (int q = 0; q < 2; ++q) {
            bool load = false;
            const int victim = large_bin_for(bin, seq, i, need[q], evict == 1, &load);
            if (!load) continue;
            bin[victim] = need[q];
            loads[q] = need[q] * 1000 + victim;  // part * 1000 + bin
        }
        pairs_out[2 * i] = seq[i].first;
        pairs_out[2 * i + 1] = seq[i].second;
        loads_out[2 * i] = loads[0];
        loads_out[2 * i + 1] = loads[1];
    }
    (void)n;
    return (int)seq.size();
}

gosh_status gosh_large_block(const gosh_csr *g, int K, int a, int b, int64_t *m_ab, int64_t *m_ba, int64_t *rp_ab,
                             int32_t *col_ab, int64_t *rp_ba, int32_t *col_ba) {
    clear_error();
    GOSH_CHECK_ARG(g && !g->on_device && g->rowptr && g->col, "needs a host CSR");
    GOSH_CHECK_ARG(g->n >= 1 && g->n < (int64_t(1) << 31), "bad n");
    GOSH_CHECK_ARG(K >= 1 && K <= g->n, "need 1 <= K <= n");
    GOSH_CHECK_ARG(0 <= b && b <= a && a < K, "need 0 <= b <= a < K");
    GOSH_CHECK_ARG(m_ab && m_ba, "m_ab and m_ba are required");
    GOSH_TRY(check_host_csr(g->rowptr, g->col, g->n, false));
    std::vector<int64_t> start(K + 1);
    for (int i = 0; i <= K; ++i) start[i] = g->n * i / K;
    EdgeBlocks eb;
    eb.plan(g->rowptr, g->col, K, start, 1);
    const size_t i = (size_t)a * (a + 1) / 2 + b;  // position of (a, b) in the inside-out order
    GOSH_CHECK_ARG(eb.order[i] == std::make_pair(a, b), "pair order mismatch");
    *m_ab = eb.blocks[i].m_ab;
    *m_ba = eb.blocks[i].m_ba;
    if (!rp_ab) return GOSH_OK;  // sizes only
    GOSH_CHECK_ARG(col_ab && (a == b || (rp_ba && col_ba)), "NULL output");
    std::vector<char> region(eb.total_bytes);
    eb.place(region.data());
    for (size_t k = 0; k < eb.items.size(); ++k)
        if (eb.sides[eb.items[k].side].blk == (int)i) eb.fill(k);
    const Block &B = eb.blocks[i];
    const int64_t na = start[a + 1] - start[a], nb = start[b + 1] - start[b];
    std::memcpy(rp_ab, B.rp_ab, sizeof(int64_t) * (na + 1));
    std::memcpy(col_ab, B.col_ab, sizeof(int32_t) * B.m_ab);
    if (a != b) {
        std::memcpy(rp_ba, B.rp_ba, sizeof(int64_t) * (nb + 1));
        std::memcpy(col_ba, B.col_ba, sizeof(int32_t) * B.m_ba);
    }
    return GOSH_OK;
}

gosh_status gosh_large_pool(const gosh_csr *g, int K, int a, int b, int round, int B, int level, uint64_t seed,
                            uint64_t graph_id, int32_t *out) {
    clear_error();
    GOSH_CHECK_ARG(g && !g->on_device && g->rowptr && g->col && out, "needs a host CSR and an output");
    GOSH_CHECK_ARG(g->n >= 1 && g->n < (int64_t(1) << 31), "bad n");
    GOSH_CHECK_ARG(K >= 1 && K <= g->n, "need 1 <= K <= n");
    GOSH_CHECK_ARG(0 <= b && b <= a && a < K, "need 0 <= b <= a < K");
    GOSH_CHECK_ARG(B >= 1 && round >= 0 && level >= 0, "bad B / round / level");
    GOSH_TRY(check_host_csr(g->rowptr, g->col, g->n, false));
    PoolDraw pd;
    pd.rowptr = g->rowptr;
    pd.col = g->col;
    pd.start.resize(K + 1);
    for (int i = 0; i <= K; ++i) pd.start[i] = g->n * i / K;
    pd.K = K;
    pd.B = B;
    pd.level = (uint32_t)level;
    pd.seed = seed;
    pd.graph = graph_id;
    pd.fill(a, b, round, 0, pd.sources(a, b), out);
    return GOSH_OK;
}

gosh_status gosh_train_level_large(const gosh_csr *g, void *M, int level, int epochs, const gosh_params *p,
                                   void *stream, gosh_large_stats *stats) {
    clear_error();
    GOSH_CHECK_ARG(g && p && M, "NULL argument");
    GOSH_TRY(check_params(p));
    GOSH_CHECK_ARG(!g->on_device, "gosh_train_level_large takes a host CSR (it streams it)");
    GOSH_CHECK_ARG(g->n >= 1 && g->n < (int64_t(1) << 31), "bad n");
    GOSH_CHECK_ARG(p->mode == GOSH_HOGWILD, "LargeGraphGPU is lock-free (GOSH_HOGWILD)");
    GOSH_CHECK_ARG(p->B >= 1 && p->B * (p->k + 1) <= kMaxSlots && p->B <= 8, "need 1 <= B <= 8 and B*(k+1) <= %d",
                   kMaxSlots);
    GOSH_CHECK_ARG(p->p_gpu >= 2 && p->s_gpu >= 1, "need P_GPU >= 2 and S_GPU >= 1");
    GOSH_CHECK_ARG(p->large_evict == 0 || p->large_evict == 1, "large_evict must be 0 or 1");
    const PairLaunch launch = pick_pair_kernel(p->dtype, p->d);
    GOSH_CHECK_ARG(launch != nullptr, "LargeGraphGPU serves FP32 / BF16 with d in {32, 64, 128}");
    GOSH_CHECK_ARG(g->rowptr && g->col, "csr pointers are NULL");
    if (p->validate) GOSH_TRY(check_host_csr(g->rowptr, g->col, g->n, false));
    const auto t_start = std::chrono::steady_clock::now();
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = g->n;
    const size_t row = (size_t)p->d * dtype_size(p->dtype);
    const int64_t nnz = g->rowptr[n];

    // ---- K from the budget (reading of "increasing P_GPU increases K") ----
    int K = p->large_parts;
    const int64_t budget = p->device_budget_bytes;
    if (K <= 0) {
        GOSH_CHECK_ARG(budget > 0, "give device_budget_bytes or large_parts");
        // edge bins take up to 40% of the budget, part bins the rest
        const double part_budget = 0.6 * (double)budget / p->p_gpu;
        K = std::max(p->p_gpu, (int)std::ceil((double)n * row / part_budget));
    }
    K = (int)std::min<int64_t>(K, n);
    std::vector<int64_t> start(K + 1);
    for (int i = 0; i <= K; ++i) start[i] = n * i / K;

    // ---- positive samples: edge blocks or host sample pools ----
    // Edge blocks (default): only the count pass and the layout run up front
    // (EdgeBlocks::plan); the blocks then sit in one pinned region (kept
    // across calls, grow-only: pinning host memory costs far more than
    // building), and their row chunks are filled by the threads that overlap
    // the stream loop below.  Sample pools (large_pools = 1): host threads
    // draw every kernel's positives, in kernel order, into a ring of pinned
    // slots, running ahead of the stream loop by up to the ring's length.
    const bool use_pools = p->large_pools != 0;
    const int nt = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    std::vector<std::pair<int, int>> order;
    large_pair_order(K, order);
    EdgeBlocks eb;
    PinnedLease lease(g_pinned);
    PoolDraw pd;
    size_t max_pool = 0;
    if (!use_pools) {
        eb.plan(g->rowptr, g->col, K, start, nt);
        GOSH_TRY(lease.acquire(eb.total_bytes, "edge blocks"));
        eb.place(lease.ptr);
    } else {
        pd.rowptr = g->rowptr;
        pd.col = g->col;
        pd.start = start;
        pd.K = K;
        pd.B = p->B;
        pd.level = (uint32_t)level;
        pd.seed = p->seed;
        pd.graph = p->graph_id;
        for (auto &pr : order)
            max_pool = std::max(max_pool, (size_t)pd.sources(pr.first, pr.second) * p->B * sizeof(int32_t));
        max_pool = (max_pool + 255) / 256 * 256;
    }
    const std::vector<Block> &blocks = eb.blocks;
    const size_t max_block = use_pools ? max_pool : eb.max_block;
    int64_t part_rows = 0;
    for (int i = 0; i < K; ++i) part_rows = std::max(part_rows, start[i + 1] - start[i]);
    const size_t bin_bytes = row * part_rows;
    const size_t need = bin_bytes * p->p_gpu + max_block * p->s_gpu;
    if (budget > 0 && (int64_t)need > budget) {
        set_error("LargeGraphGPU: %d parts need %zu bytes of bins (> budget %lld); raise K (large_parts)", K, need,
                  (long long)budget);
        return GOSH_ERR_BUDGET;
    }

    // The entries of the blocks are copied by host threads in block order
    // while the stream loop below already sends the finished blocks: block i's
    // first copy to the device waits only for block i (the items are ordered
    // by block, so the first blocks finish first).
    struct BlockGate {
        std::mutex mu;
        std::condition_variable cv;
        std::vector<int> left;
        std::atomic<size_t> next{0};
        std::vector<std::thread> th;
        void wait(int b) {
            std::unique_lock<std::mutex> lk(mu);
            cv.wait(lk, [&] { return left[b] == 0; });
        }
        ~BlockGate() {
            for (auto &x : th) x.join();
        }
    } gate;
    if (!use_pools) {
        std::vector<int> items_left(blocks.size(), 0);
        for (const auto &it : eb.items) ++items_left[eb.sides[it.side].blk];
        gate.left = items_left;
        for (int t = 0; t < nt; ++t)
            gate.th.emplace_back([&]() {
                for (size_t k = gate.next.fetch_add(1); k < eb.items.size(); k = gate.next.fetch_add(1)) {
                    eb.fill(k);
                    const int blk = eb.sides[eb.items[k].side].blk;
                    bool done;
                    {
                        std::lock_guard<std::mutex> lk(gate.mu);
                        done = --gate.left[blk] == 0;
                    }
                    if (done) gate.cv.notify_all();
                }
            });
    }

    // host M pinned for async copies (registered in place if the caller's is pageable)
    bool registered = false;
    {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, M) != cudaSuccess || at.type == cudaMemoryTypeUnregistered) {
            cudaGetLastError();
            if (cudaHostRegister(M, row * n, cudaHostRegisterDefault) == cudaSuccess) registered = true;
            else cudaGetLastError();
        }
    }
    struct Unreg {
        void *p;
        bool on;
        ~Unreg() {
            if (on) cudaHostUnregister(p);
        }
    } unreg{M, registered};

    // ---- device bins, streams, events ----
    std::vector<Scratch> pbin(p->p_gpu), ebin(p->s_gpu);
    for (auto &b : pbin) GOSH_TRY(b.alloc(bin_bytes, s));
    for (auto &b : ebin) GOSH_TRY(b.alloc(max_block, s));
    Scratch counters;
    GOSH_TRY(counters.alloc(2 * sizeof(unsigned long long), s));
    GOSH_TRY_CUDA(cudaMemsetAsync(counters.ptr, 0, 2 * sizeof(unsigned long long), s));
    GOSH_TRY_CUDA(cudaStreamSynchronize(s));
    std::vector<cudaStream_t> pstr(p->p_gpu), estr(p->s_gpu), kstr(2);
    for (auto &x : pstr) GOSH_TRY_CUDA(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
    for (auto &x : estr) GOSH_TRY_CUDA(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
    for (auto &x : kstr) GOSH_TRY_CUDA(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
    std::vector<cudaEvent_t> pool;
    auto new_event = [&](cudaStream_t st) {
        cudaEvent_t e;
        cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
        cudaEventRecord(e, st);
        pool.push_back(e);
        return e;
    };
    struct Cleanup {
        std::vector<cudaStream_t> &a, &b, &c;
        std::vector<cudaEvent_t> &ev;
        ~Cleanup() {
            for (auto *v : {&a, &b, &c})
                for (auto x : *v) {
                    cudaStreamSynchronize(x);
                    cudaStreamDestroy(x);
                }
            for (auto e : ev) cudaEventDestroy(e);
        }
    } cleanup{pstr, estr, kstr, pool};

    const int rounds = (epochs + p->B - 1) / p->B;
    std::vector<std::pair<int, int>> seq;
    for (int r = 0; r < rounds; ++r)
        for (auto &pr : order) seq.push_back(pr);

    // Sample pools: items of kPoolChunk sources of kernel i, taken by host
    // threads in kernel order; kernel i's pool goes into ring slot i % R once
    // the copy of the pool that used the slot before (kernel i - R) has
    // completed; the stream loop sends pool i when all its items are done.
    constexpr int64_t kPoolChunk = 16384;
    const int R = std::max(2, p->s_gpu + 2);
    PinnedLease pool_lease(g_pinned_pools);
    struct PoolGate {
        std::mutex mu;
        std::condition_variable cv;
        std::vector<int> left;
        std::vector<cudaEvent_t> copied;  // H2D copy of pool i (recorded by the stream loop)
        std::atomic<size_t> next{0};
        bool stop = false;
        std::vector<std::thread> th;
        ~PoolGate() {
            {
                std::lock_guard<std::mutex> lk(mu);
                stop = true;
            }
            cv.notify_all();
            for (auto &x : th) x.join();
        }
    } pgate;
    struct PoolItem {
        size_t kernel;
        int64_t s0, s1;
    };
    std::vector<PoolItem> pitems;
    if (use_pools) {
        GOSH_TRY(pool_lease.acquire(max_pool * R, "sample pools"));
        pgate.left.assign(seq.size(), 0);
        pgate.copied.assign(seq.size(), nullptr);
        for (size_t i = 0; i < seq.size(); ++i) {
            const int64_t ns = pd.sources(seq[i].first, seq[i].second);
            for (int64_t s0 = 0; s0 < ns; s0 += kPoolChunk) {
                pitems.push_back({i, s0, std::min(ns, s0 + kPoolChunk)});
                ++pgate.left[i];
            }
        }
        const size_t per_round = order.size();
        for (int t = 0; t < nt; ++t)
            pgate.th.emplace_back([&, per_round]() {
                for (size_t k = pgate.next.fetch_add(1); k < pitems.size(); k = pgate.next.fetch_add(1)) {
                    const PoolItem &it = pitems[k];
                    const size_t i = it.kernel;
                    if (i >= (size_t)R) {  // the slot's previous pool must be on the device
                        cudaEvent_t ev = nullptr;
                        {
                            std::unique_lock<std::mutex> lk(pgate.mu);
                            pgate.cv.wait(lk, [&] { return pgate.stop || pgate.copied[i - R] != nullptr; });
                            if (pgate.stop) return;
                            ev = pgate.copied[i - R];
                        }
                        cudaEventSynchronize(ev);
                    }
                    int32_t *slot = reinterpret_cast<int32_t *>(pool_lease.ptr + (i % R) * max_pool);
                    pd.fill(seq[i].first, seq[i].second, (int)(i / per_round), it.s0, it.s1, slot + it.s0 * p->B);
                    bool done;
                    {
                        std::lock_guard<std::mutex> lk(pgate.mu);
                        done = --pgate.left[i] == 0;
                    }
                    if (done) pgate.cv.notify_all();
                }
            });
    }
    std::vector<int> bin_part(p->p_gpu, -1);
    std::vector<std::vector<cudaEvent_t>> bin_users(p->p_gpu);     // kernels using the bin since its load
    std::vector<cudaEvent_t> bin_ready(p->p_gpu, nullptr);
    std::vector<cudaEvent_t> host_fresh(K, nullptr);               // D2H of part x completed
    std::vector<cudaEvent_t> ebin_free(p->s_gpu, nullptr);
    const auto t_setup = std::chrono::steady_clock::now();
    int64_t swaps = 0, h2d = 0, d2h = 0, block_bytes = 0;
    const int grid = num_sms() * 2;
    char *hM = static_cast<char *>(M);

    auto ensure = [&](int x, size_t i) -> int {
        bool load = false;
        const int victim = large_bin_for(bin_part, seq, i, x, p->large_evict == 1, &load);
        if (!load) return victim;
        cudaStream_t st = pstr[victim];
        for (cudaEvent_t e : bin_users[victim]) cudaStreamWaitEvent(st, e, 0);
        bin_users[victim].clear();
        const int old = bin_part[victim];
        if (old >= 0) {  // MST, first half: the evicted part goes home
            const size_t bytes = row * (start[old + 1] - start[old]);
            cudaMemcpyAsync(hM + row * start[old], pbin[victim].ptr, bytes, cudaMemcpyDeviceToHost, st);
            host_fresh[old] = new_event(st);
            d2h += bytes;
        }
        if (host_fresh[x]) cudaStreamWaitEvent(st, host_fresh[x], 0);
        const size_t bytes = row * (start[x + 1] - start[x]);
        cudaMemcpyAsync(pbin[victim].ptr, hM + row * start[x], bytes, cudaMemcpyHostToDevice, st);
        h2d += bytes;
        bin_ready[victim] = new_event(st);
        bin_part[victim] = x;
        ++swaps;
        return victim;
    };

    for (size_t i = 0; i < seq.size(); ++i) {
        const int a = seq[i].first, b = seq[i].second;
        const int r = (int)(i / order.size());
        const int ba = ensure(a, i);
        const int bb = ensure(b, i);
        // SCT: the edge block, or the kernel's sample pool, into the next bin
        const int eb = (int)(i % p->s_gpu);
        const Block *blk = use_pools ? nullptr : &blocks[i % order.size()];
        if (ebin_free[eb]) cudaStreamWaitEvent(estr[eb], ebin_free[eb], 0);
        cudaEvent_t e_ready;
        if (!use_pools) {
            if (i < order.size()) gate.wait((int)i);
            cudaMemcpyAsync(ebin[eb].ptr, blk->base, blk->bytes, cudaMemcpyHostToDevice, estr[eb]);
            block_bytes += blk->bytes;
            e_ready = new_event(estr[eb]);
        } else {
            {
                std::unique_lock<std::mutex> lk(pgate.mu);
                pgate.cv.wait(lk, [&] { return pgate.left[i] == 0; });
            }
            const size_t bytes = (size_t)pd.sources(a, b) * p->B * sizeof(int32_t);
            cudaMemcpyAsync(ebin[eb].ptr, pool_lease.ptr + (i % R) * max_pool, bytes, cudaMemcpyHostToDevice,
                            estr[eb]);
            block_bytes += bytes;
            e_ready = new_event(estr[eb]);
            {
                std::lock_guard<std::mutex> lk(pgate.mu);
                pgate.copied[i] = e_ready;
            }
            pgate.cv.notify_all();
        }
        // KT
        cudaStream_t ks = kstr[p->large_serial ? 0 : i % 2];
        cudaStreamWaitEvent(ks, bin_ready[ba], 0);
        cudaStreamWaitEvent(ks, bin_ready[bb], 0);
        cudaStreamWaitEvent(ks, e_ready, 0);
        PairArgs pa{};
        const char *eb0 = ebin[eb].as<char>();
        pa.Ma = pbin[ba].ptr;
        pa.Mb = pbin[bb].ptr;
        pa.na = start[a + 1] - start[a];
        pa.nb = start[b + 1] - start[b];
        pa.start_a = start[a];
        pa.start_b = start[b];
        if (!use_pools) {
            pa.rp_ab = reinterpret_cast<const int64_t *>(eb0 + ((char *)blk->rp_ab - blk->base));
            pa.col_ab = reinterpret_cast<const int32_t *>(eb0 + ((char *)blk->col_ab - blk->base));
            pa.rp_ba = reinterpret_cast<const int64_t *>(eb0 + ((char *)blk->rp_ba - blk->base));
            pa.col_ba = reinterpret_cast<const int32_t *>(eb0 + ((char *)blk->col_ba - blk->base));
        } else {
            pa.pool = reinterpret_cast<const int32_t *>(eb0);
        }
        pa.same = a == b;
        pa.B = p->B;
        pa.k = p->k;
        pa.epochs_total = epochs;
        pa.round = r;
        pa.lr = (float)p->lr;
        pa.lr_floor = (float)p->lr_floor;
        pa.seed = p->seed;
        pa.graph = p->graph_id;
        pa.tag = K == 1 ? kTagSample : (kTagLarge | ((uint64_t)(a * K + b) << 8));
        pa.level = (uint32_t)level;
        pa.positives = counters.as<unsigned long long>();
        pa.cap = (unsigned long long)epochs * (unsigned long long)n;
        pa.n_updates = counters.as<unsigned long long>() + 1;
        launch(pa, grid, ks);
        cudaEvent_t kdone = new_event(ks);
        bin_users[ba].push_back(kdone);
        if (bb != ba) bin_users[bb].push_back(kdone);
        ebin_free[eb] = kdone;
    }
    // write every resident part back
    for (int bi = 0; bi < p->p_gpu; ++bi) {
        if (bin_part[bi] < 0) continue;
        for (cudaEvent_t e : bin_users[bi]) cudaStreamWaitEvent(pstr[bi], e, 0);
        const int x = bin_part[bi];
        const size_t bytes = row * (start[x + 1] - start[x]);
        cudaMemcpyAsync(hM + row * start[x], pbin[bi].ptr, bytes, cudaMemcpyDeviceToHost, pstr[bi]);
        d2h += bytes;
    }
    unsigned long long hc[2] = {0, 0};
    for (auto x : pstr) GOSH_TRY_CUDA(cudaStreamSynchronize(x));
    for (auto x : kstr) GOSH_TRY_CUDA(cudaStreamSynchronize(x));
    for (auto x : estr) GOSH_TRY_CUDA(cudaStreamSynchronize(x));
    GOSH_TRY_CUDA(cudaMemcpy(hc, counters.ptr, sizeof(hc), cudaMemcpyDeviceToHost));
    GOSH_TRY_CUDA(cudaGetLastError());
    if (stats) {
        stats->parts = K;
        stats->rounds = rounds;
        stats->kernels = (int64_t)seq.size();
        stats->swaps = swaps;
        stats->h2d_bytes = h2d + block_bytes;
        stats->d2h_bytes = d2h;
        stats->positives = hc[0] < (unsigned long long)epochs * n ? hc[0] : (unsigned long long)epochs * n;
        stats->updates = hc[1];
        stats->device_bytes = (int64_t)need;
        stats->total_ms =
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
        stats->setup_ms = std::chrono::duration<double, std::milli>(t_setup - t_start).count();
    }
    (void)nnz;
    return GOSH_OK;
}

}  // extern "C"
