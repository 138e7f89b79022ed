// MULTIEDGECOLLAPSE (Alg. 4) on the GPU, with maps identical to the
// sequential greedy algorithm.
//
// The greedy walk in degree order makes v a cluster root ("hub") exactly when
// no earlier-ranked eligible neighbour of v is a hub, i.e. the hubs are the
// lexicographically-first maximal independent set, in rank order, of the
// graph of eligible edges (hub^2 restriction: deg(u) <= delta or deg(v) <=
// delta).  A non-hub is absorbed by the first hub that reaches it, which is
// its earliest-ranked eligible hub neighbour.  Cluster ids follow hub rank.
// So one level is:
//   1. order = stable sort by descending degree (radix sort), rank = order^-1;
//   2. rounds of the MIS rule until every vertex is decided (each round
//      decides at least the lowest-ranked undecided vertex; decisions made
//      earlier in the same round are visible, which usually settles long
//      dependency chains in a handful of rounds);
//   3. each non-hub takes its earliest-ranked eligible hub neighbour;
//      cluster id = number of hubs ranked before the hub (prefix sum);
//   4. COARSEN: coarse row c = the set of map[u] over the edges (v, u) of
//      the members v of cluster c, minus c: built in a shared-memory bitmap
//      over the coarse ids and read back in ascending order (sorted, unique);
//      above 2^19 coarse vertices, by a radix sort of packed (map v, map u)
//      keys instead.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <vector>

#include "hierarchy.cuh"

namespace gosh {
namespace {

enum : uint8_t { kUndecided = 0, kHub = 1, kNonHub = 2 };

__device__ __forceinline__ bool small_deg(int64_t deg, int64_t n, int64_t nnz) { return deg * n <= nnz; }

__global__ void invert_order(const uint32_t *__restrict__ order, int64_t n, int32_t *__restrict__ rank) {
    GOSH_DEP_WAIT();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        rank[order[i]] = (int32_t)i;
}

// Sort key (n - 1) - deg (a simple graph has deg <= n - 1): ascending keys
// are descending degrees, and the sort needs only the bits of n - 1.
// Initial MIS state: a vertex above the density (deg * n > nnz) has no
// eligible earlier-ranked neighbour (eligibility needs the other end at or
// below the density, and an earlier rank needs a degree at least as large),
// so it is a cluster root from the start; only vertices at or below the
// density (whose every edge is eligible and whose rows are at most the
// average degree long) go through the rounds.
__global__ void degree_keys(const int64_t *__restrict__ rowptr, int64_t n, uint32_t *__restrict__ key,
                            uint32_t *__restrict__ val, uint8_t *__restrict__ state) {
    GOSH_DEP_WAIT();
    const int64_t nnz = rowptr[n];
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t deg = rowptr[v + 1] - rowptr[v];
        key[v] = deg < n ? (uint32_t)(n - 1 - deg) : 0u;
        val[v] = (uint32_t)v;
        state[v] = small_deg(deg, n, nnz) ? kUndecided : kHub;
    }
}

// One round of the MIS rule, one thread per rank position (so a warp holds
// vertices of nearly equal degree): v becomes a non-hub if an earlier-ranked
// neighbour is a hub, a hub if every earlier-ranked neighbour is a non-hub,
// and stays undecided otherwise.  Decisions are final, so reading states that
// other threads set during the same round is safe and speeds convergence.
__global__ void __launch_bounds__(256) mis_round(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                                                 int64_t n, const uint32_t *__restrict__ order,
                                                 const int32_t *__restrict__ rank, uint8_t *state,
                                                 unsigned long long *__restrict__ undecided) {
    GOSH_DEP_WAIT();
    volatile uint8_t *vstate = state;
    unsigned long long left = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = (int32_t)order[i];
        if (vstate[v] != kUndecided) continue;
        bool hub_seen = false, open_seen = false;
        for (int64_t p = rowptr[v], e = rowptr[v + 1]; p < e; ++p) {
            const int32_t u = __ldg(col + p);
            if (__ldg(rank + u) >= (int32_t)i) continue;
            const uint8_t su = vstate[u];
            if (su == kHub) {
                hub_seen = true;
                break;
            }
            open_seen |= su == kUndecided;
        }
        if (hub_seen) vstate[v] = kNonHub;
        else if (!open_seen) vstate[v] = kHub;
        else ++left;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) left += __shfl_xor_sync(0xffffffffu, left, o);
    if ((threadIdx.x & 31) == 0 && left) atomicAdd(undecided, left);
}

// hub_rank[v] = rank of v for hubs; for a non-hub (always at or below the
// density, so all its edges are eligible) the earliest-ranked hub neighbour.
__global__ void attach_to_hub(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col, int64_t n,
                              const int32_t *__restrict__ rank, const uint8_t *__restrict__ state,
                              int32_t *__restrict__ hub_rank) {
    GOSH_DEP_WAIT();
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        if (state[v] == kHub) {
            hub_rank[v] = rank[v];
            continue;
        }
        int32_t best = 0x7fffffff;
        for (int64_t p = rowptr[v], e = rowptr[v + 1]; p < e; ++p) {
            const int32_t u = __ldg(col + p);
            if (state[u] == kHub) best = min(best, __ldg(rank + u));
        }
        hub_rank[v] = best;
    }
}

// The same with one warp per vertex, for dense levels (non-hub rows are up to
// the average degree long, hundreds of entries on the small levels).
__global__ void __launch_bounds__(256) attach_to_hub_warp(const int64_t *__restrict__ rowptr,
                                                          const int32_t *__restrict__ col, int64_t n,
                                                          const int32_t *__restrict__ rank,
                                                          const uint8_t *__restrict__ state,
                                                          int32_t *__restrict__ hub_rank) {
    GOSH_DEP_WAIT();
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t wstride = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = wid; v < n; v += wstride) {
        if (state[v] == kHub) {
            if (lane == 0) hub_rank[v] = rank[v];
            continue;
        }
        int32_t best = 0x7fffffff;
        for (int64_t p = rowptr[v] + lane, e = rowptr[v + 1]; p < e; p += 32) {
            const int32_t u = __ldg(col + p);
            if (state[u] == kHub) best = min(best, __ldg(rank + u));
        }
        best = __reduce_min_sync(0xffffffffu, best);
        if (lane == 0) hub_rank[v] = best;
    }
}

__global__ void hub_flags_by_rank(const uint32_t *__restrict__ order, const uint8_t *__restrict__ state, int64_t n,
                                  uint8_t *__restrict__ flag) {
    GOSH_DEP_WAIT();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = state[order[i]] == kHub ? 1 : 0;
}

// A non-hub always has an earlier eligible hub neighbour (maximality); a
// vertex without one would be a logic error: it is flagged, not followed.
__global__ void assign_map(const int32_t *__restrict__ hub_rank, const int64_t *__restrict__ cid_of_rank, int64_t n,
                           int32_t *__restrict__ map, unsigned long long *__restrict__ orphan) {
    GOSH_DEP_WAIT();
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t hr = hub_rank[v];
        if (hr >= 0 && hr < n) {
            map[v] = (int32_t)cid_of_rank[hr];
        } else {
            map[v] = 0;
            atomicAdd(orphan, 1ull);
        }
    }
}

// Key of every CSR entry (v, u): map v * nc + map u, or the sentinel nc * nc for
// a self-loop (packed so the sort needs only ceil(log2(nc^2) / 8) passes).
// Balanced over entries: each warp takes 1024 consecutive entries; a lane finds
// the row of its first entry by binary search and then walks forward.
constexpr int kEntriesPerWarp = 1024;
__global__ void __launch_bounds__(256) edge_image(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                                                  int64_t n, const int32_t *__restrict__ map, uint64_t nc,
                                                  uint64_t *__restrict__ keys) {
    GOSH_DEP_WAIT();
    const int lane = threadIdx.x & 31;
    const int64_t nnz = rowptr[n];
    const int64_t sentinel = (int64_t)(nc * nc);
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t wstride = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = wid * kEntriesPerWarp; base < nnz; base += wstride * kEntriesPerWarp) {
        int64_t p = base + lane;
        if (p >= nnz) continue;
        int64_t lo = 0, hi = n;  // last row with rowptr[row] <= p
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (__ldg(rowptr + mid) <= p) lo = mid; else hi = mid;
        }
        int64_t r = lo;
        int64_t rend = __ldg(rowptr + r + 1);
        uint64_t a = (uint64_t)__ldg(map + r);
        const int64_t end = base + kEntriesPerWarp < nnz ? base + kEntriesPerWarp : nnz;
        for (; p < end; p += 32) {
            while (rend <= p) {
                ++r;
                rend = __ldg(rowptr + r + 1);
                a = (uint64_t)__ldg(map + r);
            }
            const uint64_t b = (uint64_t)__ldg(map + __ldg(col + p));
            keys[p] = a != b ? a * nc + b : (uint64_t)sentinel;
        }
    }
}

__global__ void unique_flags(const uint64_t *__restrict__ keys, int64_t m, uint64_t sentinel, uint8_t *__restrict__ f) {
    GOSH_DEP_WAIT();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        f[i] = keys[i] != sentinel && (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
}

// Sorted unique keys -> coarse CSR.  The first entry of each row writes the
// row pointers of that row and of the empty rows before it; the last valid
// entry closes the empty rows after it.  No atomics.
__global__ void write_coarse(const uint64_t *__restrict__ keys, const uint8_t *__restrict__ f,
                             const int64_t *__restrict__ pos, int64_t nnz, uint64_t sentinel, int64_t nc,
                             int32_t *__restrict__ col_out, int64_t *__restrict__ rowptr) {
    GOSH_DEP_WAIT();
    const int64_t m = pos[nnz];
    const uint64_t unc = (uint64_t)nc;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnz; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = keys[i];
        if (key == sentinel) continue;
        const int64_t r = (int64_t)(key / unc);
        if (f[i]) col_out[pos[i]] = (int32_t)(key - (uint64_t)r * unc);
        const int64_t rprev = i == 0 ? -1 : (int64_t)(keys[i - 1] / unc);
        for (int64_t c = rprev + 1; c <= r; ++c) rowptr[c] = pos[i];
        if (i + 1 == nnz || keys[i + 1] == sentinel)
            for (int64_t c = r + 1; c <= nc; ++c) rowptr[c] = m;
    }
}

// ---- COARSEN through per-row bitmaps ----------------------------------------
// Coarse row c is the union of map[N(x)] over the members x of cluster c,
// minus c itself.  The members that have neighbours are grouped by cluster
// and their CSR rows, laid end to end, are the "virtual entries" of row c,
// cut into chunks of kChunk entries.  A block takes one chunk and sets bit
// map[y] of a shared-memory bitmap over the coarse ids (of the row's graph,
// for a union of graphs) for each entry, plus one summary bit per nonzero
// 32-bit word, then reads the set bits back in ascending order over the
// front of the row's own entry range: the row comes out sorted and
// deduplicated without a global sort, and only the words the chunk touched
// are visited.  Rows of more than one chunk OR their chunk bitmaps into a
// global bitmap that a second kernel reads back; a compaction then moves
// every row to its CSR position.  The member order inside a cluster
// (atomics) does not matter: a bitmap is a set.
constexpr int kChunk = 4096;
constexpr int kBatch = 8;                    // loads in flight per thread
constexpr int kRowThreads = 128;
constexpr int kSumGroup = 32;                // summary words read back per step
constexpr int kListCap = kSumGroup * 32;     // nonzero bitmap words per step
constexpr int64_t kBitmapMaxDefault = int64_t(1) << 19;

// Sort key of vertex v for grouping the members by cluster: map[v], or nc for
// a vertex without neighbours (it adds no entries and sorts past every cluster).
__global__ void member_keys(const int64_t *__restrict__ rowptr, int64_t n, const int32_t *__restrict__ map,
                            uint32_t nc, uint32_t *__restrict__ key, uint32_t *__restrict__ val) {
    GOSH_DEP_WAIT();
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        key[v] = rowptr[v + 1] > rowptr[v] ? (uint32_t)map[v] : nc;
        val[v] = (uint32_t)v;
    }
}

// From the members sorted by cluster: cstart[c] = first member of cluster c
// (cstart[nc] = number of members with neighbours) and each member's degree.  A position whose key differs from its
// predecessor's writes the starts of every cluster in between (clusters
// without such members are empty).
__global__ void member_layout(const uint32_t *__restrict__ key, const uint32_t *__restrict__ val,
                              const int64_t *__restrict__ rowptr, int64_t n, uint32_t nc,
                              int64_t *__restrict__ cstart, int64_t *__restrict__ mdeg) {
    GOSH_DEP_WAIT();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t v = val[i];
        const int64_t k = key[i];
        mdeg[i] = rowptr[v + 1] - rowptr[v];
        const int64_t kp = i == 0 ? -1 : (int64_t)key[i - 1];
        for (int64_t c = kp + 1; c <= k; ++c) cstart[c] = i;
        if (i == n - 1)
            for (int64_t c = k + 1; c <= (int64_t)nc; ++c) cstart[c] = n;
    }
}

// Last index i in [0, n) with a[i] <= x (a non-decreasing, a[0] <= x), found
// by the whole warp: each round probes 32 evenly spaced positions, so the
// range shrinks 32-fold per dependent load instead of 2-fold.
__device__ __forceinline__ int64_t warp_last_le(const int64_t *__restrict__ a, int64_t n, int64_t x) {
    const int lane = threadIdx.x & 31;
    int64_t lo = 0, hi = n;
    while (hi - lo > 1) {
        const int64_t step = (hi - lo + 31) / 32;
        const int64_t probe = lo + lane * step;
        const bool ok = probe < hi && __ldg(a + probe) <= x;
        const unsigned m = __ballot_sync(0xffffffffu, ok);
        const int64_t k = 31 - __clz(m);  // lane 0 always holds: a[lo] <= x
        lo += k * step;
        hi = lo + step < hi ? lo + step : hi;
    }
    return lo;
}

// Cluster id of every CSR entry, written in member order: the entries of
// member i (vertex mval[i], members sorted by cluster) go to vb[moff[i] ..
// moff[i+1]), so the entries of cluster c's members are vb[moff[cstart c] ..
// moff[cstart c+1]).  Balanced over the output: a warp takes kEntriesPerWarp
// consecutive positions, finds the member holding the first one (one
// warp-wide search), and walks batches of 32 members whose offsets sit in
// its lanes: each position finds its member by a shuffle search among them,
// so the gathers of col and map carry no dependent index loads.
__global__ void __launch_bounds__(256) member_entries(const int64_t *__restrict__ rowptr,
                                                      const int32_t *__restrict__ col, int64_t n,
                                                      const int32_t *__restrict__ map,
                                                      const uint32_t *__restrict__ mval,
                                                      const int64_t *__restrict__ moff, int32_t *__restrict__ vb) {
    GOSH_DEP_WAIT();
    constexpr int U = 4;  // positions per lane per step
    const int lane = threadIdx.x & 31;
    const int64_t total = moff[n];
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t wstride = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t o0 = wid * kEntriesPerWarp; o0 < total; o0 += wstride * kEntriesPerWarp) {
        const int64_t o1 = o0 + kEntriesPerWarp < total ? o0 + kEntriesPerWarp : total;
        int64_t i = warp_last_le(moff, n, o0);
        while (true) {
            const int64_t im = i + lane;
            const bool valid = im < n;
            const int64_t mo = valid ? __ldg(moff + im) : total;
            const int64_t me = valid ? __ldg(moff + im + 1) : total;
            const int64_t rs = valid ? __ldg(rowptr + __ldg(mval + im)) : 0;
            const int64_t first = __shfl_sync(0xffffffffu, mo, 0);
            if (i >= n || first >= o1) break;
            const int64_t lo_pos = first > o0 ? first : o0;
            const int64_t last = __shfl_sync(0xffffffffu, me, 31);
            const int64_t hi_pos = last < o1 ? last : o1;
            for (int64_t base = lo_pos; base < hi_pos; base += 32 * U) {
                int64_t src[U];
                int32_t y[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int64_t o = base + u * 32 + lane;
                    int j = 0;  // last lane whose member starts at or before o
#pragma unroll
                    for (int w = 16; w > 0; w >>= 1) {
                        const int64_t t = __shfl_sync(0xffffffffu, mo, j + w);
                        if (t <= o) j += w;
                    }
                    const int64_t s0 = __shfl_sync(0xffffffffu, rs, j);
                    const int64_t m0 = __shfl_sync(0xffffffffu, mo, j);
                    src[u] = s0 + (o - m0);
                    y[u] = o < hi_pos ? __ldg(col + src[u]) : 0;
                }
                int32_t b[U];
#pragma unroll
                for (int u = 0; u < U; ++u) b[u] = __ldg(map + y[u]);
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int64_t o = base + u * 32 + lane;
                    if (o < hi_pos) vb[o] = b[u];
                }
            }
            if (last >= o1) break;
            i += 32;
        }
    }
}

__global__ void row_chunks(const int64_t *__restrict__ cstart, const int64_t *__restrict__ moff, int64_t nc,
                           int32_t *__restrict__ nchunk, uint8_t *__restrict__ multi, int32_t *__restrict__ count) {
    GOSH_DEP_WAIT();
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x) {
        count[c] = 0;  // rows without entries keep it
        const int64_t len = moff[cstart[c + 1]] - moff[cstart[c]];
        const int64_t k = (len + kChunk - 1) / kChunk;
        nchunk[c] = (int32_t)k;
        multi[c] = k > 1 ? 1 : 0;
    }
}

// One chunk of a coarse row: entries [e0, e0 + len) of the member-order vb
// (the row's entries start at rb), cluster c, and whether the row has more
// than one chunk.  One 24-byte record per chunk instead of a chain of
// dependent index loads in the kernels that walk the chunks.
struct ChunkInfo {
    int64_t e0;
    int64_t rb;
    int32_t len;
    int32_t c;     // bit 31: the row has several chunks
    int32_t base;  // first coarse id of the row's graph (unions of graphs; else 0)
    int32_t pad;
};

__global__ void chunk_rows(const int64_t *__restrict__ chunk_start, const uint8_t *__restrict__ multi,
                           const int64_t *__restrict__ slot, const int64_t *__restrict__ cstart,
                           const int64_t *__restrict__ moff, const int32_t *__restrict__ cbase, int64_t nc,
                           ChunkInfo *__restrict__ info, int32_t *__restrict__ slot_row) {
    GOSH_DEP_WAIT();
    // a thread per cluster reads its layout; the warp then writes the
    // clusters' chunk records together (a hub's row has many chunks)
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); c0 < nc; c0 += stride) {
        const int64_t c = c0 + lane;
        int64_t rb = 0, re = 0, t0 = 0, t1 = 0;
        int32_t base = 0;
        bool many = false;
        if (c < nc) {
            if (cbase) base = cbase[c];
            rb = moff[cstart[c]];
            re = moff[cstart[c + 1]];
            t0 = chunk_start[c];
            t1 = chunk_start[c + 1];
            many = multi[c] != 0;
            if (many) slot_row[slot[c]] = (int32_t)c;
        }
        for (int j = 0; j < 32; ++j) {
            const int64_t jt0 = __shfl_sync(0xffffffffu, t0, j), jt1 = __shfl_sync(0xffffffffu, t1, j);
            const int64_t jrb = __shfl_sync(0xffffffffu, rb, j), jre = __shfl_sync(0xffffffffu, re, j);
            const bool jmany = __shfl_sync(0xffffffffu, many ? 1 : 0, j) != 0;
            const int32_t jbase = __shfl_sync(0xffffffffu, base, j);
            for (int64_t t = jt0 + lane; t < jt1; t += 32) {
                ChunkInfo ci;
                ci.e0 = jrb + (t - jt0) * kChunk;
                ci.rb = jrb;
                ci.len = (int32_t)(jre - ci.e0 < kChunk ? jre - ci.e0 : kChunk);
                ci.c = (int32_t)(c0 + j) | (jmany ? (int32_t)0x80000000 : 0);
                ci.base = jbase;
                ci.pad = 0;
                info[t] = ci;
            }
        }
    }
}

// Exclusive prefix sum over the block (kRowThreads threads); every thread
// gets the block total.  wsum: kRowThreads / 32 shared ints.
__device__ __forceinline__ int block_scan(int x, int *wsum, int &total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    int off = 0;
    total = 0;
#pragma unroll
    for (int i = 0; i < kRowThreads / 32; ++i) {
        const int t = wsum[i];
        off += i < w ? t : 0;
        total += t;
    }
    __syncthreads();
    return off + incl - x;
}

// Writes base + the set bits of bm (its nonzero words flagged in sum, n0
// summary words) in ascending order to out and returns their number (in every
// thread).  kClear: zero the visited words (shared-memory bitmaps are reused).
template <bool kClear>
__device__ int read_bits(uint32_t *bm, uint32_t *sum, int n0, int32_t *list, int *wsum, int32_t *__restrict__ out,
                         int32_t base) {
    int nout = 0;
    for (int s0 = 0; s0 < n0; s0 += kSumGroup) {
        const int s = s0 + threadIdx.x;
        const bool mine = threadIdx.x < kSumGroup && s < n0;
        uint32_t sw = mine ? sum[s] : 0u;
        if (kClear && mine) sum[s] = 0;
        int nlist;
        int k = block_scan(__popc(sw), wsum, nlist);
        while (sw) {
            list[k++] = s * 32 + (__ffs(sw) - 1);
            sw &= sw - 1;
        }
        __syncthreads();
        for (int i0 = 0; i0 < nlist; i0 += kRowThreads) {
            const int i = i0 + threadIdx.x;
            int w = 0;
            uint32_t bits = 0;
            if (i < nlist) {
                w = list[i];
                bits = bm[w];
                if (kClear) bm[w] = 0;
            }
            int tot;
            int at = nout + block_scan(__popc(bits), wsum, tot);
            while (bits) {
                out[at++] = base + w * 32 + (__ffs(bits) - 1);
                bits &= bits - 1;
            }
            nout += tot;
        }
    }
    return nout;
}

// The same read-back by one warp (shuffle scans, no block barrier): the
// chunk's words are few, so a single warp walks them faster than the block's
// barrier-separated scans.
__device__ __forceinline__ int warp_incl_scan(int x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

template <bool kClear>
__device__ int read_bits_warp(uint32_t *bm, uint32_t *sum, int n0, int32_t *list, int32_t *__restrict__ out,
                              int32_t base) {
    const int lane = threadIdx.x & 31;
    int nout = 0;
    for (int s0 = 0; s0 < n0; s0 += 32) {
        const int s = s0 + lane;
        uint32_t sw = s < n0 ? sum[s] : 0u;
        if (kClear && s < n0 && sw) sum[s] = 0;
        const int c = __popc(sw);
        const int incl = warp_incl_scan(c);
        const int nlist = __shfl_sync(0xffffffffu, incl, 31);
        int k = incl - c;
        while (sw) {
            list[k++] = s * 32 + (__ffs(sw) - 1);
            sw &= sw - 1;
        }
        __syncwarp();
        for (int i0 = 0; i0 < nlist; i0 += 32) {
            const int i = i0 + lane;
            int w = 0;
            uint32_t bits = 0;
            if (i < nlist) {
                w = list[i];
                bits = bm[w];
                if (kClear) bm[w] = 0;
            }
            const int cb = __popc(bits);
            const int ib = warp_incl_scan(cb);
            int at = nout + ib - cb;
            while (bits) {
                out[at++] = base + w * 32 + (__ffs(bits) - 1);
                bits &= bits - 1;
            }
            nout += __shfl_sync(0xffffffffu, ib, 31);
        }
        __syncwarp();
    }
    return nout;
}

// One pass over the chunks of the coarse rows (cluster ids of their member
// entries in vb).  A single-chunk row reads its bitmap back, sorted, over the
// front of its own vb range (its entries are all in the bitmap by then and no
// other block reads them) and writes its length to count[c]; rows of several
// chunks OR their chunk bitmaps into their global bitmap for
// coarse_rows_multi.  compact_rows then moves every row to its CSR position.
__global__ void __launch_bounds__(kRowThreads) coarse_rows(
    int32_t *vb, const ChunkInfo *__restrict__ info, const int64_t *__restrict__ slot, int64_t nchunks, int words,
    int n0, uint32_t *__restrict__ gbm, uint32_t *__restrict__ gsum, int32_t *__restrict__ count) {
    GOSH_DEP_WAIT();
    extern __shared__ uint32_t smem[];
    uint32_t *bm = smem;
    uint32_t *sum = bm + words;
    int32_t *list = reinterpret_cast<int32_t *>(sum + n0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < words + n0; i += kRowThreads) smem[i] = 0;
    __syncthreads();
    // Entries crowd onto the hubs' clusters, so most bits are already set: a
    // plain read first turns those into broadcast loads instead of atomics
    // serialised on one word.
    auto set_bits = [&](const int32_t *bs, int32_t c, int32_t base) {
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            if (bs[u] == c) continue;
            const int32_t b = bs[u] - base;  // id within the row's graph
            const uint32_t bit = 1u << (b & 31);
            if (bm[b >> 5] & bit) continue;
            const uint32_t old = atomicOr(bm + (b >> 5), bit);
            if (old == 0) atomicOr(sum + (b >> 10), 1u << ((b >> 5) & 31));
        }
    };
    // kBatch entries per thread from p0 on (the chunk's own id past its end)
    auto load_batch = [&](int32_t *bs, int64_t p0, int64_t e1, int32_t c) {
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int64_t p = p0 + (int64_t)u * kRowThreads;
            bs[u] = p < e1 ? vb[p] : c;
        }
    };
    // The first batch of the next chunk is loaded while this chunk is read
    // back (its range is another cluster's: the read-back never writes it).
    ChunkInfo cur;
    int32_t first[kBatch];
    if (blockIdx.x < nchunks) {
        cur = info[blockIdx.x];
        load_batch(first, cur.e0 + threadIdx.x, cur.e0 + cur.len, cur.c & 0x7fffffff);
    }
    for (int64_t t = blockIdx.x; t < nchunks; t += gridDim.x) {
        // the next chunk's record is loaded while this one is worked on
        ChunkInfo nxt = cur;
        const bool has_next = t + gridDim.x < nchunks;
        if (has_next) nxt = info[t + gridDim.x];
        const int32_t c = cur.c & 0x7fffffff;
        const bool many = cur.c < 0;
        const int64_t e0 = cur.e0, e1 = cur.e0 + cur.len;
        set_bits(first, c, cur.base);
        for (int64_t p0 = e0 + threadIdx.x + kBatch * kRowThreads; p0 < e1; p0 += kBatch * kRowThreads) {
            int32_t bs[kBatch];
            load_batch(bs, p0, e1, c);
            set_bits(bs, c, cur.base);
        }
        __syncthreads();
        if (has_next) load_batch(first, nxt.e0 + threadIdx.x, nxt.e0 + nxt.len, nxt.c & 0x7fffffff);
        if (!many) {
            if (warp == 0) {
                const int m = read_bits_warp<true>(bm, sum, n0, list, vb + cur.rb, cur.base);
                if (lane == 0) count[c] = m;
            }
        } else {
            // OR the chunk's bitmap into row c's global bitmap, every thread
            // on its own words, and clear it here
            const int64_t g = slot[c];
            uint32_t *gb = gbm + g * words;
            uint32_t *gs = gsum + g * n0;
            for (int si = threadIdx.x; si < n0; si += kRowThreads) {
                const uint32_t sw = sum[si];
                if (sw) {
                    atomicOr(gs + si, sw);
                    sum[si] = 0;
                }
            }
            for (int w = threadIdx.x; w < words; w += kRowThreads) {
                const uint32_t x = bm[w];
                if (x) {
                    atomicOr(gb + w, x);
                    bm[w] = 0;
                }
            }
        }
        __syncthreads();
        cur = nxt;
    }
}

// Rows of more than one chunk, from their global bitmaps: read back, sorted,
// over the front of the row's vb range, length to count[c].
__global__ void __launch_bounds__(kRowThreads) coarse_rows_multi(
    const int32_t *__restrict__ slot_row, int64_t nslots, int words, int n0, uint32_t *gbm, uint32_t *gsum,
    const int64_t *__restrict__ cstart, const int64_t *__restrict__ moff, const int32_t *__restrict__ cbase,
    int32_t *__restrict__ count, int32_t *__restrict__ vb) {
    GOSH_DEP_WAIT();
    __shared__ int32_t list[kListCap];
    __shared__ int wsum[kRowThreads / 32];
    for (int64_t g = blockIdx.x; g < nslots; g += gridDim.x) {
        const int32_t c = slot_row[g];
        const int m = read_bits<false>(gbm + g * words, gsum + g * n0, n0, list, wsum, vb + moff[cstart[c]],
                                       cbase ? cbase[c] : 0);
        if (threadIdx.x == 0) count[c] = m;
        __syncthreads();
    }
}

// Row c of the coarse CSR from the front of its vb range to col_out at
// rowptr[c], in the row's input chunks (a row is no longer than its entries):
// one warp per chunk, kBatch loads in flight per lane.
__global__ void compact_rows(const int32_t *__restrict__ vb, const ChunkInfo *__restrict__ info, int64_t nchunks,
                             const int64_t *__restrict__ rowptr, int32_t *__restrict__ col_out) {
    GOSH_DEP_WAIT();
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t wstride = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t = wid; t < nchunks; t += wstride) {
        const ChunkInfo ci = info[t];
        const int32_t c = ci.c & 0x7fffffff;
        const int64_t len = rowptr[c + 1] - rowptr[c];
        const int64_t j0 = ci.e0 - ci.rb;
        const int64_t j1 = j0 + kChunk < len ? j0 + kChunk : len;
        const int32_t *src = vb + ci.rb;
        int32_t *dst = col_out + rowptr[c];
        for (int64_t j = j0 + lane; j < j1; j += kBatch * 32) {
            int32_t x[kBatch];
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                const int64_t i = j + u * 32;
                x[u] = i < j1 ? src[i] : 0;
            }
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                const int64_t i = j + u * 32;
                if (i < j1) dst[i] = x[u];
            }
        }
    }
}

int grid_1d(int64_t n, int threads = 256) {
    const int64_t cap = (int64_t)num_sms() * 16;
    const int64_t g = ceil_div(n > 0 ? n : 1, threads);
    return (int)(g < cap ? g : cap);
}

int grid_warps(int64_t nwarps) {
    const int64_t cap = (int64_t)num_sms() * 8;
    const int64_t g = ceil_div(nwarps > 0 ? nwarps : 1, 8);
    return (int)(g < cap ? g : cap);
}

int bits_for(uint64_t x) {
    int b = 0;
    while (b < 64 && (uint64_t(1) << b) <= x) ++b;
    return b < 1 ? 1 : b;
}

// Largest coarse vertex count for the bitmap construction (its shared-memory
// bitmap has nc bits); GOSH_COARSEN_BITMAP_MAX overrides it (0: always sort).
int64_t bitmap_limit() {
    const char *e = getenv("GOSH_COARSEN_BITMAP_MAX");
    if (e && *e) {
        const long long v = atoll(e);
        return v < kBitmapMaxDefault ? (int64_t)v : kBitmapMaxDefault;
    }
    return kBitmapMaxDefault;
}

// Coarse CSR by sorting the packed edge keys (map v * nc + map u) of all entries.
gosh_status coarse_graph_sorted(int64_t n, const int64_t *rowptr, const int32_t *col, const int32_t *map, int64_t nc,
                                int64_t nnz, int64_t *rp, int32_t **co_out, int64_t *m_out, cudaStream_t s) {
    Scratch ek, fl, pos;
    GOSH_TRY(ek.alloc(sizeof(uint64_t) * nnz, s));
    GOSH_TRY(fl.alloc(nnz, s));
    GOSH_TRY(pos.alloc(sizeof(int64_t) * (nnz + 1), s));
    const uint64_t unc = (uint64_t)nc;
    const uint64_t sentinel = unc * unc;
    launch_dep(edge_image, grid_warps(ceil_div(nnz, kEntriesPerWarp)), 256, 0, s, rowptr, col, n, map, unc, ek.as<uint64_t>());
    int shifts[8];
    int nd = 0;
    const int kb = bits_for(sentinel);
    for (int b = 0; b < kb && nd < 8; b += 8) shifts[nd++] = b;
    GOSH_TRY(radix_sort_u64(ek.as<uint64_t>(), nullptr, nnz, shifts, nd, s));
    launch_dep(unique_flags, grid_1d(nnz), 256, 0, s, ek.as<uint64_t>(), nnz, sentinel, fl.as<uint8_t>());
    GOSH_TRY(scan_exclusive_u8_to_i64(fl.as<uint8_t>(), pos.as<int64_t>(), nnz, pos.as<int64_t>() + nnz, s));
    int64_t m = 0;
    GOSH_TRY_CUDA(cudaMemcpyAsync(&m, pos.as<int64_t>() + nnz, sizeof(m), cudaMemcpyDeviceToHost, s));
    GOSH_TRY_CUDA(cudaStreamSynchronize(s));
    GOSH_TRY_CUDA(dev_alloc((void **)co_out, sizeof(int32_t) * (m > 0 ? m : 1), s));
    GOSH_TRY_CUDA(cudaMemsetAsync(rp, 0, sizeof(int64_t) * (nc + 1), s));
    launch_dep(write_coarse, grid_1d(nnz), 256, 0, s, ek.as<uint64_t>(), fl.as<uint8_t>(), pos.as<int64_t>(), nnz, sentinel, nc, *co_out, rp);
    *m_out = m;
    return GOSH_OK;
}

// Coarse CSR through per-row bitmaps (coarse_rows); nc <= bitmap_limit().
// width: the bitmaps' span of coarse ids (nc; for a union of graphs the most
// clusters of one graph, with cbase[c] the first coarse id of row c's graph).
gosh_status coarse_graph_bitmap(int64_t n, const int64_t *rowptr, const int32_t *col, const int32_t *map, int64_t nc,
                                int64_t nnz, int64_t width, const int32_t *cbase, int64_t *rp, int32_t **co_out,
                                int64_t *m_out, cudaStream_t s) {
    const int words = (int)ceil_div(width, 32);
    const int n0 = (int)ceil_div(words, 32);
    const int list_cap = words < kListCap ? words : kListCap;
    Scratch mkey, mval, kalt, valt, cstart, mdeg, moff, vb, nchunk, multi, cstart_k, slot, count;
    GOSH_TRY(mkey.alloc(sizeof(uint32_t) * n, s));
    GOSH_TRY(mval.alloc(sizeof(uint32_t) * n, s));
    GOSH_TRY(kalt.alloc(sizeof(uint32_t) * n, s));
    GOSH_TRY(valt.alloc(sizeof(uint32_t) * n, s));
    GOSH_TRY(count.alloc(sizeof(int32_t) * nc, s));
    GOSH_TRY(cstart.alloc(sizeof(int64_t) * (nc + 1), s));
    GOSH_TRY(mdeg.alloc(sizeof(int64_t) * n, s));
    GOSH_TRY(moff.alloc(sizeof(int64_t) * (n + 1), s));
    GOSH_TRY(vb.alloc(sizeof(int32_t) * nnz, s));
    GOSH_TRY(nchunk.alloc(sizeof(int32_t) * nc, s));
    GOSH_TRY(multi.alloc(nc, s));
    GOSH_TRY(cstart_k.alloc(sizeof(int64_t) * (nc + 1), s));
    GOSH_TRY(slot.alloc(sizeof(int64_t) * (nc + 1), s));
    // members grouped by cluster (stable: ascending ids inside a cluster)
    launch_dep(member_keys, grid_1d(n), 256, 0, s, rowptr, n, map, (uint32_t)nc, mkey.as<uint32_t>(), mval.as<uint32_t>());
    bool in_alt = false;
    GOSH_TRY(radix_sort_u32_pp(mkey.as<uint32_t>(), mval.as<uint32_t>(), kalt.as<uint32_t>(), valt.as<uint32_t>(), n, 0,
                               bits_for((uint64_t)nc), s, &in_alt));
    const uint32_t *skey = in_alt ? kalt.as<uint32_t>() : mkey.as<uint32_t>();
    const uint32_t *sval = in_alt ? valt.as<uint32_t>() : mval.as<uint32_t>();
    launch_dep(member_layout, grid_1d(n), 256, 0, s, skey, sval, rowptr, n, (uint32_t)nc, cstart.as<int64_t>(),
               mdeg.as<int64_t>());
    GOSH_TRY(scan_exclusive_i64(mdeg.as<int64_t>(), moff.as<int64_t>(), n, moff.as<int64_t>() + n, s));
    launch_dep(member_entries, grid_warps(ceil_div(nnz, kEntriesPerWarp)), 256, 0, s, rowptr, col, n, map, sval,
               moff.as<int64_t>(), vb.as<int32_t>());
    launch_dep(row_chunks, grid_1d(nc), 256, 0, s, cstart.as<int64_t>(), moff.as<int64_t>(), nc, nchunk.as<int32_t>(), multi.as<uint8_t>(), count.as<int32_t>());
    GOSH_TRY(scan_exclusive_i32_to_i64(nchunk.as<int32_t>(), cstart_k.as<int64_t>(), nc, cstart_k.as<int64_t>() + nc, s));
    GOSH_TRY(scan_exclusive_u8_to_i64(multi.as<uint8_t>(), slot.as<int64_t>(), nc, slot.as<int64_t>() + nc, s));
    int64_t totals[2] = {0, 0};
    GOSH_TRY_CUDA(cudaMemcpyAsync(totals, cstart_k.as<int64_t>() + nc, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    GOSH_TRY_CUDA(cudaMemcpyAsync(totals + 1, slot.as<int64_t>() + nc, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    GOSH_TRY_CUDA(cudaStreamSynchronize(s));
    const int64_t nchunks = totals[0], nslots = totals[1];
    Scratch chunk_info, slot_row, gbm, gsum;
    GOSH_TRY(chunk_info.alloc(sizeof(ChunkInfo) * nchunks, s));
    GOSH_TRY(slot_row.alloc(sizeof(int32_t) * nslots, s));
    GOSH_TRY(gbm.alloc(sizeof(uint32_t) * nslots * words, s));
    GOSH_TRY(gsum.alloc(sizeof(uint32_t) * nslots * n0, s));
    if (nslots > 0) {
        GOSH_TRY_CUDA(cudaMemsetAsync(gbm.ptr, 0, sizeof(uint32_t) * nslots * words, s));
        GOSH_TRY_CUDA(cudaMemsetAsync(gsum.ptr, 0, sizeof(uint32_t) * nslots * n0, s));
    }
    launch_dep(chunk_rows, grid_1d(nc), 256, 0, s, cstart_k.as<int64_t>(), multi.as<uint8_t>(), slot.as<int64_t>(),
               cstart.as<int64_t>(), moff.as<int64_t>(), cbase, nc, chunk_info.as<ChunkInfo>(), slot_row.as<int32_t>());
    const size_t smem = sizeof(uint32_t) * ((size_t)words + n0 + list_cap);
    if (nchunks > 0) {
        // The attribute is process-wide state of the kernel: set it once to
        // the largest size any level can ask for, so concurrent coarsenings
        // (the batched entry runs several host threads) never lower it under
        // one another's launch.
        static std::once_flag attr_once;
        static cudaError_t attr_err = cudaSuccess;
        std::call_once(attr_once, [] {
            constexpr int64_t w = kBitmapMaxDefault / 32;
            const size_t most = sizeof(uint32_t) * (size_t)(w + ceil_div(w, 32) + kListCap);
            attr_err = cudaFuncSetAttribute(coarse_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most);
        });
        GOSH_TRY_CUDA(attr_err);
        int per_sm = 0;
        GOSH_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, coarse_rows, kRowThreads, smem));
        if (per_sm < 1) per_sm = 1;
        const int64_t cap = (int64_t)num_sms() * per_sm;
        const int grid = (int)(nchunks < cap ? nchunks : cap);
        launch_dep(coarse_rows, grid, kRowThreads, smem, s, vb.as<int32_t>(), chunk_info.as<ChunkInfo>(),
                   slot.as<int64_t>(), nchunks, words, n0, gbm.as<uint32_t>(), gsum.as<uint32_t>(),
                   count.as<int32_t>());
    }
    if (nslots > 0) {
        const int64_t cap = (int64_t)num_sms() * 8;
        const int mgrid = (int)(nslots < cap ? nslots : cap);
        launch_dep(coarse_rows_multi, mgrid, kRowThreads, 0, s, slot_row.as<int32_t>(), nslots, words, n0,
                   gbm.as<uint32_t>(), gsum.as<uint32_t>(), cstart.as<int64_t>(), moff.as<int64_t>(), cbase,
                   count.as<int32_t>(), vb.as<int32_t>());
    }
    GOSH_TRY(scan_exclusive_i32_to_i64(count.as<int32_t>(), rp, nc, rp + nc, s));
    int64_t m = 0;
    GOSH_TRY_CUDA(cudaMemcpyAsync(&m, rp + nc, sizeof(m), cudaMemcpyDeviceToHost, s));
    GOSH_TRY_CUDA(cudaStreamSynchronize(s));
    GOSH_TRY_CUDA(dev_alloc((void **)co_out, sizeof(int32_t) * (m > 0 ? m : 1), s));
    if (m > 0)
        launch_dep(compact_rows, grid_warps(nchunks), 256, 0, s, vb.as<int32_t>(), chunk_info.as<ChunkInfo>(),
                   nchunks, rp, *co_out);
    *m_out = m;
    return GOSH_OK;
}

// ---------------------------------------------------------------------------
// Unions of graphs.  Many graphs are coarsened as one disjoint union: slot j
// holds the vertices [vo[j], vo[j+1]) (ids graph-major).  The degree order
// sorts by (slot, descending degree, id), so every graph keeps its own rank
// order, its hubs are numbered consecutively from the union's count of hubs
// in earlier slots, and each graph's maps and coarse CSR equal those of
// coarsening it alone once that first id is subtracted.
// ---------------------------------------------------------------------------

// Last i in [0, n) with a[i] <= x (a non-decreasing, a[0] <= x).
__device__ __forceinline__ int last_le(const int64_t *__restrict__ a, int n, int64_t x) {
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(a + mid) <= x) lo = mid; else hi = mid;
    }
    return lo;
}

// Key (slot << bn) | (nmax - 1 - deg): graph-major, descending degree inside
// a graph; the density test uses the vertex's own graph.
__global__ void degree_keys_union(const int64_t *__restrict__ rowptr, int64_t n, const int32_t *__restrict__ vslot,
                                  const int64_t *__restrict__ slot_n, const int64_t *__restrict__ slot_nnz,
                                  int64_t nmax, int bn, uint32_t *__restrict__ key, uint32_t *__restrict__ val,
                                  uint8_t *__restrict__ state) {
    GOSH_DEP_WAIT();
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t deg = rowptr[v + 1] - rowptr[v];
        const int j = vslot[v];
        key[v] = ((uint32_t)j << bn) | (deg < nmax ? (uint32_t)(nmax - 1 - deg) : 0u);
        val[v] = (uint32_t)v;
        state[v] = small_deg(deg, slot_n[j], slot_nnz[j]) ? kUndecided : kHub;
    }
}

// out[j] = src[idx[j]] for j < m
__global__ void gather_at(const int64_t *__restrict__ src, const int64_t *__restrict__ idx, int m,
                          int64_t *__restrict__ out) {
    GOSH_DEP_WAIT();
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) out[j] = src[idx[j]];
}

// cbase[c] = first coarse id of the slot holding cluster c
__global__ void fill_cbase(const int64_t *__restrict__ cid_at, int nslots, int64_t nc, int32_t *__restrict__ cbase) {
    GOSH_DEP_WAIT();
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x)
        cbase[c] = (int32_t)cid_at[last_le(cid_at, nslots, c)];
}

struct SlotIn {
    const int64_t *rowptr;
    const int32_t *col;
};
struct SlotOut {
    int32_t *map;
    int64_t *rp;
    int32_t *col;
};

// union CSR rows (and the slot of every vertex)
__global__ void union_rows(const SlotIn *__restrict__ in, const int64_t *__restrict__ vo,
                           const int64_t *__restrict__ eo, int nslots, int64_t n, int64_t nnz,
                           int64_t *__restrict__ rowptr_u, int32_t *__restrict__ vslot) {
    GOSH_DEP_WAIT();
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r <= n; r += (int64_t)gridDim.x * blockDim.x) {
        if (r == n) {
            rowptr_u[n] = nnz;
            continue;
        }
        const int j = last_le(vo, nslots, r);
        rowptr_u[r] = eo[j] + in[j].rowptr[r - vo[j]];
        vslot[r] = j;
    }
}

// union CSR entries: neighbour ids shifted by their graph's first vertex
__global__ void union_cols(const SlotIn *__restrict__ in, const int64_t *__restrict__ vo,
                           const int64_t *__restrict__ eo, int nslots, int64_t nnz, int32_t *__restrict__ col_u) {
    GOSH_DEP_WAIT();
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
        const int j = last_le(eo, nslots, e);
        col_u[e] = in[j].col[e - eo[j]] + (int32_t)vo[j];
    }
}

// per-graph maps (cluster ids minus the graph's first cluster id)
__global__ void split_maps(const int32_t *__restrict__ map_u, const int32_t *__restrict__ vslot,
                           const int64_t *__restrict__ vo, const int64_t *__restrict__ cid_at, int64_t n,
                           const SlotOut *__restrict__ out) {
    GOSH_DEP_WAIT();
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const int j = vslot[r];
        out[j].map[r - vo[j]] = map_u[r] - (int32_t)cid_at[j];
    }
}

// per-graph coarse row pointers (rows [cid_at[j], cid_at[j+1]) of the union,
// entries from ceo[j]); thread t < nslots also writes graph t's final pointer
__global__ void split_rows(const int64_t *__restrict__ rp_u, const int64_t *__restrict__ cid_at,
                           const int64_t *__restrict__ ceo, int nslots, int64_t nc, const SlotOut *__restrict__ out) {
    GOSH_DEP_WAIT();
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nc + nslots;
         c += (int64_t)gridDim.x * blockDim.x) {
        if (c < nc) {
            const int j = last_le(cid_at, nslots, c);
            out[j].rp[c - cid_at[j]] = rp_u[c] - ceo[j];
        } else {
            const int j = (int)(c - nc);
            out[j].rp[cid_at[j + 1] - cid_at[j]] = ceo[j + 1] - ceo[j];
        }
    }
}

// per-graph coarse entries
__global__ void split_cols(const int32_t *__restrict__ co_u, const int64_t *__restrict__ ceo,
                           const int64_t *__restrict__ cid_at, int nslots, int64_t m,
                           const SlotOut *__restrict__ out) {
    GOSH_DEP_WAIT();
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const int j = last_le(ceo, nslots, e);
        out[j].col[e - ceo[j]] = co_u[e] - (int32_t)cid_at[j];
    }
}

}  // namespace

// One level: map (device, caller-allocated int32[n]); the coarse CSR is
// allocated with cudaMalloc into *rp_out / *col_out.  Synchronous.
// A union of graphs for mec_level (device arrays; cid_at is returned).
struct UnionLevel {
    int nslots = 0;
    int64_t nmax = 0;                  // most vertices of one graph
    const int32_t *vslot = nullptr;    // slot of every vertex
    const int64_t *slot_n = nullptr;   // vertices of every slot
    const int64_t *slot_nnz = nullptr; // entries of every slot
    const int64_t *vo = nullptr;       // nslots + 1 first vertices
    std::vector<int64_t> cid_at;       // out: nslots + 1 first cluster ids
};

gosh_status mec_level(int64_t n, const int64_t *rowptr, const int32_t *col, int64_t nnz, int32_t *map,
                      int64_t *nc_out, int64_t **rp_out, int32_t **col_out, int64_t *nnz_out, int *rounds_out,
                      cudaStream_t s, UnionLevel *u) {
    Scratch keys, vals, kalt, valt, rank, state, hub_rank, flags, cid, counter;
    GOSH_TRY(keys.alloc(sizeof(uint32_t) * n, s));
    GOSH_TRY(vals.alloc(sizeof(uint32_t) * n, s));
    GOSH_TRY(kalt.alloc(sizeof(uint32_t) * n, s));
    GOSH_TRY(valt.alloc(sizeof(uint32_t) * n, s));
    GOSH_TRY(rank.alloc(sizeof(int32_t) * n, s));
    GOSH_TRY(state.alloc(n, s));
    GOSH_TRY(hub_rank.alloc(sizeof(int32_t) * n, s));
    GOSH_TRY(flags.alloc(n, s));
    GOSH_TRY(cid.alloc(sizeof(int64_t) * (n + 1), s));
    GOSH_TRY(counter.alloc(sizeof(unsigned long long) * 2, s));

    // 1. degree order (and the initial MIS state)
    int key_bits = bits_for((uint64_t)(n - 1));
    if (u) {
        const int bn = bits_for((uint64_t)(u->nmax - 1));
        key_bits = bn + bits_for((uint64_t)(u->nslots - 1));
        launch_dep(degree_keys_union, grid_1d(n), 256, 0, s, rowptr, n, u->vslot, u->slot_n, u->slot_nnz, u->nmax, bn,
                   keys.as<uint32_t>(), vals.as<uint32_t>(), state.as<uint8_t>());
    } else {
        launch_dep(degree_keys, grid_1d(n), 256, 0, s, rowptr, n, keys.as<uint32_t>(), vals.as<uint32_t>(),
                   state.as<uint8_t>());
    }
    bool in_alt = false;
    GOSH_TRY(radix_sort_u32_pp(keys.as<uint32_t>(), vals.as<uint32_t>(), kalt.as<uint32_t>(), valt.as<uint32_t>(), n, 0,
                               key_bits, s, &in_alt));
    const uint32_t *order = in_alt ? valt.as<uint32_t>() : vals.as<uint32_t>();
    launch_dep(invert_order, grid_1d(n), 256, 0, s, order, n, rank.as<int32_t>());

    // 2. MIS rounds, two per check of the undecided count (most levels settle
    // in two; a round after settling does nothing)
    unsigned long long left[2] = {1, 1};
    int rounds = 0;
    while (left[1] > 0) {
        if (rounds > n + 1) {
            set_error("coarsening did not settle after %d rounds", rounds);
            return GOSH_ERR_CUDA;
        }
        GOSH_TRY_CUDA(cudaMemsetAsync(counter.ptr, 0, sizeof(unsigned long long) * 2, s));
        for (int r = 0; r < 2; ++r)
            launch_dep(mis_round, grid_1d(n), 256, 0, s, rowptr, col, n, order, rank.as<int32_t>(), state.as<uint8_t>(), counter.as<unsigned long long>() + r);
        GOSH_TRY_CUDA(cudaMemcpyAsync(left, counter.ptr, sizeof(left), cudaMemcpyDeviceToHost, s));
        GOSH_TRY_CUDA(cudaStreamSynchronize(s));
        rounds += 2;
    }
    if (rounds_out) *rounds_out = rounds;

    // 3. attach non-hubs, number the clusters by hub rank
    if (nnz > 64 * n)
        launch_dep(attach_to_hub_warp, grid_warps(n), 256, 0, s, rowptr, col, n, rank.as<int32_t>(), state.as<uint8_t>(), hub_rank.as<int32_t>());
    else
        launch_dep(attach_to_hub, grid_1d(n), 256, 0, s, rowptr, col, n, rank.as<int32_t>(), state.as<uint8_t>(), hub_rank.as<int32_t>());
    launch_dep(hub_flags_by_rank, grid_1d(n), 256, 0, s, order, state.as<uint8_t>(), n, flags.as<uint8_t>());
    GOSH_TRY(scan_exclusive_u8_to_i64(flags.as<uint8_t>(), cid.as<int64_t>(), n, cid.as<int64_t>() + n, s));
    GOSH_TRY_CUDA(cudaMemsetAsync(counter.ptr, 0, sizeof(unsigned long long), s));
    launch_dep(assign_map, grid_1d(n), 256, 0, s, hub_rank.as<int32_t>(), cid.as<int64_t>(), n, map, counter.as<unsigned long long>());
    int64_t nc = 0;
    unsigned long long orphans = 0;
    Scratch cid_at;
    if (u) {
        // first cluster id of every slot (its hubs come after all earlier slots')
        GOSH_TRY(cid_at.alloc(sizeof(int64_t) * (u->nslots + 1), s));
        launch_dep(gather_at, grid_1d(u->nslots + 1), 256, 0, s, cid.as<int64_t>(), u->vo, u->nslots + 1,
                   cid_at.as<int64_t>());
        u->cid_at.assign(u->nslots + 1, 0);
        GOSH_TRY_CUDA(cudaMemcpyAsync(u->cid_at.data(), cid_at.ptr, sizeof(int64_t) * (u->nslots + 1),
                                      cudaMemcpyDeviceToHost, s));
    }
    GOSH_TRY_CUDA(cudaMemcpyAsync(&nc, cid.as<int64_t>() + n, sizeof(nc), cudaMemcpyDeviceToHost, s));
    GOSH_TRY_CUDA(cudaMemcpyAsync(&orphans, counter.ptr, sizeof(orphans), cudaMemcpyDeviceToHost, s));
    GOSH_TRY_CUDA(cudaStreamSynchronize(s));
    if (orphans) {
        set_error("coarsening: %llu vertices without a cluster root", orphans);
        return GOSH_ERR_CUDA;
    }
    // bitmap span: the most clusters of one graph (ids taken from the graph's first)
    int64_t width = nc;
    Scratch cbase;
    if (u) {
        width = 0;
        for (int j = 0; j < u->nslots; ++j) width = std::max<int64_t>(width, u->cid_at[j + 1] - u->cid_at[j]);
        GOSH_TRY(cbase.alloc(sizeof(int32_t) * (nc > 0 ? nc : 1), s));
        launch_dep(fill_cbase, grid_1d(nc), 256, 0, s, cid_at.as<int64_t>(), u->nslots, nc, cbase.as<int32_t>());
    }
    keys.release();
    vals.release();
    rank.release();
    state.release();
    hub_rank.release();
    flags.release();
    cid.release();

    // 4. COARSEN
    int64_t *rp = nullptr;
    int32_t *co = nullptr;
    // hierarchy buffers come from the stream-ordered pool (no device-wide sync)
    GOSH_TRY_CUDA(dev_alloc((void **)&rp, sizeof(int64_t) * (nc + 1), s));
    int64_t m = 0;
    if (nnz > 0 && width <= bitmap_limit()) {
        GOSH_TRY(coarse_graph_bitmap(n, rowptr, col, map, nc, nnz, width, u ? cbase.as<int32_t>() : nullptr, rp, &co,
                                     &m, s));
    } else if (nnz > 0) {
        GOSH_TRY(coarse_graph_sorted(n, rowptr, col, map, nc, nnz, rp, &co, &m, s));
    } else {
        GOSH_TRY_CUDA(dev_alloc((void **)&co, sizeof(int32_t), s));
        GOSH_TRY_CUDA(cudaMemsetAsync(rp, 0, sizeof(int64_t) * (nc + 1), s));
    }
    *nc_out = nc;
    *rp_out = rp;
    *col_out = co;
    *nnz_out = m;
    return GOSH_OK;
}

gosh_status coarsen_impl(const gosh_csr *g0, int threshold, double shrink, int max_levels, cudaStream_t s,
                         gosh_hierarchy **out) {
    keep_pool_memory();
    gosh_hierarchy *h = new gosh_hierarchy();
    int64_t nnz0 = 0;
    cudaError_t e = cudaMemcpyAsync(&nnz0, g0->rowptr + g0->n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        delete h;
        set_error("reading rowptr[n]: %s", cudaGetErrorString(e));
        return GOSH_ERR_CUDA;
    }
    h->n.push_back(g0->n);
    h->nnz.push_back(nnz0);
    h->rowptr.push_back(const_cast<int64_t *>(g0->rowptr));
    h->col.push_back(const_cast<int32_t *>(g0->col));
    if (max_levels < 2) max_levels = 2;
    while (true) {
        const size_t i = h->n.size() - 1;
        const int64_t n = h->n[i];
        int32_t *map = nullptr;
        if (dev_alloc((void **)&map, sizeof(int32_t) * (n > 0 ? n : 1), s) != cudaSuccess) {
            delete h;
            set_error("allocation of map_%zu failed", i);
            return GOSH_ERR_OOM;
        }
        h->map.push_back(map);
        h->owned.push_back(device_owner(map));
        int64_t nc = 0, m = 0;
        int64_t *rp = nullptr;
        int32_t *co = nullptr;
        gosh_status st = mec_level(n, h->rowptr[i], h->col[i], h->nnz[i], map, &nc, &rp, &co, &m, nullptr, s, nullptr);
        if (st != GOSH_OK) {
            delete h;
            return st;
        }
        h->n.push_back(nc);
        h->nnz.push_back(m);
        h->rowptr.push_back(rp);
        h->col.push_back(co);
        h->owned.push_back(device_owner(rp));
        h->owned.push_back(device_owner(co));
        const bool more = nc > threshold && (double)nc <= std::floor(shrink * (double)n);
        if (!more || (int)h->n.size() >= max_levels) break;
    }
    const cudaError_t e2 = cudaStreamSynchronize(s);
    if (e2 != cudaSuccess) {
        delete h;
        set_error("coarsening: %s", cudaGetErrorString(e2));
        return GOSH_ERR_CUDA;
    }
    *out = h;
    return GOSH_OK;
}


namespace {

// sizes of the G input graphs' CSRs: nnz[g] = rowptr_g[n_g]
__global__ void input_nnz(const SlotIn *__restrict__ in, const int64_t *__restrict__ n, int G,
                          int64_t *__restrict__ nnz) {
    GOSH_DEP_WAIT();
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) nnz[g] = in[g].rowptr[n[g]];
}

// One level of the graphs in `slots` (each at its hierarchy's last level),
// coarsened as one union; appends the map and the coarse level to each.
gosh_status union_level(const std::vector<int> &slots, std::vector<gosh_hierarchy *> &hs, cudaStream_t s) {
    const int A = (int)slots.size();
    std::vector<int64_t> vo(A + 1, 0), eo(A + 1, 0), sn(A), snnz(A);
    std::vector<SlotIn> in(A);
    int64_t nmax = 0;
    for (int j = 0; j < A; ++j) {
        const gosh_hierarchy *h = hs[slots[j]];
        const size_t i = h->n.size() - 1;
        sn[j] = h->n[i];
        snnz[j] = h->nnz[i];
        in[j] = {h->rowptr[i], h->col[i]};
        vo[j + 1] = vo[j] + sn[j];
        eo[j + 1] = eo[j] + snnz[j];
        nmax = std::max(nmax, sn[j]);
    }
    const int64_t N = vo[A], E = eo[A];
    // device tables: SlotIn[A] | vo[A+1] | eo[A+1] | n[A] | nnz[A]
    const size_t tbytes = sizeof(SlotIn) * A + sizeof(int64_t) * (2 * (A + 1) + 2 * A);
    std::vector<char> host(tbytes);
    char *hp = host.data();
    std::memcpy(hp, in.data(), sizeof(SlotIn) * A);
    hp += sizeof(SlotIn) * A;
    for (auto *v : {&vo, &eo, &sn, &snnz}) {
        std::memcpy(hp, v->data(), sizeof(int64_t) * v->size());
        hp += sizeof(int64_t) * v->size();
    }
    Scratch tab, rowptr_u, col_u, vslot, map_u;
    GOSH_TRY(tab.alloc(tbytes, s));
    GOSH_TRY_CUDA(cudaMemcpyAsync(tab.ptr, host.data(), tbytes, cudaMemcpyHostToDevice, s));
    const SlotIn *d_in = tab.as<SlotIn>();
    const int64_t *d_vo = reinterpret_cast<const int64_t *>(tab.as<char>() + sizeof(SlotIn) * A);
    const int64_t *d_eo = d_vo + (A + 1);
    const int64_t *d_n = d_eo + (A + 1);
    const int64_t *d_nnz = d_n + A;
    GOSH_TRY(rowptr_u.alloc(sizeof(int64_t) * (N + 1), s));
    GOSH_TRY(col_u.alloc(sizeof(int32_t) * (E > 0 ? E : 1), s));
    GOSH_TRY(vslot.alloc(sizeof(int32_t) * N, s));
    GOSH_TRY(map_u.alloc(sizeof(int32_t) * N, s));
    launch_dep(union_rows, grid_1d(N + 1), 256, 0, s, d_in, d_vo, d_eo, A, N, E, rowptr_u.as<int64_t>(),
               vslot.as<int32_t>());
    if (E > 0) launch_dep(union_cols, grid_1d(E), 256, 0, s, d_in, d_vo, d_eo, A, E, col_u.as<int32_t>());

    UnionLevel u;
    u.nslots = A;
    u.nmax = nmax;
    u.vslot = vslot.as<int32_t>();
    u.slot_n = d_n;
    u.slot_nnz = d_nnz;
    u.vo = d_vo;
    int64_t NC = 0, M = 0;
    int64_t *rp_u = nullptr;
    int32_t *co_u = nullptr;
    GOSH_TRY(mec_level(N, rowptr_u.as<int64_t>(), col_u.as<int32_t>(), E, map_u.as<int32_t>(), &NC, &rp_u, &co_u, &M,
                       nullptr, s, &u));
    std::shared_ptr<void> rp_own = device_owner(rp_u), co_own = device_owner(co_u);
    rowptr_u.release();
    col_u.release();

    // every graph's first coarse entry (ceo) and its first cluster id (cid_at)
    Scratch at;
    GOSH_TRY(at.alloc(sizeof(int64_t) * 2 * (A + 1), s));
    GOSH_TRY_CUDA(cudaMemcpyAsync(at.ptr, u.cid_at.data(), sizeof(int64_t) * (A + 1), cudaMemcpyHostToDevice, s));
    const int64_t *d_cid = at.as<int64_t>();
    int64_t *d_ceo = at.as<int64_t>() + (A + 1);
    launch_dep(gather_at, grid_1d(A + 1), 256, 0, s, static_cast<const int64_t *>(rp_u), d_cid, A + 1, d_ceo);
    std::vector<int64_t> ceo(A + 1);
    GOSH_TRY_CUDA(cudaMemcpyAsync(ceo.data(), d_ceo, sizeof(int64_t) * (A + 1), cudaMemcpyDeviceToHost, s));
    GOSH_TRY_CUDA(cudaStreamSynchronize(s));

    // the graphs' new levels: one buffer each for maps, row pointers and
    // entries, shared by the hierarchies
    int32_t *maps = nullptr, *cols = nullptr;
    int64_t *rps = nullptr;
    GOSH_TRY_CUDA(dev_alloc((void **)&maps, sizeof(int32_t) * N, s));
    std::shared_ptr<void> maps_own = device_owner(maps);
    GOSH_TRY_CUDA(dev_alloc((void **)&rps, sizeof(int64_t) * (NC + A), s));
    std::shared_ptr<void> rps_own = device_owner(rps);
    GOSH_TRY_CUDA(dev_alloc((void **)&cols, sizeof(int32_t) * (M > 0 ? M : 1), s));
    std::shared_ptr<void> cols_own = device_owner(cols);
    std::vector<SlotOut> out(A);
    for (int j = 0; j < A; ++j)
        out[j] = {maps + vo[j], rps + u.cid_at[j] + j, cols + ceo[j]};
    Scratch otab;
    GOSH_TRY(otab.alloc(sizeof(SlotOut) * A, s));
    GOSH_TRY_CUDA(cudaMemcpyAsync(otab.ptr, out.data(), sizeof(SlotOut) * A, cudaMemcpyHostToDevice, s));
    launch_dep(split_maps, grid_1d(N), 256, 0, s, static_cast<const int32_t *>(map_u.as<int32_t>()),
               static_cast<const int32_t *>(vslot.as<int32_t>()), d_vo, d_cid, N, otab.as<SlotOut>());
    launch_dep(split_rows, grid_1d(NC + A), 256, 0, s, static_cast<const int64_t *>(rp_u), d_cid,
               static_cast<const int64_t *>(d_ceo), A, NC, otab.as<SlotOut>());
    if (M > 0)
        launch_dep(split_cols, grid_1d(M), 256, 0, s, static_cast<const int32_t *>(co_u),
                   static_cast<const int64_t *>(d_ceo), d_cid, A, M, otab.as<SlotOut>());
    for (int j = 0; j < A; ++j) {
        gosh_hierarchy *h = hs[slots[j]];
        h->map.push_back(out[j].map);
        h->n.push_back(u.cid_at[j + 1] - u.cid_at[j]);
        h->nnz.push_back(ceo[j + 1] - ceo[j]);
        h->rowptr.push_back(out[j].rp);
        h->col.push_back(out[j].col);
        h->owned.push_back(maps_own);
        h->owned.push_back(rps_own);
        h->owned.push_back(cols_own);
    }
    return GOSH_OK;
}

}  // namespace

// Coarsens G graphs (device CSRs) level by level as unions of the graphs
// still coarsening; each hierarchy equals coarsen_impl's for its graph.
gosh_status coarsen_batch_impl(const gosh_csr *graphs, int G, int threshold, double shrink, int max_levels,
                               cudaStream_t s, std::vector<gosh_hierarchy *> &out) {
    keep_pool_memory();
    out.assign(G, nullptr);
    struct Fail {
        std::vector<gosh_hierarchy *> &v;
        bool armed = true;
        ~Fail() {
            if (!armed) return;
            for (auto *&h : v) {
                delete h;
                h = nullptr;
            }
        }
    } fail{out};
    for (int g = 0; g < G; ++g) out[g] = new gosh_hierarchy();
    {
        // level 0: the callers' CSRs
        std::vector<SlotIn> in(G);
        std::vector<int64_t> n(G), nnz(G);
        for (int g = 0; g < G; ++g) {
            in[g] = {graphs[g].rowptr, graphs[g].col};
            n[g] = graphs[g].n;
        }
        Scratch tab;
        const size_t tb = sizeof(SlotIn) * G + sizeof(int64_t) * 2 * G;
        GOSH_TRY(tab.alloc(tb, s));
        GOSH_TRY_CUDA(cudaMemcpyAsync(tab.ptr, in.data(), sizeof(SlotIn) * G, cudaMemcpyHostToDevice, s));
        int64_t *d_n = reinterpret_cast<int64_t *>(tab.as<char>() + sizeof(SlotIn) * G);
        GOSH_TRY_CUDA(cudaMemcpyAsync(d_n, n.data(), sizeof(int64_t) * G, cudaMemcpyHostToDevice, s));
        launch_dep(input_nnz, grid_1d(G), 256, 0, s, static_cast<const SlotIn *>(tab.as<SlotIn>()),
                   static_cast<const int64_t *>(d_n), G, d_n + G);
        GOSH_TRY_CUDA(cudaMemcpyAsync(nnz.data(), d_n + G, sizeof(int64_t) * G, cudaMemcpyDeviceToHost, s));
        GOSH_TRY_CUDA(cudaStreamSynchronize(s));
        for (int g = 0; g < G; ++g) {
            out[g]->n.push_back(n[g]);
            out[g]->nnz.push_back(nnz[g]);
            out[g]->rowptr.push_back(const_cast<int64_t *>(graphs[g].rowptr));
            out[g]->col.push_back(const_cast<int32_t *>(graphs[g].col));
        }
    }
    if (max_levels < 2) max_levels = 2;
    std::vector<int> active(G);
    for (int g = 0; g < G; ++g) active[g] = g;
    while (!active.empty()) {
        // unions within the limits of 32-bit ids and 32-bit sort keys
        std::vector<std::vector<int>> groups(1);
        int64_t sum_n = 0, nmax = 0;
        for (int g : active) {
            const int64_t ng = out[g]->n.back();
            const int64_t nm = std::max(nmax, ng);
            const size_t cnt = groups.back().size() + 1;
            const bool fits = sum_n + ng < (int64_t(1) << 31) - 1 &&
                              bits_for((uint64_t)(nm - 1)) + bits_for((uint64_t)(cnt - 1)) <= 32;
            if (!groups.back().empty() && !fits) {
                groups.emplace_back();
                sum_n = 0;
                nmax = 0;
            }
            groups.back().push_back(g);
            sum_n += ng;
            nmax = std::max(nmax, ng);
        }
        for (auto &grp : groups) GOSH_TRY(union_level(grp, out, s));
        std::vector<int> next;
        for (int g : active) {
            const gosh_hierarchy *h = out[g];
            const int64_t nc = h->n.back(), nf = h->n[h->n.size() - 2];
            const bool more = nc > threshold && (double)nc <= std::floor(shrink * (double)nf);
            if (more && (int)h->n.size() < max_levels) next.push_back(g);
        }
        active.swap(next);
    }
    GOSH_TRY_CUDA(cudaStreamSynchronize(s));
    fail.armed = false;
    return GOSH_OK;
}

}  // namespace gosh
