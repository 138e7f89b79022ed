// Lock-free training step with the sample rows staged by the Tensor Memory
// Accelerator (cp.async.bulk, 1-D bulk copies into shared memory).
//
// Per warp: a tile of 32 sources; lanes draw the samples as in train_kernel.
// Then the warp walks the tile in rounds of G = 32/L sources with a two-stage
// shared-memory ring: while round q computes from stage q%2, the bulk copies
// of round q+1 (the G source rows and their k+1 sample rows, one copy per
// row) land in the other stage and complete on that stage's mbarrier.  A
// round therefore exposes no load latency once the pipeline is full, and the
// registers hold only the source row and the current sample row (the paper
// stages the source row in shared memory; here every row is staged).
// Sample-row changes go straight to global memory as atomic vector additions
// (16-bit tables: of the stochastically rounded new row minus the staged
// one), or as plain stores in the store mode; a later draw of the same
// row by the same source continues from the staged copy, which the lanes
// overwrite with the updated values.  Every mbarrier wait is bounded: on
// time-out the warp raises the error word, waits (bounded) for its copies
// and leaves the tile.
#pragma once

#include "tcgen05.cuh"
#include "train_kernels.cuh"

namespace gosh {

constexpr int kTmaWarps = 4;
constexpr uint32_t kTmaWaitPolls = 1u << 24;

__device__ __forceinline__ void bulk_g2s(uint32_t dst_smem, const void *src, uint32_t bytes, uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst_smem),
        "l"(src), "r"(bytes), "r"(mbar)
        : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity, uint32_t limit) {
    for (uint32_t i = 0; i < limit; ++i) {
        uint32_t done = 0;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Bytes of shared memory per warp: 2 stages x G sources x (1 + KS) rows.
template <typename T, int D, int L, int KS>
constexpr int tma_stage_bytes() {
    return (32 / L) * (1 + KS) * D * (int)sizeof(T);
}

template <typename T, int D, int L, int KS, int MODE>
__global__ void __launch_bounds__(kTmaWarps * 32) train_tma_kernel(TrainArgs a) {
    constexpr bool RED = MODE == kModeRed;
    constexpr bool RED16 = RED && !std::is_same<T, float>::value;
    static_assert(MODE == kModeRed || MODE == kModeStore, "lock-free modes only");
    constexpr int E = D / L;
    constexpr int PV = Store<T>::kPerVec;
    constexpr int G = 32 / L;
    constexpr int R = D * (int)sizeof(T);        // bytes per row
    constexpr int SLOTS = 1 + KS;                // source row + samples
    constexpr int STAGE = G * SLOTS * R;         // bytes per stage
    static_assert(E % PV == 0 && R % 16 == 0, "16-byte vectors");
    extern __shared__ __align__(128) uint8_t dsm[];
    __shared__ int32_t s_u[kTmaWarps][32 * kSlotStride];
    __shared__ uint32_t s_sr[kTmaWarps][32];
    __shared__ __align__(8) uint64_t s_bar[kTmaWarps][2];

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int grp = lane / L, gl = lane % L;
    const int ns = a.k + 1;
    uint8_t *stage_base = dsm + (size_t)warp * 2 * STAGE;
    const uint32_t bar0 = tc::smem_addr(&s_bar[warp][0]), bar1 = tc::smem_addr(&s_bar[warp][1]);
    if (lane == 0) {
        tc::mbar_init(&s_bar[warp][0], 1);
        tc::mbar_init(&s_bar[warp][1], 1);
    }
    __syncwarp();
    T *__restrict__ M = static_cast<T *>(a.M);
    uint32_t phase[2] = {0, 0};
    unsigned long long applied = 0;
    double loss_acc = 0.0;
    const bool want_loss = a.loss_partials != nullptr;
    const int64_t ntiles = (a.src_end - a.src_begin + a.tile - 1) / a.tile;
    const int rounds = a.tile / G;
    bool failed = false;

    // issues the copies of round q of the tile starting at v0 into stage st
    auto issue = [&](int64_t v0, int q, int st) {
        const uint32_t bar = st ? bar1 : bar0;
        const uint32_t sbase = tc::smem_addr(stage_base + st * STAGE);
        uint32_t bytes = 0;
        for (int t = lane; t < G * SLOTS; t += 32) {
            const int j = q * G + t / SLOTS, s = t % SLOTS;
            const int64_t v = v0 + j;
            if (v < a.src_end && (s == 0 || s <= ns)) {
                const int32_t id = s == 0 ? (int32_t)v : s_u[warp][j * kSlotStride + s - 1];
                if (id >= 0) bytes += R;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) bytes += __shfl_xor_sync(0xffffffffu, bytes, o);
        tc::fence_proxy_async();
        if (lane == 0) mbar_expect_tx(bar, bytes);
        __syncwarp();
        for (int t = lane; t < G * SLOTS; t += 32) {
            const int j = q * G + t / SLOTS, s = t % SLOTS;
            const int64_t v = v0 + j;
            if (v < a.src_end && (s == 0 || s <= ns)) {
                const int32_t id = s == 0 ? (int32_t)v : s_u[warp][j * kSlotStride + s - 1];
                if (id >= 0) bulk_g2s(sbase + (uint32_t)(((t / SLOTS) * SLOTS + s) * R), M + (int64_t)id * D, R, bar);
            }
        }
    };

    // draws of the tile starting at v0 (as in train_tile); they read only the CSR
    auto draw = [&](int64_t v0) {
        {
            const uint64_t ctr2 = ((uint64_t)a.level << 32) | a.epoch;
            const int64_t v = v0 + lane;
            if (lane < a.tile && v < a.src_end) {
                const int64_t off = a.rowptr[v];
                const int64_t deg = a.rowptr[v + 1] - off;
                for (int blk = 0; blk * 4 < ns; ++blk) {
                    const Philox4 w = philox4x64_10((uint64_t)v, (uint64_t)blk, ctr2, kTagSample, a.seed, a.graph);
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) {
                        const int t = blk * 4 + jj;
                        if (t < ns) {
                            int32_t u;
                            if (t == 0) {
                                u = deg > 0 ? __ldg(a.col + off + (int64_t)uniform_index(w.w[0], (uint64_t)deg)) : -1;
                            } else {
                                const int64_t x = (int64_t)uniform_index(w.w[jj], (uint64_t)a.n);
                                u = x == v ? -1 : (int32_t)x;
                            }
                            s_u[warp][lane * kSlotStride + t] = u;
                        }
                    }
                }
                if (!std::is_same<T, float>::value)
                    s_sr[warp][lane] = sr_source_seed(a.seed, a.graph, a.level, a.epoch, v);
            }
        }
        __syncwarp();
    };

    // The first tile's draws are taken while the previous kernel of the
    // stream (the previous epoch) still runs; the rows only after it ended.
    // (One call site of the draws: a second copy costs registers.)
    bool waited = false;
    for (int64_t tile = (int64_t)blockIdx.x * kTmaWarps + warp;; tile += (int64_t)gridDim.x * kTmaWarps) {
        const bool more = tile < ntiles && !failed;
        const int64_t v0 = a.src_begin + tile * a.tile;
        if (more) draw(v0);
        if (!waited) {
            GOSH_DEP_WAIT();
            // let the next epoch start early only where every warp owns one
            // tile (small levels); on large grids it cost throughput
            if (ntiles <= (int64_t)gridDim.x * kTmaWarps) GOSH_DEP_TRIGGER();
            waited = true;
        }
        if (!more) break;
        issue(v0, 0, 0);
#pragma unroll 1
        for (int q = 0; q < rounds; ++q) {
            const int st = q & 1;
            if (q + 1 < rounds) issue(v0, q + 1, st ^ 1);
            if (!mbar_try(st ? bar1 : bar0, phase[st], kTmaWaitPolls)) {
                failed = true;
                if (lane == 0 && a.err) atomicExch(a.err, 1);
                mbar_try(st ? bar1 : bar0, phase[st], kTmaWaitPolls);
                if (q + 1 < rounds) mbar_try(st ? bar0 : bar1, phase[st ^ 1], kTmaWaitPolls);
                break;
            }
            phase[st] ^= 1;
            const int j = q * G + grp;
            const int64_t v = v0 + j;
            const bool active = v < a.src_end;
            const uint32_t sr = std::is_same<T, float>::value ? 0u : s_sr[warp][j];
            uint8_t *sb = stage_base + st * STAGE + grp * SLOTS * R;  // this source's rows
            float r[E], r0[RED ? E : 1];
            if (active) {
                const uint4 *q4 = reinterpret_cast<const uint4 *>(sb) + gl;
#pragma unroll
                for (int x = 0; x < E / PV; ++x) Store<T>::unpack(q4[x * L], r + x * PV);
            } else {
#pragma unroll
                for (int e = 0; e < E; ++e) r[e] = 0.0f;
            }
            if (RED) {
#pragma unroll
                for (int e = 0; e < E; ++e) r0[e] = r[e];
            }
#pragma unroll 1
            for (int t = 0; t < ns; ++t) {
                const int32_t uid = active ? s_u[warp][j * kSlotStride + t] : -1;
                const bool ok = uid >= 0;
                float row[E];
                uint4 *rs = reinterpret_cast<uint4 *>(sb + (1 + t) * R) + gl;
                if (ok) {
#pragma unroll
                    for (int x = 0; x < E / PV; ++x) Store<T>::unpack(rs[x * L], row + x * PV);
                } else {
#pragma unroll
                    for (int e = 0; e < E; ++e) row[e] = 0.0f;
                }
                const float part = dot2<E>(r, row);
                const float x = group_sum<L>(part);
                const float b = t == 0 ? 1.0f : 0.0f;
                const float score = ok ? (b - sigmoid_f(x)) * a.lr : 0.0f;
                axpy2<E>(r, row, score);
                float old16[RED16 ? E : 1];
                if (RED16) {
#pragma unroll
                    for (int e = 0; e < E; ++e) old16[e] = row[e];
                }
                axpy2<E>(row, r, score);
                if (ok) {
                    if constexpr (RED16) {
                        red_row16<T, D, E, L>(M + (int64_t)uid * D, row, old16, sr, t, gl);
                    } else if (RED) {
                        float c[E];
#pragma unroll
                        for (int e = 0; e < E; ++e) c[e] = r[e] * score;
                        red_row<E, L>(reinterpret_cast<float *>(M) + (int64_t)uid * D, c, gl);
                    } else {
                        store_row<T, D, E, L>(M + (int64_t)uid * D, row, sr, t, gl);
                    }
                    // a later draw of the same row by this source continues from here
                    for (int t2 = t + 1; t2 < ns; ++t2)
                        if (s_u[warp][j * kSlotStride + t2] == uid) {
                            uint4 *d4 = reinterpret_cast<uint4 *>(sb + (1 + t2) * R) + gl;
#pragma unroll
                            for (int xx = 0; xx < E / PV; ++xx) {
                                float tmp[PV];
#pragma unroll
                                for (int e = 0; e < PV; ++e) tmp[e] = row[xx * PV + e];
                                d4[xx * L] = Store<T>::pack(tmp, 0u, 0u);  // values already rounded by the store
                            }
                        }
                    if (gl == 0) {
                        ++applied;
                        if (want_loss) loss_acc += (double)softplus_f(t == 0 ? -x : x);
                    }
                }
            }
            if (active) {
                if constexpr (RED16) {
                    red_row16<T, D, E, L>(M + v * D, r, r0, sr, ns, gl);
                } else if (RED) {
                    float dr[E];
#pragma unroll
                    for (int e = 0; e < E; ++e) dr[e] = r[e] - r0[RED ? e : 0];
                    red_row<E, L>(reinterpret_cast<float *>(M) + v * D, dr, gl);
                } else {
                    store_row<T, D, E, L>(M + v * D, r, sr, ns, gl);
                }
            }
            __syncwarp();
        }
        __syncwarp();
    }

    if (a.n_updates) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) applied += __shfl_xor_sync(0xffffffffu, applied, o);
        if (lane == 0 && applied) atomicAdd(a.n_updates, applied);
    }
    if (want_loss) {
        __shared__ double s_loss[kTmaWarps];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) loss_acc += __shfl_xor_sync(0xffffffffu, loss_acc, o);
        if (lane == 0) s_loss[warp] = loss_acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < kTmaWarps; ++w) t += s_loss[w];
            a.loss_partials[blockIdx.x] = t;
        }
    }
}

template <typename T, int D, int L, int KS, int MODE>
void launch_train_tma(const TrainArgs &a, int grid, cudaStream_t s) {
    constexpr int smem = kTmaWarps * 2 * tma_stage_bytes<T, D, L, KS>();
    launch_dep(train_tma_kernel<T, D, L, KS, MODE>, grid, kTmaWarps * 32, smem, s, a);
}

template <typename T, int D, int L, int KS, int MODE>
TrainKernel make_train_tma_kernel() {
    constexpr int smem = kTmaWarps * 2 * tma_stage_bytes<T, D, L, KS>();
    TrainKernel k;
    k.launch = &launch_train_tma<T, D, L, KS, MODE>;
    k.launch_epochs = nullptr;
    k.epochs_blocks_per_sm = 0;
    cudaFuncSetAttribute(train_tma_kernel<T, D, L, KS, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    k.blocks_per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k.blocks_per_sm, train_tma_kernel<T, D, L, KS, MODE>,
                                                  kTmaWarps * 32, smem);
    if (k.blocks_per_sm < 1) k.blocks_per_sm = 1;
    k.lanes = L;
    k.pass = -KS;  // negative pass = all k+1 <= KS samples staged by TMA
    k.warps = kTmaWarps;
    return k;
}

}  // namespace gosh
