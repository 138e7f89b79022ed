// Kernel templates of the training step; instantiated per storage type in
// train_f32.cu, train_bf16.cu and train_f16.cu.
#pragma once

#include <type_traits>

#include "train.cuh"

namespace gosh {

// Stochastic-rounding seed of one source in one epoch.
__device__ __forceinline__ uint32_t sr_source_seed(uint64_t seed, uint64_t graph, uint32_t level,
                                                   uint32_t epoch, int64_t v) {
    uint32_t h = mix32((uint32_t)v ^ mix32((uint32_t)((uint64_t)v >> 32)));
    h = mix32(h ^ (level << 20) ^ epoch);
    h = mix32(h ^ (uint32_t)graph ^ mix32((uint32_t)(graph >> 32)));
    h = mix32(h ^ (uint32_t)seed ^ mix32((uint32_t)(seed >> 32)));
    return h;
}

// sigma(x) = 1 / (1 + e^-x) with the fast exponential and the fast
// reciprocal (MUFU rcp: within 2 ulps, 0 for an infinite denominator); the
// correctly rounded reciprocal costs a slow path that made it a tenth of
// the level-0 step.
__device__ __forceinline__ float sigmoid_f(float x) { return __fdividef(1.0f, 1.0f + __expf(-x)); }

__device__ __forceinline__ float softplus_f(float z) {
    return fmaxf(z, 0.0f) + log1pf(__expf(-fabsf(z)));
}

// A lane holds E values of a row as E/PV 16-byte vectors (PV values each):
// its vector v is the row's vector v*L + gl (gl = lane within the L lanes of a
// source), so consecutive lanes take consecutive vectors and one load of the
// L lanes covers L * 16 contiguous bytes: whole 32-byte sectors.
template <typename T, int L>
__device__ __forceinline__ int lane_col(int gl, int v) {
    return (v * L + gl) * Store<T>::kPerVec;
}

template <typename T, int E, int L>
__device__ __forceinline__ void load_row(const T *__restrict__ row, int gl, float *f) {
    constexpr int PV = Store<T>::kPerVec;
    const uint4 *q = reinterpret_cast<const uint4 *>(row) + gl;
#pragma unroll
    for (int v = 0; v < E / PV; ++v) Store<T>::unpack(__ldcg(q + v * L), f + v * PV);
}

template <typename T, int E, int L>
__device__ __forceinline__ void load_row_snapshot(const T *__restrict__ row, int gl, float *f) {
    constexpr int PV = Store<T>::kPerVec;
    const uint4 *q = reinterpret_cast<const uint4 *>(row) + gl;
#pragma unroll
    for (int v = 0; v < E / PV; ++v) Store<T>::unpack(__ldg(q + v * L), f + v * PV);
}

// Stores the lane's E values of row-slot `slot` (columns lane_col); f is
// replaced by the stored (rounded) values.  The rounding bits of a pair of
// values depend on (slot, column) only.
template <typename T, int D, int E, int L>
__device__ __forceinline__ void store_row(T *__restrict__ row, float *f, uint32_t sr, int slot, int gl) {
    constexpr int PV = Store<T>::kPerVec;
    uint4 *q = reinterpret_cast<uint4 *>(row) + gl;
#pragma unroll
    for (int v = 0; v < E / PV; ++v) {
        const uint32_t base = (uint32_t)((slot * D + lane_col<T, L>(gl, v)) >> 1);
        q[v * L] = Store<T>::pack(f + v * PV, sr, base);
    }
}

// FP32 copies of the lane's values (vectors of PV values at columns lane_col
// of storage type T) into a row of an FP32 buffer.
template <typename T, int E, int L>
__device__ __forceinline__ void store_f32(float *__restrict__ row, const float *f, int gl) {
    constexpr int PV = Store<T>::kPerVec;
#pragma unroll
    for (int v = 0; v < E / PV; ++v) {
        float4 *q = reinterpret_cast<float4 *>(row + lane_col<T, L>(gl, v));
#pragma unroll
        for (int k = 0; k < PV / 4; ++k)
            q[k] = make_float4(f[v * PV + 4 * k], f[v * PV + 4 * k + 1], f[v * PV + 4 * k + 2], f[v * PV + 4 * k + 3]);
    }
}

// ... and back: FP32 buffer row -> the lane's values
template <typename T, int E, int L>
__device__ __forceinline__ void load_f32(const float *__restrict__ row, float *f, int gl) {
    constexpr int PV = Store<T>::kPerVec;
#pragma unroll
    for (int v = 0; v < E / PV; ++v) {
        const float4 *q = reinterpret_cast<const float4 *>(row + lane_col<T, L>(gl, v));
#pragma unroll
        for (int k = 0; k < PV / 4; ++k) {
            const float4 x = __ldg(q + k);
            f[v * PV + 4 * k] = x.x;
            f[v * PV + 4 * k + 1] = x.y;
            f[v * PV + 4 * k + 2] = x.z;
            f[v * PV + 4 * k + 3] = x.w;
        }
    }
}

// Atomic vector addition at L2 (fire-and-forget): M[p..p+3] += f[0..3].
__device__ __forceinline__ void red_add_v4(float *p, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d)
                 : "memory");
}

// 16-bit tables, atomic mode: the new values f are stochastically rounded in
// place and new - old, rounded to nearest, is added to the stored row at L2.
// Without a concurrent writer the stored old value becomes exactly the rounded
// new one whenever new - old fits the 16-bit significand (always when the
// change is below 256 ulps of the value, which covers the small updates that
// stochastic rounding exists for), else within one ulp of it; with a
// concurrent writer both changes are kept instead of one overwriting the other.
template <typename T, int D, int E, int L>
__device__ __forceinline__ void red_row16(T *__restrict__ row, float *f, const float *old, uint32_t sr, int slot,
                                          int gl) {
    constexpr int PV = Store<T>::kPerVec;
#pragma unroll
    for (int v = 0; v < E / PV; ++v) {
        const int col = lane_col<T, L>(gl, v);
        const uint32_t base = (uint32_t)((slot * D + col) >> 1);
        const uint4 nw = Store<T>::pack(f + v * PV, sr, base);
        Store<T>::red_add(row + col, Store<T>::change(nw, old + v * PV));
    }
}

template <int E, int L>
__device__ __forceinline__ void red_row(float *row, const float *f, int gl) {
#pragma unroll
    for (int v = 0; v < E / 4; ++v) {
        float *p = row + lane_col<float, L>(gl, v);
        red_add_v4(p, f[4 * v], f[4 * v + 1], f[4 * v + 2], f[4 * v + 3]);
    }
}

// d = a * b + c on two FP32 lanes at once (fma.rn.f32x2, sm_100 and later).
__device__ __forceinline__ void ffma2(float &d0, float &d1, float a0, float a1, float b0, float b1, float c0, float c1) {
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\t"
        "mov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d0), "=f"(d1)
        : "f"(a0), "f"(a1), "f"(b0), "f"(b1), "f"(c0), "f"(c1));
}

// sum over e of x[e] * y[e] (E even): two interleaved partial sums.
template <int E>
__device__ __forceinline__ float dot2(const float *x, const float *y) {
    float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
    for (int e = 0; e < E; e += 2) ffma2(s0, s1, x[e], x[e + 1], y[e], y[e + 1], s0, s1);
    return s0 + s1;
}

// y[e] += a * x[e] (E even).
template <int E>
__device__ __forceinline__ void axpy2(float *y, const float *x, float a) {
#pragma unroll
    for (int e = 0; e < E; e += 2) ffma2(y[e], y[e + 1], x[e], x[e + 1], a, a, y[e], y[e + 1]);
}

template <int L>
__device__ __forceinline__ float group_sum(float x) {
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Phases of a tile: the draws (sample ids and rounding seeds into shared
// memory; they read only the CSR) and the rounds (the row updates).
constexpr int kTileDraws = 1, kTileRounds = 2;

/*
 * One epoch (Hogwild) or one snapshot batch (deterministic) over sources
 * [src_begin, src_end).  Template: storage T, dimension D, L lanes per source,
 * P sample rows gathered per pass, MODE:
 *   kModeStore  lock-free epoch, rows written back with plain stores (the
 *               paper's scheme; concurrent writers to one row may lose updates);
 *   kModeRed    lock-free epoch, rows changed by atomic vector additions of
 *               the update (M[u] += score * M[v]; M[v] += its net change;
 *               16-bit tables add the difference of the stochastically
 *               rounded new row and the row read), so concurrent updates are
 *               kept, only read stale;
 *   kModeDet    snapshot batch, changes written to R/C/keys (needs P >= k+1).
 */
// Position i of an epoch's walk pairs visited i-th (Sec. 3.2, "shuffled"):
// a 4-round Feistel network on 2h-bit words (2^(2h) >= P) with round
// function mix32(x ^ k_r) & (2^h - 1), k_r = mix32(key + r), repeated until the
// value falls below P (cycle walking keeps it a bijection of [0, P)).
__host__ __device__ __forceinline__ uint64_t walk_position(uint64_t i, uint64_t P, uint32_t key, int h) {
    const uint32_t mask = h >= 32 ? 0xffffffffu : ((1u << h) - 1u);
    uint64_t x = i;
    do {
        uint32_t lo = (uint32_t)(x & mask), hi = (uint32_t)(x >> h);
#pragma unroll
        for (uint32_t r = 0; r < 4; ++r) {
            const uint32_t t = hi ^ (mix32(lo ^ mix32(key + r)) & mask);
            hi = lo;
            lo = t;
        }
        x = ((uint64_t)hi << h) | lo;
    } while (x >= P);
    return x;
}

template <typename T, int D, int L, int P, int MODE, int PHASES = kTileDraws | kTileRounds, bool PAIRS = false>
__device__ __forceinline__ void train_tile(const TrainArgs &a, const int64_t v0, int32_t *s_u_w, uint32_t *s_sr_w,
                                           double &loss_acc, unsigned long long &applied,
                                           int32_t *s_src_w = nullptr) {
    constexpr bool DET = MODE == kModeDet;
    constexpr bool RED = MODE == kModeRed;
    constexpr bool RED16 = RED && !std::is_same<T, float>::value;
    constexpr int E = D / L;
    constexpr int PV = Store<T>::kPerVec;
    constexpr int G = 32 / L;
    static_assert(E % PV == 0, "lane slice must be whole 16-byte vectors");
    static_assert(32 % L == 0, "L must divide the warp");
    static_assert(!DET || E % 4 == 0, "float4 stores of the change buffers");
    static_assert(!(DET && PAIRS), "walk pairs are trained lock-free");

    const int lane = threadIdx.x & 31;
    const int grp = lane / L, gl = lane % L;
    const int ns = a.k + 1;
    T *__restrict__ M = static_cast<T *>(a.M);
    const uint64_t ctr2 = ((uint64_t)a.level << 32) | a.epoch;
    const bool want_loss = a.loss_partials != nullptr;
    {
        // ---- draws: lane j -> source v0 + j ----
        if constexpr ((PHASES & kTileDraws) != 0 && PAIRS) {
            // walk pairs: slot v0 + lane visits position q; its source and
            // positive come from the pair table, the negatives from the
            // position's own Philox block (word 0 unused)
            const int64_t i = v0 + lane;
            if (lane < a.tile && i < a.src_end) {
                const uint64_t q = walk_position((uint64_t)i, (uint64_t)a.src_end, a.walk_key, a.walk_h);
                const int2 pr = __ldg(reinterpret_cast<const int2 *>(a.pairs) + q);
                s_src_w[lane] = pr.x;
                for (int blk = 0; blk * 4 < ns; ++blk) {
                    const Philox4 w = philox4x64_10(q, (uint64_t)blk, ctr2, kTagWalkNeg, a.seed, a.graph);
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int t = blk * 4 + j;
                        if (t < ns) {
                            int32_t u;
                            if (pr.x < 0) {
                                u = -1;
                            } else if (t == 0) {
                                u = pr.y;
                            } else {
                                const int64_t x = (int64_t)uniform_index(w.w[j], (uint64_t)a.n);
                                u = x == pr.x ? -1 : (int32_t)x;
                            }
                            s_u_w[lane * kSlotStride + t] = u;
                        }
                    }
                }
                if (!std::is_same<T, float>::value)
                    s_sr_w[lane] = sr_source_seed(a.seed, a.graph, a.level, a.epoch, (int64_t)q);
            }
        } else if constexpr ((PHASES & kTileDraws) != 0) {
            const int64_t v = v0 + lane;
            if (lane < a.tile && v < a.src_end) {
                const int64_t off = a.rowptr[v];
                const int64_t deg = a.rowptr[v + 1] - off;
                for (int blk = 0; blk * 4 < ns; ++blk) {
                    const Philox4 w = philox4x64_10((uint64_t)v, (uint64_t)blk, ctr2, kTagSample, a.seed, a.graph);
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int t = blk * 4 + j;
                        if (t < ns) {
                            int32_t u;
                            if (t == 0) {
                                u = deg > 0 ? __ldg(a.col + off + (int64_t)uniform_index(w.w[0], (uint64_t)deg)) : -1;
                            } else {
                                const int64_t x = (int64_t)uniform_index(w.w[j], (uint64_t)a.n);
                                u = x == v ? -1 : (int32_t)x;
                            }
                            s_u_w[lane * kSlotStride + t] = u;
                        }
                    }
                }
                if (!std::is_same<T, float>::value)
                    s_sr_w[lane] = sr_source_seed(a.seed, a.graph, a.level, a.epoch, v);
            }
        }
        __syncwarp();
        if constexpr ((PHASES & kTileRounds) == 0) return;
        // ---- rounds: G sources at a time, L lanes each (tile / G rounds) ----
        const int rounds = a.tile / G;
#pragma unroll 1
        for (int q = 0; q < rounds; ++q) {
            const int j = q * G + grp;
            int64_t v = v0 + j;
            bool active = v < a.src_end;
            if constexpr (PAIRS) {
                v = active ? s_src_w[j] : -1;  // the pair's source row (-1: a hole)
                active = v >= 0;
            }
            const uint32_t sr = std::is_same<T, float>::value ? 0u : s_sr_w[j];
            if constexpr (RED16) {
                // 16-bit tables, atomic changes: the rows as read stay packed
                // (their values are exact in T) and are unpacked where used,
                // so a lane holds E/2 words per row instead of E floats; same
                // operations in the same order as the unpacked form below
                constexpr int NV = E / PV;
                const uint4 z4 = make_uint4(0u, 0u, 0u, 0u);
                uint4 r0p[NV];
                float r[E];
                if (active) {
                    const uint4 *q4 = reinterpret_cast<const uint4 *>(M + v * D) + gl;
#pragma unroll
                    for (int x = 0; x < NV; ++x) {
                        r0p[x] = __ldcg(q4 + x * L);
                        Store<T>::unpack(r0p[x], r + x * PV);
                    }
                } else {
#pragma unroll
                    for (int x = 0; x < NV; ++x) r0p[x] = z4;
#pragma unroll
                    for (int e = 0; e < E; ++e) r[e] = 0.0f;
                }
#pragma unroll 1
                for (int p0 = 0; p0 < ns; p0 += P) {
                    int32_t us[P];
                    uint4 rowp[P][NV];
#pragma unroll
                    for (int s = 0; s < P; ++s) {
                        const int t = p0 + s;
                        us[s] = (active && t < ns) ? s_u_w[j * kSlotStride + t] : -1;
                    }
#pragma unroll
                    for (int s = 0; s < P; ++s) {
                        const uint4 *q4 = reinterpret_cast<const uint4 *>(M + (int64_t)(us[s] >= 0 ? us[s] : 0) * D) + gl;
#pragma unroll
                        for (int x = 0; x < NV; ++x) rowp[s][x] = us[s] >= 0 ? __ldcg(q4 + x * L) : z4;
                    }
#pragma unroll
                    for (int s = 0; s < P; ++s) {
                        const int t = p0 + s;
                        const bool ok = us[s] >= 0;
                        float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
                        for (int x = 0; x < NV; ++x) {
                            float tmp[PV];
                            Store<T>::unpack(rowp[s][x], tmp);
#pragma unroll
                            for (int e = 0; e < PV; e += 2)
                                ffma2(s0, s1, r[x * PV + e], r[x * PV + e + 1], tmp[e], tmp[e + 1], s0, s1);
                        }
                        const float xd = group_sum<L>(s0 + s1);
                        const float b = t == 0 ? 1.0f : 0.0f;
                        const float sig = sigmoid_f(xd);
                        const float score = ok ? (b - sig) * a.lr : 0.0f;
#pragma unroll
                        for (int x = 0; x < NV; ++x) {
                            float tmp[PV];
                            Store<T>::unpack(rowp[s][x], tmp);
#pragma unroll
                            for (int e = 0; e < PV; e += 2)
                                ffma2(r[x * PV + e], r[x * PV + e + 1], tmp[e], tmp[e + 1], score, score,
                                      r[x * PV + e], r[x * PV + e + 1]);
                        }
                        if (ok) {
                            T *row = M + (int64_t)us[s] * D;
#pragma unroll
                            for (int x = 0; x < NV; ++x) {
                                float tmp[PV];
                                Store<T>::unpack(rowp[s][x], tmp);
#pragma unroll
                                for (int e = 0; e < PV; e += 2)
                                    ffma2(tmp[e], tmp[e + 1], r[x * PV + e], r[x * PV + e + 1], score, score, tmp[e],
                                          tmp[e + 1]);
                                const int col = lane_col<T, L>(gl, x);
                                const uint4 nw = Store<T>::pack(tmp, sr, (uint32_t)((t * D + col) >> 1));
                                Store<T>::red_add(row + col, Store<T>::change_packed(nw, rowp[s][x]));
                                // a later sample of this pass with the same id continues from this row
#pragma unroll
                                for (int s2 = s + 1; s2 < P; ++s2)
                                    if (us[s2] == us[s]) rowp[s2][x] = nw;
                            }
                            if (gl == 0) {
                                ++applied;
                                if (want_loss) loss_acc += (double)softplus_f(t == 0 ? -xd : xd);
                            }
                        }
                    }
                }
                if (active) {
#pragma unroll
                    for (int x = 0; x < NV; ++x) {
                        const int col = lane_col<T, L>(gl, x);
                        const uint4 nw = Store<T>::pack(r + x * PV, sr, (uint32_t)((ns * D + col) >> 1));
                        Store<T>::red_add(M + v * D + col, Store<T>::change_packed(nw, r0p[x]));
                    }
                }
                continue;
            }
            float r[E];
            if (active) {
                if (DET) load_row_snapshot<T, E, L>(M + v * D, gl, r);
                else load_row<T, E, L>(M + v * D, gl, r);
            } else {
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
                for (int s = 0; s < P; ++s) {
                    const int t = p0 + s;
                    us[s] = (active && t < ns) ? s_u_w[j * kSlotStride + t] : -1;
                }
#pragma unroll
                for (int s = 0; s < P; ++s) {
                    if (us[s] >= 0) {
                        if (DET) load_row_snapshot<T, E, L>(M + (int64_t)us[s] * D, gl, row[s]);
                        else load_row<T, E, L>(M + (int64_t)us[s] * D, gl, row[s]);
                    } else {
#pragma unroll
                        for (int e = 0; e < E; ++e) row[s][e] = 0.0f;
                    }
                }
#pragma unroll
                for (int s = 0; s < P; ++s) {
                    const int t = p0 + s;
                    const bool ok = us[s] >= 0;
                    const float part = dot2<E>(r, row[s]);
                    const float x = group_sum<L>(part);
                    const float b = t == 0 ? 1.0f : 0.0f;
                    const float sig = sigmoid_f(x);
                    const float score = ok ? (b - sig) * a.lr : 0.0f;
                    axpy2<E>(r, row[s], score);
                    float old16[RED16 ? E : 1];
                    if (RED16) {
#pragma unroll
                        for (int e = 0; e < E; ++e) old16[e] = row[s][e];
                    }
                    axpy2<E>(row[s], r, score);
                    if (ok) {
                        if constexpr (RED16) {
                            red_row16<T, D, E, L>(M + (int64_t)us[s] * D, row[s], old16, sr, t, gl);
                        } else if (DET) {
                            const int64_t slot = (v - a.src_begin) * ns + t;
                            float c[E];
#pragma unroll
                            for (int e = 0; e < E; ++e) c[e] = r[e] * score;
                            store_f32<T, E, L>(a.C + slot * D, c, gl);
                            if (gl == 0) a.keys[slot] = (uint32_t)us[s];
                        } else if (RED) {
                            float c[E];
#pragma unroll
                            for (int e = 0; e < E; ++e) c[e] = r[e] * score;
                            red_row<E, L>(reinterpret_cast<float *>(M) + (int64_t)us[s] * D, c, gl);
                        } else {
                            store_row<T, D, E, L>(M + (int64_t)us[s] * D, row[s], sr, t, gl);
                        }
                        if (gl == 0) {
                            ++applied;
                            if (want_loss) loss_acc += (double)softplus_f(t == 0 ? -x : x);
                        }
                    } else if (DET && active && t < ns && gl == 0) {
                        a.keys[(v - a.src_begin) * ns + t] = (uint32_t)a.n;
                    }
                    // a later sample of this pass with the same id continues from this row
#pragma unroll
                    for (int s2 = s + 1; s2 < P; ++s2) {
                        if (ok && us[s2] == us[s]) {
#pragma unroll
                            for (int e = 0; e < E; ++e) row[s2][e] = row[s][e];
                        }
                    }
                }
            }
            if (active) {
                if constexpr (RED16) {
                    red_row16<T, D, E, L>(M + v * D, r, r0, sr, ns, gl);
                } else if (DET) {
                    store_f32<T, E, L>(a.R + (v - a.src_begin) * D, r, gl);
                } else if (RED) {
                    float dr[E];
#pragma unroll
                    for (int e = 0; e < E; ++e) dr[e] = r[e] - r0[RED ? e : 0];
                    red_row<E, L>(reinterpret_cast<float *>(M) + v * D, dr, gl);
                } else {
                    store_row<T, D, E, L>(M + v * D, r, sr, ns, gl);
                }
            }
        }
        __syncwarp();
    }
}

// Resident blocks the register allocation must allow: three (80 registers,
// 24 warps per SM) for lock-free variants whose lanes hold at most 8 values of
// a row, and for 16-bit tables with atomic changes (rows kept packed) up to 16;
// two (128 registers) otherwise: longer slices and the deterministic mode's
// larger passes would spill under three.
template <typename T>
constexpr int train_min_blocks(int values_per_lane, int mode) {
    return (mode != kModeDet && (values_per_lane <= 8 ||
                                 (mode == kModeRed && !std::is_same<T, float>::value && values_per_lane <= 16)))
               ? 3
               : 2;
}

/*
 * One epoch (Hogwild) or one snapshot batch (deterministic): the warps of the
 * grid take tiles of consecutive sources of [src_begin, src_end) in turn.
 */
template <typename T, int D, int L, int P, int MODE>
__global__ void __launch_bounds__(kTrainWarps * 32, train_min_blocks<T>(D / L, MODE)) train_kernel(TrainArgs a) {
    __shared__ int32_t s_u[kTrainWarps][32 * kSlotStride];
    __shared__ uint32_t s_sr[kTrainWarps][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t ntiles = (a.src_end - a.src_begin + a.tile - 1) / a.tile;
    const int64_t wstride = (int64_t)gridDim.x * kTrainWarps;
    const bool want_loss = a.loss_partials != nullptr;
    double loss_acc = 0.0;
    unsigned long long applied = 0;
    // The first tile's draws read only the CSR: taken while the previous
    // kernel of the stream (the previous epoch) still runs.
    const int64_t first = (int64_t)blockIdx.x * kTrainWarps + warp;
    if (first < ntiles)
        train_tile<T, D, L, P, MODE, kTileDraws>(a, a.src_begin + first * a.tile, s_u[warp], s_sr[warp], loss_acc,
                                                 applied);
    GOSH_DEP_WAIT();
    // the next epoch may start early where every warp owns one tile
    if (ntiles <= wstride) GOSH_DEP_TRIGGER();
    for (int64_t tile = first; tile < ntiles; tile += wstride) {
        if (tile == first)
            train_tile<T, D, L, P, MODE, kTileRounds>(a, a.src_begin + tile * a.tile, s_u[warp], s_sr[warp], loss_acc,
                                                      applied);
        else
            train_tile<T, D, L, P, MODE>(a, a.src_begin + tile * a.tile, s_u[warp], s_sr[warp], loss_acc, applied);
    }

    // ---- monitors ----
    if (a.n_updates) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) applied += __shfl_xor_sync(0xffffffffu, applied, o);
        if (lane == 0 && applied) atomicAdd(a.n_updates, applied);
    }
    if (want_loss) {
        __shared__ double s_loss[kTrainWarps];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) loss_acc += __shfl_xor_sync(0xffffffffu, loss_acc, o);
        if (lane == 0) s_loss[warp] = loss_acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < kTrainWarps; ++w) t += s_loss[w];
            a.loss_partials[blockIdx.x] = t;
        }
    }
}

template <typename T, int D, int L, int P, int MODE>
void launch_train(const TrainArgs &a, int grid, cudaStream_t s) {
    launch_dep(train_kernel<T, D, L, P, MODE>, grid, kTrainWarps * 32, 0, s, a);
}

constexpr uint32_t kEpochBarrierPolls = 1u << 22;

/*
 * Every epoch of a lock-free level in one cooperative launch: the warps run
 * their tiles of epoch j (learning rate lr * max(1 - j/epochs, lr_floor), as
 * the host would pass it), then the blocks meet at a grid barrier (a
 * monotonic arrival counter: epoch j waits for (j+1) * gridDim.x arrivals)
 * before epoch j+1, so an epoch sees every update of the previous one (Alg. 3
 * serialises epochs).  Small levels are bound by launch latency, not work.
 * The barrier wait is bounded: on time-out the block raises the error word
 * and goes on.
 */
template <typename T, int D, int L, int P, int MODE>
__global__ void __launch_bounds__(kTrainWarps * 32, train_min_blocks<T>(D / L, MODE))
    train_epochs_kernel(TrainArgs a, int epochs, double lr, double lr_floor, unsigned int *barrier) {
    GOSH_DEP_WAIT();
    __shared__ int32_t s_u[kTrainWarps][32 * kSlotStride];
    __shared__ uint32_t s_sr[kTrainWarps][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t ntiles = (a.src_end - a.src_begin + a.tile - 1) / a.tile;
    const int64_t wstride = (int64_t)gridDim.x * kTrainWarps;
    double loss_acc = 0.0;
    unsigned long long applied = 0;
    // A warp that owns at most one tile draws the samples of epoch j+1 (they
    // read only the CSR) before the barrier that closes epoch j, so an epoch
    // after the barrier starts with the row loads.
    const int64_t my_tile = (int64_t)blockIdx.x * kTrainWarps + warp;
    const bool one_tile = ntiles <= wstride;
    const int64_t my_v0 = a.src_begin + my_tile * a.tile;
    for (int j = 0; j < epochs; ++j) {
        const double f = 1.0 - (double)j / (double)epochs;
        a.lr = (float)(lr * (f > lr_floor ? f : lr_floor));
        a.epoch = (uint32_t)j;
        if (one_tile) {
            if (my_tile < ntiles) {
                if (j == 0)
                    train_tile<T, D, L, P, MODE, kTileDraws>(a, my_v0, s_u[warp], s_sr[warp], loss_acc, applied);
                train_tile<T, D, L, P, MODE, kTileRounds>(a, my_v0, s_u[warp], s_sr[warp], loss_acc, applied);
                if (j + 1 < epochs) {
                    a.epoch = (uint32_t)(j + 1);
                    train_tile<T, D, L, P, MODE, kTileDraws>(a, my_v0, s_u[warp], s_sr[warp], loss_acc, applied);
                }
            }
        } else {
            for (int64_t tile = my_tile; tile < ntiles; tile += wstride)
                train_tile<T, D, L, P, MODE>(a, a.src_begin + tile * a.tile, s_u[warp], s_sr[warp], loss_acc, applied);
        }
        if (j + 1 == epochs) break;
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(barrier, 1u);
            const unsigned int target = (unsigned int)(j + 1) * gridDim.x;
            uint32_t polls = 0;
            while (*reinterpret_cast<volatile unsigned int *>(barrier) < target) {
                if (++polls > kEpochBarrierPolls) {
                    if (a.err) atomicExch(a.err, 1);
                    break;
                }
            }
            __threadfence();
        }
        __syncthreads();
    }
    if (a.n_updates) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) applied += __shfl_xor_sync(0xffffffffu, applied, o);
        if (lane == 0 && applied) atomicAdd(a.n_updates, applied);
    }
}

template <typename T, int D, int L, int P, int MODE>
cudaError_t launch_train_epochs(const TrainArgs &a, int grid, int epochs, double lr, double lr_floor,
                                unsigned int *barrier, cudaStream_t s) {
    TrainArgs args = a;
    void *params[] = {&args, &epochs, &lr, &lr_floor, &barrier};
    const cudaError_t e = cudaLaunchCooperativeKernel((const void *)train_epochs_kernel<T, D, L, P, MODE>, dim3(grid),
                                                      dim3(kTrainWarps * 32), params, 0, s);
    if (e == cudaSuccess) note_launch();
    return e;
}

template <typename T, int D, int L, int P, int MODE>
TrainKernel make_train_kernel() {
    TrainKernel k;
    k.launch = &launch_train<T, D, L, P, MODE>;
    k.launch_epochs = nullptr;
    k.epochs_blocks_per_sm = 0;
    k.blocks_per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k.blocks_per_sm, train_kernel<T, D, L, P, MODE>,
                                                  kTrainWarps * 32, 0);
    if (k.blocks_per_sm < 1) k.blocks_per_sm = 1;
    if constexpr (MODE != kModeDet) {
        k.launch_epochs = &launch_train_epochs<T, D, L, P, MODE>;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k.epochs_blocks_per_sm, train_epochs_kernel<T, D, L, P, MODE>,
                                                      kTrainWarps * 32, 0);
    }
    k.lanes = L;
    k.pass = P;
    k.warps = kTrainWarps;
    return k;
}

// ---------------------------------------------------------------------------
// Deterministic mode, end of batch.  Sorted (target row, slot) pairs group the
// sample-row changes of each row in slot order = (source, sample) order.
// One L-lane group per sorted position; a group that starts a segment sums it.
// ---------------------------------------------------------------------------
template <typename T, int D, int L>
__global__ void __launch_bounds__(256) det_apply_segments(const uint32_t *__restrict__ skeys,
                                                          const uint32_t *__restrict__ sidx, int64_t nslots,
                                                          const float *__restrict__ C, const float *__restrict__ R,
                                                          T *__restrict__ M, int64_t n, int64_t b0, int64_t b1,
                                                          uint8_t *__restrict__ src_done, uint32_t sr_seed) {
    GOSH_DEP_WAIT();
    constexpr int E = D / L;
    const int gl = threadIdx.x % L;
    const int64_t gid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / L;
    const int64_t gstride = (int64_t)gridDim.x * blockDim.x / L;
    for (int64_t i = gid; i < nslots; i += gstride) {
        const uint32_t key = skeys[i];
        if ((int64_t)key >= n) continue;
        if (i > 0 && skeys[i - 1] == key) continue;
        const int64_t x = key;
        float acc[E];
        if (x >= b0 && x < b1) {
            load_f32<T, E, L>(R + (x - b0) * D, acc, gl);
            if (gl == 0) src_done[x - b0] = 1;
        } else {
            load_row_snapshot<T, E, L>(M + x * D, gl, acc);
        }
        for (int64_t jj = i; jj < nslots && skeys[jj] == key; ++jj) {
            float c[E];
            load_f32<T, E, L>(C + (int64_t)sidx[jj] * D, c, gl);
#pragma unroll
            for (int e = 0; e < E; ++e) acc[e] += c[e];
        }
        store_row<T, D, E, L>(M + x * D, acc, mix32(sr_seed ^ (uint32_t)x), 0, gl);
    }
}

template <typename T, int D, int L>
__global__ void __launch_bounds__(256) det_apply_sources(const float *__restrict__ R, T *__restrict__ M,
                                                         int64_t b0, int64_t b1,
                                                         const uint8_t *__restrict__ src_done, uint32_t sr_seed) {
    GOSH_DEP_WAIT();
    constexpr int E = D / L;
    const int gl = threadIdx.x % L;
    const int64_t gid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / L;
    const int64_t gstride = (int64_t)gridDim.x * blockDim.x / L;
    for (int64_t i = gid; i < b1 - b0; i += gstride) {
        if (src_done[i]) continue;
        float acc[E];
        load_f32<T, E, L>(R + i * D, acc, gl);
        store_row<T, D, E, L>(M + (b0 + i) * D, acc, mix32(sr_seed ^ (uint32_t)(b0 + i)), 0, gl);
    }
}

template <typename T, int D>
void launch_det_apply_t(const uint32_t *skeys, const uint32_t *sidx, int64_t nslots, const float *C,
                        const float *R, void *M, int64_t n, int64_t b0, int64_t b1, uint8_t *src_done,
                        uint32_t sr_seed, cudaStream_t s) {
    constexpr int L = (D * (int)sizeof(T) / 16) < 1 ? 1 : (D * (int)sizeof(T) / 16);
    constexpr int LL = (D / L) % 4 == 0 ? L : L / 2;  // float4 slices of the FP32 buffers
    const int64_t groups_per_block = 256 / LL;
    const int64_t g1 = ceil_div(nslots, groups_per_block);
    const int64_t g2 = ceil_div(b1 - b0, groups_per_block);
    const int cap = num_sms() * 8;
    if (nslots > 0)
        launch_dep(det_apply_segments<T, D, LL>, (int)(g1 < cap ? (g1 > 0 ? g1 : 1) : cap), 256, 0, s,
            skeys, sidx, nslots, C, R, static_cast<T *>(M), n, b0, b1, src_done, sr_seed);
    if (b1 > b0)
        launch_dep(det_apply_sources<T, D, LL>, (int)(g2 < cap ? (g2 > 0 ? g2 : 1) : cap), 256, 0, s,
            R, static_cast<T *>(M), b0, b1, src_done, sr_seed ^ 0x9e3779b9u);
}

}  // namespace gosh
