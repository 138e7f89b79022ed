// BF16 GEMM on the tcgen05 tensor cores: acc[m][n] = sum_k A[m][k] * B[n][k]
// (A and B row-major with K contiguous, FP32 accumulation in tensor memory),
// with the epilogue fused: FP32 store, FP32 atomic addition (split-K),
// bias + ReLU to BF16, or the learned projection's residual update of an
// embedding table.
//
// One CTA (4 warps) computes a 128 x NT tile.  Operands arrive by TMA: each
// stage holds 64 K-columns of the A and B tiles, one 2-D box of {64 columns,
// rows} per operand written with the 128-byte swizzle (rows of 128 bytes,
// 8-row atoms of 1024 bytes), the tensor cores' K-major swizzled layout: one
// copy per operand and stage instead of eight 16-byte-wide boxes.  Thread
// 0 of warp 0 runs the TMA producer over a ring of S stages (full/empty
// mbarriers), thread 0 of warp 1 issues the MMAs (one elected thread) and
// frees each stage with tcgen05.commit; after the last commit all four warps
// read their 32 accumulator lanes back with tcgen05.ld and apply the
// epilogue.  Every wait is bounded: on time-out the CTA raises *err, waits
// (bounded) for its MMAs and copies, frees its tensor memory and leaves the
// output unwritten.
#include <cuda.h>

#include <type_traits>

#include "common.cuh"
#include "tcgen05.cuh"

namespace gosh {

constexpr int kGemmThreads = 128;
constexpr int kGemmKStage = 64;  // K columns per pipeline stage
constexpr uint32_t kGemmWaitPolls = 1u << 22;

enum : int { kEpiStore = 0, kEpiAtomic = 1, kEpiBiasRelu = 2, kEpiResidual = 3 };

// Epilogue operands (unused fields stay null).
struct GemmEpi {
    float *C = nullptr;               // kEpiStore / kEpiAtomic: C[m][n], row stride ldc
    int64_t ldc = 0;
    const float *bias = nullptr;      // kEpiBiasRelu / kEpiResidual: bias[n]
    __nv_bfloat16 *H = nullptr;       // kEpiBiasRelu: H[m][n] = relu(acc + bias), row stride ldh
    int64_t ldh = 0;
    const int32_t *map = nullptr;     // kEpiResidual: Mf[v][n] = Mc[map v][n] + acc + bias, v = v0 + m
    const void *Mc = nullptr;
    void *Mf = nullptr;
    int64_t v0 = 0;
    int d = 0;                        // kEpiResidual: row length of Mc / Mf
};

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(mbar)
        : "memory");
}

// The box at {x, y} into L2 only (no shared memory, no completion).
__device__ __forceinline__ void tma_prefetch_2d(const CUtensorMap *map, int x, int y) {
    asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_addr(mbar)), "r"(bytes)
                 : "memory");
}

// relu(a + b) for two pairs, rounded to BF16 and packed (a0 + b0 in the low
// half): one paired FP32 add and one converting ReLU.
__device__ __forceinline__ uint32_t bias_relu_bf16x2(float a0, float a1, float b0, float b1) {
    uint64_t x, y, z;
    asm("mov.b64 %0, {%1, %2};" : "=l"(x) : "f"(a0), "f"(a1));
    asm("mov.b64 %0, {%1, %2};" : "=l"(y) : "f"(b0), "f"(b1));
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(z) : "l"(x), "l"(y));
    float s0, s1;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(s0), "=f"(s1) : "l"(z));
    uint32_t r;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(s1), "f"(s0));
    return r;
}

template <typename T>
__device__ __forceinline__ float to_f(T x) { return (float)x; }
template <>
__device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 x) { return __bfloat162float(x); }
template <>
__device__ __forceinline__ float to_f<__half>(__half x) { return __half2float(x); }
template <typename T>
__device__ __forceinline__ T from_f(float x) { return (T)x; }
template <>
__device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
template <>
__device__ __forceinline__ __half from_f<__half>(float x) { return __float2half_rn(x); }

// Pipeline stages: as many 64-column stages (2..4) as fit in 96 KB, so two
// CTAs share an SM (two 256-column accumulators fill its tensor memory).
template <int NT>
struct GemmShape {
    static constexpr int kStageBytes = (128 + NT) * kGemmKStage * 2;
    static constexpr int kFit = 98304 / kStageBytes;
    static constexpr int kStages = kFit < 2 ? 2 : (kFit > 4 ? 4 : kFit);
    // + 1024: the stages start at the first 1024-byte boundary (swizzle atoms)
    static constexpr size_t kSmem = (size_t)kStages * kStageBytes + 1024;
};

template <int NT, int EPI, typename T>
__global__ void __launch_bounds__(kGemmThreads) tma_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                                                                const __grid_constant__ CUtensorMap tmB, GemmEpi ep,
                                                                int M, int N, int K, int k_per_split,
                                                                int *__restrict__ err) {
    GOSH_DEP_WAIT();
    static_assert(NT % 16 == 0 && NT >= 16 && NT <= 256, "M = 128 needs N in [16, 256], multiple of 16");
    constexpr int S = GemmShape<NT>::kStages;
    constexpr uint32_t kCols = NT <= 32 ? 32 : (NT <= 64 ? 64 : (NT <= 128 ? 128 : 256));
    constexpr int A_BYTES = 128 * kGemmKStage * 2, B_BYTES = NT * kGemmKStage * 2;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    // the 128-byte swizzle needs 1024-byte aligned atoms: round the base up
    uint8_t *smem = smem_raw + ((1024u - (tc::smem_addr(smem_raw) & 1023u)) & 1023u);
    __shared__ __align__(8) uint64_t full[S], empty[S], done;
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * 128, n0 = blockIdx.y * NT;
    const int kb = blockIdx.z * k_per_split;
    const int ke = min(K, kb + k_per_split);
    const int nk = (ke - kb + kGemmKStage - 1) / kGemmKStage;

    if (warp == 0) tc::tmem_alloc(&tmem_base, kCols);
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_init(&done, 1);
        s_fail = 0;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base;
    int issued[S];  // loads issued per stage (producer thread)
#pragma unroll
    for (int s = 0; s < S; ++s) issued[s] = 0;

    if (warp == 0 && lane == 0) {
        // ---- TMA producer ----
        for (int k = 0; k < nk; ++k) {
            const int st = k % S;
            if (k >= S && !tc::mbar_wait(&empty[st], ((k / S) - 1) & 1, kGemmWaitPolls)) {
                atomicExch(&s_fail, 1);
                break;
            }
            const int k0 = kb + k * kGemmKStage;
            // whole boxes arrive (columns past K read as zero); the MMA
            // steps below stop at this split's end
            mbar_arrive_expect_tx(&full[st], (uint32_t)(A_BYTES + B_BYTES));
            const uint32_t sa = tc::smem_addr(smem + (size_t)st * (A_BYTES + B_BYTES));
            const uint32_t sb = sa + A_BYTES;
            tma_load_2d(sa, &tmA, k0, m0, tc::smem_addr(&full[st]));
            tma_load_2d(sb, &tmB, k0, n0, tc::smem_addr(&full[st]));
            ++issued[st];
        }
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer ----
        const uint32_t idesc = tc::make_idesc_bf16(128, NT);
        bool ok = true;
        for (int k = 0; k < nk && ok; ++k) {
            const int st = k % S;
            if (!tc::mbar_wait(&full[st], (k / S) & 1, kGemmWaitPolls) || *(volatile int *)&s_fail) {
                atomicExch(&s_fail, 1);
                ok = false;
                break;
            }
            tc::fence_after_sync();
            const int k0 = kb + k * kGemmKStage;
            const int steps = min(kGemmKStage, ke - k0) / 16;
            const uint32_t sa = tc::smem_addr(smem + (size_t)st * (A_BYTES + B_BYTES));
            const uint32_t sb = sa + A_BYTES;
            for (int j = 0; j < steps; ++j) {
                const uint64_t ad = tc::make_desc_sw128(sa + 32 * j);
                const uint64_t bd = tc::make_desc_sw128(sb + 32 * j);
                tc::mma_bf16(tmem, ad, bd, idesc, (k > 0 || j > 0) ? 1u : 0u);
            }
            tc::mma_commit(&empty[st]);
        }
        tc::mma_commit(&done);  // arrives once every MMA issued above has completed
    }
    __syncwarp();
    const bool finished = tc::mbar_wait(&done, 0, kGemmWaitPolls);
    const int ok = __syncthreads_and(finished && !s_fail ? 1 : 0);
    tc::fence_after_sync();
    if (!ok) {
        if (tid == 0) {
            atomicExch(err, 1);
            // Let copies still in flight land before the CTA's shared memory
            // goes away.  A stage is refilled only after its previous load was
            // consumed, so at most its last load (phase issued - 1) is pending.
            for (int s = 0; s < S; ++s)
                if (issued[s] > 0) tc::mbar_wait(&full[s], (uint32_t)(issued[s] - 1) & 1u, kGemmWaitPolls);
        }
    } else if (nk > 0) {
        const int row = m0 + warp * 32 + lane;
#pragma unroll 1
        for (int c = 0; c < NT; c += 16) {
            float v[16];
            tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
            if (row >= M) continue;
            const int col0 = n0 + c;
            if (EPI == kEpiStore || EPI == kEpiAtomic) {
                float *out = ep.C + (int64_t)row * ep.ldc + col0;
#pragma unroll
                for (int j = 0; j < 16; j += 4) {
                    if (col0 + j + 3 < N) {
                        if (EPI == kEpiAtomic) {
                            asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(out + j), "f"(v[j]),
                                         "f"(v[j + 1]), "f"(v[j + 2]), "f"(v[j + 3])
                                         : "memory");
                        } else {
                            *reinterpret_cast<float4 *>(out + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                        }
                    } else {
                        for (int q = j; q < j + 4; ++q)
                            if (col0 + q < N) {
                                if (EPI == kEpiAtomic) atomicAdd(out + q, v[q]);
                                else out[q] = v[q];
                            }
                    }
                }
            } else if (EPI == kEpiBiasRelu) {
                __nv_bfloat16 *out = ep.H + (int64_t)row * ep.ldh + col0;
                if (col0 + 15 < N) {
                    uint32_t w[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const __nv_bfloat162 h = __floats2bfloat162_rn(fmaxf(v[2 * j] + ep.bias[col0 + 2 * j], 0.0f),
                                                                       fmaxf(v[2 * j + 1] + ep.bias[col0 + 2 * j + 1], 0.0f));
                        w[j] = *reinterpret_cast<const uint32_t *>(&h);
                    }
                    uint4 *o4 = reinterpret_cast<uint4 *>(out);
                    o4[0] = make_uint4(w[0], w[1], w[2], w[3]);
                    o4[1] = make_uint4(w[4], w[5], w[6], w[7]);
                } else {
                    for (int q = 0; q < 16; ++q)
                        if (col0 + q < N) out[q] = __float2bfloat16_rn(fmaxf(v[q] + ep.bias[col0 + q], 0.0f));
                }
            } else {  // kEpiResidual: N == d, a multiple of 16 (16 values = whole 16-byte vectors)
                constexpr int PV = 16 / (int)sizeof(T);
                const int64_t vv = ep.v0 + row;
                const uint4 *src = reinterpret_cast<const uint4 *>(static_cast<const T *>(ep.Mc) +
                                                                   (int64_t)__ldg(ep.map + vv) * ep.d + col0);
                uint4 *dst = reinterpret_cast<uint4 *>(static_cast<T *>(ep.Mf) + vv * ep.d + col0);
#pragma unroll
                for (int x = 0; x < 16 / PV; ++x) {
                    union {
                        uint4 u;
                        T t[PV];
                    } pk;
                    pk.u = __ldg(src + x);
#pragma unroll
                    for (int q = 0; q < PV; ++q)
                        pk.t[q] = from_f<T>(to_f<T>(pk.t[q]) + v[x * PV + q] + __ldg(ep.bias + col0 + x * PV + q));
                    dst[x] = pk.u;
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kCols);
}

// ---------------------------------------------------------------------------
// The learned projection of one chunk of fine vertices in one persistent
// kernel (both layers of the MLP; the hidden layer never leaves the SM):
//
//   acc1   = X W1^T                    tensor memory, lanes = tile rows, columns [0, hid)
//   H      = relu(acc1 + b1)           BF16, shared memory
//   acc2^T = W2 H^T                    tensor memory, lanes = output dimensions, columns = tile rows
//   Mf[v0 + m][o] = Mc[map[v0 + m]][o] + acc2^T[o][m] + b2[o]
//
// Layer 2 runs transposed so that W2 stays resident in tensor memory as the
// A operand (lanes = its rows, zero rows up to 128, the K = hid values of a
// row packed two per 32-bit column) and H, the B operand, is read in place
// from shared memory; the weights streamed per tile are then W1's alone.
// Its epilogue gives lane o of a warp output dimension o of a row, so the
// coarse-row loads and the fine-row stores of a warp are contiguous.
//
// One CTA per SM walks the chunk's 128-row tiles (tile = blockIdx.x + i *
// gridDim.x).  Roles: warps 0-15 run the epilogues (four warps per 32
// tensor-memory lanes, each a quarter of the columns; warps 0-3 first write
// W2 into tensor memory, while layer 1 of the first tile runs), warp 16
// loads the ring of S stages (each: one 64-column block of the X tile and
// the matching block of W1, both as one 128-byte-swizzled TMA box; the
// 16-column tail of K as two 8-column boxes per operand without swizzle),
// stages one more block per tile in H's buffer (idle during layer 1) and
// prefetches the next tile's X rows into L2, warp 17 issues the MMAs.  The
// epilogue warps bring the residual's coarse rows into L2 at the start of a
// tile, so their latency hides behind layer 1.
//
// Barriers: full / empty per stage, hs_full (the K block staged in H's
// buffer arrived), acc1_full (layer 1 done), h_full (acc1 read out and H
// written and fenced for the tensor cores), w2_ready (W2 in tensor memory),
// acc2_full (layer 2 done: H's buffer free for the next tile's staged
// block), acc2_empty (acc2 read out).  Every wait is bounded; on time-out
// the CTA raises *err, every role stops, the producer waits (bounded) for
// its copies in flight and the tensor memory is freed.
constexpr int kMlpEpiWarps = 16;
constexpr int kMlpParts = kMlpEpiWarps / 4;  // epilogue warps sharing each 32 tensor-memory lanes
constexpr int kMlpThreads = (kMlpEpiWarps + 2) * 32;
constexpr int kMlpXBlock = 128 * kGemmKStage * 2;  // one 64-column block of a 128-row tile
constexpr int kMlpKS = kGemmKStage;                 // K columns per ring stage (128-byte swizzled rows)
constexpr int kMlpXPart = kMlpXBlock;               // the X part of a stage
constexpr int kMlpMaxHid = 256;
constexpr int kMlpMaxStages = 8;
constexpr size_t kMlpSmemLimit = 232448 - 4096;    // dynamic shared memory left beside the static part

struct MlpDims {
    int hid, kp, nkb1, hbytes, stage, S;
    uint32_t c_w2, c_acc2, cols;
    __host__ __device__ MlpDims(int hid_, int kp_)
        : hid(hid_), kp(kp_), nkb1((kp_ + kMlpKS - 1) / kMlpKS), hbytes(128 * hid_ * 2),
          stage(kMlpXPart + hid_ * kMlpKS * 2), S(0), c_w2((uint32_t)hid_), c_acc2((uint32_t)(hid_ + hid_ / 2)),
          cols(32) {
        const long room = (long)kMlpSmemLimit - 1024 - hbytes;
        S = (int)(room / stage);
        if (S > kMlpMaxStages) S = kMlpMaxStages;
        while (cols < c_acc2 + 128u) cols <<= 1;
    }
    __host__ __device__ size_t smem() const { return (size_t)hbytes + (size_t)S * stage + 1024; }
};

template <typename T, int D>
__global__ void __launch_bounds__(kMlpThreads, 1)
    mlp_project_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmW1,
                       const __grid_constant__ CUtensorMap tmXt, const __grid_constant__ CUtensorMap tmW1t,
                       const __nv_bfloat16 *__restrict__ W2b, const float *__restrict__ b1,
                       const float *__restrict__ b2, const int32_t *__restrict__ map, const T *__restrict__ Mc,
                       T *__restrict__ Mf, int64_t v0, int M, int hid, int kp, int *__restrict__ err) {
    GOSH_DEP_WAIT();
    static_assert(D == 32 || D == 64 || D == 128, "D in {32, 64, 128}");
    const MlpDims dm(hid, kp);
    const int S = dm.S;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = smem_raw + ((1024u - (tc::smem_addr(smem_raw) & 1023u)) & 1023u);
    const uint32_t hbuf = tc::smem_addr(smem);
    const uint32_t ring0 = hbuf + (uint32_t)dm.hbytes;
    __shared__ __align__(8) uint64_t full[kMlpMaxStages], empty[kMlpMaxStages];
    __shared__ __align__(8) uint64_t acc1_full, h_full, acc2_full, acc2_empty, w2_ready, hs_full, fin;
    __shared__ __align__(16) float sb1[kMlpMaxHid];
    __shared__ float sb2[128];
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntiles = (M + 127) / 128;
    const int T_n = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
#define MLP_TILE_ROW0(t) (((int)blockIdx.x + (t) * (int)gridDim.x) * 128)

    if (warp == kMlpEpiWarps) tc::tmem_alloc(&tmem_base, dm.cols);
    if (tid == 0) {
        for (int i = 0; i < S; ++i) {
            tc::mbar_init(&full[i], 1);
            tc::mbar_init(&empty[i], 1);
        }
        tc::mbar_init(&acc1_full, 1);
        tc::mbar_init(&h_full, kMlpEpiWarps);
        tc::mbar_init(&acc2_full, 1);
        tc::mbar_init(&acc2_empty, kMlpEpiWarps);
        tc::mbar_init(&w2_ready, 4);
        tc::mbar_init(&hs_full, 1);
        tc::mbar_init(&fin, 1);
        s_fail = 0;
    }
    for (int i = tid; i < hid; i += kMlpThreads) sb1[i] = b1[i];
    for (int i = tid; i < 128; i += kMlpThreads) sb2[i] = i < D ? b2[i] : 0.0f;
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base;
    volatile int *vfail = &s_fail;
    // K block kh of every tile is staged in the hidden tile's buffer, idle
    // from the end of layer 2 of one tile to the hidden-layer epilogue of the
    // next: one more stage in flight during layer 1 (the last full block, so
    // that its load, which waits for the previous tile's layer 2, starts a
    // few stages before it is needed); none when a tile has fewer than three
    const int kh = dm.nkb1 >= 3 ? dm.nkb1 - 2 : -1;

    // W2 into tensor memory (warps 0-3, while layer 1 of the first tile
    // runs): warp w writes lanes 32 w .. 32 w + 31, row o of W2 (zero past
    // D) packed two BF16 per column; layer 2 waits for w2_ready
    if (warp < 4) {
        const int o = warp * 32 + lane;
        const uint4 *src = reinterpret_cast<const uint4 *>(W2b + (int64_t)(o < D ? o : 0) * hid);
        for (int c = 0; c < hid / 2; c += 32) {
            uint32_t r[32];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const uint4 q = o < D ? __ldg(src + c / 4 + i) : make_uint4(0, 0, 0, 0);
                r[4 * i] = q.x;
                r[4 * i + 1] = q.y;
                r[4 * i + 2] = q.z;
                r[4 * i + 3] = q.w;
            }
            tc::tmem_st32(tmem + ((uint32_t)(warp * 32) << 16) + dm.c_w2 + (uint32_t)c, r);
        }
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&w2_ready);
    }

    if (warp == kMlpEpiWarps) {
        // ---- producer: per tile nkb1 stages of (X block, W1 block) ----
        if (lane == 0) {
            int issued[kMlpMaxStages];
            for (int i = 0; i < kMlpMaxStages; ++i) issued[i] = 0;
            int st = 0, round = 0;  // ring position: stage st, pass `round` over the ring
            int h_issued = 0;       // loads into the hidden tile's buffer
            bool ok = true;
            for (int t = 0; t < T_n && ok; ++t) {
                const int m0 = MLP_TILE_ROW0(t);
                if (t + 1 < T_n) {  // the next tile's rows into L2 while this one is computed
                    const int m1 = MLP_TILE_ROW0(t + 1);
                    for (int kb = 0; kb < dm.nkb1; ++kb) tma_prefetch_2d(&tmX, kb * kMlpKS, m1);
                }
                for (int kb = 0; kb < dm.nkb1; ++kb) {
                    if (kb == kh) {
                        // the hidden tile's buffer is free once layer 2 of tile t - 1 is done
                        if (*vfail || (t > 0 && !tc::mbar_wait(&acc2_full, (t - 1) & 1, kGemmWaitPolls))) {
                            atomicExch(&s_fail, 1);
                            ok = false;
                            break;
                        }
                        const uint32_t hb = tc::smem_addr(&hs_full);
                        mbar_arrive_expect_tx(&hs_full, (uint32_t)dm.stage);
                        tma_load_2d(hbuf, &tmX, kb * kMlpKS, m0, hb);
                        tma_load_2d(hbuf + kMlpXPart, &tmW1, kb * kMlpKS, 0, hb);
                        ++h_issued;
                        continue;
                    }
                    if (*vfail || (round > 0 && !tc::mbar_wait(&empty[st], (round - 1) & 1, kGemmWaitPolls))) {
                        atomicExch(&s_fail, 1);
                        ok = false;
                        break;
                    }
                    const uint32_t sx = ring0 + (uint32_t)(st * dm.stage);
                    const uint32_t fb = tc::smem_addr(&full[st]);
                    const int k0 = kb * kMlpKS;
                    if (kp - k0 >= kMlpKS) {
                        mbar_arrive_expect_tx(&full[st], (uint32_t)dm.stage);
                        tma_load_2d(sx, &tmX, k0, m0, fb);
                        tma_load_2d(sx + kMlpXPart, &tmW1, k0, 0, fb);
                    } else {
                        // the last 16 columns: two 8-column boxes per operand (no swizzle)
                        mbar_arrive_expect_tx(&full[st], (uint32_t)(2 * 128 * 16 + 2 * hid * 16));
                        tma_load_2d(sx, &tmXt, k0, m0, fb);
                        tma_load_2d(sx + 128 * 16, &tmXt, k0 + 8, m0, fb);
                        tma_load_2d(sx + kMlpXPart, &tmW1t, k0, 0, fb);
                        tma_load_2d(sx + kMlpXPart + (uint32_t)(hid * 16), &tmW1t, k0 + 8, 0, fb);
                    }
                    ++issued[st];
                    if (++st == S) {
                        st = 0;
                        ++round;
                    }
                }
            }
            // every copy has landed before shared memory goes away (at once
            // when the MMAs consumed them)
            for (int st = 0; st < S; ++st)
                if (issued[st] > 0) tc::mbar_wait(&full[st], (uint32_t)(issued[st] - 1) & 1u, kGemmWaitPolls);
            if (h_issued > 0) tc::mbar_wait(&hs_full, (uint32_t)(h_issued - 1) & 1u, kGemmWaitPolls);
        }
    } else if (warp == kMlpEpiWarps + 1) {
        // ---- MMA issuer ----
        if (lane == 0) {
            const uint32_t idesc1 = tc::make_idesc_bf16(128, hid);
            const uint32_t idesc2 = tc::make_idesc_bf16(128, 128);
            int st = 0, round = 0;
            bool ok = true;
            for (int t = 0; t < T_n && ok; ++t) {
                // layer 1 (acc1 was read out before h_full of tile t - 1)
                for (int kb = 0; kb < dm.nkb1; ++kb) {
                    const bool in_h = kb == kh;  // staged in the hidden tile's buffer
                    if (*vfail || !tc::mbar_wait(in_h ? &hs_full : &full[st], (uint32_t)(in_h ? t : round) & 1u,
                                                 kGemmWaitPolls)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t sx = in_h ? hbuf : ring0 + (uint32_t)(st * dm.stage);
                    if (kp - kb * kMlpKS >= kMlpKS) {
#pragma unroll
                        for (int j = 0; j < kMlpKS / 16; ++j)
                            tc::mma_bf16(tmem, tc::make_desc_sw128(sx + (uint32_t)(32 * j)),
                                         tc::make_desc_sw128(sx + (uint32_t)(kMlpXPart + 32 * j)), idesc1,
                                         (kb > 0 || j > 0) ? 1u : 0u);
                    } else {  // 16-column tail: K-major core matrices, the two 8-column halves LBO apart
                        tc::mma_bf16(tmem, tc::make_desc(sx, 128 * 16, 128),
                                     tc::make_desc(sx + kMlpXPart, (uint32_t)(hid * 16), 128), idesc1,
                                     kb > 0 ? 1u : 0u);
                    }
                    if (in_h) continue;  // freed by acc2_full of this tile instead
                    tc::mma_commit(&empty[st]);
                    if (++st == S) {
                        st = 0;
                        ++round;
                    }
                }
                if (!ok) break;
                tc::mma_commit(&acc1_full);
                // layer 2: H(t) written, acc2 read out for tile t - 1
                ok = tc::mbar_wait(&h_full, t & 1, kGemmWaitPolls) &&
                     (t > 0 || tc::mbar_wait(&w2_ready, 0, kGemmWaitPolls)) &&
                     (t == 0 || tc::mbar_wait(&acc2_empty, (t - 1) & 1, kGemmWaitPolls)) && !*vfail;
                if (!ok) break;
                tc::fence_after_sync();
                for (int j = 0; j < hid / 16; ++j)
                    tc::mma_bf16_tmem_a(tmem + dm.c_acc2, tmem + dm.c_w2 + (uint32_t)(8 * j),
                                        tc::make_desc_sw128(hbuf + (uint32_t)((j / 4) * kMlpXBlock + 32 * (j % 4))),
                                        idesc2, j > 0 ? 1u : 0u);
                tc::mma_commit(&acc2_full);
            }
            if (!ok) atomicExch(&s_fail, 1);
            tc::mma_commit(&fin);  // every MMA issued above has completed when this arrives
            tc::mbar_wait(&fin, 0, kGemmWaitPolls);
        }
    } else {
        // ---- epilogues ----
        // layer 1: warp w reads tile rows 32 (w % 4) .. + 31, part w / 4 of the hidden columns
        // layer 2: warp w reads output dimensions 32 (w % 4) .. + 31, part w / 4 of the tile rows
        constexpr int RW = 128 / kMlpParts;  // tile rows per warp in layer 2
        const int quarter = warp & 3, part = warp >> 2;
        const uint32_t lane_addr = (uint32_t)(quarter * 32) << 16;
        const int r = quarter * 32 + lane;
        const int hc0 = part * (hid / kMlpParts), hc1 = hc0 + hid / kMlpParts;
        const int o = quarter * 32 + lane;  // output dimension in layer 2
        const bool dim_ok = o < D;
        const bool warp_dims = quarter * 32 < D;
        const float bo = sb2[o];
        for (int t = 0; t < T_n; ++t) {
            const int m0 = MLP_TILE_ROW0(t);
            // the residual's coarse rows do not depend on the MMAs: bring
            // this warp's piece of each into L2 now (lane l: rows rb0 + l,
            // rb0 + 32 + l, ...), its latency hides behind layer 1
            const int rb0 = m0 + RW * part;
            int32_t mv[RW / 32];
#pragma unroll
            for (int c = 0; c < RW / 32; ++c) mv[c] = 0;
            if (warp_dims) {
#pragma unroll
                for (int c = 0; c < RW / 32; ++c) {
                    const int rl = rb0 + 32 * c + lane;
                    if (rl < M) {
                        mv[c] = __ldg(map + v0 + rl);
                        asm volatile("prefetch.global.L2 [%0];" ::"l"(Mc + (int64_t)mv[c] * D + quarter * 32));
                    }
                }
            }
            if (!__all_sync(0xffffffffu, tc::mbar_wait(&acc1_full, t & 1, kGemmWaitPolls) && !*vfail)) {
                atomicExch(&s_fail, 1);
                break;
            }
            tc::fence_after_sync();
            // H = relu(acc1 + b1) -> BF16, 128-byte swizzle: 16-byte chunk c of
            // row r of a 64-column block sits at chunk c ^ (r mod 8)
            for (int c0 = hc0; c0 < hc1; c0 += 32) {
                float v[32];
                tc::tmem_ld32(tmem + lane_addr + (uint32_t)c0, v);
                uint32_t w[16];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float4 bb = reinterpret_cast<const float4 *>(sb1 + c0)[j];
                    w[2 * j] = bias_relu_bf16x2(v[4 * j], v[4 * j + 1], bb.x, bb.y);
                    w[2 * j + 1] = bias_relu_bf16x2(v[4 * j + 2], v[4 * j + 3], bb.z, bb.w);
                }
                const uint32_t base = hbuf + (uint32_t)((c0 / kGemmKStage) * kMlpXBlock + r * 128);
                const int cc = (c0 % kGemmKStage) / 8;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint32_t a = base + (uint32_t)((((cc + q) ^ (r & 7)) & 7) << 4);
                    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(w[4 * q]), "r"(w[4 * q + 1]),
                                 "r"(w[4 * q + 2]), "r"(w[4 * q + 3])
                                 : "memory");
                }
            }
            tc::fence_before_sync();
            tc::fence_proxy_async();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&h_full);
            if (!__all_sync(0xffffffffu, tc::mbar_wait(&acc2_full, t & 1, kGemmWaitPolls) && !*vfail)) {
                atomicExch(&s_fail, 1);
                break;
            }
            tc::fence_after_sync();
            // residual: row rb0 + i, lane o = output dimension (contiguous per warp);
            // 32 rows per tensor-memory load
            const int nrow = M - rb0;
            T *dst = Mf + (v0 + rb0) * D + o;
#pragma unroll
            for (int c = 0; c < RW / 32; ++c) {
                float y[32];
                if (warp_dims) tc::tmem_ld32(tmem + lane_addr + dm.c_acc2 + (uint32_t)(RW * part + 32 * c), y);
                if (c == RW / 32 - 1) {
                    tc::fence_before_sync();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&acc2_empty);
                }
                if (!warp_dims || !dim_ok) continue;
                T own[32];
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const int32_t mi = __shfl_sync(0xffffffffu, mv[c], i);
                    own[i] = 32 * c + i < nrow ? __ldg(Mc + (int64_t)mi * D + o) : from_f<T>(0.0f);
                }
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    if (32 * c + i >= nrow) break;
                    dst[(int64_t)(32 * c + i) * D] = from_f<T>(to_f<T>(own[i]) + y[i] + bo);
                }
            }
        }
    }
    __syncwarp();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (s_fail && tid == 0) atomicExch(err, 1);
    if (warp == kMlpEpiWarps) tc::tmem_dealloc(tmem, dm.cols);
#undef MLP_TILE_ROW0
}

namespace {

typedef CUresult (*EncodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

gosh_status encoder(EncodeTiled *out) {
    static EncodeTiled fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p) {
            set_error("cuTensorMapEncodeTiled is not available from the driver");
            return GOSH_ERR_CUDA;
        }
        fn = reinterpret_cast<EncodeTiled>(p);
    }
    *out = fn;
    return GOSH_OK;
}

// Row-major BF16 matrix (rows x cols, row stride ld elements) read in boxes of
// {box_cols columns, box_rows rows}: 64 columns written with the 128-byte
// swizzle, or 8 columns (one 16-byte core-matrix column, no swizzle);
// out-of-range rows and columns read as zero.
gosh_status make_map(CUtensorMap *m, const __nv_bfloat16 *base, int64_t rows, int64_t cols, int64_t ld, int box_rows,
                     int box_cols = kGemmKStage) {
    EncodeTiled enc = nullptr;
    GOSH_TRY(encoder(&enc));
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(base), dims, strides, box,
                           estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           box_cols == kGemmKStage ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d) for a %lld x %lld operand, stride %lld", (int)r, (long long)rows,
                  (long long)cols, (long long)ld);
        return GOSH_ERR_CUDA;
    }
    return GOSH_OK;
}

template <int NT, int EPI, typename T>
gosh_status launch_nt(const __nv_bfloat16 *A, int64_t lda, const __nv_bfloat16 *B, int64_t ldb, const GemmEpi &ep,
                      int M, int N, int K, int splits, int *err, cudaStream_t s) {
    constexpr size_t smem = GemmShape<NT>::kSmem;
    static bool attr = false;
    if (!attr) {
        GOSH_TRY_CUDA(cudaFuncSetAttribute(tma_gemm_kernel<NT, EPI, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem));
        attr = true;
    }
    CUtensorMap ma, mb;
    GOSH_TRY(make_map(&ma, A, M, K, lda, 128));
    GOSH_TRY(make_map(&mb, B, N, K, ldb, NT));
    int kps = (int)ceil_div(K, splits);
    kps = (int)ceil_div(kps, 16) * 16;
    const int zs = (int)ceil_div(K, kps);
    dim3 grid((unsigned)ceil_div(M, 128), (unsigned)ceil_div(N, NT), (unsigned)zs);
    launch_dep(tma_gemm_kernel<NT, EPI, T>, grid, kGemmThreads, smem, s, ma, mb, ep, M, N, K, kps, err);
    GOSH_TRY_CUDA(cudaGetLastError());
    return GOSH_OK;
}

template <int EPI, typename T>
gosh_status launch(const __nv_bfloat16 *A, int64_t lda, const __nv_bfloat16 *B, int64_t ldb, const GemmEpi &ep, int M,
                   int N, int K, int splits, int *err, cudaStream_t s) {
    if (N <= 16) return launch_nt<16, EPI, T>(A, lda, B, ldb, ep, M, N, K, splits, err, s);
    if (N <= 32) return launch_nt<32, EPI, T>(A, lda, B, ldb, ep, M, N, K, splits, err, s);
    if (N <= 64) return launch_nt<64, EPI, T>(A, lda, B, ldb, ep, M, N, K, splits, err, s);
    if (N <= 128) return launch_nt<128, EPI, T>(A, lda, B, ldb, ep, M, N, K, splits, err, s);
    return launch_nt<256, EPI, T>(A, lda, B, ldb, ep, M, N, K, splits, err, s);
}

gosh_status check_operands(const void *A, int64_t lda, const void *B, int64_t ldb, int M, int N, int K) {
    GOSH_CHECK_ARG(M > 0 && N > 0 && N <= 256 && K > 0 && K % 16 == 0,
                   "GEMM needs M > 0, 0 < N <= 256 and K a positive multiple of 16");
    GOSH_CHECK_ARG(lda % 8 == 0 && ldb % 8 == 0 && lda >= K && ldb >= K, "row strides must be >= K and keep 16-byte alignment");
    GOSH_CHECK_ARG(((uintptr_t)A & 15) == 0 && ((uintptr_t)B & 15) == 0, "GEMM operands must be 16-byte aligned");
    return GOSH_OK;
}

template <typename T, int D>
gosh_status launch_mlp(const CUtensorMap &mx, const CUtensorMap &m1, const CUtensorMap &mxt, const CUtensorMap &m1t,
                       const __nv_bfloat16 *W2b, const float *b1, const float *b2, const int32_t *map, const void *Mc,
                       void *Mf, int64_t v0, int M, int hid, int kp, int *err, cudaStream_t s) {
    const MlpDims dm(hid, kp);
    const size_t smem = dm.smem();
    static size_t attr = 0;
    if (attr < smem) {
        GOSH_TRY_CUDA(
            cudaFuncSetAttribute(mlp_project_kernel<T, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = smem;
    }
    const int ntiles = (int)ceil_div(M, 128);
    const int grid = ntiles < num_sms() ? ntiles : num_sms();
    launch_dep(mlp_project_kernel<T, D>, grid, kMlpThreads, smem, s, mx, m1, mxt, m1t, W2b, b1, b2, map,
               static_cast<const T *>(Mc), static_cast<T *>(Mf), v0, M, hid, kp, err);
    GOSH_TRY_CUDA(cudaGetLastError());
    return GOSH_OK;
}

}  // namespace

// Whether tc_mlp_project takes these shapes: d in {32, 64, 128}, hidden 128
// or 256 (acc1, W2 and acc2 in one SM's tensor memory; whole 32-column
// loads for each epilogue warp), at least two ring stages beside the hidden
// tile in shared memory.
bool tc_mlp_fused_ok(int d, int hid, int kp) {
    if (!(d == 32 || d == 64 || d == 128) || !(hid == 64 || hid == 128 || hid == 256) || kp % 16 != 0 || kp <= 0)
        return false;
    const MlpDims dm(hid, kp);
    // (the hidden tile's buffer also holds one ring stage: hbytes >= stage)
    return kp % kMlpKS == 16 && hid / kMlpParts % 32 == 0 && dm.S >= 2 && dm.cols <= 512 && dm.hbytes >= dm.stage;
}

// Mf[v0 + m] = Mc[map[v0 + m]] + relu(X[m] W1^T + b1) W2^T + b2 for m < M:
// X (M x kp, BF16, row stride kp), W1b (hid x kp), W2b (d x hid), both BF16
// row-major; the hidden layer is rounded to BF16 as the two-GEMM path does.
gosh_status tc_mlp_project(const __nv_bfloat16 *X, const __nv_bfloat16 *W1b, const __nv_bfloat16 *W2b,
                           const float *b1, const float *b2, const int32_t *map, const void *Mc, void *Mf, int64_t v0,
                           int d, int hid, int kp, gosh_dtype dt, int M, int *err, cudaStream_t s) {
    GOSH_CHECK_ARG(M > 0 && tc_mlp_fused_ok(d, hid, kp), "fused projection: unsupported shape");
    GOSH_CHECK_ARG(((uintptr_t)X & 15) == 0 && ((uintptr_t)W1b & 15) == 0 && ((uintptr_t)W2b & 3) == 0,
                   "fused projection: operands must be 16-byte aligned");
    CUtensorMap mx, m1, mxt, m1t;
    GOSH_TRY(make_map(&mx, X, M, kp, kp, 128, kMlpKS));
    GOSH_TRY(make_map(&m1, W1b, hid, kp, kp, hid, kMlpKS));
    GOSH_TRY(make_map(&mxt, X, M, kp, kp, 128, 8));
    GOSH_TRY(make_map(&m1t, W1b, hid, kp, kp, hid, 8));
    auto go = [&](auto *tp) -> gosh_status {
        using T = std::remove_pointer_t<decltype(tp)>;
        switch (d) {
        case 32: return launch_mlp<T, 32>(mx, m1, mxt, m1t, W2b, b1, b2, map, Mc, Mf, v0, M, hid, kp, err, s);
        case 64: return launch_mlp<T, 64>(mx, m1, mxt, m1t, W2b, b1, b2, map, Mc, Mf, v0, M, hid, kp, err, s);
        default: return launch_mlp<T, 128>(mx, m1, mxt, m1t, W2b, b1, b2, map, Mc, Mf, v0, M, hid, kp, err, s);
        }
    };
    switch (dt) {
    case GOSH_F32: return go((float *)nullptr);
    case GOSH_BF16: return go((__nv_bfloat16 *)nullptr);
    case GOSH_F16: return go((__half *)nullptr);
    }
    set_error("unknown dtype");
    return GOSH_ERR_INVALID_ARG;
}

// C (M x N, FP32, row stride ldc) = A (M x K) . B (N x K)^T, or += when splits > 1
// (split-K over `splits` CTAs per tile, C must then hold the addend).  N <= 256.
gosh_status tc_gemm(const __nv_bfloat16 *A, int64_t lda, const __nv_bfloat16 *B, int64_t ldb, float *C, int64_t ldc,
                    int M, int N, int K, int splits, int *err, cudaStream_t s) {
    GOSH_TRY(check_operands(A, lda, B, ldb, M, N, K));
    GOSH_CHECK_ARG(ldc % 4 == 0 && ((uintptr_t)C & 15) == 0, "C must keep 16-byte alignment");
    if (splits < 1) splits = 1;
    GemmEpi ep;
    ep.C = C;
    ep.ldc = ldc;
    if (splits > 1) return launch<kEpiAtomic, float>(A, lda, B, ldb, ep, M, N, K, splits, err, s);
    return launch<kEpiStore, float>(A, lda, B, ldb, ep, M, N, K, 1, err, s);
}

// H (M x N, BF16, row stride ldh) = relu(A . B^T + bias).  N <= 256.
gosh_status tc_gemm_bias_relu(const __nv_bfloat16 *A, int64_t lda, const __nv_bfloat16 *B, int64_t ldb,
                              const float *bias, __nv_bfloat16 *H, int64_t ldh, int M, int N, int K, int *err,
                              cudaStream_t s) {
    GOSH_TRY(check_operands(A, lda, B, ldb, M, N, K));
    GOSH_CHECK_ARG(ldh % 8 == 0 && ((uintptr_t)H & 15) == 0, "H must keep 16-byte alignment");
    GemmEpi ep;
    ep.bias = bias;
    ep.H = H;
    ep.ldh = ldh;
    return launch<kEpiBiasRelu, float>(A, lda, B, ldb, ep, M, N, K, 1, err, s);
}

// Mf[v0 + m][n] = Mc[map[v0 + m]][n] + (A . B^T)[m][n] + bias[n] for m < M,
// n < d (storage type of Mc/Mf: dt; d a multiple of 16, at most 256; rows
// 16-byte aligned).
gosh_status tc_gemm_residual(const __nv_bfloat16 *A, int64_t lda, const __nv_bfloat16 *B, int64_t ldb,
                             const float *bias, const int32_t *map, const void *Mc, void *Mf, int64_t v0, int d,
                             gosh_dtype dt, int M, int K, int *err, cudaStream_t s) {
    GOSH_TRY(check_operands(A, lda, B, ldb, M, d, K));
    GOSH_CHECK_ARG(d % 16 == 0 && ((uintptr_t)Mc & 15) == 0 && ((uintptr_t)Mf & 15) == 0,
                   "residual epilogue needs d a multiple of 16 and 16-byte aligned tables");
    GemmEpi ep;
    ep.bias = bias;
    ep.map = map;
    ep.Mc = Mc;
    ep.Mf = Mf;
    ep.v0 = v0;
    ep.d = d;
    switch (dt) {
    case GOSH_F32: return launch<kEpiResidual, float>(A, lda, B, ldb, ep, M, d, K, 1, err, s);
    case GOSH_BF16: return launch<kEpiResidual, __nv_bfloat16>(A, lda, B, ldb, ep, M, d, K, 1, err, s);
    case GOSH_F16: return launch<kEpiResidual, __half>(A, lda, B, ldb, ep, M, d, K, 1, err, s);
    }
    set_error("unknown dtype");
    return GOSH_ERR_INVALID_ARG;
}

}  // namespace gosh

using namespace gosh;

extern "C" gosh_status gosh_tc_gemm_bf16(const void *A, int64_t lda, const void *B, int64_t ldb, float *C, int64_t ldc,
                                         int M, int N, int K, int splits, void *stream) {
    clear_error();
    GOSH_CHECK_ARG(A && B && C, "NULL operand");
    cudaStream_t s = (cudaStream_t)stream;
    Scratch err;
    GOSH_TRY(err.alloc(sizeof(int), s));
    GOSH_TRY_CUDA(cudaMemsetAsync(err.ptr, 0, sizeof(int), s));
    const int nt_max = 256;
    for (int n0 = 0; n0 < N; n0 += nt_max) {
        const int nn = N - n0 < nt_max ? N - n0 : nt_max;
        GOSH_TRY(tc_gemm(static_cast<const __nv_bfloat16 *>(A), lda,
                         static_cast<const __nv_bfloat16 *>(B) + (int64_t)n0 * ldb, ldb, C + n0, ldc, M, nn, K, splits,
                         err.as<int>(), s));
    }
    int herr = 0;
    GOSH_TRY_CUDA(cudaMemcpyAsync(&herr, err.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
    GOSH_TRY_CUDA(cudaStreamSynchronize(s));
    if (herr) {
        set_error("tensor-core GEMM: an MMA or copy completion wait timed out");
        return GOSH_ERR_TIMEOUT;
    }
    return GOSH_OK;
}
