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

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_addr(mbar)), "r"(bytes)
                 : "memory");
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
// kernel (both layers of the MLP, the hidden layer never leaves the SM):
//
//   acc1 = X W1^T                 tensor memory columns [0, HID)
//   H    = relu(acc1 + b1)        BF16, written to shared memory
//   acc2 = H W2^T                 tensor memory columns [HID, HID + D)
//   Mf[v0 + m] = Mc[map[v0 + m]] + acc2 + b2
//
// One CTA per SM walks the chunk's 128-row tiles (tile = blockIdx.x + i *
// gridDim.x).  Roles: warps 0-7 run the epilogues (warps w and w + 4 read
// the same 32 tensor-memory lanes, each half of the columns), warp 8 loads
// the X tiles (two tile buffers, the next tile's rows arrive while this
// one is computed), warp 9 streams the weights through a two-slot ring in
// 64-column blocks (W1 blocks for layer 1, W2 blocks for layer 2, in the
// order the MMAs consume them) and warp 10 issues the MMAs.  H of tile t is
// written over X of tile t (layer 1 has consumed it), in the same 128-byte
// swizzled K-major layout the TMA writes, so layer 2 reads it in place.
// Every operand and tile buffer starts on a 1024-byte boundary.
//
// Barriers: x_full / x_empty per tile buffer, w_full / w_empty per ring
// slot, acc1_full (layer 1 done), acc1_empty (acc1 read out), h_full (H
// written and fenced for the tensor cores), acc2_full (layer 2 done: H and
// its buffer free), acc2_empty (acc2 read out).  Every wait is bounded; on
// time-out the CTA raises *err, every role stops, the producers wait
// (bounded) for their copies in flight and the tensor memory is freed.
constexpr int kMlpEpiWarps = 8;
constexpr int kMlpThreads = (kMlpEpiWarps + 3) * 32;
constexpr int kMlpTileBytes = 128 * kGemmKStage * 2;  // one 64-column block of a 128-row tile

struct MlpDims {
    int hid, kp, nkb1, nkb2, xbytes, slot;
    __host__ __device__ MlpDims(int D, int hid_, int kp_)
        : hid(hid_), kp(kp_), nkb1((kp_ + kGemmKStage - 1) / kGemmKStage), nkb2(hid_ / kGemmKStage),
          xbytes((nkb1 > nkb2 ? nkb1 : nkb2) * kMlpTileBytes), slot((hid_ > D ? hid_ : D) * kGemmKStage * 2) {}
    __host__ __device__ size_t smem() const { return (size_t)2 * xbytes + (size_t)2 * slot + 1024; }
};

// The MMA issue order: layer 1 of tile i then layer 2 of tile i.  The
// weight producer loads the ring in the same order.
template <typename T, int D>
__global__ void __launch_bounds__(kMlpThreads, 1)
    mlp_project_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmW1,
                       const __grid_constant__ CUtensorMap tmW2, const float *__restrict__ b1,
                       const float *__restrict__ b2, const int32_t *__restrict__ map, const T *__restrict__ Mc,
                       T *__restrict__ Mf, int64_t v0, int M, int hid, int kp, uint32_t tmem_cols,
                       int *__restrict__ err) {
    GOSH_DEP_WAIT();
    static_assert(D == 32 || D == 64 || D == 128, "D in {32, 64, 128}");
    const MlpDims dm(D, hid, kp);
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = smem_raw + ((1024u - (tc::smem_addr(smem_raw) & 1023u)) & 1023u);
    const uint32_t xbuf0 = tc::smem_addr(smem);
    const uint32_t ring0 = xbuf0 + 2u * (uint32_t)dm.xbytes;
    __shared__ __align__(8) uint64_t x_full[2], x_empty[2], w_full[2], w_empty[2];
    __shared__ __align__(8) uint64_t acc1_full, acc1_empty, h_full, acc2_full, acc2_empty, fin;
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntiles = (M + 127) / 128;
    const int T_n = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

    if (warp == kMlpEpiWarps) tc::tmem_alloc(&tmem_base, tmem_cols);
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&x_full[i], 1);
            tc::mbar_init(&x_empty[i], 1);
            tc::mbar_init(&w_full[i], 1);
            tc::mbar_init(&w_empty[i], 1);
        }
        tc::mbar_init(&acc1_full, 1);
        tc::mbar_init(&acc1_empty, kMlpEpiWarps);
        tc::mbar_init(&h_full, kMlpEpiWarps);
        tc::mbar_init(&acc2_full, 1);
        tc::mbar_init(&acc2_empty, kMlpEpiWarps);
        tc::mbar_init(&fin, 1);
        s_fail = 0;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base;
    volatile int *vfail = &s_fail;

    if (warp == kMlpEpiWarps) {
        // ---- X tiles: buffer t & 1, reused once layer 2 of tile t - 2 is done ----
        if (lane == 0) {
            int issued[2] = {0, 0};
            for (int t = 0; t < T_n; ++t) {
                const int b = t & 1;
                if (*vfail) break;
                if (t >= 2 && !tc::mbar_wait(&x_empty[b], ((t >> 1) - 1) & 1, kGemmWaitPolls)) {
                    atomicExch(&s_fail, 1);
                    break;
                }
                const int m0 = ((int)blockIdx.x + t * (int)gridDim.x) * 128;
                mbar_arrive_expect_tx(&x_full[b], (uint32_t)(dm.nkb1 * kMlpTileBytes));
                for (int kb = 0; kb < dm.nkb1; ++kb)
                    tma_load_2d(xbuf0 + (uint32_t)(b * dm.xbytes + kb * kMlpTileBytes), &tmX, kb * kGemmKStage, m0,
                                tc::smem_addr(&x_full[b]));
                ++issued[b];
            }
            // every copy has landed before shared memory goes away (at once
            // when the MMAs consumed them)
            for (int b = 0; b < 2; ++b)
                if (issued[b] > 0) tc::mbar_wait(&x_full[b], (uint32_t)(issued[b] - 1) & 1u, kGemmWaitPolls);
        }
    } else if (warp == kMlpEpiWarps + 1) {
        // ---- weight ring: per tile nkb1 W1 blocks, then nkb2 W2 blocks ----
        if (lane == 0) {
            int issued[2] = {0, 0};
            int it = 0;
            bool ok = true;
            for (int t = 0; t < T_n && ok; ++t) {
                for (int layer = 0; layer < 2 && ok; ++layer) {
                    const int nb = layer == 0 ? dm.nkb1 : dm.nkb2;
                    const uint32_t bytes = (uint32_t)((layer == 0 ? hid : D) * kGemmKStage * 2);
                    for (int kb = 0; kb < nb; ++kb, ++it) {
                        const int sl = it & 1;
                        if (*vfail || (it >= 2 && !tc::mbar_wait(&w_empty[sl], ((it >> 1) - 1) & 1, kGemmWaitPolls))) {
                            atomicExch(&s_fail, 1);
                            ok = false;
                            break;
                        }
                        mbar_arrive_expect_tx(&w_full[sl], bytes);
                        tma_load_2d(ring0 + (uint32_t)(sl * dm.slot), layer == 0 ? &tmW1 : &tmW2, kb * kGemmKStage, 0,
                                    tc::smem_addr(&w_full[sl]));
                        ++issued[sl];
                    }
                }
            }
            for (int sl = 0; sl < 2; ++sl)
                if (issued[sl] > 0) tc::mbar_wait(&w_full[sl], (uint32_t)(issued[sl] - 1) & 1u, kGemmWaitPolls);
        }
    } else if (warp == kMlpEpiWarps + 2) {
        // ---- MMA issuer ----
        if (lane == 0) {
            const uint32_t idesc1 = tc::make_idesc_bf16(128, hid);
            const uint32_t idesc2 = tc::make_idesc_bf16(128, D);
            int it = 0;
            bool ok = true;
            for (int t = 0; t < T_n && ok; ++t) {
                const int b = t & 1;
                const uint32_t xb = xbuf0 + (uint32_t)(b * dm.xbytes);
                // layer 1: X(t) and acc1 free (read out for tile t - 1)
                ok = tc::mbar_wait(&x_full[b], (t >> 1) & 1, kGemmWaitPolls) &&
                     (t == 0 || tc::mbar_wait(&acc1_empty, (t - 1) & 1, kGemmWaitPolls));
                for (int kb = 0; kb < dm.nkb1 && ok; ++kb, ++it) {
                    const int sl = it & 1;
                    if (*vfail || !tc::mbar_wait(&w_full[sl], (it >> 1) & 1, kGemmWaitPolls)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const int k0 = kb * kGemmKStage;
                    const int steps = min(kGemmKStage, kp - k0) / 16;
                    const uint32_t wb = ring0 + (uint32_t)(sl * dm.slot);
                    for (int j = 0; j < steps; ++j)
                        tc::mma_bf16(tmem, tc::make_desc_sw128(xb + (uint32_t)(kb * kMlpTileBytes + 32 * j)),
                                     tc::make_desc_sw128(wb + (uint32_t)(32 * j)), idesc1, (kb > 0 || j > 0) ? 1u : 0u);
                    tc::mma_commit(&w_empty[sl]);
                }
                if (!ok) break;
                tc::mma_commit(&acc1_full);
                // layer 2: H(t) written, acc2 free (read out for tile t - 1)
                ok = tc::mbar_wait(&h_full, t & 1, kGemmWaitPolls) &&
                     (t == 0 || tc::mbar_wait(&acc2_empty, (t - 1) & 1, kGemmWaitPolls));
                for (int kb = 0; kb < dm.nkb2 && ok; ++kb, ++it) {
                    const int sl = it & 1;
                    if (*vfail || !tc::mbar_wait(&w_full[sl], (it >> 1) & 1, kGemmWaitPolls)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t wb = ring0 + (uint32_t)(sl * dm.slot);
                    for (int j = 0; j < kGemmKStage / 16; ++j)
                        tc::mma_bf16(tmem + (uint32_t)hid, tc::make_desc_sw128(xb + (uint32_t)(kb * kMlpTileBytes + 32 * j)),
                                     tc::make_desc_sw128(wb + (uint32_t)(32 * j)), idesc2, (kb > 0 || j > 0) ? 1u : 0u);
                    tc::mma_commit(&w_empty[sl]);
                }
                if (!ok) break;
                tc::mma_commit(&acc2_full);
                tc::mma_commit(&x_empty[b]);
            }
            if (!ok) atomicExch(&s_fail, 1);
            tc::mma_commit(&fin);  // every MMA issued above has completed when this arrives
            tc::mbar_wait(&fin, 0, kGemmWaitPolls);
        }
    } else {
        // ---- epilogues: warp w reads lanes 32 (w % 4) .. + 31, column half w / 4 ----
        const int quarter = warp & 3, half = warp >> 2;
        const uint32_t lane_addr = (uint32_t)(quarter * 32) << 16;
        const int r = quarter * 32 + lane;  // row of the tile
        const int hc0 = half * (hid / 2), hc1 = hc0 + hid / 2;
        constexpr int DH = D / 2;                       // acc2 columns of this warp
        constexpr int PV = 16 / (int)sizeof(T);         // table values per 16-byte vector
        constexpr int NV = DH / PV;                     // 16-byte vectors of this warp's part of a row
        const int dc0 = half * DH;
        for (int t = 0; t < T_n; ++t) {
            const int b = t & 1;
            const uint32_t xb = xbuf0 + (uint32_t)(b * dm.xbytes);
            const int row = ((int)blockIdx.x + t * (int)gridDim.x) * 128 + r;
            // the coarse rows of the residual do not depend on the MMAs: fetch them first
            uint4 own[NV];
            const int64_t vv = v0 + row;
            if (row < M) {
                const uint4 *src = reinterpret_cast<const uint4 *>(Mc + (int64_t)__ldg(map + vv) * D + dc0);
#pragma unroll
                for (int x = 0; x < NV; ++x) own[x] = __ldg(src + x);
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
                for (int j = 0; j < 16; ++j) {
                    const float2 bb = __ldg(reinterpret_cast<const float2 *>(b1 + c0) + j);
                    const __nv_bfloat162 h =
                        __floats2bfloat162_rn(fmaxf(v[2 * j] + bb.x, 0.0f), fmaxf(v[2 * j + 1] + bb.y, 0.0f));
                    w[j] = *reinterpret_cast<const uint32_t *>(&h);
                }
                const uint32_t base = xb + (uint32_t)((c0 / kGemmKStage) * kMlpTileBytes + r * 128);
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
            if (lane == 0) {
                tc::mbar_arrive(&acc1_empty);
                tc::mbar_arrive(&h_full);
            }
            if (!__all_sync(0xffffffffu, tc::mbar_wait(&acc2_full, t & 1, kGemmWaitPolls) && !*vfail)) {
                atomicExch(&s_fail, 1);
                break;
            }
            tc::fence_after_sync();
            float y[DH];
#pragma unroll
            for (int c = 0; c < DH; c += 16) tc::tmem_ld16(tmem + lane_addr + (uint32_t)(hid + dc0 + c), y + c);
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&acc2_empty);
            if (row < M) {
                uint4 *dst = reinterpret_cast<uint4 *>(Mf + vv * D + dc0);
#pragma unroll
                for (int x = 0; x < NV; ++x) {
                    union {
                        uint4 u;
                        T t[PV];
                    } pk;
                    pk.u = own[x];
#pragma unroll
                    for (int q = 0; q < PV; ++q)
                        pk.t[q] = from_f<T>(to_f<T>(pk.t[q]) + y[x * PV + q] + __ldg(b2 + dc0 + x * PV + q));
                    dst[x] = pk.u;
                }
            }
        }
    }
    __syncwarp();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (s_fail && tid == 0) atomicExch(err, 1);
    if (warp == kMlpEpiWarps) tc::tmem_dealloc(tmem, tmem_cols);
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
// {64 columns, box_rows rows} with the 128-byte swizzle; out-of-range rows
// and columns read as zero.
gosh_status make_map(CUtensorMap *m, const __nv_bfloat16 *base, int64_t rows, int64_t cols, int64_t ld, int box_rows) {
    EncodeTiled enc = nullptr;
    GOSH_TRY(encoder(&enc));
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kGemmKStage, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(base), dims, strides, box,
                           estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
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
gosh_status launch_mlp(const CUtensorMap &mx, const CUtensorMap &m1, const CUtensorMap &m2, const float *b1,
                       const float *b2, const int32_t *map, const void *Mc, void *Mf, int64_t v0, int M, int hid, int kp,
                       int *err, cudaStream_t s) {
    const MlpDims dm(D, hid, kp);
    const size_t smem = dm.smem();
    static size_t attr = 0;
    if (attr < smem) {
        GOSH_TRY_CUDA(
            cudaFuncSetAttribute(mlp_project_kernel<T, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = smem;
    }
    uint32_t cols = 32;
    while (cols < (uint32_t)(hid + D)) cols <<= 1;
    const int ntiles = (int)ceil_div(M, 128);
    const int grid = ntiles < num_sms() ? ntiles : num_sms();
    launch_dep(mlp_project_kernel<T, D>, grid, kMlpThreads, smem, s, mx, m1, m2, b1, b2, map, static_cast<const T *>(Mc),
               static_cast<T *>(Mf), v0, M, hid, kp, cols, err);
    GOSH_TRY_CUDA(cudaGetLastError());
    return GOSH_OK;
}

}  // namespace

// Whether tc_mlp_project takes these shapes: d in {32, 64, 128}, hidden a
// multiple of 64 up to 256 (both accumulators in one SM's tensor memory).
bool tc_mlp_fused_ok(int d, int hid, int kp) {
    if (!(d == 32 || d == 64 || d == 128) || hid % 64 != 0 || hid < 64 || hid > 256 || kp % 16 != 0 || kp <= 0)
        return false;
    return MlpDims(d, hid, kp).smem() <= 232448 - 1024;
}

// Mf[v0 + m] = Mc[map[v0 + m]] + relu(X[m] W1^T + b1) W2^T + b2 for m < M:
// X (M x kp, BF16, row stride kp), W1b (hid x kp), W2b (d x hid), both BF16
// row-major; the hidden layer is rounded to BF16 as the two-GEMM path does.
gosh_status tc_mlp_project(const __nv_bfloat16 *X, const __nv_bfloat16 *W1b, const __nv_bfloat16 *W2b,
                           const float *b1, const float *b2, const int32_t *map, const void *Mc, void *Mf, int64_t v0,
                           int d, int hid, int kp, gosh_dtype dt, int M, int *err, cudaStream_t s) {
    GOSH_CHECK_ARG(M > 0 && tc_mlp_fused_ok(d, hid, kp), "fused projection: unsupported shape");
    GOSH_CHECK_ARG(((uintptr_t)X & 15) == 0 && ((uintptr_t)W1b & 15) == 0 && ((uintptr_t)W2b & 15) == 0 &&
                       ((uintptr_t)Mc & 15) == 0 && ((uintptr_t)Mf & 15) == 0 && ((uintptr_t)b1 & 7) == 0,
                   "fused projection: operands must be 16-byte aligned");
    CUtensorMap mx, m1, m2;
    GOSH_TRY(make_map(&mx, X, M, kp, kp, 128));
    GOSH_TRY(make_map(&m1, W1b, hid, kp, kp, hid));
    GOSH_TRY(make_map(&m2, W2b, d, hid, hid, d));
    auto go = [&](auto *tp) -> gosh_status {
        using T = std::remove_pointer_t<decltype(tp)>;
        switch (d) {
        case 32: return launch_mlp<T, 32>(mx, m1, m2, b1, b2, map, Mc, Mf, v0, M, hid, kp, err, s);
        case 64: return launch_mlp<T, 64>(mx, m1, m2, b1, b2, map, Mc, Mf, v0, M, hid, kp, err, s);
        default: return launch_mlp<T, 128>(mx, m1, m2, b1, b2, map, Mc, Mf, v0, M, hid, kp, err, s);
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
