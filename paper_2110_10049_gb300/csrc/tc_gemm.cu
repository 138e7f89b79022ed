// BF16 GEMM on the tcgen05 tensor cores: C[m][n] = sum_k A[m][k] * B[n][k]
// (A and B row-major with K contiguous, FP32 accumulation in tensor memory).
//
// One CTA (4 warps) computes a 128 x NT tile over a K range: 64-wide K chunks
// of A and B are copied into shared memory in the canonical no-swizzle K-major
// layout, one thread issues the K/16 MMAs, tcgen05.commit signals an mbarrier
// and the four warps read their 32 accumulator lanes back with tcgen05.ld.
// Split-K launches add their partial tiles into C with vector atomics.
// Every wait is bounded: on time-out the CTA raises *err, waits (bounded) for
// its MMAs, frees its tensor memory and leaves C unwritten.
#include "common.cuh"
#include "tcgen05.cuh"

namespace gosh {

constexpr int kGemmThreads = 128;
constexpr int kGemmKChunk = 64;
constexpr uint32_t kGemmWaitPolls = 1u << 22;

template <int NT>
__global__ void __launch_bounds__(kGemmThreads) tc_gemm_kernel(const __nv_bfloat16 *__restrict__ A, int64_t lda,
                                                               const __nv_bfloat16 *__restrict__ B, int64_t ldb,
                                                               float *__restrict__ C, int64_t ldc, int M, int N,
                                                               int K, int k_per_split, int atomic_add,
                                                               int *__restrict__ err) {
    static_assert(NT % 16 == 0 && NT >= 16 && NT <= 256, "M = 128 needs N in [16, 256], multiple of 16");
    constexpr uint32_t kCols = NT <= 32 ? 32 : (NT <= 64 ? 64 : (NT <= 128 ? 128 : 256));
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint64_t mbar;
    __shared__ uint32_t tmem_base;
    uint8_t *sA = smem;                  // 128 rows x 64 K x 2 B = 16 KB
    uint8_t *sB = smem + 128 * 128;      // NT rows x 64 K x 2 B
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * 128, n0 = blockIdx.y * NT;
    const int kb = blockIdx.z * k_per_split;
    const int ke = min(K, kb + k_per_split);

    if (warp == 0) tc::tmem_alloc(&tmem_base, kCols);
    if (tid == 0) tc::mbar_init(&mbar, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = tc::make_idesc_bf16(128, NT);

    uint32_t phase = 0;
    int ok = 1, issued = 0;
    for (int k0 = kb; k0 < ke && ok; k0 += kGemmKChunk) {
        const int kc = min(kGemmKChunk, ke - k0);  // multiple of 16
        const int nv = kc / 8;                       // core matrices along K
        for (int i = tid; i < 128 * nv; i += kGemmThreads) {
            const int r = i / nv, c = i % nv;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (m0 + r < M) v = *reinterpret_cast<const uint4 *>(A + (int64_t)(m0 + r) * lda + k0 + c * 8);
            *reinterpret_cast<uint4 *>(sA + (r >> 3) * (nv * 128) + c * 128 + (r & 7) * 16) = v;
        }
        for (int i = tid; i < NT * nv; i += kGemmThreads) {
            const int r = i / nv, c = i % nv;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (n0 + r < N) v = *reinterpret_cast<const uint4 *>(B + (int64_t)(n0 + r) * ldb + k0 + c * 8);
            *reinterpret_cast<uint4 *>(sB + (r >> 3) * (nv * 128) + c * 128 + (r & 7) * 16) = v;
        }
        tc::fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            for (int s = 0; s < kc / 16; ++s) {
                const uint64_t ad = tc::make_desc(tc::smem_addr(sA) + s * 256, 128, nv * 128);
                const uint64_t bd = tc::make_desc(tc::smem_addr(sB) + s * 256, 128, nv * 128);
                tc::mma_bf16(tmem, ad, bd, idesc, (k0 > kb || s > 0) ? 1u : 0u);
            }
            tc::mma_commit(&mbar);
        }
        issued = 1;
        const bool done = tc::mbar_wait(&mbar, phase, kGemmWaitPolls);
        ok = __syncthreads_and(done ? 1 : 0);
        phase ^= 1;
        tc::fence_after_sync();
    }
    if (!ok) {
        // the last commit never arrived: give the MMAs one more bounded wait
        tc::mbar_wait(&mbar, phase ^ 1, kGemmWaitPolls);
        if (tid == 0) atomicExch(err, 1);
    } else if (issued) {
        const int row = m0 + warp * 32 + lane;
#pragma unroll 1
        for (int c = 0; c < NT; c += 16) {
            float v[16];
            tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
            if (row < M) {
                float *out = C + (int64_t)row * ldc + n0 + c;
#pragma unroll
                for (int j = 0; j < 16; j += 4) {
                    if (n0 + c + j + 3 < N) {
                        if (atomic_add) {
                            asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(out + j), "f"(v[j]),
                                         "f"(v[j + 1]), "f"(v[j + 2]), "f"(v[j + 3])
                                         : "memory");
                        } else {
                            *reinterpret_cast<float4 *>(out + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                        }
                    } else {
                        for (int q = j; q < j + 4; ++q)
                            if (n0 + c + q < N) {
                                if (atomic_add) atomicAdd(out + q, v[q]);
                                else out[q] = v[q];
                            }
                    }
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kCols);
}

template <int NT>
gosh_status launch_tc_gemm_nt(const __nv_bfloat16 *A, int64_t lda, const __nv_bfloat16 *B, int64_t ldb, float *C,
                              int64_t ldc, int M, int N, int K, int splits, int *err, cudaStream_t s) {
    const size_t smem = 128 * 128 + NT * 128;
    static bool attr = false;
    if (!attr) {
        GOSH_TRY_CUDA(cudaFuncSetAttribute(tc_gemm_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = true;
    }
    int kps = (int)ceil_div(K, splits);
    kps = (int)ceil_div(kps, 16) * 16;
    const int zs = (int)ceil_div(K, kps);
    dim3 grid((unsigned)ceil_div(M, 128), (unsigned)ceil_div(N, NT), (unsigned)zs);
    (tc_gemm_kernel<NT><<<grid, kGemmThreads, smem, s>>>(A, lda, B, ldb, C, ldc, M, N, K, kps, splits > 1 ? 1 : 0,
                                                         err),
     note_launch());
    GOSH_TRY_CUDA(cudaGetLastError());
    return GOSH_OK;
}

// C (M x N, FP32, row stride ldc) = A (M x K) . B (N x K)^T, or += when splits > 1
// (split-K over `splits` CTAs per tile, C must then hold the addend).
gosh_status tc_gemm(const __nv_bfloat16 *A, int64_t lda, const __nv_bfloat16 *B, int64_t ldb, float *C, int64_t ldc,
                    int M, int N, int K, int splits, int *err, cudaStream_t s) {
    GOSH_CHECK_ARG(M > 0 && N > 0 && K > 0 && K % 16 == 0, "GEMM needs M, N > 0 and K a positive multiple of 16");
    GOSH_CHECK_ARG(lda % 8 == 0 && ldb % 8 == 0 && ldc % 4 == 0, "row strides must keep 16-byte alignment");
    GOSH_CHECK_ARG(((uintptr_t)A & 15) == 0 && ((uintptr_t)B & 15) == 0 && ((uintptr_t)C & 15) == 0,
                   "GEMM operands must be 16-byte aligned");
    if (splits < 1) splits = 1;
    if (N <= 16) return launch_tc_gemm_nt<16>(A, lda, B, ldb, C, ldc, M, N, K, splits, err, s);
    if (N <= 32) return launch_tc_gemm_nt<32>(A, lda, B, ldb, C, ldc, M, N, K, splits, err, s);
    if (N <= 64) return launch_tc_gemm_nt<64>(A, lda, B, ldb, C, ldc, M, N, K, splits, err, s);
    if (N <= 128) return launch_tc_gemm_nt<128>(A, lda, B, ldb, C, ldc, M, N, K, splits, err, s);
    return launch_tc_gemm_nt<256>(A, lda, B, ldb, C, ldc, M, N, K, splits, err, s);
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
        set_error("tensor-core GEMM: an MMA completion wait timed out");
        return GOSH_ERR_TIMEOUT;
    }
    return GOSH_OK;
}
