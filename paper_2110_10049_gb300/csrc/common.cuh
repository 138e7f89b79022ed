// Shared device/host helpers of libgosh: error reporting, storage-type
// conversion with stochastic rounding, a device Philox4x64-10, and a
// stream-ordered scratch buffer.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <utility>

#include "gosh.h"

namespace gosh {

// ---------------------------------------------------------------------------
// Errors: a thread-local message plus the status code returned through the ABI.
// ---------------------------------------------------------------------------
void set_error(const char *fmt, ...);
void clear_error();

// Process-wide count of kernel launches made by this library (diagnostics).
void note_launch();

#define GOSH_TRY_CUDA(expr)                                                              \
    do {                                                                                 \
        cudaError_t e_ = (expr);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            ::gosh::set_error("%s:%d %s: %s", __FILE__, __LINE__, #expr,                 \
                              cudaGetErrorString(e_));                                   \
            return e_ == cudaErrorMemoryAllocation ? GOSH_ERR_OOM : GOSH_ERR_CUDA;       \
        }                                                                                \
    } while (0)

#define GOSH_TRY(expr)                                                                   \
    do {                                                                                 \
        gosh_status s_ = (expr);                                                         \
        if (s_ != GOSH_OK) return s_;                                                    \
    } while (0)

#define GOSH_CHECK_ARG(cond, ...)                                                        \
    do {                                                                                 \
        if (!(cond)) {                                                                   \
            ::gosh::set_error(__VA_ARGS__);                                              \
            return GOSH_ERR_INVALID_ARG;                                                 \
        }                                                                                \
    } while (0)

// Keeps freed stream-ordered memory cached in the device's default pool
// (release threshold = unlimited) so repeated calls do not re-map physical
// pages for their scratch; done once per device.
void keep_pool_memory();

// Device memory of the library: from the caller's allocator when one is set
// (gosh_set_allocator), else cudaMallocAsync on the stream-ordered pool.
// dev_free returns a block to whichever allocator provided it.
cudaError_t dev_alloc(void **p, size_t bytes, cudaStream_t s);
void dev_free(void *p, cudaStream_t s);

// Stream-ordered device scratch, released on the same stream when it leaves scope.
struct Scratch {
    void *ptr = nullptr;
    cudaStream_t stream = nullptr;
    Scratch() = default;
    Scratch(const Scratch &) = delete;
    Scratch &operator=(const Scratch &) = delete;
    ~Scratch() { release(); }
    gosh_status alloc(size_t bytes, cudaStream_t s) {
        release();
        stream = s;
        if (bytes == 0) bytes = 16;
        cudaError_t e = dev_alloc(&ptr, bytes, s);
        if (e != cudaSuccess) {
            ptr = nullptr;
            set_error("device allocation of %zu bytes: %s", bytes, cudaGetErrorString(e));
            return GOSH_ERR_OOM;
        }
        return GOSH_OK;
    }
    void release() {
        if (ptr) dev_free(ptr, stream);
        ptr = nullptr;
    }
    template <typename T> T *as() const { return static_cast<T *>(ptr); }
};

// Programmatic dependent launch: the next kernel in the stream is scheduled
// while this one drains, and waits at GOSH_DEP_WAIT() for it to finish (its
// writes visible) before touching anything.  Every kernel started through
// launch_dep must begin with GOSH_DEP_WAIT(); for a plain launch it is a no-op.
// The one exception is a training epoch, which may draw its samples first:
// they read only the CSR, which no kernel of a training run writes.
// GOSH_DEP_TRIGGER() (after the wait) lets the next kernel start while this
// one still runs; only training epochs of small levels use it, so at most two
// grids overlap, and the next one's pre-wait part reads nothing the running
// one writes.
#define GOSH_DEP_WAIT() asm volatile("griddepcontrol.wait;" ::: "memory")
#define GOSH_DEP_TRIGGER() asm volatile("griddepcontrol.launch_dependents;" ::: "memory")

template <typename... KArgs, typename... Args>
inline void launch_dep(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
    note_launch();
}

inline int num_sms() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

inline size_t dtype_size(gosh_dtype t) { return t == GOSH_F32 ? 4 : 2; }

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon et al., SC'11): ten rounds of two 64x64->128-bit
// multiplies; the key is bumped by the Weyl constants between rounds.
// ---------------------------------------------------------------------------
struct Philox4 {
    uint64_t w[4];
};

// High 64 bits of a 64 x 64-bit product (device: one instruction; host: the
// compiler's 128-bit integer), so the host threads that draw random walks
// produce the same words as the kernels.
__host__ __device__ __forceinline__ uint64_t mulhi64(uint64_t a, uint64_t b) {
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

__host__ __device__ __forceinline__ Philox4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2,
                                                          uint64_t c3, uint64_t k0, uint64_t k1) {
    const uint64_t kMul0 = 0xD2E7470EE14C6C93ull, kMul1 = 0xCA5A826395121157ull;
    const uint64_t kWeyl0 = 0x9E3779B97F4A7C15ull, kWeyl1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0hi = mulhi64(kMul0, c0), p0lo = kMul0 * c0;
        const uint64_t p1hi = mulhi64(kMul1, c2), p1lo = kMul1 * c2;
        const uint64_t n0 = p1hi ^ c1 ^ k0;
        const uint64_t n2 = p0hi ^ c3 ^ k1;
        c0 = n0;
        c1 = p1lo;
        c2 = n2;
        c3 = p0lo;
        k0 += kWeyl0;
        k1 += kWeyl1;
    }
    Philox4 o;
    o.w[0] = c0;
    o.w[1] = c1;
    o.w[2] = c2;
    o.w[3] = c3;
    return o;
}

// Uniform integer in [0, n): floor(w * n / 2^64).
__host__ __device__ __forceinline__ uint64_t uniform_index(uint64_t w, uint64_t n) { return mulhi64(w, n); }

enum : uint64_t { kTagSample = 0, kTagInit = 1, kTagWalk = 4, kTagWalkNeg = 5 };

// 32-bit integer finaliser "lowbias32" (C. Wellons, hash-prospector, public
// domain): used as a counter-based source of stochastic-rounding bits.
__host__ __device__ __forceinline__ uint32_t mix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// ---------------------------------------------------------------------------
// Storage types: 16-byte vectors of T unpacked to / packed from FP32.
// ---------------------------------------------------------------------------
template <typename T> struct Store;

template <> struct Store<float> {
    static constexpr int kPerVec = 4;
    __device__ __forceinline__ static void unpack(const uint4 &v, float *f) {
        f[0] = __uint_as_float(v.x);
        f[1] = __uint_as_float(v.y);
        f[2] = __uint_as_float(v.z);
        f[3] = __uint_as_float(v.w);
    }
    // Exact store; `f` already holds the stored values.
    __device__ __forceinline__ static uint4 pack(float *f, uint32_t /*rnd_seed*/, uint32_t /*base*/) {
        return make_uint4(__float_as_uint(f[0]), __float_as_uint(f[1]), __float_as_uint(f[2]),
                          __float_as_uint(f[3]));
    }
    __device__ __forceinline__ static float round_nearest(float x) { return x; }
};

// BF16 stochastic rounding: add 16 random bits below the BF16 mantissa of the
// FP32 pattern, then truncate.  Rounds |x| up with probability equal to its
// distance from the lower neighbour (unbiased).  An infinity's low half is
// zero, so the addition cannot carry out of it, and a NaN keeps its exponent
// and a nonzero mantissa: specials pass unchanged without a test; the largest
// finite value may round up to infinity, as rounding away from zero must.
__device__ __forceinline__ uint32_t bf16_sr_bits(float x, uint32_t r16) {
    return (__float_as_uint(x) + (r16 & 0xffffu)) >> 16;
}

// 32 random bits for the pair of values with counter c (seed-relative): an
// odd multiply and an xorshift, both bijections, so every 16-bit half is
// uniform when the seed is (the per-source seed is a full hash).
__device__ __forceinline__ uint32_t sr_pair_bits(uint32_t c) {
    c *= 0x9e3779b1u;
    return c ^ (c >> 15);
}

template <> struct Store<__nv_bfloat16> {
    static constexpr int kPerVec = 8;
    __device__ __forceinline__ static void unpack(const uint4 &v, float *f) {
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            f[2 * i] = __uint_as_float(w[i] << 16);
            f[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
        }
    }
    // Stochastic rounding with bits sr_pair_bits(seed + base + i/2) (two 16-bit
    // halves per word, as bf16_sr_bits); one byte permute keeps the upper
    // halves of both sums.  `f` is overwritten with the stored values.
    __device__ __forceinline__ static uint4 pack(float *f, uint32_t seed, uint32_t base) {
        uint32_t w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint32_t r = sr_pair_bits(seed + base + (uint32_t)i);
            const uint32_t a = __float_as_uint(f[2 * i]) + (r & 0xffffu);
            const uint32_t b = __float_as_uint(f[2 * i + 1]) + (r >> 16);
            w[i] = __byte_perm(a, b, 0x7632);
            f[2 * i] = __uint_as_float(w[i] << 16);
            f[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
        }
        return make_uint4(w[0], w[1], w[2], w[3]);
    }
    __device__ __forceinline__ static float round_nearest(float x) {
        return __bfloat162float(__float2bfloat16_rn(x));
    }
    // Packed differences nw - old of 8 values (nw packed; old exact BF16
    // values as floats, packed losslessly by one byte permute per pair), by a
    // packed BF16 subtraction rounded to nearest: exact when a difference
    // needs at most 8 significant bits, e.g. a few ulps.
    __device__ __forceinline__ static uint4 change(const uint4 &nw, const float *old) {
        const uint32_t n4[4] = {nw.x, nw.y, nw.z, nw.w};
        uint32_t w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint32_t o = __byte_perm(__float_as_uint(old[2 * i]), __float_as_uint(old[2 * i + 1]), 0x7632);
            const __nv_bfloat162 d = __hsub2(*reinterpret_cast<const __nv_bfloat162 *>(&n4[i]),
                                             *reinterpret_cast<const __nv_bfloat162 *>(&o));
            w[i] = *reinterpret_cast<const uint32_t *>(&d);
        }
        return make_uint4(w[0], w[1], w[2], w[3]);
    }
    // The same difference with `old` still packed (its 8 values are exact
    // BF16): the identical packed subtraction, without unpacking.
    __device__ __forceinline__ static uint4 change_packed(const uint4 &nw, const uint4 &old) {
        const uint32_t n4[4] = {nw.x, nw.y, nw.z, nw.w}, o4[4] = {old.x, old.y, old.z, old.w};
        uint32_t w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const __nv_bfloat162 d = __hsub2(*reinterpret_cast<const __nv_bfloat162 *>(&n4[i]),
                                             *reinterpret_cast<const __nv_bfloat162 *>(&o4[i]));
            w[i] = *reinterpret_cast<const uint32_t *>(&d);
        }
        return make_uint4(w[0], w[1], w[2], w[3]);
    }
    // Atomic addition of 8 packed values at L2 (no flush to zero).
    __device__ __forceinline__ static void red_add(__nv_bfloat16 *p, const uint4 &d) {
        asm volatile("red.global.add.noftz.v4.bf16x2 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(d.x), "r"(d.y),
                     "r"(d.z), "r"(d.w)
                     : "memory");
    }
};

// FP16 stochastic rounding: between the toward-zero neighbour and the next
// value away from zero, pick the upper one with probability proportional to
// the distance (16-bit resolution).
__device__ __forceinline__ uint32_t f16_sr_bits(float x, uint32_t r16) {
    const __half t = __float2half_rz(x);
    const uint16_t tb = __half_as_ushort(t);
    if ((tb & 0x7c00u) == 0x7c00u) return tb;  // inf / nan
    const float lo = __half2float(t);
    const __half u = __ushort_as_half((uint16_t)(tb + 1));
    const float hi = __half2float(u);
    // fast division (within 2 ulps; 0 past the largest finite value, where hi
    // is infinite): the IEEE division's slow path is not worth a 2^-16 decision
    const float frac = __fdividef(fabsf(x) - fabsf(lo), fabsf(hi) - fabsf(lo));
    return ((float)(r16 & 0xffffu) * (1.0f / 65536.0f) < frac) ? (uint32_t)(tb + 1) : (uint32_t)tb;
}

template <> struct Store<__half> {
    static constexpr int kPerVec = 8;
    __device__ __forceinline__ static void unpack(const uint4 &v, float *f) {
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            f[2 * i] = __half2float(__ushort_as_half((uint16_t)(w[i] & 0xffffu)));
            f[2 * i + 1] = __half2float(__ushort_as_half((uint16_t)(w[i] >> 16)));
        }
    }
    __device__ __forceinline__ static uint4 pack(float *f, uint32_t seed, uint32_t base) {
        uint32_t w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint32_t r = sr_pair_bits(seed + base + (uint32_t)i);
            const uint32_t lo = f16_sr_bits(f[2 * i], r & 0xffffu);
            const uint32_t hi = f16_sr_bits(f[2 * i + 1], r >> 16);
            w[i] = lo | (hi << 16);
            f[2 * i] = __half2float(__ushort_as_half((uint16_t)lo));
            f[2 * i + 1] = __half2float(__ushort_as_half((uint16_t)hi));
        }
        return make_uint4(w[0], w[1], w[2], w[3]);
    }
    __device__ __forceinline__ static float round_nearest(float x) {
        return __half2float(__float2half_rn(x));
    }
    // Packed differences nw - old (old exact FP16 values as floats), by a packed
    // FP16 subtraction rounded to nearest.
    __device__ __forceinline__ static uint4 change(const uint4 &nw, const float *old) {
        const uint32_t n4[4] = {nw.x, nw.y, nw.z, nw.w};
        uint32_t w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const __half2 o = __floats2half2_rn(old[2 * i], old[2 * i + 1]);
            const __half2 d = __hsub2(*reinterpret_cast<const __half2 *>(&n4[i]), o);
            w[i] = *reinterpret_cast<const uint32_t *>(&d);
        }
        return make_uint4(w[0], w[1], w[2], w[3]);
    }
    // The same difference with `old` still packed (exact FP16 values).
    __device__ __forceinline__ static uint4 change_packed(const uint4 &nw, const uint4 &old) {
        const uint32_t n4[4] = {nw.x, nw.y, nw.z, nw.w}, o4[4] = {old.x, old.y, old.z, old.w};
        uint32_t w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const __half2 d = __hsub2(*reinterpret_cast<const __half2 *>(&n4[i]),
                                      *reinterpret_cast<const __half2 *>(&o4[i]));
            w[i] = *reinterpret_cast<const uint32_t *>(&d);
        }
        return make_uint4(w[0], w[1], w[2], w[3]);
    }
    __device__ __forceinline__ static void red_add(__half *p, const uint4 &d) {
        asm volatile("red.global.add.noftz.v4.f16x2 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(d.x), "r"(d.y),
                     "r"(d.z), "r"(d.w)
                     : "memory");
    }
};

// Device word raised by bounded waits that gave up (capi.cu); read by gosh_device_check.
int *device_error_word();
// The same for gosh_train_level_noalloc's static word (noalloc.cu): *raised = 1
// if it was set since the last read (then cleared).
gosh_status noalloc_take_error(int *raised);

// The parameter checks every training entry point makes: dtype, d in
// {16, 32, 64, 128}, 0 <= k <= 15, a positive finite lr, lr_floor in [0, 1],
// mode, epochs >= 0, p in [0, 1], shrink in (0, 1].
gosh_status check_params(const gosh_params *p);

// Per-level epoch counts of Alg. 2 (Sec. 3 split; with unit 1 the total first
// converted from Sec. 6's |E|-draw epochs to passes); the body of gosh_level_epochs.
gosh_status level_epochs(int e, double p, int D, int unit, const int64_t *n, const int64_t *nnz, int *out);

// Content check of a HOST CSR, the host counterpart of gosh_validate_csr:
// rowptr starts at 0 and never decreases, every column lies in [0, n), rows
// are strictly ascending and hold no self-loop, and (if `symmetric`) every
// (v, u) has its (u, v).  Sets the error line and returns
// GOSH_ERR_INVALID_ARG naming the first bad row.
gosh_status check_host_csr(const int64_t *rowptr, const int32_t *col, int64_t n, bool symmetric);

// Free the idle pinned regions kept across calls by LargeGraphGPU (edge
// blocks) and walk training (pair tables); each returns the bytes freed.
size_t large_release_pinned();
size_t walks_release_pinned();

// ---------------------------------------------------------------------------
// Device primitives (primitives.cu).
// ---------------------------------------------------------------------------
// Exclusive prefix sum of n values; `total` (device, nullable) receives the sum.
gosh_status scan_exclusive_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *total,
                               cudaStream_t s);
gosh_status scan_exclusive_u8_to_i64(const uint8_t *in, int64_t *out, int64_t n,
                                     int64_t *total, cudaStream_t s);
gosh_status scan_exclusive_i32_to_i64(const int32_t *in, int64_t *out, int64_t n,
                                      int64_t *total, cudaStream_t s);

// Stable LSD radix sort on the bit ranges [lo_bits[i], hi_bits[i]) of the key.
// keys/vals are sorted in place (vals may be null); scratch is taken internally.
gosh_status radix_sort_u32(uint32_t *keys, uint32_t *vals, int64_t n, int begin_bit, int end_bit,
                           cudaStream_t s);
// The same into caller-provided alternate buffers, without the copy back:
// *in_alt tells where the sorted data ended.
gosh_status radix_sort_u32_pp(uint32_t *keys, uint32_t *vals, uint32_t *kalt, uint32_t *valt, int64_t n, int begin_bit,
                              int end_bit, cudaStream_t s, bool *in_alt);
gosh_status radix_sort_u64(uint64_t *keys, uint32_t *vals, int64_t n, const int *digit_bits,
                           int ndigits, cudaStream_t s);

}  // namespace gosh
