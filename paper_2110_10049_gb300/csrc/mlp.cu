// Learned coarse-to-fine projection: a residual two-layer MLP trained on the
// (coarse embedding, degree, neighbour mean) -> fine embedding pairs that the
// multi-level method itself produces, replacing the copy of EXPANDEMBEDDING
// (Alg. 2) between levels.
//
//   f(v) = [ Mc[map v] | log(1 + deg v) | mean_{w in Gamma(v)} Mc[map w] | 0 pad ]   (kp = round16(2d+1))
//   Z1 = f W1^T + b1,  H = relu(Z1),  Y = H W2^T + b2,  Mf[v] = Mc[map v] + Y
//
// All contractions of a training step (Z1, Y, dW2 = dY^T H, dH = dY W2,
// dW1 = dZ1^T f) and of the projection run on the TMA-fed tcgen05 GEMM with
// BF16 operands and FP32 accumulation; bias + ReLU is fused into the first
// layer's epilogue and the residual update of the fine table into the second
// layer's; masters and Adam moments are FP32.  W2 = b2 = 0 at creation,
// so an untrained network is exactly the copy projection.
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "common.cuh"

namespace gosh {
gosh_status tc_gemm(const __nv_bfloat16 *A, int64_t lda, const __nv_bfloat16 *B, int64_t ldb, float *C, int64_t ldc,
                    int M, int N, int K, int splits, int *err, cudaStream_t s);
gosh_status tc_gemm_bias_relu(const __nv_bfloat16 *A, int64_t lda, const __nv_bfloat16 *B, int64_t ldb,
                              const float *bias, __nv_bfloat16 *H, int64_t ldh, int M, int N, int K, int *err,
                              cudaStream_t s);
gosh_status tc_gemm_residual(const __nv_bfloat16 *A, int64_t lda, const __nv_bfloat16 *B, int64_t ldb,
                             const float *bias, const int32_t *map, const void *Mc, void *Mf, int64_t v0, int d,
                             gosh_dtype dt, int M, int K, int *err, cudaStream_t s);
bool tc_mlp_fused_ok(int d, int hid, int kp);
gosh_status tc_mlp_project(const __nv_bfloat16 *X, const __nv_bfloat16 *W1b, const __nv_bfloat16 *W2b,
                           const float *b1, const float *b2, const int32_t *map, const void *Mc, void *Mf, int64_t v0,
                           int d, int hid, int kp, gosh_dtype dt, int M, int *err, cudaStream_t s);
}

struct gosh_mlp {
    int d = 0, din = 0, kp = 0, hid = 0;
    float *W1 = nullptr, *b1 = nullptr, *W2 = nullptr, *b2 = nullptr;
    float *mo[4] = {nullptr, nullptr, nullptr, nullptr}, *ve[4] = {nullptr, nullptr, nullptr, nullptr};
    __nv_bfloat16 *W1b = nullptr, *W2b = nullptr, *W2tb = nullptr;
    int *err = nullptr;
    int64_t t = 0;
    // Feature rows kept by a projection for the next training on the same
    // level (gosh_embed only): rows v = j * stride of the graph with row
    // pointer `key_rowptr`, features from the table `key_Mc` through `key_map`.
    __nv_bfloat16 *Xc = nullptr;
    int64_t Xc_cap = 0;
    const void *key_Mc = nullptr;
    const int64_t *key_rowptr = nullptr;
    const int32_t *key_map = nullptr;
    int64_t key_n = 0, key_stride = 0;
    ~gosh_mlp() {
        void *ps[] = {W1, b1, W2, b2, mo[0], mo[1], mo[2], mo[3], ve[0], ve[1], ve[2], ve[3], W1b, W2b, W2tb, err, Xc};
        for (void *p : ps)
            if (p) cudaFree(p);
    }
};

namespace gosh {
namespace {

constexpr uint64_t kTagMlp = 2;
constexpr int kRowsPerChunk = 1 << 18;

inline int round16(int x) { return (x + 15) / 16 * 16; }

int grid_for(int64_t work) {
    const int64_t cap = (int64_t)num_sms() * 16;
    const int64_t g = ceil_div(work > 0 ? work : 1, 256);
    return (int)(g < cap ? g : cap);
}

__global__ void mlp_init_kernel(float *W1, int hid, int din, int kp, uint64_t seed, float a) {
    GOSH_DEP_WAIT();
    const int64_t total = (int64_t)hid * kp;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t h = i / kp;
        const int k = (int)(i % kp);
        float x = 0.0f;
        if (k < din) {
            const Philox4 w = philox4x64_10((uint64_t)h, (uint64_t)(k / 4), 0, kTagMlp, seed, 0);
            const double unit = (double)(w.w[k % 4] >> 11) * 0x1.0p-53;
            x = (float)((2.0 * unit - 1.0) * a);
        }
        W1[i] = x;
    }
}

// BF16 working copies: W1b (hid x kp), W2b (d x hid), W2tb (hid x d).
__global__ void refresh_bf16(const float *W1, const float *W2, __nv_bfloat16 *W1b, __nv_bfloat16 *W2b,
                             __nv_bfloat16 *W2tb, int hid, int kp, int d) {
    GOSH_DEP_WAIT();
    const int64_t n1 = (int64_t)hid * kp, n2 = (int64_t)d * hid;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n1 + n2; i += (int64_t)gridDim.x * blockDim.x) {
        if (i < n1) {
            W1b[i] = __float2bfloat16_rn(W1[i]);
        } else {
            const int64_t j = i - n1;  // W2 index: row o (0..d), col h
            const int o = (int)(j / hid), h = (int)(j % hid);
            const __nv_bfloat16 b = __float2bfloat16_rn(W2[j]);
            W2b[j] = b;
            W2tb[(int64_t)h * d + o] = b;
        }
    }
}

// f(v) for the selected fine vertices v_r = v0 + r * stride, r < rows.
//
// The neighbour mean is an entry-balanced gather: the selected rows' CSR
// entries are laid end to end (voff = prefix sum of their degrees) and cut
// into spans of kFeatSpan entries, one warp per span, so a hub's row is
// spread over many warps instead of holding one.  A warp walks the row
// segments of its span; rows read as 16-byte vectors (V = d * sizeof(T) / 16
// per row, 32 / V neighbours per step, four steps in flight), FP32 sums,
// lanes holding the same vector added in a fixed order.  A row inside one
// span is written at once; a row crossing spans leaves its partial sums in
// the span's slots (0: the span's first row, 1: its last row) and
// feat_fixup adds them in span order.  Deterministic throughout.
constexpr int kFeatSpan = 1024;

__global__ void feat_degrees(const int64_t *__restrict__ rowptr, int64_t v0, int64_t rows, int64_t stride,
                             int64_t *__restrict__ deg) {
    GOSH_DEP_WAIT();
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = v0 + r * stride;
        deg[r] = rowptr[v + 1] - rowptr[v];
    }
}

// Own row, log-degree and padding of every selected row; the mean part is
// zero for a row without neighbours (the spans never visit it).
template <typename T>
__global__ void __launch_bounds__(256) feat_own(const int32_t *__restrict__ map, const T *__restrict__ Mc,
                                                const int64_t *__restrict__ voff, int d, int kp, int64_t v0,
                                                int64_t rows, int64_t stride, __nv_bfloat16 *__restrict__ X) {
    GOSH_DEP_WAIT();
    constexpr int PV = Store<T>::kPerVec;
    const int lane = threadIdx.x & 31;
    const int V = d / PV;
    const uint4 *M4 = reinterpret_cast<const uint4 *>(Mc);
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = wid; r < rows; r += nw) {
        const int64_t v = v0 + r * stride;
        const int64_t deg = voff[r + 1] - voff[r];
        __nv_bfloat16 *x = X + r * kp;
        if (lane < V) {
            float own[PV];
            Store<T>::unpack(__ldg(M4 + (int64_t)__ldg(map + v) * V + lane), own);
#pragma unroll
            for (int i = 0; i < PV; ++i) {
                x[lane * PV + i] = __float2bfloat16_rn(own[i]);
                if (deg == 0) x[d + 1 + lane * PV + i] = __float2bfloat16_rn(0.0f);
            }
        }
        if (lane == 0) x[d] = __float2bfloat16_rn(log1pf((float)deg));
        for (int c = 2 * d + 1 + lane; c < kp; c += 32) x[c] = __float2bfloat16_rn(0.0f);
    }
}

template <typename T>
__global__ void __launch_bounds__(256) feat_spans(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                                                  const int32_t *__restrict__ map, const T *__restrict__ Mc,
                                                  const int64_t *__restrict__ voff, int d, int kp, int64_t v0,
                                                  int64_t rows, int64_t stride, __nv_bfloat16 *__restrict__ X,
                                                  float *__restrict__ slots) {
    GOSH_DEP_WAIT();
    constexpr int PV = Store<T>::kPerVec;
    const int lane = threadIdx.x & 31;
    const int V = d / PV;
    const int R = 32 / V;
    const int sub = lane / V, vec = lane % V;
    const uint4 *M4 = reinterpret_cast<const uint4 *>(Mc);
    const int64_t total = voff[rows];
    const int64_t nspans = (total + kFeatSpan - 1) / kFeatSpan;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t sp = wid; sp < nspans; sp += nw) {
        const int64_t lo = sp * kFeatSpan, hi = lo + kFeatSpan < total ? lo + kFeatSpan : total;
        int64_t a = 0, b = rows;  // last row with voff[row] <= lo
        while (b - a > 1) {
            const int64_t mid = (a + b) >> 1;
            if (__ldg(voff + mid) <= lo) a = mid; else b = mid;
        }
        const int64_t first = a;
        for (int64_t r = first; r < rows && __ldg(voff + r) < hi; ++r) {
            const int64_t rb = __ldg(voff + r), re = __ldg(voff + r + 1);
            if (re == rb) continue;
            const int64_t sb = rb > lo ? rb : lo, se = re < hi ? re : hi;
            const int64_t cbase = __ldg(rowptr + v0 + r * stride) - rb;  // CSR index of virtual entry p: cbase + p
            float acc[PV];
#pragma unroll
            for (int i = 0; i < PV; ++i) acc[i] = 0.0f;
            for (int64_t p0 = sb; p0 < se; p0 += 32) {
                const int cnt = (int)(se - p0 < 32 ? se - p0 : 32);
                const int32_t cid = lane < cnt ? __ldg(map + __ldg(col + cbase + p0 + lane)) : 0;
                for (int q0 = 0; q0 < cnt; q0 += 4 * R) {
                    uint4 w[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int q = q0 + u * R + sub;
                        const int32_t c = __shfl_sync(0xffffffffu, cid, q & 31);
                        w[u] = q < cnt ? __ldg(M4 + (int64_t)c * V + vec) : make_uint4(0, 0, 0, 0);
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        float f[PV];
                        Store<T>::unpack(w[u], f);
#pragma unroll
                        for (int i = 0; i < PV; ++i) acc[i] += f[i];
                    }
                }
            }
            for (int o = V; o < 32; o <<= 1)
#pragma unroll
                for (int i = 0; i < PV; ++i) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], o);
            if (lane < V) {
                if (rb >= lo && re <= hi) {
                    const float inv = 1.0f / (float)(re - rb);
                    __nv_bfloat16 *x = X + r * kp + d + 1 + vec * PV;
#pragma unroll
                    for (int i = 0; i < PV; ++i) x[i] = __float2bfloat16_rn(acc[i] * inv);
                } else {
                    float *sl = slots + (sp * 2 + (r == first ? 0 : 1)) * d + vec * PV;
#pragma unroll
                    for (int i = 0; i < PV; ++i) sl[i] = acc[i];
                }
            }
        }
    }
}

// Rows whose entries cross span boundaries: add the span partials in order.
__global__ void __launch_bounds__(256) feat_fixup(const int64_t *__restrict__ voff, int d, int kp, int64_t rows,
                                                  const float *__restrict__ slots, __nv_bfloat16 *__restrict__ X) {
    GOSH_DEP_WAIT();
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = wid; r < rows; r += nw) {
        const int64_t rb = voff[r], re = voff[r + 1];
        if (re == rb) continue;
        const int64_t s0 = rb / kFeatSpan, s1 = (re - 1) / kFeatSpan;
        if (s0 == s1) continue;
        const float inv = 1.0f / (float)(re - rb);
        for (int c = lane; c < d; c += 32) {
            float t = 0.0f;
            for (int64_t sp = s0; sp <= s1; ++sp) {
                const int slot = (sp == s0 && rb != sp * kFeatSpan) ? 1 : 0;
                t += slots[(sp * 2 + slot) * d + c];
            }
            X[r * kp + d + 1 + c] = __float2bfloat16_rn(t * inv);
        }
    }
}

// R[r][c] = Mf[v][c] - Mc[map v][c], v = v0 + r.
template <typename T>
__global__ void residual_kernel(const int32_t *__restrict__ map, const T *__restrict__ Mc, const T *__restrict__ Mf,
                                int d, int64_t v0, int64_t rows, int64_t stride, float *__restrict__ R) {
    GOSH_DEP_WAIT();
    const int64_t total = rows * d;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / d;
        const int c = (int)(i % d);
        const int64_t v = v0 + r * stride;
        R[i] = (float)Mf[v * d + c] - (float)Mc[(int64_t)map[v] * d + c];
    }
}

// Y = Yacc + b2; diff = Y - R; G = 2 diff / B (FP32 and BF16); per-block loss sums.
__global__ void out_grad_kernel(const float *__restrict__ Yacc, const float *__restrict__ b2,
                                const float *__restrict__ R, int64_t rows, int d, float scale,
                                float *__restrict__ G, __nv_bfloat16 *__restrict__ Gb, double *__restrict__ parts) {
    GOSH_DEP_WAIT();
    __shared__ double s[256];
    double acc = 0.0;
    const int64_t total = rows * d;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const float diff = Yacc[i] + b2[i % d] - R[i];
        acc += (double)diff * (double)diff;
        const float g = scale * diff;
        G[i] = g;
        Gb[i] = __float2bfloat16_rn(g);
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) parts[blockIdx.x] = s[0];
}

// dZ1 = dH * (H > 0): FP32 (for the bias gradient) and BF16 (for dW1).
__global__ void relu_grad_kernel(const float *__restrict__ dH, const __nv_bfloat16 *__restrict__ H, int64_t total,
                                 float *__restrict__ dZ, __nv_bfloat16 *__restrict__ dZb) {
    GOSH_DEP_WAIT();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const float g = __bfloat162float(H[i]) > 0.0f ? dH[i] : 0.0f;
        dZ[i] = g;
        dZb[i] = __float2bfloat16_rn(g);
    }
}

// Column sums out[c] = sum over rows of G[r][c] in two fixed-order passes:
// block (x, y) of 32 x 32 threads sums rows y*kColRows .. of 32 columns
// (thread row ty takes rows ty, ty + 32, ...; then the 32 partials in order)
// into part[y][c]; colsum_finish adds the row blocks' partials in order.
constexpr int kColRows = 512;

__global__ void __launch_bounds__(1024) colsum_kernel(const float *__restrict__ G, int64_t rows, int cols,
                                                      float *__restrict__ part) {
    GOSH_DEP_WAIT();
    __shared__ float p[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + tx;
    const int64_t r0 = (int64_t)blockIdx.y * kColRows, r1 = r0 + kColRows < rows ? r0 + kColRows : rows;
    float s = 0.0f;
    if (c < cols)
        for (int64_t r = r0 + ty; r < r1; r += 32) s += G[r * cols + c];
    p[ty][tx] = s;
    __syncthreads();
    if (ty == 0 && c < cols) {
        float t = 0.0f;
        for (int i = 0; i < 32; ++i) t += p[i][tx];
        part[(int64_t)blockIdx.y * cols + c] = t;
    }
}

__global__ void colsum_finish(const float *__restrict__ part, int nparts, int cols, float *__restrict__ out) {
    GOSH_DEP_WAIT();
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cols; c += gridDim.x * blockDim.x) {
        float t = 0.0f;
        for (int i = 0; i < nparts; ++i) t += part[(int64_t)i * cols + c];
        out[c] = t;
    }
}

// out (cols x ldo) = in^T for in (rows x cols); columns rows..ldo-1 of out are zero.
__global__ void transpose_bf16(const __nv_bfloat16 *__restrict__ in, int64_t rows, int cols, int64_t ldo,
                               __nv_bfloat16 *__restrict__ out) {
    GOSH_DEP_WAIT();
    __shared__ __nv_bfloat16 tile[32][33];
    const int64_t r0 = (int64_t)blockIdx.x * 32;
    const int c0 = blockIdx.y * 32;
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int64_t r = r0 + j;
        const int c = c0 + threadIdx.x;
        tile[j][threadIdx.x] = (r < rows && c < cols) ? in[r * cols + c] : __float2bfloat16_rn(0.0f);
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int c = c0 + j;
        const int64_t r = r0 + threadIdx.x;
        if (c < cols && r < ldo) out[(int64_t)c * ldo + r] = tile[threadIdx.x][j];
    }
}

__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, int64_t n, float lr, float c1, float c2) {
    GOSH_DEP_WAIT();
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// Copies the chunk rows v = j * stride (v in [v0, v0 + rows)) of X into row j
// of Xc (16-byte vectors; kp * 2 bytes is a multiple of 16).
__global__ void keep_rows(const __nv_bfloat16 *__restrict__ X, int kp, int64_t v0, int64_t rows, int64_t stride,
                          __nv_bfloat16 *__restrict__ Xc) {
    GOSH_DEP_WAIT();
    const int vpr = kp * 2 / 16;
    const int64_t j0 = (v0 + stride - 1) / stride, j1 = (v0 + rows + stride - 1) / stride;
    const int64_t total = (j1 - j0) * vpr;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = j0 + i / vpr;
        const int q = (int)(i % vpr);
        reinterpret_cast<uint4 *>(Xc + j * kp)[q] = reinterpret_cast<const uint4 *>(X + (j * stride - v0) * kp)[q];
    }
}

template <typename T> struct TypeOf;

template <typename F>
gosh_status by_dtype(gosh_dtype t, F &&f) {
    switch (t) {
    case GOSH_F32: f((float *)nullptr); return GOSH_OK;
    case GOSH_BF16: f((__nv_bfloat16 *)nullptr); return GOSH_OK;
    case GOSH_F16: f((__half *)nullptr); return GOSH_OK;
    }
    set_error("unknown dtype");
    return GOSH_ERR_INVALID_ARG;
}

// GEMM over N in chunks of 256 columns.
gosh_status gemm(const __nv_bfloat16 *A, int64_t lda, const __nv_bfloat16 *B, int64_t ldb, float *C, int64_t ldc, int M,
                 int N, int K, int splits, int *err, cudaStream_t s) {
    for (int n0 = 0; n0 < N; n0 += 256) {
        const int nn = N - n0 < 256 ? N - n0 : 256;
        GOSH_TRY(tc_gemm(A, lda, B + (int64_t)n0 * ldb, ldb, C + n0, ldc, M, nn, K, splits, err, s));
    }
    return GOSH_OK;
}

// H = relu(A . B^T + bias) in BF16, over N in chunks of 256 columns.
gosh_status gemm_bias_relu(const __nv_bfloat16 *A, int64_t lda, const __nv_bfloat16 *B, int64_t ldb, const float *bias,
                           __nv_bfloat16 *H, int64_t ldh, int M, int N, int K, int *err, cudaStream_t s) {
    for (int n0 = 0; n0 < N; n0 += 256) {
        const int nn = N - n0 < 256 ? N - n0 : 256;
        GOSH_TRY(tc_gemm_bias_relu(A, lda, B + (int64_t)n0 * ldb, ldb, bias + n0, H + n0, ldh, M, nn, K, err, s));
    }
    return GOSH_OK;
}

// Workspace of one training batch of up to B rows.
struct Work {
    Scratch H, Y, G, Gb, Gt, Ht, dH, dZ, dZb, dZt, Xt, dW1, db1, dW2, db2, parts, loss, cpart;
    int B = 0;
    gosh_status alloc(const gosh_mlp *m, int B_, cudaStream_t s) {
        B = B_;
        const int64_t Bp = round16(B);
        GOSH_TRY(H.alloc(sizeof(__nv_bfloat16) * B * m->hid, s));
        GOSH_TRY(Y.alloc(sizeof(float) * B * m->d, s));
        GOSH_TRY(G.alloc(sizeof(float) * B * m->d, s));
        GOSH_TRY(Gb.alloc(sizeof(__nv_bfloat16) * B * m->d, s));
        GOSH_TRY(Gt.alloc(sizeof(__nv_bfloat16) * m->d * Bp, s));
        GOSH_TRY(Ht.alloc(sizeof(__nv_bfloat16) * m->hid * Bp, s));
        GOSH_TRY(dH.alloc(sizeof(float) * B * m->hid, s));
        GOSH_TRY(dZ.alloc(sizeof(float) * B * m->hid, s));
        GOSH_TRY(dZb.alloc(sizeof(__nv_bfloat16) * B * m->hid, s));
        GOSH_TRY(dZt.alloc(sizeof(__nv_bfloat16) * m->hid * Bp, s));
        GOSH_TRY(Xt.alloc(sizeof(__nv_bfloat16) * m->kp * Bp, s));
        GOSH_TRY(dW1.alloc(sizeof(float) * m->hid * m->kp, s));
        GOSH_TRY(db1.alloc(sizeof(float) * m->hid, s));
        GOSH_TRY(dW2.alloc(sizeof(float) * m->d * m->hid, s));
        GOSH_TRY(db2.alloc(sizeof(float) * m->d, s));
        GOSH_TRY(parts.alloc(sizeof(double) * num_sms() * 16, s));
        GOSH_TRY(loss.alloc(sizeof(double), s));
        GOSH_TRY(cpart.alloc(sizeof(float) * ceil_div(B, kColRows) * std::max(m->d, m->hid), s));
        return GOSH_OK;
    }
};

void colsum(const float *G, int64_t rows, int cols, float *part, float *out, cudaStream_t s) {
    const int nparts = (int)ceil_div(rows, kColRows);
    dim3 grid((unsigned)ceil_div(cols, 32), (unsigned)nparts);
    launch_dep(colsum_kernel, grid, 1024, 0, s, G, rows, cols, part);
    launch_dep(colsum_finish, (int)ceil_div(cols, 256), 256, 0, s, part, nparts, cols, out);
}

void transpose(const __nv_bfloat16 *in, int64_t rows, int cols, int64_t ldo, __nv_bfloat16 *out, cudaStream_t s) {
    dim3 grid((unsigned)ceil_div(ldo, 32), (unsigned)ceil_div(cols, 32));
    launch_dep(transpose_bf16, grid, dim3(32, 8), 0, s, in, rows, cols, ldo, out);
}

__global__ void sum_parts_kernel(const double *__restrict__ parts, int n, double *__restrict__ out, int accumulate) {
    GOSH_DEP_WAIT();
    __shared__ double s[256];
    double t = 0.0;
    for (int i = threadIdx.x; i < n; i += 256) t += parts[i];
    s[threadIdx.x] = t;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = accumulate ? *out + s[0] : s[0];
}

// Forward + backward of one batch (X: rows x kp BF16, R: rows x d FP32).
// Gradients land in w.dW1/db1/dW2/db2; the batch's summed squared error is
// added to *loss_acc (device) when loss_acc is not null.
gosh_status batch_grads(gosh_mlp *m, const __nv_bfloat16 *X, const float *R, int rows, Work &w, double *loss_acc,
                        int accumulate_loss, cudaStream_t s) {
    const int hid = m->hid, d = m->d, kp = m->kp;
    const int Kb = round16(rows);
    const int splits = (int)std::max<int64_t>(1, std::min<int64_t>(32, Kb / 256));
    const int g = grid_for((int64_t)rows * hid);
    // forward (bias and ReLU fused into the first GEMM's epilogue)
    GOSH_TRY(gemm_bias_relu(X, kp, m->W1b, kp, m->b1, w.H.as<__nv_bfloat16>(), hid, rows, hid, kp, m->err, s));
    GOSH_TRY(gemm(w.H.as<__nv_bfloat16>(), hid, m->W2b, hid, w.Y.as<float>(), d, rows, d, hid, 1, m->err, s));
    const int go = grid_for((int64_t)rows * d);
    launch_dep(out_grad_kernel, go, 256, 0, s, w.Y.as<float>(), m->b2, R, rows, d, 2.0f / (float)rows, w.G.as<float>(),
                                        w.Gb.as<__nv_bfloat16>(), w.parts.as<double>());
    if (loss_acc) launch_dep(sum_parts_kernel, 1, 256, 0, s, w.parts.as<double>(), go, loss_acc, accumulate_loss);
    // backward
    transpose(w.Gb.as<__nv_bfloat16>(), rows, d, Kb, w.Gt.as<__nv_bfloat16>(), s);
    transpose(w.H.as<__nv_bfloat16>(), rows, hid, Kb, w.Ht.as<__nv_bfloat16>(), s);
    GOSH_TRY_CUDA(cudaMemsetAsync(w.dW2.ptr, 0, sizeof(float) * d * hid, s));
    GOSH_TRY(gemm(w.Gt.as<__nv_bfloat16>(), Kb, w.Ht.as<__nv_bfloat16>(), Kb, w.dW2.as<float>(), hid, d, hid, Kb,
                  splits, m->err, s));
    colsum(w.G.as<float>(), rows, d, w.cpart.as<float>(), w.db2.as<float>(), s);
    GOSH_TRY(gemm(w.Gb.as<__nv_bfloat16>(), d, m->W2tb, d, w.dH.as<float>(), hid, rows, hid, d, 1, m->err, s));
    launch_dep(relu_grad_kernel, g, 256, 0, s, w.dH.as<float>(), w.H.as<__nv_bfloat16>(), (int64_t)rows * hid,
                                        w.dZ.as<float>(), w.dZb.as<__nv_bfloat16>());
    colsum(w.dZ.as<float>(), rows, hid, w.cpart.as<float>(), w.db1.as<float>(), s);
    transpose(w.dZb.as<__nv_bfloat16>(), rows, hid, Kb, w.dZt.as<__nv_bfloat16>(), s);
    transpose(X, rows, kp, Kb, w.Xt.as<__nv_bfloat16>(), s);
    GOSH_TRY_CUDA(cudaMemsetAsync(w.dW1.ptr, 0, sizeof(float) * hid * kp, s));
    GOSH_TRY(gemm(w.dZt.as<__nv_bfloat16>(), Kb, w.Xt.as<__nv_bfloat16>(), Kb, w.dW1.as<float>(), kp, hid, kp, Kb,
                  splits, m->err, s));
    return GOSH_OK;
}

void adam_all(gosh_mlp *m, Work &w, float lr, cudaStream_t s) {
    m->t += 1;
    const float c1 = 1.0f - std::pow(0.9f, (float)m->t), c2 = 1.0f - std::pow(0.999f, (float)m->t);
    float *P[4] = {m->W1, m->b1, m->W2, m->b2};
    float *Gs[4] = {w.dW1.as<float>(), w.db1.as<float>(), w.dW2.as<float>(), w.db2.as<float>()};
    const int64_t N[4] = {(int64_t)m->hid * m->kp, m->hid, (int64_t)m->d * m->hid, m->d};
    for (int i = 0; i < 4; ++i)
        launch_dep(adam_kernel, grid_for(N[i]), 256, 0, s, P[i], Gs[i], m->mo[i], m->ve[i], N[i], lr, c1, c2);
    (refresh_bf16<<<grid_for((int64_t)m->hid * m->kp + (int64_t)m->d * m->hid), 256, 0, s>>>(
         m->W1, m->W2, m->W1b, m->W2b, m->W2tb, m->hid, m->kp, m->d),
     note_launch());
}

gosh_status check_err(gosh_mlp *m, cudaStream_t s) {
    int herr = 0;
    GOSH_TRY_CUDA(cudaMemcpyAsync(&herr, m->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    GOSH_TRY_CUDA(cudaStreamSynchronize(s));
    if (herr) {
        set_error("tensor-core GEMM: an MMA completion wait timed out");
        return GOSH_ERR_TIMEOUT;
    }
    return GOSH_OK;
}

gosh_status features(const gosh_csr *g, const int32_t *map, const void *Mc, int d, gosh_dtype dt, int kp, int64_t v0,
                     int64_t rows, __nv_bfloat16 *X, cudaStream_t s, int64_t stride = 1) {
    if (rows <= 0) return GOSH_OK;
    Scratch deg, voff;
    GOSH_TRY(deg.alloc(sizeof(int64_t) * rows, s));
    GOSH_TRY(voff.alloc(sizeof(int64_t) * (rows + 1), s));
    launch_dep(feat_degrees, grid_for(rows), 256, 0, s, g->rowptr, v0, rows, stride, deg.as<int64_t>());
    GOSH_TRY(scan_exclusive_i64(deg.as<int64_t>(), voff.as<int64_t>(), rows, voff.as<int64_t>() + rows, s));
    int64_t total = 0;
    GOSH_TRY_CUDA(cudaMemcpyAsync(&total, voff.as<int64_t>() + rows, sizeof(total), cudaMemcpyDeviceToHost, s));
    GOSH_TRY_CUDA(cudaStreamSynchronize(s));
    const int64_t nspans = ceil_div(total, kFeatSpan);
    Scratch slots;
    GOSH_TRY(slots.alloc(sizeof(float) * 2 * d * (nspans > 0 ? nspans : 1), s));
    const int64_t cap = (int64_t)num_sms() * 8;
    const int own_blocks = (int)std::min<int64_t>(ceil_div(rows * 32, 256), cap);
    const int span_blocks = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(nspans * 32, 256), cap));
    return by_dtype(dt, [&](auto *tp) {
        using T = std::remove_pointer_t<decltype(tp)>;
        const T *M = static_cast<const T *>(Mc);
        launch_dep(feat_own<T>, own_blocks, 256, 0, s, map, M, voff.as<int64_t>(), d, kp, v0, rows, stride, X);
        if (nspans > 0) {
            launch_dep(feat_spans<T>, span_blocks, 256, 0, s, g->rowptr, g->col, map, M, voff.as<int64_t>(), d, kp, v0, rows,
                                                      stride, X, slots.as<float>());
            launch_dep(feat_fixup, own_blocks, 256, 0, s, voff.as<int64_t>(), d, kp, rows, slots.as<float>(), X);
        }
    });
}

}  // namespace

gosh_status mlp_create(int d, int hidden, uint64_t seed, gosh_mlp **out) {
    gosh_mlp *m = new gosh_mlp();
    m->d = d;
    m->din = 2 * d + 1;
    m->kp = round16(m->din);
    m->hid = hidden;
    const int64_t n1 = (int64_t)hidden * m->kp, n2 = (int64_t)d * hidden;
    const int64_t sizes[4] = {n1, hidden, n2, d};
    bool ok = cudaMalloc(&m->W1, sizeof(float) * n1) == cudaSuccess && cudaMalloc(&m->b1, sizeof(float) * hidden) == cudaSuccess &&
              cudaMalloc(&m->W2, sizeof(float) * n2) == cudaSuccess && cudaMalloc(&m->b2, sizeof(float) * d) == cudaSuccess &&
              cudaMalloc(&m->W1b, sizeof(__nv_bfloat16) * n1) == cudaSuccess &&
              cudaMalloc(&m->W2b, sizeof(__nv_bfloat16) * n2) == cudaSuccess &&
              cudaMalloc(&m->W2tb, sizeof(__nv_bfloat16) * n2) == cudaSuccess && cudaMalloc(&m->err, sizeof(int)) == cudaSuccess;
    for (int i = 0; i < 4 && ok; ++i)
        ok = cudaMalloc(&m->mo[i], sizeof(float) * sizes[i]) == cudaSuccess &&
             cudaMalloc(&m->ve[i], sizeof(float) * sizes[i]) == cudaSuccess;
    if (!ok) {
        delete m;
        set_error("gosh_mlp_create: device allocation failed");
        return GOSH_ERR_OOM;
    }
    const float a = std::sqrt(6.0f / (float)(m->din + hidden));  // Glorot-uniform bound
    (mlp_init_kernel<<<grid_for(n1), 256>>>(m->W1, hidden, m->din, m->kp, seed, a), note_launch());
    cudaMemset(m->b1, 0, sizeof(float) * hidden);
    cudaMemset(m->W2, 0, sizeof(float) * n2);
    cudaMemset(m->b2, 0, sizeof(float) * d);
    cudaMemset(m->err, 0, sizeof(int));
    for (int i = 0; i < 4; ++i) {
        cudaMemset(m->mo[i], 0, sizeof(float) * sizes[i]);
        cudaMemset(m->ve[i], 0, sizeof(float) * sizes[i]);
    }
    (refresh_bf16<<<grid_for(n1 + n2), 256>>>(m->W1, m->W2, m->W1b, m->W2b, m->W2tb, hidden, m->kp, d), note_launch());
    GOSH_TRY_CUDA(cudaDeviceSynchronize());
    *out = m;
    return GOSH_OK;
}

// Trains on (features of g's vertices from Mc, residual Mf - copy) pairs.
// At most max_rows vertices take part (every stride-th vertex of the level).
int64_t train_stride(int64_t nlev, int64_t max_rows) {
    return (max_rows > 0 && nlev > max_rows) ? (nlev + max_rows - 1) / max_rows : 1;
}

// use_kept: take the feature rows a preceding projection kept for this level
// (same graph, map, source table and stride) instead of gathering them again.
gosh_status mlp_train(gosh_mlp *m, const gosh_csr *g, const int32_t *map, const void *Mc, const void *Mf,
                      gosh_dtype dt, int epochs, double lr, int batch, int64_t max_rows, cudaStream_t s,
                      double *final_loss, bool use_kept) {
    const int64_t nlev = g->n;
    const int64_t stride = train_stride(nlev, max_rows);
    const int64_t n = (nlev + stride - 1) / stride;
    const int d = m->d, kp = m->kp;
    if (batch <= 0) batch = 4096;
    batch = round16(batch);
    if (batch > n) batch = (int)round16((int)n);
    Scratch Xs, R, loss;
    GOSH_TRY(R.alloc(sizeof(float) * n * d, s));
    GOSH_TRY(loss.alloc(sizeof(double), s));
    const __nv_bfloat16 *X = nullptr;
    if (use_kept && m->Xc && m->key_Mc == Mc && m->key_rowptr == g->rowptr && m->key_map == map &&
        m->key_n == nlev && m->key_stride == stride) {
        X = m->Xc;
    } else {
        GOSH_TRY(Xs.alloc(sizeof(__nv_bfloat16) * n * kp, s));
        GOSH_TRY(features(g, map, Mc, d, dt, kp, 0, n, Xs.as<__nv_bfloat16>(), s, stride));
        X = Xs.as<__nv_bfloat16>();
    }
    m->key_Mc = nullptr;  // the kept rows serve one training
    GOSH_TRY(by_dtype(dt, [&](auto *tp) {
        using T = std::remove_pointer_t<decltype(tp)>;
        launch_dep(residual_kernel<T>, grid_for(n * d), 256, 0, s, map, static_cast<const T *>(Mc),
                                                            static_cast<const T *>(Mf), d, 0, n, stride,
                                                            R.as<float>());
    }));
    Work w;
    GOSH_TRY(w.alloc(m, batch, s));
    for (int ep = 0; ep < epochs; ++ep) {
        const bool last = ep + 1 == epochs;
        for (int64_t r0 = 0; r0 < n; r0 += batch) {
            const int rows = (int)std::min<int64_t>(batch, n - r0);
            if (rows < 16) continue;  // a sliver batch adds noise, not signal
            GOSH_TRY(batch_grads(m, X + r0 * kp, R.as<float>() + r0 * d, rows, w, last ? loss.as<double>() : nullptr,
                                 r0 > 0, s));
            adam_all(m, w, (float)lr, s);
        }
    }
    GOSH_TRY(check_err(m, s));
    if (final_loss) {
        double hl = 0.0;
        if (epochs > 0) GOSH_TRY_CUDA(cudaMemcpy(&hl, loss.ptr, sizeof(double), cudaMemcpyDeviceToHost));
        *final_loss = hl / (double)n;
    }
    return GOSH_OK;
}

// Mf = copy + MLP(features), in chunks of kRowsPerChunk fine vertices.
// keep_rows_of > 0: keep the feature rows a training with max_rows =
// keep_rows_of will use on this level (gosh_embed only).
gosh_status mlp_project(gosh_mlp *m, const void *Mc, const int32_t *map, const gosh_csr *g, void *Mf, gosh_dtype dt,
                        cudaStream_t s, int64_t keep_rows_of) {
    const int64_t n = g->n;
    const int d = m->d, kp = m->kp, hid = m->hid;
    const int64_t chunk = std::min<int64_t>(n, kRowsPerChunk);
    const int64_t stride = train_stride(n, keep_rows_of);
    const int64_t nkeep = (n + stride - 1) / stride;
    m->key_Mc = nullptr;
    if (keep_rows_of != 0 && nkeep > m->Xc_cap) {
        GOSH_TRY_CUDA(cudaStreamSynchronize(s));
        if (m->Xc) cudaFree(m->Xc);
        m->Xc = nullptr;
        m->Xc_cap = 0;
        GOSH_TRY_CUDA(cudaMalloc(&m->Xc, sizeof(__nv_bfloat16) * nkeep * kp));
        m->Xc_cap = nkeep;
    }
    // both layers in one persistent kernel where the accumulators fit one
    // SM's tensor memory; else two GEMMs with the hidden layer in memory
    const bool fused = tc_mlp_fused_ok(d, hid, kp);
    Scratch X, H;
    GOSH_TRY(X.alloc(sizeof(__nv_bfloat16) * chunk * kp, s));
    if (!fused) GOSH_TRY(H.alloc(sizeof(__nv_bfloat16) * chunk * hid, s));
    for (int64_t v0 = 0; v0 < n; v0 += chunk) {
        const int rows = (int)std::min<int64_t>(chunk, n - v0);
        GOSH_TRY(features(g, map, Mc, d, dt, kp, v0, rows, X.as<__nv_bfloat16>(), s));
        if (keep_rows_of != 0)
            launch_dep(keep_rows, grid_for(ceil_div(rows, stride) * (kp / 8)), 256, 0, s, X.as<__nv_bfloat16>(), kp, v0, rows,
                                                                                  stride, m->Xc);
        if (fused) {
            GOSH_TRY(tc_mlp_project(X.as<__nv_bfloat16>(), m->W1b, m->W2b, m->b1, m->b2, map, Mc, Mf, v0, d, hid, kp, dt,
                                    rows, m->err, s));
            continue;
        }
        GOSH_TRY(gemm_bias_relu(X.as<__nv_bfloat16>(), kp, m->W1b, kp, m->b1, H.as<__nv_bfloat16>(), hid, rows, hid, kp,
                                m->err, s));
        // Mf[v] = Mc[map v] + H W2^T + b2, written by the second GEMM's epilogue
        GOSH_TRY(tc_gemm_residual(H.as<__nv_bfloat16>(), hid, m->W2b, hid, m->b2, map, Mc, Mf, v0, d, dt, rows, hid,
                                  m->err, s));
    }
    if (keep_rows_of != 0) {
        m->key_Mc = Mc;
        m->key_rowptr = g->rowptr;
        m->key_map = map;
        m->key_n = n;
        m->key_stride = stride;
    }
    return check_err(m, s);
}

}  // namespace gosh

using namespace gosh;

extern "C" {

gosh_status gosh_mlp_create(int d, int hidden, uint64_t seed, gosh_mlp **out) {
    clear_error();
    GOSH_CHECK_ARG(out != nullptr, "out is NULL");
    GOSH_CHECK_ARG(d == 32 || d == 64 || d == 128, "d must be 32, 64 or 128");
    GOSH_CHECK_ARG(hidden >= 16 && hidden % 16 == 0 && hidden <= 1024, "hidden must be a multiple of 16 in [16, 1024]");
    return mlp_create(d, hidden, seed, out);
}

void gosh_mlp_free(gosh_mlp *m) { delete m; }

int gosh_mlp_feature_stride(int d) { return round16(2 * d + 1); }

gosh_status gosh_mlp_get_weights(const gosh_mlp *m, float *W1, float *b1, float *W2, float *b2) {
    clear_error();
    GOSH_CHECK_ARG(m != nullptr, "mlp is NULL");
    GOSH_TRY_CUDA(cudaDeviceSynchronize());
    if (W1)
        GOSH_TRY_CUDA(cudaMemcpy2D(W1, sizeof(float) * m->din, m->W1, sizeof(float) * m->kp, sizeof(float) * m->din, m->hid,
                                   cudaMemcpyDeviceToHost));
    if (b1) GOSH_TRY_CUDA(cudaMemcpy(b1, m->b1, sizeof(float) * m->hid, cudaMemcpyDeviceToHost));
    if (W2) GOSH_TRY_CUDA(cudaMemcpy(W2, m->W2, sizeof(float) * m->d * m->hid, cudaMemcpyDeviceToHost));
    if (b2) GOSH_TRY_CUDA(cudaMemcpy(b2, m->b2, sizeof(float) * m->d, cudaMemcpyDeviceToHost));
    return GOSH_OK;
}

gosh_status gosh_mlp_set_weights(gosh_mlp *m, const float *W1, const float *b1, const float *W2, const float *b2) {
    clear_error();
    GOSH_CHECK_ARG(m != nullptr && W1 && b1 && W2 && b2, "NULL argument");
    GOSH_TRY_CUDA(cudaMemset(m->W1, 0, sizeof(float) * m->hid * m->kp));
    GOSH_TRY_CUDA(cudaMemcpy2D(m->W1, sizeof(float) * m->kp, W1, sizeof(float) * m->din, sizeof(float) * m->din, m->hid,
                               cudaMemcpyHostToDevice));
    GOSH_TRY_CUDA(cudaMemcpy(m->b1, b1, sizeof(float) * m->hid, cudaMemcpyHostToDevice));
    GOSH_TRY_CUDA(cudaMemcpy(m->W2, W2, sizeof(float) * m->d * m->hid, cudaMemcpyHostToDevice));
    GOSH_TRY_CUDA(cudaMemcpy(m->b2, b2, sizeof(float) * m->d, cudaMemcpyHostToDevice));
    (refresh_bf16<<<grid_for((int64_t)m->hid * m->kp + (int64_t)m->d * m->hid), 256>>>(m->W1, m->W2, m->W1b, m->W2b,
                                                                                        m->W2tb, m->hid, m->kp, m->d),
     note_launch());
    GOSH_TRY_CUDA(cudaDeviceSynchronize());
    return GOSH_OK;
}

gosh_status gosh_mlp_features(const gosh_csr *g_fine, const int32_t *map, const void *M_coarse, int d, gosh_dtype dtype,
                              void *X, void *stream) {
    clear_error();
    GOSH_CHECK_ARG(g_fine && g_fine->on_device && map && M_coarse && X, "NULL or host argument");
    GOSH_CHECK_ARG(d == 32 || d == 64 || d == 128, "bad d");
    return features(g_fine, map, M_coarse, d, dtype, round16(2 * d + 1), 0, g_fine->n,
                    static_cast<__nv_bfloat16 *>(X), (cudaStream_t)stream);
}

gosh_status gosh_mlp_grads(gosh_mlp *m, const void *X, const float *R, int64_t n, float *dW1, float *db1, float *dW2,
                           float *db2, double *loss, void *stream) {
    clear_error();
    GOSH_CHECK_ARG(m && X && R && n >= 16 && n <= (1 << 20), "bad arguments (n in [16, 2^20])");
    cudaStream_t s = (cudaStream_t)stream;
    Work w;
    GOSH_TRY(w.alloc(m, (int)n, s));
    GOSH_TRY(batch_grads(m, static_cast<const __nv_bfloat16 *>(X), R, (int)n, w, w.loss.as<double>(), 0, s));
    GOSH_TRY(check_err(m, s));
    std::vector<float> tmp((size_t)m->hid * m->kp);
    if (dW1) {
        GOSH_TRY_CUDA(cudaMemcpy(tmp.data(), w.dW1.ptr, sizeof(float) * tmp.size(), cudaMemcpyDeviceToHost));
        for (int h = 0; h < m->hid; ++h)
            for (int k = 0; k < m->din; ++k) dW1[(size_t)h * m->din + k] = tmp[(size_t)h * m->kp + k];
    }
    if (db1) GOSH_TRY_CUDA(cudaMemcpy(db1, w.db1.ptr, sizeof(float) * m->hid, cudaMemcpyDeviceToHost));
    if (dW2) GOSH_TRY_CUDA(cudaMemcpy(dW2, w.dW2.ptr, sizeof(float) * m->d * m->hid, cudaMemcpyDeviceToHost));
    if (db2) GOSH_TRY_CUDA(cudaMemcpy(db2, w.db2.ptr, sizeof(float) * m->d, cudaMemcpyDeviceToHost));
    if (loss) {
        double hl = 0.0;
        GOSH_TRY_CUDA(cudaMemcpy(&hl, w.loss.ptr, sizeof(double), cudaMemcpyDeviceToHost));
        *loss = hl / (double)n;
    }
    return GOSH_OK;
}

gosh_status gosh_mlp_train(gosh_mlp *m, const gosh_csr *g_fine, const int32_t *map, const void *M_coarse,
                           const void *M_fine, int d, gosh_dtype dtype, int epochs, double lr, int batch,
                           int64_t max_rows, void *stream, double *final_loss) {
    clear_error();
    GOSH_CHECK_ARG(m && g_fine && g_fine->on_device && map && M_coarse && M_fine, "NULL or host argument");
    GOSH_CHECK_ARG(d == m->d, "d (%d) differs from the network's (%d)", d, m->d);
    GOSH_CHECK_ARG(epochs >= 0 && lr > 0, "bad epochs / lr");
    return mlp_train(m, g_fine, map, M_coarse, M_fine, dtype, epochs, lr, batch, max_rows, (cudaStream_t)stream,
                     final_loss, false);
}

gosh_status gosh_project_learned(gosh_mlp *m, const void *M_coarse, const int32_t *map, const gosh_csr *g_fine,
                                 void *M_fine, int d, gosh_dtype dtype, void *stream) {
    clear_error();
    GOSH_CHECK_ARG(m && g_fine && g_fine->on_device && map && M_coarse && M_fine, "NULL or host argument");
    GOSH_CHECK_ARG(d == m->d, "d (%d) differs from the network's (%d)", d, m->d);
    return mlp_project(m, M_coarse, map, g_fine, M_fine, dtype, (cudaStream_t)stream, 0);
}

}  // extern "C"
