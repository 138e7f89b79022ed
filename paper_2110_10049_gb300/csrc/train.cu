// Host side of the training step: variant registry, the epoch loop of Alg. 3
// (one launch per epoch, so epochs are serialised as Sec. 3.1 requires) and the
// batch loop of the deterministic mode.
#include <algorithm>
#include <mutex>
#include <vector>

#include "train.cuh"

namespace gosh {
namespace {

struct Registry {
    std::vector<TrainEntry> entries;
    std::vector<TrainKernel> made;
    std::vector<bool> ready;
    std::mutex mu;
    Registry() {
        int c = 0;
        const TrainEntry *e = train_entries_f32(&c);
        entries.insert(entries.end(), e, e + c);
        e = train_entries_bf16(&c);
        entries.insert(entries.end(), e, e + c);
        e = train_entries_f16(&c);
        entries.insert(entries.end(), e, e + c);
        e = train_tma_entries_f32(&c);
        entries.insert(entries.end(), e, e + c);
        e = train_tma_entries_bf16(&c);
        entries.insert(entries.end(), e, e + c);
        made.resize(entries.size());
        ready.assign(entries.size(), false);
    }
};

Registry &registry() {
    static Registry r;
    return r;
}

__global__ void loss_finalize(const double *__restrict__ parts, int nparts, double *__restrict__ out,
                              int accumulate) {
    GOSH_DEP_WAIT();
    __shared__ double s[256];
    double t = 0.0;
    for (int i = threadIdx.x; i < nparts; i += 256) t += parts[i];
    s[threadIdx.x] = t;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = accumulate ? *out + s[0] : s[0];
}

__global__ void iota_u32(uint32_t *__restrict__ p, int64_t n) {
    GOSH_DEP_WAIT();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = (uint32_t)i;
}

int bits_for(int64_t x) {  // bits needed to hold values 0..x
    int b = 0;
    while (b < 63 && (int64_t(1) << b) <= x) ++b;
    return b < 1 ? 1 : b;
}

void det_apply(gosh_dtype dtype, int d, const uint32_t *skeys, const uint32_t *sidx, int64_t nslots,
               const float *C, const float *R, void *M, int64_t n, int64_t b0, int64_t b1,
               uint8_t *src_done, uint32_t sr_seed, cudaStream_t s) {
    if (dtype == GOSH_F32) det_apply_f32(d, skeys, sidx, nslots, C, R, M, n, b0, b1, src_done, sr_seed, s);
    else if (dtype == GOSH_BF16) det_apply_bf16(d, skeys, sidx, nslots, C, R, M, n, b0, b1, src_done, sr_seed, s);
    else det_apply_f16(d, skeys, sidx, nslots, C, R, M, n, b0, b1, src_done, sr_seed, s);
}

}  // namespace

const TrainKernel *find_train_kernel(gosh_dtype dtype, int d, int lanes, int pass, int mode) {
    Registry &r = registry();
    std::lock_guard<std::mutex> lock(r.mu);
    for (size_t i = 0; i < r.entries.size(); ++i) {
        const TrainEntry &e = r.entries[i];
        if (e.dtype == dtype && e.d == d && e.lanes == lanes && e.pass == pass && e.mode == mode) {
            if (!r.ready[i]) {
                r.made[i] = e.make();
                r.ready[i] = true;
            }
            return &r.made[i];
        }
    }
    return nullptr;
}

int list_train_variants(gosh_dtype dtype, int d, int mode, int *lanes, int *pass, int cap) {
    Registry &r = registry();
    int c = 0;
    for (const TrainEntry &e : r.entries)
        if (e.dtype == dtype && e.d == d && e.mode == mode && c < cap) {
            lanes[c] = e.lanes;
            pass[c] = e.pass;
            ++c;
        }
    return c;
}

// Natural lanes per row: one 16-byte vector per lane.
int natural_lanes(gosh_dtype dtype, int d) { return d * (int)dtype_size(dtype) / 16; }

// Sources per warp tile.  A warp walks its tile in tile / (32/L) dependent
// rounds, so small levels (few tiles, far fewer than the GPU's warps) take
// short tiles (4 below 2^16 rows; below 2^19, 8 for 16-bit tables with plain
// stores, 16 in the deterministic mode, 32 lock-free with atomic changes);
// from 2^19 rows 16 for the lock-free modes with atomic changes (one more
// wave of tiles than 32 evens out the tail; measured on R-MAT 20 level 0:
// BF16 231 vs 234 us, FP32 362 vs 373 us), else 32 to amortise the draws.
// A multiple of 32/L in [32/L, 32]; params->vertices_per_warp overrides.
int tile_vertices(const gosh_params *p, int64_t n, int lanes, int pass) {
    const int G = 32 / lanes;
    int t = p->vertices_per_warp;
    if (t <= 0 && pass < 0 && n < (int64_t(1) << 14)) {
        // TMA-staged kernel on a small level: about 2048 warps of single
        // rounds (G sources each), fewer rounds per warp than a fixed tile
        t = (int)(ceil_div(n, (int64_t)G * 2048) * G);
    }
    const bool red16 = p->dtype != GOSH_F32 && p->mode != GOSH_DETERMINISTIC && !p->plain_stores;
    const bool f32_lockfree = p->dtype == GOSH_F32 && p->mode != GOSH_DETERMINISTIC;
    const bool atomic_lockfree = (red16 || f32_lockfree) && !p->plain_stores;
    const int mid = atomic_lockfree ? 32 : (p->dtype != GOSH_F32 && p->mode != GOSH_DETERMINISTIC ? 8 : 16);
    // 16-bit atomic levels: 28 from 2^19 rows, 32 from 2^21 (per-epoch BF16
    // sweep of tiles 12-32, two repeats: R-MAT 20 level 0, 614 k rows, 204.3
    // us at 28 against 207.5 at 16 and 32; R-MAT 22 level 0, 2.27 M rows,
    // 880 us at 32 against 885 at 28 and 911 at 16)
    const int large =
        atomic_lockfree ? (red16 ? (n >= (int64_t(1) << 21) ? 32 : 28) : 16) : 32;
    // atomic lock-free levels of 2^14 to 2^16 rows: 8 (level 2 of R-MAT 20,
    // 22k rows: 10.4 us per BF16 epoch against 12.6 at 4)
    const int small = atomic_lockfree && n >= (int64_t(1) << 14) ? 8 : 4;
    if (t <= 0) t = n >= (int64_t(1) << 19) ? large : (n >= (int64_t(1) << 16) ? mid : small);
    t = t < G ? G : (t > 32 ? 32 : t);
    return t / G * G;
}

// Kernel mode for the parameters: deterministic batches, or the lock-free
// epoch with atomic row changes (16-bit tables: the stochastically rounded
// change) unless plain stores are requested.
int train_mode(const gosh_params *p) {
    if (p->mode == GOSH_DETERMINISTIC) return kModeDet;
    return p->plain_stores ? kModeStore : kModeRed;
}

gosh_status pick_train_kernel(gosh_dtype dtype, int d, int k, int mode, int lanes, int pass, int64_t n,
                              const TrainKernel **out) {
    const bool det = mode == kModeDet;
    const int ns = k + 1;
    const int nat = natural_lanes(dtype, d);
    // Defaults by level size, from per-level sweeps of lanes per row L,
    // samples per pass P and tile on the R-MAT 20 hierarchy (d = 128, k = 3;
    // L0 = one 16-byte vector per lane; P < 0: rows staged by TMA):
    //  - FP32 lock-free: from 2^19 rows registers, L0/2 lanes, P = 4 (361 us
    //    per level-0 epoch against 444 TMA-staged); from 2^16 registers, L0
    //    lanes, P = 4; from 2^12 registers, L0/2 lanes, P = 2 (level 2, 22k
    //    rows: 14.9 us against 16.3 with P = 4; level 3, 6.4k rows: 6.5 us
    //    against 7.7 TMA-staged); below, TMA-staged with L0 lanes (a
    //    latency-bound level: every row of a round in flight at once; 3.7 us
    //    against 3.9 with L0/2 lanes);
    //  - BF16 tables (atomic changes): registers, L0/2 lanes (two vectors per
    //    lane, more sources in flight), P = 2 at every size (levels of 6.4k,
    //    1.6k and 1.3k rows: 5.1, 4.0 and 3.9 us against 5.7, 4.2 and 4.1
    //    TMA-staged); FP16 tables the same from 2^14 rows, below L0 lanes,
    //    P = 4; with plain stores, L0/2 lanes and P = 4 except L0 lanes from
    //    2^16 to 2^19 rows.
    const bool defaulted = lanes <= 0 && pass == 0;
    if (!det && defaulted) {
        const int staged = ns <= 4 ? -4 : -6;
        const int half = nat >= 4 ? nat / 2 : nat;
        if (dtype == GOSH_F32 && mode == kModeRed) {
            if (n >= (int64_t(1) << 19)) {
                lanes = half;
                pass = 4;
            } else if (n >= (int64_t(1) << 16)) {
                lanes = nat;
                pass = 4;
            } else if (n >= (int64_t(1) << 12)) {
                lanes = half;
                pass = 2;
            } else {
                lanes = nat;
                pass = ns <= 6 ? staged : 4;
            }
        } else if (dtype != GOSH_F32 && mode == kModeRed) {
            if (n >= (int64_t(1) << 14) || dtype == GOSH_BF16) {
                lanes = half;
                pass = 2;
            } else {
                lanes = nat;
                pass = 4;
            }
        } else if (dtype != GOSH_F32) {
            const bool mid = n >= (int64_t(1) << 16) && n < (int64_t(1) << 19);
            lanes = (mid || nat < 4) ? nat : nat / 2;
            pass = 4;
        }
    }
    if (lanes <= 0) lanes = (!det && dtype != GOSH_F32 && nat >= 4) ? nat / 2 : nat;
    if (pass == 0) pass = det ? (ns <= 4 ? 4 : 8) : 2;
    if (pass < 0 && (det || ns > -pass)) {
        set_error("TMA-staged kernels (samples_per_pass = -S) serve the lock-free mode with k+1 <= S (k+1 = %d)", ns);
        return GOSH_ERR_UNSUPPORTED;
    }
    if (det && pass < ns) {
        set_error("deterministic mode gathers all k+1 samples in one pass: samples_per_pass %d < k+1 = %d",
                  pass, ns);
        return GOSH_ERR_UNSUPPORTED;
    }
    const TrainKernel *kern = find_train_kernel(dtype, d, lanes, pass, mode);
    if (!kern && defaulted && pass < 0) {
        // no TMA-staged variant for this width (d = 16): registers, 4 samples per pass
        pass = 4;
        kern = find_train_kernel(dtype, d, lanes, pass, mode);
    }
    if (!kern) {
        set_error("no training kernel for dtype %d, d %d, lanes_per_row %d, samples_per_pass %d, mode %d",
                  (int)dtype, d, lanes, pass, mode);
        return GOSH_ERR_UNSUPPORTED;
    }
    *out = kern;
    return GOSH_OK;
}

gosh_status train_level_impl(const gosh_csr *g, void *M, int level, int epochs, const gosh_params *p,
                             cudaStream_t s, double *loss_per_epoch, unsigned long long *n_updates) {
    const bool det = p->mode == GOSH_DETERMINISTIC;
    if (p->k > 7 && det) {
        set_error("deterministic mode supports k <= 7 (got %d)", p->k);
        return GOSH_ERR_UNSUPPORTED;
    }
    const TrainKernel *kern = nullptr;
    GOSH_TRY(pick_train_kernel(p->dtype, p->d, p->k, train_mode(p), p->lanes_per_row, p->samples_per_pass, g->n,
                               &kern));
    const int64_t n = g->n;
    if (epochs <= 0 || n <= 0) return GOSH_OK;
    const int ns = p->k + 1;
    const int cap_blocks = num_sms() * kern->blocks_per_sm;

    TrainArgs a{};
    a.rowptr = g->rowptr;
    a.col = g->col;
    a.M = M;
    a.n = n;
    a.k = p->k;
    a.seed = p->seed;
    a.graph = p->graph_id;
    a.level = (uint32_t)level;
    a.n_updates = n_updates;
    a.err = device_error_word();
    a.tile = tile_vertices(p, n, kern->lanes, kern->pass);

    auto grid_for = [&](int64_t nsrc) {
        const int64_t tiles = ceil_div(nsrc, a.tile);
        const int64_t want = ceil_div(tiles, kern->warps);
        return (int)(want < cap_blocks ? (want > 0 ? want : 1) : cap_blocks);
    };

    Scratch parts;
    if (loss_per_epoch) GOSH_TRY(parts.alloc(sizeof(double) * cap_blocks, s));
    a.loss_partials = loss_per_epoch ? parts.as<double>() : nullptr;

    if (!det) {
        a.src_begin = 0;
        a.src_end = n;
        // On request (cooperative_epochs), every epoch in one cooperative
        // launch, where one wave holds every tile (more would make warps
        // loop); by default one launch per epoch, whose programmatic
        // overlap measured faster than a grid barrier per epoch.
        const int coop_cap = num_sms() * kern->epochs_blocks_per_sm;
        const int grid = grid_for(n);
        if (p->cooperative_epochs && kern->launch_epochs && !loss_per_epoch && epochs > 1 &&
            kern->epochs_blocks_per_sm > 0 &&
            ceil_div(ceil_div(n, a.tile), kern->warps) <= coop_cap) {
            const int g = grid;
            Scratch bar;
            GOSH_TRY(bar.alloc(sizeof(unsigned int), s));
            GOSH_TRY_CUDA(cudaMemsetAsync(bar.ptr, 0, sizeof(unsigned int), s));
            const cudaError_t e = kern->launch_epochs(a, g, epochs, p->lr, p->lr_floor, bar.as<unsigned int>(), s);
            if (e == cudaSuccess) return GOSH_OK;
            cudaGetLastError();  // not co-resident here: fall back to one launch per epoch
        }
        // Epoch overlap (off by default; Sec. 6.3 leaves concurrent epochs on
        // large levels as future work): on a level of at least
        // overlap_min_vertices, epoch j runs on stream j mod c and so waits
        // only for epoch j - c; the streams fork from s and join it again.
        const int c = (!loss_per_epoch && p->epoch_overlap > 1 && n >= p->overlap_min_vertices && epochs > 1)
                          ? std::min(p->epoch_overlap, epochs)
                          : 1;
        cudaStream_t side[8] = {};
        cudaEvent_t ev[8] = {};
        struct SideCleanup {
            cudaStream_t *side;
            cudaEvent_t *ev;
            ~SideCleanup() {
                for (int i = 0; i < 8; ++i) {
                    if (side[i]) cudaStreamDestroy(side[i]);  // released once its work is done
                    if (ev[i]) cudaEventDestroy(ev[i]);
                }
            }
        } side_cleanup{side, ev};
        for (int i = 1; i < c; ++i) {
            GOSH_TRY_CUDA(cudaStreamCreateWithFlags(&side[i], cudaStreamNonBlocking));
            GOSH_TRY_CUDA(cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming));
        }
        if (c > 1) {
            GOSH_TRY_CUDA(cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming));
            GOSH_TRY_CUDA(cudaEventRecord(ev[0], s));
            for (int i = 1; i < c; ++i) GOSH_TRY_CUDA(cudaStreamWaitEvent(side[i], ev[0], 0));
        }
        for (int j = 0; j < epochs; ++j) {
            const double f = 1.0 - (double)j / (double)epochs;
            a.lr = (float)(p->lr * (f > p->lr_floor ? f : p->lr_floor));
            a.epoch = (uint32_t)j;
            kern->launch(a, grid, j % c == 0 ? s : side[j % c]);
            if (loss_per_epoch)
                launch_dep(loss_finalize, 1, 256, 0, s, parts.as<double>(), grid, loss_per_epoch + j, 0);
        }
        for (int i = 1; i < c; ++i) {
            GOSH_TRY_CUDA(cudaEventRecord(ev[i], side[i]));
            GOSH_TRY_CUDA(cudaStreamWaitEvent(s, ev[i], 0));
        }
        GOSH_TRY_CUDA(cudaGetLastError());
        return GOSH_OK;
    }

    // deterministic: snapshot batches of m consecutive sources
    const int64_t m = p->det_batch > 0 ? (p->det_batch < n ? p->det_batch : n) : n;
    const int64_t slots = m * ns;
    if (slots >= (int64_t(1) << 32)) {
        set_error("det_batch * (k+1) must stay below 2^32");
        return GOSH_ERR_INVALID_ARG;
    }
    Scratch R, C, keys, idx, done;
    GOSH_TRY(R.alloc(sizeof(float) * m * p->d, s));
    GOSH_TRY(C.alloc(sizeof(float) * slots * p->d, s));
    GOSH_TRY(keys.alloc(sizeof(uint32_t) * slots, s));
    GOSH_TRY(idx.alloc(sizeof(uint32_t) * slots, s));
    GOSH_TRY(done.alloc(m, s));
    a.R = R.as<float>();
    a.C = C.as<float>();
    a.keys = keys.as<uint32_t>();
    const int kbits = bits_for(n);
    for (int j = 0; j < epochs; ++j) {
        const double f = 1.0 - (double)j / (double)epochs;
        a.lr = (float)(p->lr * (f > p->lr_floor ? f : p->lr_floor));
        a.epoch = (uint32_t)j;
        for (int64_t b0 = 0; b0 < n; b0 += m) {
            const int64_t b1 = b0 + m < n ? b0 + m : n;
            const int64_t nsl = (b1 - b0) * ns;
            a.src_begin = b0;
            a.src_end = b1;
            const int grid = grid_for(b1 - b0);
            kern->launch(a, grid, s);
            if (loss_per_epoch)
                launch_dep(loss_finalize, 1, 256, 0, s, parts.as<double>(), grid, loss_per_epoch + j, b0 > 0);
            launch_dep(iota_u32, (int)std::min<int64_t>(ceil_div(nsl, 256), 4096), 256, 0, s, idx.as<uint32_t>(), nsl);
            GOSH_TRY(radix_sort_u32(keys.as<uint32_t>(), idx.as<uint32_t>(), nsl, 0, kbits, s));
            GOSH_TRY_CUDA(cudaMemsetAsync(done.ptr, 0, (size_t)(b1 - b0), s));
            const uint32_t sr = mix32((uint32_t)p->seed ^ mix32((uint32_t)(level << 20) ^ (uint32_t)j)) ^
                                mix32((uint32_t)(b0 >> 5));
            det_apply(p->dtype, p->d, keys.as<uint32_t>(), idx.as<uint32_t>(), nsl, C.as<float>(), R.as<float>(),
                      M, n, b0, b1, done.as<uint8_t>(), sr, s);
        }
    }
    GOSH_TRY_CUDA(cudaGetLastError());
    return GOSH_OK;
}

}  // namespace gosh
