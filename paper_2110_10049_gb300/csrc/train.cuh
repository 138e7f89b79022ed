// Training-step kernels of libgosh (Alg. 1 inside the epoch loop of Alg. 3).
//
// Mapping (GB300): a warp takes a tile of 32 consecutive sources.  First each
// lane draws the samples of one source of the tile (one Philox4x64-10 block
// per four samples, computed once per source instead of once per lane of the
// row) and parks the sample ids in shared memory.  Then the warp walks the
// tile in rounds: L lanes share one source (G = 32/L sources per round); each
// lane owns E = D/L contiguous elements of every row and moves them with
// 16-byte loads/stores.  The source row stays in registers across its k+1
// updates (the paper stages it in shared memory); the sample rows of one pass
// (P of them) are gathered together before any arithmetic so that their loads
// overlap; dot products are reduced with xor-shuffles inside the L-lane group.
#pragma once

#include "common.cuh"

namespace gosh {

constexpr int kMaxK = 15;        // negatives per positive
constexpr int kTrainWarps = 8;   // warps per block
constexpr int kSlotStride = kMaxK + 2;  // padded per-source sample-id slots in smem

// How a kernel writes its row changes (see train_kernels.cuh).
enum : int { kModeStore = 0, kModeRed = 1, kModeDet = 2 };

struct TrainArgs {
    const int64_t *rowptr;
    const int32_t *col;
    void *M;
    int64_t n;                 // |V_i|
    int k;                     // negatives per positive
    uint64_t seed, graph;      // Philox key
    uint32_t level, epoch;     // Philox counter word 2 = level << 32 | epoch
    float lr;                  // lr' of this epoch
    int64_t src_begin, src_end;
    int tile;                  // sources per warp tile (a multiple of 32/L, <= 32)
    // deterministic mode (snapshot batch [src_begin, src_end))
    float *R;                  // [(src_end-src_begin) x D]  final source rows
    float *C;                  // [(src_end-src_begin)*(k+1) x D] sample-row changes
    uint32_t *keys;            // [(src_end-src_begin)*(k+1)] target row or n (skipped)
    // monitors
    double *loss_partials;     // [gridDim.x] or null
    unsigned long long *n_updates;  // or null
    int *err;                  // device error word raised by a timed-out wait, or null
    // walk pairs (Sec. 3.2): int32 (source, positive) per position, source -1
    // for a hole; src_end = positions; visited in walk_position order
    const int32_t *pairs;
    uint32_t walk_key;
    int walk_h;
};

// Per-device error word of the library (lazily allocated; read and cleared
// by gosh_device_check).
int *device_error_word();

// Host-side launcher for one epoch (Hogwild) or one snapshot batch (deterministic).
struct TrainKernel {
    void (*launch)(const TrainArgs &, int grid, cudaStream_t);
    // all epochs in one cooperative launch with a grid barrier between them
    // (null where not compiled); returns the launch's error
    cudaError_t (*launch_epochs)(const TrainArgs &, int grid, int epochs, double lr, double lr_floor,
                                 unsigned int *barrier, cudaStream_t);
    int epochs_blocks_per_sm;
    int blocks_per_sm;
    int lanes;     // L
    int pass;      // P (negative: all of up to -P samples staged by TMA)
    int warps;     // warps per block
};

// One compiled variant: its key and a factory (the factory queries occupancy,
// so it runs lazily once a device is current).
struct TrainEntry {
    gosh_dtype dtype;
    int d, lanes, pass;
    int mode;
    TrainKernel (*make)();
};
const TrainEntry *train_entries_f32(int *count);
const TrainEntry *train_entries_bf16(int *count);
const TrainEntry *train_entries_f16(int *count);
const TrainEntry *train_tma_entries_f32(int *count);
const TrainEntry *train_tma_entries_bf16(int *count);
void det_apply_f32(int d, const uint32_t *skeys, const uint32_t *sidx, int64_t nslots, const float *C,
                   const float *R, void *M, int64_t n, int64_t b0, int64_t b1, uint8_t *src_done,
                   uint32_t sr_seed, cudaStream_t s);
void det_apply_bf16(int d, const uint32_t *skeys, const uint32_t *sidx, int64_t nslots, const float *C,
                    const float *R, void *M, int64_t n, int64_t b0, int64_t b1, uint8_t *src_done,
                    uint32_t sr_seed, cudaStream_t s);
void det_apply_f16(int d, const uint32_t *skeys, const uint32_t *sidx, int64_t nslots, const float *C,
                   const float *R, void *M, int64_t n, int64_t b0, int64_t b1, uint8_t *src_done,
                   uint32_t sr_seed, cudaStream_t s);

// Looks up the kernel for (dtype, d, lanes-per-row, samples-per-pass, mode).
// Returns nullptr if that combination is not compiled.
const TrainKernel *find_train_kernel(gosh_dtype dtype, int d, int lanes, int pass, int mode);

// Lists the lanes-per-row and samples-per-pass variants compiled for (dtype, d, mode).
int list_train_variants(gosh_dtype dtype, int d, int mode, int *lanes, int *pass, int cap);

}  // namespace gosh
