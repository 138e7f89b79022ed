/*
 * gosh.h -- C ABI of libgosh, a GB300 (sm_103a) implementation of the
 * multi-level graph embedding of GOSH ("Boosting Graph Embedding on a Single
 * GPU", arxiv 2110.10049).
 *
 * Conventions for every entry point
 *  - Graphs are CSR: row pointer int64[n+1] (rowptr[0] = 0, rowptr[n] = nnz),
 *    neighbour ids int32[nnz], strictly ascending inside each row, no
 *    self-loops, symmetric (undirected graph stored in both directions).
 *  - Embedding matrices are row-major n x d, element type given by gosh_dtype,
 *    row stride d elements, base address 16-byte aligned.  d is 8, 16, 32, 64
 *    or 128 for the resident entry points (initialisation, training, copy
 *    projection, gosh_embed with the copy projection, scores); 32, 64 or 128
 *    for LargeGraphGPU, the batched entry and the learned projection.  At
 *    d = 16 a warp updates 8 (FP32) or 16 (16-bit tables) sources at once, at
 *    d = 8 16 or 32 (Sec. 3.1.1's small-d mapping).
 *  - Every pointer is a device pointer unless its comment says otherwise.  The
 *    caller owns every buffer it passes; the library owns hierarchy handles.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Entry points are asynchronous on that stream unless marked
 *    "synchronous".  Temporary device memory is taken with cudaMallocAsync on
 *    the same stream (or from the caller's allocator, gosh_set_allocator)
 *    and released before return.
 *  - No exception crosses the ABI.  Each call returns a gosh_status; on error
 *    gosh_last_error() (thread-local) holds a one-line message.  Argument
 *    errors are detected before any kernel is launched.
 */
#ifndef GOSH_H
#define GOSH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gosh_status {
    GOSH_OK = 0,
    GOSH_ERR_INVALID_ARG = 1,  /* bad pointer, size, layout or CSR */
    GOSH_ERR_OOM = 2,          /* device or pinned allocation failed */
    GOSH_ERR_BUDGET = 3,       /* the work does not fit the device budget */
    GOSH_ERR_CUDA = 4,         /* a CUDA call failed */
    GOSH_ERR_TIMEOUT = 5,      /* a bounded device-side wait gave up */
    GOSH_ERR_UNSUPPORTED = 6   /* valid request the library does not serve */
} gosh_status;

typedef enum gosh_dtype { GOSH_F32 = 0, GOSH_BF16 = 1, GOSH_F16 = 2 } gosh_dtype;

/* GOSH_HOGWILD: the lock-free epoch of Sec. 3.1 (concurrent sources race on
 * shared sample rows).  GOSH_DETERMINISTIC: sources in batches of det_batch
 * consecutive ids read a snapshot of M taken at the batch start; the row
 * changes are summed in a fixed order (source, then sample) at the batch end,
 * so results do not depend on scheduling.  det_batch = 1 is the sequential
 * epoch of Alg. 3. */
typedef enum gosh_mode { GOSH_HOGWILD = 0, GOSH_DETERMINISTIC = 1 } gosh_mode;

typedef struct gosh_csr {
    int64_t n;              /* |V| */
    const int64_t *rowptr;  /* [n+1] */
    const int32_t *col;     /* [rowptr[n]] */
    int on_device;          /* 1: device pointers; 0: host pointers (gosh_embed copies them in) */
} gosh_csr;

typedef struct gosh_params {
    int d;                  /* embedding dimension: 8, 16, 32, 64 or 128 (LargeGraphGPU, walks, the
                               batched entry and the learned projection: 32, 64 or 128) */
    int k;                  /* negatives per positive, n_s (0..15; deterministic mode <= 7,
                               walks <= 3, LargeGraphGPU B * (k+1) <= 32) */
    double lr;              /* initial learning rate of every level */
    double lr_floor;        /* lr' = lr * max(1 - j/e_i, lr_floor); paper: 1e-4 */
    int epochs;             /* e: total epochs over all levels (unit: epoch_unit) */
    double p;               /* smoothing ratio of the epoch split */
    int threshold;          /* coarsening stops once |V_i| <= threshold (paper: 100) */
    double shrink;          /* ... or once |V_{i+1}| > shrink * |V_i| (paper: 0.8) */
    int max_levels;         /* cap on the number of graphs; 1 = no coarsening */
    gosh_dtype dtype;       /* storage type of M */
    gosh_mode mode;
    int64_t det_batch;      /* sources per snapshot batch (GOSH_DETERMINISTIC) */
    uint64_t seed;          /* Philox key word 0 */
    uint64_t graph_id;      /* Philox key word 1 (distinguishes graphs of a batch) */
    int lanes_per_row;      /* lanes that share one source row; 0 = automatic */
    int samples_per_pass;   /* sample rows gathered at once per source; 0 = automatic */
    int64_t device_budget_bytes; /* 0 = unlimited */
    int validate;           /* 1: check the CSR before use (costs one pass; host CSRs of
                               gosh_train_level_large and _walks are checked on the host) */
    int plain_stores;       /* GOSH_HOGWILD: 0 (default) applies every row change as an atomic
                               vector addition at L2 (16-bit tables: the stochastically
                               rounded new row minus the row read, rounded to nearest; without
                               a racing writer this leaves exactly the rounded row whenever the
                               change fits the 16-bit significand, e.g. any change below 256
                               ulps, else within one ulp), so concurrent updates of one row are
                               never lost; 1 writes rows back with plain (16-bit:
                               stochastically rounded) stores as the paper does (a racing
                               writer may overwrite an update). */
    int projection;         /* gosh_embed between levels: 0 = copy (EXPANDEMBEDDING, Alg. 2),
                               1 = learned residual MLP (gosh_project_learned), trained after
                               every level on that level's (coarse, fine) pairs */
    int mlp_hidden;         /* hidden width of the projection MLP (default 256) */
    int mlp_epochs;         /* passes over a level's training rows per MLP training (default 1) */
    double mlp_lr;          /* Adam step size (default 1e-3) */
    int mlp_batch;          /* vertices per MLP training step (default 8192) */
    int64_t mlp_max_rows;   /* training rows per level: every ceil(n/max)-th vertex (default 32768; 0 = all) */
    int p_gpu;              /* LargeGraphGPU: part (submatrix) bins on the device (paper: 3) */
    int s_gpu;              /* LargeGraphGPU: edge-block bins on the device (paper: 2) */
    int B;                  /* LargeGraphGPU: positives per vertex per part pair per round (paper: 5) */
    int large_parts;        /* LargeGraphGPU: K; 0 = derive from device_budget_bytes */
    int persistent_small_levels; /* gosh_embed, lock-free with copy projection and automatic
                               kernels: 1 trains every level with |V_i| <= 2^17 in one
                               persistent launch (as gosh_embed_batch does; built for many
                               graphs at once, it is slower for one: R-MAT 20, 835 against
                               347 ms per embed); 0 (default) launches every epoch separately */
    int vertices_per_warp;  /* sources a warp takes per tile (<= 32, rounded to a multiple
                               of 32/lanes_per_row); 0 = by level size (8 / 16 / 32) */
    int walk_length;        /* gosh_train_level_walks: vertices per random walk, l (default 8) */
    int walk_window;        /* gosh_train_level_walks: pairs within distance g (default 3) */
    int large_serial;       /* LargeGraphGPU: 1 runs the part-pair kernels one after another on
                               one stream (a reproducible kernel order: with FP32 d = 128, whose
                               kernel gives each source a whole warp, a part pair of at most 32
                               sources is then trained exactly in the sequential order); 0
                               (default) alternates two streams so that kernels of independent
                               pairs overlap */
    int large_evict;        /* LargeGraphGPU part-bin choice when a part must come in: 0
                               (default) the part next used farthest ahead (fewest copies); 1
                               the same, but sparing the parts of the previous kernel while
                               another bin is eligible, so that the copy overlaps that kernel
                               (Sec. 5.2's example), at the cost of more copies */
    int64_t overlap_min_vertices; /* epoch_overlap applies to levels with at least this many
                               vertices (default 65536); smaller levels stay serialised */
    int epoch_overlap;      /* lock-free per-epoch launches: c in 1..8 consecutive epochs of a
                               large level may run at once (epoch j waits only for epoch j-c:
                               the concurrency that Sec. 6.3 leaves as future work); 1
                               (default) serialises every epoch as the paper does.  Levels
                               trained in one cooperative launch (cooperative_epochs), and
                               calls that request per-epoch losses, stay serialised. */
    int large_pools;        /* LargeGraphGPU positives: 0 (default) drawn on the device from edge
                               blocks streamed from the host; 1 drawn on host threads into sample
                               pools (B per source per kernel, Sec. 5's scheme) streamed instead;
                               the same samples either way */
    int epoch_unit;         /* unit of `epochs` in gosh_embed and gosh_embed_batch: 0 (default)
                               one pass over V_i (Alg. 3); 1 |E| positive draws, the unit of the
                               paper's experiments (Sec. 6 setup): e becomes round(e * nnz_0 /
                               |V_0|) passes, split over the levels as usual (gosh_level_epochs).
                               gosh_train_level always counts passes. */
    int cooperative_epochs; /* lock-free levels whose tiles fit one wave of the register
                               kernel: 1 runs all their epochs in one cooperative launch (a
                               grid barrier between epochs); 0 (default) one launch per epoch,
                               consecutive launches overlapping their drain and start, which
                               measured faster (R-MAT 20 level 1: 347 against 356 ms per embed) */
} gosh_params;

typedef struct gosh_walk_stats {
    int64_t positions;      /* pair positions per epoch: |V| * W, W = pairs of a full walk */
    int epochs;
    double host_ms;         /* walks drawn on host threads (overlapped with the device) */
    double total_ms;        /* wall time of the call */
    int64_t h2d_bytes;      /* pair tables copied to the device */
} gosh_walk_stats;

typedef struct gosh_large_stats {
    int parts;              /* K */
    int rounds;             /* ceil(e / B) */
    int64_t kernels;        /* part-pair kernels launched (rounds * K(K+1)/2) */
    int64_t swaps;          /* part loads into bins */
    int64_t h2d_bytes;      /* parts + edge blocks copied to the device */
    int64_t d2h_bytes;      /* parts copied back */
    unsigned long long positives;  /* positive samples used (<= e * |V|) */
    unsigned long long updates;    /* UPDATEEMBED applications */
    int64_t device_bytes;   /* bins allocated on the device */
    double total_ms;        /* wall time of the call */
    double setup_ms;        /* of which: edge blocks built (host threads, pinned) and bins allocated */
} gosh_large_stats;

#define GOSH_MAX_LEVELS 64

typedef struct gosh_stats {
    int levels;                           /* D */
    int64_t n[GOSH_MAX_LEVELS];           /* |V_i| */
    int64_t nnz[GOSH_MAX_LEVELS];         /* CSR entries of G_i */
    int epochs[GOSH_MAX_LEVELS];          /* e_i */
    double train_ms[GOSH_MAX_LEVELS];     /* device time of level i's training */
    double coarsen_ms;                    /* device time of the whole coarsening */
    double project_ms;                    /* device time of all projections */
    double total_ms;                      /* wall time of gosh_embed */
    unsigned long long updates;           /* UPDATEEMBED applications */
} gosh_stats;

typedef struct gosh_hierarchy gosh_hierarchy;

/* Fills *p with the paper's defaults: d 128, k 3, lr 0.035, lr_floor 1e-4,
 * e 200, p 0.3 (the "normal" row of the configuration table, Sec. 7),
 * threshold 100 and shrink 0.8 (Sec. 4), FP32 Hogwild, det_batch 4096. */
gosh_status gosh_params_default(gosh_params *p);

/* The epoch schedule of gosh_embed (Alg. 2, Sec. 3) for D graphs, host only.
 * With epoch_unit = 1 (an epoch is |E| positive draws, the paper's
 * experimental unit, Sec. 6; one Alg. 3 pass makes |V| of them) the total e
 * first becomes floor((2 e nnz_0 + n_0) / (2 n_0)) passes (e * nnz_0 / n_0
 * rounded half up, at least 1 when e >= 1; nnz_0 = CSR entries of G_0).
 * Then a fraction p of the total goes uniformly to the levels and the rest
 * geometrically (each level twice its finer neighbour):
 *   e_i = floor(p*e/D + (1-p)*e*2^i/(2^D-1)) for i >= 1,  e_0 = e - sum of the others.
 * n, nnz: host int64[D] sizes of the graphs (only G_0's are read, and only
 * with epoch_unit = 1; may be NULL otherwise); out: host int[D] passes.
 * GOSH_ERR_INVALID_ARG for D < 1, epochs < 0, p outside [0, 1], an unknown
 * unit, or a pass count beyond INT_MAX. */
gosh_status gosh_level_epochs(int epochs, double p, int D, int epoch_unit, const int64_t *n, const int64_t *nnz,
                              int *out);

/* Caller-provided device memory.  alloc(bytes, stream, ctx) returns device
 * memory of at least `bytes` bytes, 256-byte aligned, usable in stream order on
 * `stream` (a cudaStream_t, NULL = legacy default stream), or NULL when it
 * cannot; free(ptr, bytes, stream, ctx) takes it back in stream order.  A
 * framework that owns device memory through its own caching allocator (e.g.
 * PyTorch's) installs it here so that the library's working buffers come from
 * it: every call's workspaces (deterministic-mode batches, LargeGraphGPU
 * bins, gosh_embed's level tables, coarsening temporaries) and the coarse
 * levels a hierarchy handle holds.  Not routed: the learned projection's
 * weights (created with the network), the prefix sum's cached per-stream
 * status words (a few KB) and the 4-byte device error word.  Process-wide;
 * both functions, or neither (NULL, NULL: back to the stream-ordered pool).
 * Each block is returned to the allocator that provided it, so the allocator
 * may change between calls, but not while a call runs. */
typedef void *(*gosh_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*gosh_free_fn)(void *ptr, size_t bytes, void *stream, void *ctx);
gosh_status gosh_set_allocator(gosh_alloc_fn alloc, gosh_free_fn free, void *ctx);

/* Thread-local message of the last failed call ("" if none). */
const char *gosh_last_error(void);

/* Synchronises `stream`, then reads and clears the current device's error
 * word, which a kernel raises when one of its bounded waits (TMA copy or MMA
 * completion) gave up.  GOSH_ERR_TIMEOUT if it was raised since the last
 * check.  gosh_embed checks it before returning. */
gosh_status gosh_device_check(void *stream);

/* Number of CUDA kernels this library has launched in this process so far
 * (all threads, all devices).  A diagnostic for profiling and benchmarking. */
unsigned long long gosh_kernel_launches(void);

/* LargeGraphGPU and walk training keep their pinned host buffers (edge
 * blocks, walk pair tables) across calls, since pinning costs far more than
 * filling.  This frees those not held by a running call and returns the
 * bytes freed; later calls pin again.  No device work. */
unsigned long long gosh_release_host_buffers(void);

/* Checks a device CSR against the layout above (row pointer monotone,
 * neighbour ids in range, ascending, no self-loop, symmetric).  Synchronous.
 * Returns GOSH_ERR_INVALID_ARG with a message naming the first violation. */
gosh_status gosh_validate_csr(const gosh_csr *g, void *stream);

/*
 * MULTIEDGECOLLAPSE (Alg. 4, Sec. 4).  Builds G_1, G_2, ... from the device
 * CSR g0: per level, vertices are ordered by degree (descending, ties by
 * ascending id); in that order each unmapped vertex opens a new cluster and
 * absorbs its unmapped neighbours u for which deg(v) <= delta or deg(u) <= delta
 * (hub^2 restriction, delta = nnz_i / |V_i|); G_{i+1} is the image of E_i
 * without self-loops and duplicates.  Continues while |V_{i+1}| > threshold
 * and |V_{i+1}| <= floor(shrink * |V_i|); the last graph built is kept; the
 * body always runs once.  max_levels caps the number of graphs (>= 2).
 * The maps are identical to the sequential algorithm's (cluster ids in
 * discovery order).  Synchronous (reads level sizes back).
 * *out receives a library-owned handle; level 0 aliases g0 (not copied), so
 * g0 must outlive the handle.
 */
gosh_status gosh_coarsen(const gosh_csr *g0, int threshold, double shrink, int max_levels,
                         void *stream, gosh_hierarchy **out);

/*
 * gosh_coarsen for n_graphs independent graphs at once (Alg. 4 per graph):
 * each level is computed for all graphs still coarsening as one disjoint
 * union (vertex ids graph after graph; the degree order sorts by graph
 * first), so one sequence of kernels serves every graph.  out[g] receives a
 * handle equal, level by level, to gosh_coarsen(&graphs[g], ...): the same
 * maps and coarse CSRs, bit for bit, and the same stopping rule per graph.
 * graphs: device CSRs with n >= 1 (each must outlive its handle); out:
 * n_graphs handles, each freed with gosh_hierarchy_free (levels coarsened
 * together share device buffers, released with the last handle holding
 * them).  Synchronous.  On error no handle is returned (all are NULL).
 */
gosh_status gosh_coarsen_batch(const gosh_csr *graphs, int n_graphs, int threshold, double shrink,
                               int max_levels, void *stream, gosh_hierarchy **out);

/* Number of graphs D in the hierarchy (G_0 .. G_{D-1}). */
int gosh_hierarchy_levels(const gosh_hierarchy *h);

/* Level i of the hierarchy: g_i (device CSR, library-owned) and map_i, the
 * device int32[|V_i|] fine-to-coarse map from G_i to G_{i+1} (NULL for the
 * last level). */
gosh_status gosh_hierarchy_level(const gosh_hierarchy *h, int i, gosh_csr *g_i,
                                 const int32_t **map_i);

/* Sizes of level i: *n = |V_i|, *nnz = CSR entries of G_i (either may be NULL). */
gosh_status gosh_hierarchy_sizes(const gosh_hierarchy *h, int i, int64_t *n, int64_t *nnz);

/* Copies level i to host memory: rowptr int64[n+1], col int32[nnz], map
 * int32[n] (any may be NULL; map is left untouched for the last level).
 * Synchronous on `stream`. */
gosh_status gosh_hierarchy_copy_level(const gosh_hierarchy *h, int i, int64_t *rowptr, int32_t *col,
                                      int32_t *map, void *stream);

void gosh_hierarchy_free(gosh_hierarchy *h);

/* Random initialisation of M_{D-1} (Alg. 2): M[v][c] = ((w >> 11) * 2^-53 - 0.5) / d
 * rounded to the storage type, with w word c%4 of Philox4x64-10 at counter
 * (v, c/4, level, 1) and key (seed, graph_id): uniform on [-0.5/d, 0.5/d). */
gosh_status gosh_init_embedding(void *M, int64_t n, int d, gosh_dtype dtype, int level,
                                uint64_t seed, uint64_t graph_id, void *stream);

/*
 * TRAININGPU (Alg. 3) for one level: `epochs` epochs over the sources of g;
 * in epoch j every source v draws one positive (uniform over Gamma(v)) and k
 * negatives (uniform over V) and applies UPDATEEMBED (Alg. 1) to M[v] and each
 * sample row in turn with lr' = lr * max(1 - j/epochs, lr_floor) and
 * score = (b - sigmoid(M[v].M[u])) * lr'.  Epochs are serialised (Sec. 3.1).
 * Draws: Philox4x64-10 at counter (v, blk, level << 32 | j, 0) with key
 * (seed, graph_id); word 0 picks the positive as col[rowptr[v] + floor(w * deg / 2^64)],
 * word t picks negative t as floor(w * n / 2^64).  A source without
 * neighbours skips its positive; a negative equal to the source is skipped.
 * M: device n x d, updated in place.
 * loss_per_epoch: device double[epochs] or NULL; receives the summed NLL of
 *   every applied update (pre-update dot), accumulated in FP64.
 * n_updates: device uint64 or NULL; incremented by the number of applied updates.
 * Uses params->{d,k,lr,lr_floor,dtype,mode,det_batch,seed,graph_id,
 * lanes_per_row,samples_per_pass}.
 */
gosh_status gosh_train_level(const gosh_csr *g, void *M, int level, int epochs,
                             const gosh_params *params, void *stream,
                             double *loss_per_epoch, unsigned long long *n_updates);

/*
 * gosh_train_level for callers that cannot allocate device memory (the paper
 * has no counterpart; this is a deployment variant).  Callers that run inside
 * a framework or server owning all device memory through its own arena, or
 * that must never let a library call cudaMalloc/cudaFree (which can
 * synchronise the device), use this entry point: it allocates nothing.  The
 * caller still passes the graph, M, loss_per_epoch and n_updates buffers,
 * with the same meaning, layout and results as gosh_train_level.
 * Limits and behaviour:
 *  - GOSH_HOGWILD only; GOSH_DETERMINISTIC returns GOSH_ERR_UNSUPPORTED (its
 *    scratch grows with det_batch).
 *  - The per-block loss partial sums live in one static device array of 4096
 *    FP64 values (32 KB), held by every GPU that loads the library until the
 *    process exits.  A launch needing more blocks than that returns
 *    GOSH_ERR_INVALID_ARG before any kernel runs (a launch uses at most SMs x
 *    resident blocks of the chosen kernel: on a GB300 152 x 8 = 1216 for the
 *    256-thread register kernels, at most 152 x 16 = 2432 for the 128-thread
 *    staged ones).
 *  - A bounded device-side wait that gives up (the staged kernels' copy
 *    completion) raises a second static device word, not the library's
 *    allocated one; gosh_device_check reads and clears it, returning
 *    GOSH_ERR_TIMEOUT, exactly as for the other entry points.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture starts.
 *  - All calls on a device share the array and it keeps the last call's
 *    contents (each launch overwrites the slots it reads, so nothing needs
 *    clearing).  Calls whose work overlaps on the GPU (different streams or
 *    threads at the same time) race on it: serialise them.
 */
gosh_status gosh_train_level_noalloc(const gosh_csr *g, void *M, int level, int epochs,
                                     const gosh_params *params, void *stream,
                                     double *loss_per_epoch, unsigned long long *n_updates);

/*
 * LargeGraphGPU (Sec. 5): TRAININGPU for a level whose graph and embedding
 * exceed the device budget.  V is split into K contiguous parts (K =
 * params->large_parts, or derived from device_budget_bytes: part bins get 60%
 * of the budget); a round runs kernel K_{a,b} for every part pair in
 * inside-out order (0,0),(1,0),(1,1),(2,0),...: each u in V^a with neighbours
 * in V^b takes B positives uniform over Gamma(u) & V^b, each followed by k
 * negatives uniform over V^b, and symmetrically for V^b when a != b;
 * ceil(epochs/B) rounds; a device counter stops positives at epochs * |V|.
 * Positive t = round*B + j of a source uses lr * max(1 - t/epochs, lr_floor)
 * and Philox counter (u, blk, level << 32 | t, tag) with tag 0 when K = 1
 * (so K = 1, B = 1 draws exactly the samples of gosh_train_level) and
 * 3 | (a*K+b) << 8 otherwise.  Parts move between pinned host memory and
 * params->p_gpu device bins (farthest-next-use eviction), edge blocks
 * (built once on host threads) or, with params->large_pools = 1, each
 * kernel's sample pool (its positives drawn on host threads, the same
 * samples; gosh_large_pool) through params->s_gpu bins, all
 * asynchronously on per-bin streams with cudaEvent dependencies; kernels
 * alternate over two streams and may overlap (lock-free, as in the paper),
 * or run one after another on one stream when params->large_serial is 1.
 * g: HOST CSR; M: HOST n x d (FP32 or BF16; pinned in place if pageable),
 * updated in place.  Lock-free mode only.  stats: host pointer or NULL.
 * GOSH_ERR_BUDGET if K parts do not fit the budget.  Synchronous.
 */
gosh_status gosh_train_level_large(const gosh_csr *g, void *M, int level, int epochs,
                                   const gosh_params *params, void *stream, gosh_large_stats *stats);

/*
 * Random-walk positives (Sec. 3.2, the paper's GOSHW): each epoch draws one
 * walk of l = params->walk_length vertices from every vertex on host threads
 * (step t of the walk from v: a uniform neighbour from Philox block
 * (v, t/4, level<<32 | epoch, 4), word t%4; a vertex without neighbours ends
 * the walk) and takes every pair (w_i, w_j) with 0 < j - i <= g =
 * params->walk_window as a positive with source w_i.  The walk from v fills
 * positions v*W .. v*W+W-1 (W = pairs of a full walk, i ascending then j);
 * positions past a shorter walk and pairs with equal ends are skipped.  The
 * GPU visits the positions in a pseudo-random order (the shuffle: a 4-round
 * Feistel permutation of [0, |V| W) keyed by seed, graph, level and epoch)
 * and applies Alg. 1 to the positive and to k <= 3 negatives drawn uniformly
 * over V_i from Philox block (position, blk, level<<32 | epoch, 5), words
 * 1..k (a negative equal to the source is skipped); lr decays per epoch as in
 * gosh_train_level.  The host fills the pair table of epoch j+1 while the
 * device copies and trains epoch j.
 * g: CSR (host, or device: copied back once); M: device |V| x d, FP32 or
 * BF16, d in {32, 64, 128}, updated in place.  Lock-free mode only.
 * n_updates: device counter or NULL (incremented).  stats: host or NULL.
 * Synchronous on `stream`.
 */
gosh_status gosh_train_level_walks(const gosh_csr *g, void *M, int level, int epochs, const gosh_params *params,
                                   void *stream, unsigned long long *n_updates, gosh_walk_stats *stats);

/* The pair table gosh_train_level_walks uses for one epoch, drawn on the
 * calling thread (no device involved): pairs = host int32[|V| * W * 2] of
 * (source, positive) per position, -1 for holes, W = pairs of a full walk
 * (sum over i < l-1 of min(g, l-1-i)).  g: host CSR, checked first (rowptr
 * from 0 and non-decreasing, columns in range, rows strictly ascending, no
 * self-loops; GOSH_ERR_INVALID_ARG otherwise). */
gosh_status gosh_walk_pairs(const gosh_csr *g, int walk_length, int walk_window, int level, int epoch,
                            uint64_t seed, uint64_t graph_id, int32_t *pairs);

/* The order in which the device visits an epoch's positions (the shuffle):
 * order = host int64[positions], order[i] = position visited i-th.  Host only. */
gosh_status gosh_walk_order(int64_t positions, int level, int epoch, uint64_t seed, uint64_t graph_id,
                            int64_t *order);

/* The edge block of part pair (a, b), 0 <= b <= a < K, exactly as
 * gosh_train_level_large builds it on host threads and streams it (no GPU
 * use): V is split into K contiguous parts (part i = [n*i/K, n*(i+1)/K));
 * rp_ab [n_a+1] / col_ab [m_ab] hold, for every u in V^a, its neighbours in
 * V^b as ids local to V^b (rows from 0); rp_ba / col_ba the same for V^b
 * against V^a (left untouched when a == b).  Call with rp_ab = NULL to get
 * m_ab and m_ba only.  g: host CSR, checked as by gosh_walk_pairs. */
gosh_status gosh_large_block(const gosh_csr *g, int K, int a, int b, int64_t *m_ab, int64_t *m_ba, int64_t *rp_ab,
                             int32_t *col_ab, int64_t *rp_ba, int32_t *col_ba);

/* The sample pool of part pair (a, b), 0 <= b <= a < K, in round `round`,
 * exactly as gosh_train_level_large with large_pools = 1 draws it on host
 * threads (no GPU use): V is split into K contiguous parts; for every source
 * u of the pair (V^a, then V^b when a != b) and j < B, out[s * B + j] is the
 * local id (in the opposite part) of a neighbour of u drawn uniformly from
 * its neighbours in the opposite part with Philox word 0 of block
 * (u, 0, level << 32 | round*B + j, tag), tag 0 when K = 1 and
 * 3 | (a*K + b) << 8 otherwise; -1 when u has no neighbour there.
 * out: host int32[(|V^a| + (a != b ? |V^b| : 0)) * B].  g: host CSR, checked
 * as by gosh_walk_pairs. */
gosh_status gosh_large_pool(const gosh_csr *g, int K, int a, int b, int round, int B, int level, uint64_t seed,
                            uint64_t graph_id, int32_t *out);

/* Host-only simulation of the LargeGraphGPU part-bin schedule (no GPU use):
 * for `rounds` rounds over K parts and p_gpu bins, with the bin choice
 * `evict` (params->large_evict), writes for every kernel i
 * its pair (pairs_out[2i], pairs_out[2i+1]) = (a, b) and the loads done
 * before it (loads_out[2i], loads_out[2i+1]: part * 1000 + bin, or -1),
 * choosing bins exactly as gosh_train_level_large does.  Returns the kernel
 * count, -1 if it exceeds cap_tasks, or -2 for invalid arguments (K < 1,
 * p_gpu outside [2, 999], rounds < 0, evict not 0 or 1, NULL outputs). */
int gosh_large_plan(int64_t n, int K, int p_gpu, int rounds, int evict, int *pairs_out, int *loads_out,
                    int cap_tasks);

/* Stochastic rounding of FP32 values to a 16-bit table type (dtype GOSH_BF16
 * or GOSH_F16), exactly as the training kernels round every value they write
 * (16-bit tables with FP32 arithmetic; the paper trains in FP32): value i is rounded
 * away from zero with probability equal to its distance from the value toward
 * zero divided by the gap between the two, using 16 random bits from a 32-bit
 * hash of (seed, i / 2); infinities and NaNs pass unchanged.
 * x: device float[n]; out: device 16-bit[n]; both 4-byte aligned.
 * Asynchronous on `stream`.  No counterpart in the paper. */
gosh_status gosh_round_stochastic(const float *x, void *out, int64_t n, gosh_dtype dtype, uint64_t seed,
                                  void *stream);

/* EXPANDEMBEDDING (Alg. 2, Sec. 3): M_fine[v] = M_coarse[map[v]] for v < n_fine.
 * map: device int32[n_fine] with values in [0, n_coarse). */
gosh_status gosh_project(const void *M_coarse, int64_t n_coarse, const int32_t *map,
                         void *M_fine, int64_t n_fine, int d, gosh_dtype dtype, void *stream);

/*
 * Learned coarse-to-fine projection (not in the paper, whose projection is the
 * copy of Alg. 2; MILE's learned projection is the paper's point of
 * comparison, Sec. 7).  A residual two-layer MLP on per-vertex features
 *   f(v) = [ M_c[map v] | log(1 + deg v) | mean_{w in Gamma(v)} M_c[map w] ]  (2d+1 values)
 *   M_f[v] = M_c[map v] + W2 relu(W1 f(v) + b1) + b2
 * with BF16 weights/activations for the tensor-core GEMMs, FP32 accumulation
 * and FP32 master weights with Adam.  W2 = b2 = 0 at creation, so an
 * untrained network is exactly the copy projection.
 */
typedef struct gosh_mlp gosh_mlp;

/* Creates a network for dimension d (32, 64, 128) with `hidden` units (a
 * multiple of 16); W1 is Glorot-uniform from Philox (key seed). */
gosh_status gosh_mlp_create(int d, int hidden, uint64_t seed, gosh_mlp **out);
void gosh_mlp_free(gosh_mlp *m);

/* Row stride (BF16 elements) of a feature matrix: 2d+1 rounded up to 16. */
int gosh_mlp_feature_stride(int d);

/* Host copies of the FP32 master weights: W1 hidden x (2d+1), b1 hidden,
 * W2 d x hidden, b2 d (row-major).  Any pointer may be NULL (get). */
gosh_status gosh_mlp_get_weights(const gosh_mlp *m, float *W1, float *b1, float *W2, float *b2);
gosh_status gosh_mlp_set_weights(gosh_mlp *m, const float *W1, const float *b1, const float *W2, const float *b2);

/* Feature rows of every vertex of g_fine (device CSR) from M_coarse through
 * map (device int32[n_fine]); X: device BF16 n_fine x gosh_mlp_feature_stride(d). */
gosh_status gosh_mlp_features(const gosh_csr *g_fine, const int32_t *map, const void *M_coarse, int d,
                              gosh_dtype dtype, void *X, void *stream);

/* Mean-squared-error loss L = (1/n) sum_v |Y(v) - R(v)|^2 and its gradients
 * for one batch of n rows (16 <= n <= 2^20): X device BF16 features, R device
 * FP32 n x d residual targets; gradients to host buffers (shapes as in
 * gosh_mlp_get_weights), loss to *loss (host).  No update.  Synchronous. */
gosh_status gosh_mlp_grads(gosh_mlp *m, const void *X, const float *R, int64_t n, float *dW1, float *db1,
                           float *dW2, float *db2, double *loss, void *stream);

/* Trains on the pairs of one level: inputs f(v) from M_coarse, targets
 * M_fine[v] - M_coarse[map v], `epochs` passes in batches of `batch` vertices
 * with Adam (step size lr).  max_rows > 0 trains on every ceil(n/max_rows)-th
 * vertex only (0 = all).  final_loss (host, nullable): mean squared error per
 * vertex over the last pass.  Synchronous. */
gosh_status gosh_mlp_train(gosh_mlp *m, const gosh_csr *g_fine, const int32_t *map, const void *M_coarse,
                           const void *M_fine, int d, gosh_dtype dtype, int epochs, double lr, int batch,
                           int64_t max_rows, void *stream, double *final_loss);

/* M_fine[v] = M_coarse[map v] + MLP(f(v)) for every vertex of g_fine,
 * rounded to nearest in the storage type.  The hidden layer is rounded to
 * BF16.  For d in {32, 64, 128} and hidden width 128 or 256 both layers run
 * in one persistent tensor-core kernel per chunk of 2^18 vertices (the
 * hidden layer never leaves the SM); other shapes take two GEMMs.
 * Synchronous. */
gosh_status gosh_project_learned(gosh_mlp *m, const void *M_coarse, const int32_t *map,
                                 const gosh_csr *g_fine, void *M_fine, int d, gosh_dtype dtype,
                                 void *stream);

/*
 * GOSH (Alg. 2) end to end: coarsen g0 (unless params->max_levels == 1),
 * initialise M_{D-1}, then for i = D-1 .. 0 train level i for e_i epochs and,
 * for i > 0, project onto level i-1.  The epoch split gives a fraction p of
 * `epochs` uniformly to the D levels and the rest geometrically (each level
 * twice its finer neighbour): e_i = floor(p*e/D + (1-p)*e*2^i/(2^D-1)) for
 * i >= 1, e_0 = e - sum of the others.  Every level, level 0 included, is
 * trained.
 * g0: device CSR (on_device = 1) or host CSR (on_device = 0, copied in).
 * M0_out: n x d of params->dtype; device or host memory (host: copied out).
 * stats: host pointer or NULL.  Synchronous.
 */
gosh_status gosh_embed(const gosh_csr *g0, const gosh_params *params, void *M0_out,
                       void *stream, gosh_stats *stats);

/* The tensor-core (tcgen05) GEMM behind the learned projection, exported so
 * it can be verified on its own: C[m][n] = sum_k A[m][k] * B[n][k] for
 * m < M, n < N, with A (M x K) and B (N x K) BF16 row-major (row strides lda,
 * ldb elements, K contiguous) and C FP32 row-major (stride ldc).  K must be a
 * multiple of 16; strides keep rows 16-byte aligned.  splits > 1 splits K
 * over that many thread blocks per tile and ADDS into C (which must hold the
 * addend, e.g. zeros).  Synchronous; GOSH_ERR_TIMEOUT if an MMA completion
 * wait gave up. */
gosh_status gosh_tc_gemm_bf16(const void *A, int64_t lda, const void *B, int64_t ldb, float *C, int64_t ldc,
                              int M, int N, int K, int splits, void *stream);

typedef struct gosh_batch_stats {
    int graphs;                 /* graphs in the batch */
    int64_t phases;             /* scheduled phases (inits, epochs, projections) */
    int64_t level0_vertices;    /* sum of |V_0| */
    int lanes_per_row;          /* variant used (autotuned when params asked for 0) */
    int samples_per_pass;
    int sources_per_item;       /* sources (rows) per work item of a warp */
    int autotuned;              /* 1 if this call ran the autotuner */
    double coarsen_ms;          /* host wall time of the per-graph coarsening */
    double train_ms;            /* device time of the persistent launch */
    double total_ms;            /* wall time of the call */
    unsigned long long updates; /* UPDATEEMBED applications */
} gosh_batch_stats;

/*
 * Many independent graphs embedded at once (GOSH, Alg. 2, per graph): every
 * graph is coarsened (gosh_coarsen), then ALL graphs' levels are trained in
 * one persistent kernel launch, captured in a CUDA graph.  Each graph follows
 * its own schedule -- initialise M_{D-1}, the epochs of each level in order
 * (epochs serialised, Sec. 3.1), copy projection between levels -- while
 * different graphs proceed concurrently; warps take work items (chunks of
 * sources or rows) from whichever graph has work.  Graph g draws its samples
 * with Philox key (seed, graph_id + g), so its random stream is that of a
 * standalone gosh_embed with graph_id + g.
 * graphs: n_graphs device CSRs; M_out[g]: device n_g x d of params->dtype
 * (FP32 or BF16).  Lock-free mode only (GOSH_HOGWILD), copy projection.
 * params->lanes_per_row / samples_per_pass = 0 ask the autotuner to time the
 * compiled (lanes per row, samples per pass, sources per item) variants on
 * this batch once per (dtype, d, k) and keep the fastest (cached per
 * process).  A warp that finds no work for 4 s stops the launch with
 * GOSH_ERR_TIMEOUT.  stats: host pointer or NULL.  Synchronous.
 */
gosh_status gosh_embed_batch(int n_graphs, const gosh_csr *graphs, const gosh_params *params,
                             void *const *M_out, void *stream, gosh_batch_stats *stats);

/* Scores of vertex pairs, out[i] = M[pairs[2i]] . M[pairs[2i+1]] in FP32.
 * pairs: device int32[2*npairs]; out: device float[npairs]. */
gosh_status gosh_pair_scores(const void *M, int d, gosh_dtype dtype, const int32_t *pairs,
                             int64_t npairs, float *out, void *stream);

/* Link-prediction AUCROC (Sec. 6.1) with dot-product scores: the Mann-Whitney
 * statistic over the positive and negative pairs, a tie counting 1/2, summed
 * in FP64.  pos/neg: device int32[2*npos] / [2*nneg].  auc: host double.
 * Synchronous. */
gosh_status gosh_link_auc(const void *M, int d, gosh_dtype dtype, const int32_t *pos,
                          int64_t npos, const int32_t *neg, int64_t nneg, void *stream,
                          double *auc);

#ifdef __cplusplus
}
#endif

#endif /* GOSH_H */
