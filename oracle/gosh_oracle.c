/*
 * gosh_oracle.c -- plain, slow, single-threaded FP64 CPU oracle for the GOSH
 * per-level embedding step (arxiv 2110.10049).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant generator with the CUDA library; the only thing
 * the two sides have in common is the seeded input graph that the tests hand
 * to both.
 *
 * Every function follows one passage of the paper, cited next to it:
 *   Alg. 1  UPDATEEMBED                (Sec. 2)
 *   Alg. 3  TRAININGPU epoch loop      (Sec. 3.1)
 *   Alg. 4  MULTIEDGECOLLAPSE          (Sec. 4)
 *   Sec. 3  EXPANDEMBEDDING (copy projection), epoch split, lr decay
 *   Sec. 3.2 random-walk positive sampling (GOSHW)
 *   Sec. 6.1 link-prediction AUC protocol
 * Where the paper is silent the reading used is written beside the code.
 *
 * Compiled with -ffp-contract=off so that every a*b+c is two rounded
 * operations, exactly as written.
 *
 * Parity unpinned: lock-free (Hogwild) training beyond one warp with one
 * source per round, whose update order is not reproducible, is compared with
 * orc_train_sequential only through link-prediction AUC; LargeGraphGPU beyond
 * one part (orc_train_large) is pinned here on the CPU; the device runs the
 * kernels of part pairs on two streams that may overlap, so its default
 * schedule is compared with the resident step through AUC (with the kernels
 * on one stream, graphs whose part pairs fit one tile are compared with
 * orc_train_large itself).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* ------------------------------------------------------------------------ */
/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11).  Counter-based: out = f_key(counter).           */
/* ------------------------------------------------------------------------ */
#define PHILOX_M0 0xD2E7470EE14C6C93ULL
#define PHILOX_M1 0xCA5A826395121157ULL
#define PHILOX_W0 0x9E3779B97F4A7C15ULL /* golden ratio */
#define PHILOX_W1 0xBB67AE8584CAA73BULL /* sqrt(3) - 1 */

static void mul128(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo) {
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void orc_philox4x64(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4]) {
    uint64_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
        uint64_t hi0, lo0, hi1, lo1;
        mul128(PHILOX_M0, c0, &hi0, &lo0);
        mul128(PHILOX_M1, c2, &hi1, &lo1);
        uint64_t n0 = hi1 ^ c1 ^ k0;
        uint64_t n1 = lo1;
        uint64_t n2 = hi0 ^ c3 ^ k1;
        uint64_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform integer in [0, n) from a 64-bit word: floor(w * n / 2^64). */
static uint64_t uniform_below(uint64_t w, uint64_t n) {
    uint64_t hi, lo;
    mul128(w, n, &hi, &lo);
    return hi;
}

/* Stream tags: which use a Philox block serves (fourth counter word). */
enum { TAG_SAMPLE = 0, TAG_INIT = 1 };

/* The words used by source v in epoch `epoch` of level `level`:
 * counter (v, blk, level<<32 | epoch, TAG_SAMPLE), key (seed, graph). */
static void sample_words(uint64_t seed, uint64_t graph, int level, int epoch,
                         int64_t v, int nwords, uint64_t *w) {
    uint64_t key[2] = {seed, graph};
    for (int blk = 0; blk * 4 < nwords; ++blk) {
        uint64_t ctr[4] = {(uint64_t)v, (uint64_t)blk,
                           ((uint64_t)(uint32_t)level << 32) | (uint32_t)epoch, TAG_SAMPLE};
        uint64_t o[4];
        orc_philox4x64(ctr, key, o);
        for (int j = 0; j < 4 && blk * 4 + j < nwords; ++j) w[blk * 4 + j] = o[j];
    }
}

/*
 * The k+1 sample vertices of source v (Alg. 3, Sec. 3.1): word 0 draws the
 * positive uniformly from Gamma(v) (adjacency similarity, Q(u,v)=1 iff
 * (u,v) in E), words 1..k draw negatives uniformly over V_i.
 * Reading: a source without neighbours has no positive (u[0] = -1); a
 * negative equal to the source is skipped (u[t] = -1).  Neighbours are not
 * rejected as negatives (uniform noise).
 */
void orc_draw_samples(int64_t n, const int64_t *rowptr, const int32_t *col, int k,
                      int level, int epoch, uint64_t seed, uint64_t graph,
                      int64_t v, int32_t *u) {
    uint64_t w[64];
    sample_words(seed, graph, level, epoch, v, k + 1, w);
    int64_t deg = rowptr[v + 1] - rowptr[v];
    u[0] = deg > 0 ? col[rowptr[v] + (int64_t)uniform_below(w[0], (uint64_t)deg)] : -1;
    for (int t = 1; t <= k; ++t) {
        int64_t x = (int64_t)uniform_below(w[t], (uint64_t)n);
        u[t] = (x == v) ? -1 : (int32_t)x;
    }
}

/* ------------------------------------------------------------------------ */
/* Alg. 1 UPDATEEMBED and the NCE loss (Sec. 2).                              */
/* ------------------------------------------------------------------------ */
static double sigmoid(double x) { return 1.0 / (1.0 + exp(-x)); }

/* softplus(z) = log(1 + e^z), evaluated without overflow. */
static double softplus(double z) { return (z > 0 ? z : 0.0) + log1p(exp(-fabs(z))); }

/* Negative log-likelihood of one sample (Sec. 2): -log sigma(x) for a
 * positive (b = 1), -log sigma(-x) = -log(1 - sigma(x)) for a negative. */
double orc_sample_loss(double x, int b) { return b ? softplus(-x) : softplus(x); }

static double dot(const double *a, const double *b, int d) {
    double s = 0.0;
    for (int j = 0; j < d; ++j) s += a[j] * b[j];
    return s;
}

/*
 * One UPDATEEMBED (Alg. 1).  Reading of the first line: score = (b - sigma(x)) * lr
 * (the printed precedence would make the step ~1 regardless of lr).  The
 * second line updates M[v]; the third updates M[sample] with the UPDATED M[v],
 * literally in that order.  Returns x, the dot product before the update.
 */
double orc_update_embed(double *mv, double *mu, int d, int b, double lr) {
    double x = dot(mv, mu, d);
    double score = ((double)b - sigmoid(x)) * lr;
    for (int j = 0; j < d; ++j) {
        double step = mu[j] * score;
        mv[j] = mv[j] + step;
    }
    for (int j = 0; j < d; ++j) {
        double step = mv[j] * score;
        mu[j] = mu[j] + step;
    }
    return x;
}

/* lr' = lr * max(1 - j/e_i, floor) (Sec. 3, Alg. 3). */
double orc_epoch_lr(double lr, double lr_floor, int j, int e_i) {
    double f = 1.0 - (double)j / (double)e_i;
    return lr * (f > lr_floor ? f : lr_floor);
}

/*
 * TRAININGPU (Alg. 3) executed sequentially: for each epoch j, for each source
 * v in id order, one positive update (b = 1) then k negative updates (b = 0),
 * each an UPDATEEMBED on the current M.  M is |V| x d row-major FP64.
 * loss_per_epoch[j] (nullable) sums the NLL of every applied update, taken
 * from the pre-update dot product.  n_updates (nullable) counts applied
 * updates.
 */
void orc_train_sequential(int64_t n, const int64_t *rowptr, const int32_t *col,
                          double *M, int d, int k, int level, int epochs,
                          double lr, double lr_floor, uint64_t seed, uint64_t graph,
                          double *loss_per_epoch, int64_t *n_updates) {
    int32_t u[64];
    int64_t applied = 0;
    for (int j = 0; j < epochs; ++j) {
        double lrj = orc_epoch_lr(lr, lr_floor, j, epochs);
        double loss = 0.0;
        for (int64_t v = 0; v < n; ++v) {
            orc_draw_samples(n, rowptr, col, k, level, j, seed, graph, v, u);
            for (int t = 0; t <= k; ++t) {
                if (u[t] < 0) continue;
                double x = orc_update_embed(M + v * d, M + (int64_t)u[t] * d, d, t == 0, lrj);
                loss += orc_sample_loss(x, t == 0);
                ++applied;
            }
        }
        if (loss_per_epoch) loss_per_epoch[j] = loss;
    }
    if (n_updates) *n_updates = applied;
}

/*
 * Deterministic (snapshot) mode.  Not in the paper: it is the reproducible
 * counterpart of the lock-free epoch.  Sources are taken in batches of m
 * consecutive ids; S is M at the start of the batch.  Each source v of the
 * batch runs its k+1 UPDATEEMBEDs on private copies: r starts at S[v]; the
 * sample row starts at S[u] (or at this source's own updated copy of it when
 * the same u was already drawn earlier by v, so that m = 1 is exactly the
 * sequential epoch); the change of the sample row, c = score * r_new, is
 * recorded.  At the end of the batch every row x becomes
 *     base(x) + c_1 + c_2 + ...     (summed left to right)
 * with base(x) = r_x if x is a source of the batch, else S[x], and the
 * contributions to x taken in order of (source ascending, sample ascending).
 *
 * orc_det_batch applies one batch [b0, b1) whose samples are given:
 * samples[(v-b0)*(k+1) + t] is sample t of source v (t = 0 the positive,
 * b = 1; t >= 1 negatives, b = 0; -1 = skipped).  The NLL of every applied
 * update is added to *loss (nullable) in update order; *n_applied
 * (nullable) is incremented.
 */
void orc_det_batch(double *M, int d, int64_t b0, int64_t b1, int k, const int32_t *samples, double lrj,
                   double *loss, int64_t *n_applied) {
    const int64_t m = b1 - b0;
    int64_t applied = 0;
    /* M itself is the snapshot S: nothing writes M until the batch ends. */
    double *R = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1) * d);            /* r of each source */
    double *C = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1) * (k + 1) * d);  /* contributions */
    double *rows = (double *)malloc(sizeof(double) * (size_t)(k + 1) * d);                  /* private sample rows */
    for (int64_t v = b0; v < b1; ++v) {
        double *r = R + (v - b0) * d;
        memcpy(r, M + v * d, sizeof(double) * d);
        const int32_t *u = samples + (v - b0) * (k + 1);
        for (int t = 0; t <= k; ++t) {
            if (u[t] < 0) continue;
            double *row = rows + t * d;
            int prev = -1;
            for (int s = 0; s < t; ++s) if (u[s] == u[t]) prev = s;
            memcpy(row, prev >= 0 ? rows + prev * d : M + (int64_t)u[t] * d, sizeof(double) * d);
            double x = orc_update_embed(r, row, d, t == 0, lrj);
            /* the sample row received row + r_new * score: record r_new * score */
            double score = ((double)(t == 0) - sigmoid(x)) * lrj;
            double *c = C + ((v - b0) * (k + 1) + t) * d;
            for (int q = 0; q < d; ++q) c[q] = r[q] * score;
            if (loss) *loss += orc_sample_loss(x, t == 0);
            ++applied;
        }
    }
    /* write back: bases of the sources first, then contributions in order */
    for (int64_t v = b0; v < b1; ++v) memcpy(M + v * d, R + (v - b0) * d, sizeof(double) * d);
    for (int64_t i = 0; i < m * (k + 1); ++i) {
        int32_t x = samples[i];
        if (x < 0) continue;
        const double *c = C + i * d;
        for (int q = 0; q < d; ++q) M[(int64_t)x * d + q] = M[(int64_t)x * d + q] + c[q];
    }
    free(R); free(C); free(rows);
    if (n_applied) *n_applied += applied;
}

void orc_train_deterministic(int64_t n, const int64_t *rowptr, const int32_t *col,
                             double *M, int d, int k, int level, int epochs,
                             double lr, double lr_floor, uint64_t seed, uint64_t graph,
                             int64_t m, double *loss_per_epoch, int64_t *n_updates) {
    int64_t applied = 0;
    int32_t *tgt = (int32_t *)malloc(sizeof(int32_t) * (size_t)m * (k + 1));
    for (int j = 0; j < epochs; ++j) {
        double lrj = orc_epoch_lr(lr, lr_floor, j, epochs);
        double loss = 0.0;
        for (int64_t b0 = 0; b0 < n; b0 += m) {
            int64_t b1 = b0 + m < n ? b0 + m : n;
            for (int64_t v = b0; v < b1; ++v)
                orc_draw_samples(n, rowptr, col, k, level, j, seed, graph, v, tgt + (v - b0) * (k + 1));
            orc_det_batch(M, d, b0, b1, k, tgt, lrj, &loss, &applied);
        }
        if (loss_per_epoch) loss_per_epoch[j] = loss;
    }
    free(tgt);
    if (n_updates) *n_updates = applied;
}

/* ------------------------------------------------------------------------ */
/* Random initialisation of M_{D-1} (Alg. 2, "Randomly initialize"):         */
/* U(-0.5/d, 0.5/d) from Philox.  Element c of row v takes word c%4 of the   */
/* block with counter (v, c/4, level, TAG_INIT), key (seed, graph):          */
/*   x = ((w >> 11) * 2^-53 - 0.5) / d        (exact except the division)   */
/* ------------------------------------------------------------------------ */
void orc_init_uniform(int64_t n, int d, int level, uint64_t seed, uint64_t graph, double *M) {
    uint64_t key[2] = {seed, graph};
    for (int64_t v = 0; v < n; ++v) {
        for (int c0 = 0; c0 < d; c0 += 4) {
            uint64_t ctr[4] = {(uint64_t)v, (uint64_t)(c0 / 4), (uint64_t)(uint32_t)level, TAG_INIT};
            uint64_t o[4];
            orc_philox4x64(ctr, key, o);
            for (int j = 0; j < 4 && c0 + j < d; ++j) {
                double unit = (double)(o[j] >> 11) * 0x1.0p-53;
                M[v * d + c0 + j] = (unit - 0.5) / (double)d;
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Alg. 4 MULTIEDGECOLLAPSE, one level: SORT (ordering heuristic), then the */
/* greedy mapping with the hub^2 restriction.                                */
/* ------------------------------------------------------------------------ */

/*
 * SORT: counting sort by degree, larger neighbourhoods first.  Reading: the
 * sort is stable, so vertices of equal degree keep ascending id order.
 */
void orc_degree_order(int64_t n, const int64_t *rowptr, int32_t *order) {
    int64_t maxdeg = 0;
    for (int64_t v = 0; v < n; ++v) {
        int64_t dv = rowptr[v + 1] - rowptr[v];
        if (dv > maxdeg) maxdeg = dv;
    }
    int64_t *start = (int64_t *)calloc((size_t)maxdeg + 2, sizeof(int64_t));
    for (int64_t v = 0; v < n; ++v) start[rowptr[v + 1] - rowptr[v]]++;
    /* exclusive positions, highest degree first */
    int64_t pos = 0;
    for (int64_t dd = maxdeg; dd >= 0; --dd) {
        int64_t c = start[dd];
        start[dd] = pos;
        pos += c;
    }
    for (int64_t v = 0; v < n; ++v) order[start[rowptr[v + 1] - rowptr[v]]++] = (int32_t)v;
    free(start);
}

/*
 * The mapping loop of Alg. 4.  delta = |E_i| / |V_i| where |E_i| is the number
 * of CSR entries (both directions of each undirected edge), i.e. the average
 * degree.  "|Gamma(x)| <= delta" is evaluated exactly as deg(x) * |V_i| <= nnz_i.
 * Clusters are numbered by a counter in discovery order.
 * Returns |V_{i+1}|.
 */
int64_t orc_mec_map(int64_t n, const int64_t *rowptr, const int32_t *col, int32_t *map) {
    int64_t nnz = rowptr[n];
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    orc_degree_order(n, rowptr, order);
    for (int64_t v = 0; v < n; ++v) map[v] = -1;
    int64_t cluster = 0;
    for (int64_t i = 0; i < n; ++i) {
        int32_t v = order[i];
        if (map[v] != -1) continue;
        map[v] = (int32_t)cluster++;
        int64_t dv = rowptr[v + 1] - rowptr[v];
        int v_small = dv * n <= nnz;
        for (int64_t e = rowptr[v]; e < rowptr[v + 1]; ++e) {
            int32_t u = col[e];
            int64_t du = rowptr[u + 1] - rowptr[u];
            int u_small = du * n <= nnz;
            if (v_small || u_small) {
                if (map[u] == -1) map[u] = map[v];
            }
        }
    }
    free(order);
    return cluster;
}

static int cmp_u64(const void *a, const void *b) {
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/*
 * COARSEN(G_i, map_i) (Alg. 4): G_{i+1} has an edge (map u, map v) for every
 * edge (u, v) of G_i with map u != map v; duplicates collapse (the coarse
 * graph is simple and unweighted).  Output CSR rows hold neighbours in
 * ascending order.  col_out must hold nnz_i entries.  Returns nnz_{i+1}.
 */
int64_t orc_coarsen(int64_t n, const int64_t *rowptr, const int32_t *col,
                    const int32_t *map, int64_t nc, int64_t *rowptr_out, int32_t *col_out) {
    int64_t nnz = rowptr[n];
    uint64_t *pairs = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(nnz > 0 ? nnz : 1));
    int64_t m = 0;
    for (int64_t v = 0; v < n; ++v)
        for (int64_t e = rowptr[v]; e < rowptr[v + 1]; ++e) {
            uint32_t a = (uint32_t)map[v], b = (uint32_t)map[col[e]];
            if (a != b) pairs[m++] = ((uint64_t)a << 32) | b;
        }
    qsort(pairs, (size_t)m, sizeof(uint64_t), cmp_u64);
    int64_t w = 0;
    for (int64_t i = 0; i < m; ++i)
        if (i == 0 || pairs[i] != pairs[i - 1]) pairs[w++] = pairs[i];
    for (int64_t c = 0; c <= nc; ++c) rowptr_out[c] = 0;
    for (int64_t i = 0; i < w; ++i) {
        rowptr_out[(pairs[i] >> 32) + 1]++;
        col_out[i] = (int32_t)(pairs[i] & 0xffffffffu);
    }
    for (int64_t c = 0; c < nc; ++c) rowptr_out[c + 1] += rowptr_out[c];
    free(pairs);
    return w;
}

/* EXPANDEMBEDDING (Alg. 2, Sec. 3): M_i[v] = M_{i+1}[map_i[v]]. */
void orc_project_copy(int64_t n_fine, const int32_t *map, const double *Mc, double *Mf, int d) {
    for (int64_t v = 0; v < n_fine; ++v)
        memcpy(Mf + v * d, Mc + (int64_t)map[v] * d, sizeof(double) * d);
}

/* ------------------------------------------------------------------------ */
/* Link-prediction scores and AUCROC (Sec. 6.1).  Reading: the score of a    */
/* pair is the dot product M[u].M[v]; the AUC is the Mann-Whitney statistic */
/* U / (n+ n-), a tie counting one half.                                      */
/* ------------------------------------------------------------------------ */
void orc_pair_scores(const double *M, int d, int64_t npairs, const int32_t *pairs, double *out) {
    for (int64_t i = 0; i < npairs; ++i)
        out[i] = dot(M + (int64_t)pairs[2 * i] * d, M + (int64_t)pairs[2 * i + 1] * d, d);
}

typedef struct { double s; int pos; } scored;
static int cmp_scored(const void *a, const void *b) {
    double x = ((const scored *)a)->s, y = ((const scored *)b)->s;
    return x < y ? -1 : (x > y ? 1 : 0);
}

double orc_auc(int64_t npos, const double *pos, int64_t nneg, const double *neg) {
    int64_t tot = npos + nneg;
    scored *a = (scored *)malloc(sizeof(scored) * (size_t)(tot > 0 ? tot : 1));
    for (int64_t i = 0; i < npos; ++i) { a[i].s = pos[i]; a[i].pos = 1; }
    for (int64_t i = 0; i < nneg; ++i) { a[npos + i].s = neg[i]; a[npos + i].pos = 0; }
    qsort(a, (size_t)tot, sizeof(scored), cmp_scored);
    /* walk tie groups: each positive gains (#neg strictly below) + 0.5 (#neg tied) */
    double U = 0.0;
    int64_t neg_below = 0;
    for (int64_t i = 0; i < tot;) {
        int64_t j = i, gp = 0, gn = 0;
        while (j < tot && a[j].s == a[i].s) { if (a[j].pos) ++gp; else ++gn; ++j; }
        U += (double)gp * ((double)neg_below + 0.5 * (double)gn);
        neg_below += gn;
        i = j;
    }
    free(a);
    return U / ((double)npos * (double)nneg);
}

/* ------------------------------------------------------------------------ */
/* Random-walk sampling (Sec. 3.2, GOSHW): positive pairs from walks.        */
/* The paper gives neither the walk length l nor the distance g, nor how the */
/* walks are drawn and shuffled.  Readings:                                  */
/*  - each epoch starts one walk of l vertices at every vertex v; step t      */
/*    moves to a uniform neighbour of w_t (Philox block (v, t/4, level<<32 |  */
/*    epoch, TAG_WALK), word t%4); a vertex without neighbours ends the walk; */
/*  - every pair (w_i, w_j) with 0 < j - i <= g is a positive (source w_i);  */
/*    the pairs of a full walk are ranked i ascending, then j ascending, and */
/*    pair rank r of the walk from v sits at position v*W + r (W = pairs of a */
/*    full walk); positions past the end of a shorter walk, and pairs whose   */
/*    two ends are the same vertex, are holes (no update);                   */
/*  - "shuffled": the epoch visits the positions in the order of a pseudo-    */
/*    random permutation (a 4-round Feistel network on 2h-bit words,          */
/*    2^(2h) >= P, round function lowbias32(x ^ key_r) & (2^h - 1), applied   */
/*    again until the value is below P);                                     */
/*  - each positive comes with k negatives uniform over V (Philox block      */
/*    (position, blk, level<<32 | epoch, TAG_WALK_NEG), words 1..k; word 0   */
/*    unused); a negative equal to the source is skipped.                    */
/* ------------------------------------------------------------------------ */
enum { TAG_WALK = 4, TAG_WALK_NEG = 5 };

/* lowbias32 (C. Wellons, hash-prospector): xorshift-multiply integer hash. */
static uint32_t lowbias32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}

/* pairs of a walk of l vertices with window g */
int64_t orc_walk_pairs_per_walk(int l, int g) {
    int64_t w = 0;
    for (int i = 0; i + 1 < l; ++i) w += (l - 1 - i) < g ? (l - 1 - i) : g;
    return w;
}

/* Walk of up to l vertices from v; returns its length. */
static int walk_from(const int64_t *rowptr, const int32_t *col, int64_t v, int l, int level, int epoch,
                     uint64_t seed, uint64_t graph, int32_t *w) {
    uint64_t key[2] = {seed, graph};
    uint64_t words[4];
    w[0] = (int32_t)v;
    int len = 1;
    for (int t = 0; t + 1 < l; ++t) {
        if (t % 4 == 0) {
            uint64_t ctr[4] = {(uint64_t)v, (uint64_t)(t / 4),
                               ((uint64_t)(uint32_t)level << 32) | (uint32_t)epoch, TAG_WALK};
            orc_philox4x64(ctr, key, words);
        }
        int64_t cur = w[t];
        int64_t deg = rowptr[cur + 1] - rowptr[cur];
        if (deg == 0) break;
        w[t + 1] = col[rowptr[cur] + (int64_t)uniform_below(words[t % 4], (uint64_t)deg)];
        ++len;
    }
    return len;
}

/* The epoch's position table: pairs[2*pos] = source (or -1 for a hole),
 * pairs[2*pos+1] = positive.  n*W positions. */
void orc_walk_pairs(int64_t n, const int64_t *rowptr, const int32_t *col, int l, int g, int level, int epoch,
                    uint64_t seed, uint64_t graph, int32_t *pairs) {
    const int64_t W = orc_walk_pairs_per_walk(l, g);
    int32_t *w = (int32_t *)malloc(sizeof(int32_t) * (size_t)l);
    for (int64_t v = 0; v < n; ++v) {
        int len = walk_from(rowptr, col, v, l, level, epoch, seed, graph, w);
        int64_t r = 0;
        for (int i = 0; i + 1 < l; ++i)
            for (int j = i + 1; j < l && j - i <= g; ++j, ++r) {
                int32_t *pp = pairs + 2 * (v * W + r);
                if (j < len && w[i] != w[j]) {
                    pp[0] = w[i];
                    pp[1] = w[j];
                } else {
                    pp[0] = -1;
                    pp[1] = -1;
                }
            }
    }
    free(w);
}

/* Permutation key of an epoch, and the permutation itself. */
uint32_t orc_walk_perm_key(uint64_t seed, uint64_t graph, int level, int epoch) {
    uint32_t k = lowbias32((uint32_t)seed ^ ((uint32_t)level << 24));
    k = lowbias32(k ^ (uint32_t)(seed >> 32) ^ (uint32_t)epoch);
    return lowbias32(k ^ lowbias32((uint32_t)graph ^ (uint32_t)(graph >> 32)));
}

uint64_t orc_walk_perm(uint64_t i, uint64_t P, uint32_t key) {
    int h = 1;
    while (((uint64_t)1 << (2 * h)) < P) ++h;
    const uint32_t mask = h >= 32 ? 0xffffffffU : (((uint32_t)1 << h) - 1);
    uint64_t x = i;
    do {
        uint32_t lo = (uint32_t)(x & mask), hi = (uint32_t)(x >> h);
        for (uint32_t r = 0; r < 4; ++r) {
            uint32_t f = lowbias32(lo ^ lowbias32(key + r)) & mask;
            uint32_t t = hi ^ f;
            hi = lo;
            lo = t;
        }
        x = ((uint64_t)hi << h) | lo;
    } while (x >= P);
    return x;
}

/* Sequential epochs of walk-based positives (Alg. 1 per sample, the epoch
 * visiting the positions in permuted order). */
void orc_train_walks(int64_t n, const int64_t *rowptr, const int32_t *col, double *M, int d, int k, int level,
                     int epochs, double lr, double lr_floor, uint64_t seed, uint64_t graph, int l, int g,
                     double *loss_per_epoch, int64_t *n_updates) {
    const int64_t W = orc_walk_pairs_per_walk(l, g);
    const uint64_t P = (uint64_t)(n * W);
    int32_t *pairs = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)(P > 0 ? P : 1));
    uint64_t key[2] = {seed, graph};
    int64_t applied = 0;
    for (int j = 0; j < epochs; ++j) {
        double lrj = orc_epoch_lr(lr, lr_floor, j, epochs);
        double loss = 0.0;
        orc_walk_pairs(n, rowptr, col, l, g, level, j, seed, graph, pairs);
        const uint32_t pk = orc_walk_perm_key(seed, graph, level, j);
        for (uint64_t i = 0; i < P; ++i) {
            const uint64_t q = orc_walk_perm(i, P, pk);
            const int32_t src = pairs[2 * q], pos = pairs[2 * q + 1];
            if (src < 0) continue;
            uint64_t w[64];
            for (int blk = 0; blk * 4 < k + 1; ++blk) {
                uint64_t ctr[4] = {q, (uint64_t)blk, ((uint64_t)(uint32_t)level << 32) | (uint32_t)j, TAG_WALK_NEG};
                orc_philox4x64(ctr, key, w + 4 * blk);
            }
            for (int t = 0; t <= k; ++t) {
                int64_t u;
                if (t == 0) {
                    u = pos;
                } else {
                    u = (int64_t)uniform_below(w[t], (uint64_t)n);
                    if (u == src) continue;
                }
                double x = orc_update_embed(M + (int64_t)src * d, M + u * d, d, t == 0, lrj);
                loss += orc_sample_loss(x, t == 0);
                ++applied;
            }
        }
        if (loss_per_epoch) loss_per_epoch[j] = loss;
    }
    free(pairs);
    if (n_updates) *n_updates = applied;
}

/* ------------------------------------------------------------------------ */
/* LargeGraphGPU (Sec. 5), run sequentially.  Readings (the section gives    */
/* the pair schedule and the sampling rule, not the streams):                */
/*  - V is cut into K contiguous parts, part i = [floor(n i/K), floor(n(i+1)/K));*/
/*  - rounds r = 0 .. ceil(e/B)-1; each round visits the part pairs (a, b),   */
/*    a >= b, in row-major lower-triangle order (Sec. 5.1);                  */
/*  - in pair (a, b) the sources are the vertices of V^a, then (a != b) those */
/*    of V^b, in id order; a source u draws B positives uniformly from its    */
/*    neighbours in the opposite part, each followed by k negatives uniform   */
/*    over the opposite part (a negative equal to u is skipped when a == b);  */
/*    positive j of round r uses Philox block (u, blk, level<<32 | (r*B+j),   */
/*    tag) with tag = TAG_SAMPLE for K = 1, else 3 | ((a*K+b) << 8), word 0   */
/*    for the positive and words 1..k for the negatives, and the rate         */
/*    lr * max(1 - (r*B+j)/e, lr_floor);                                      */
/*  - "a global counter" of positive updates bounds the work at e*|V|: the   */
/*    count rises by one with every positive applied, and once it has        */
/*    reached e*|V| every later slot group (a positive with its negatives)   */
/*    is dropped.  A source without a neighbour in the opposite part has no  */
/*    positive; its negatives are applied while the count is below the cap. */
/* ------------------------------------------------------------------------ */
enum { TAG_LARGE = 3 };

/* The positives that pair (a, b) of round r draws for each of its sources
 * (V^a, then V^b when a != b): out[s*B + j] = the local id (in the opposite
 * part) of the positive of slot group j, drawn as orc_train_large draws it,
 * or -1 when the source has no neighbour in the opposite part.  (Sec. 5
 * draws these on the host and sends them as sample pools.) */
void orc_large_pool(int64_t n, const int64_t *rowptr, const int32_t *col, int K, int a, int b, int r, int B,
                    int level, uint64_t seed, uint64_t graph, int32_t *out) {
    uint64_t key[2] = {seed, graph};
    const uint64_t tag = K == 1 ? (uint64_t)TAG_SAMPLE : ((uint64_t)TAG_LARGE | ((uint64_t)(a * K + b) << 8));
    const int64_t a0 = n * a / K, a1 = n * (a + 1) / K, b0 = n * b / K, b1 = n * (b + 1) / K;
    int64_t s = 0;
    for (int side = 0; side < (a == b ? 1 : 2); ++side) {
        const int64_t own0 = side == 0 ? a0 : b0, own1 = side == 0 ? a1 : b1;
        const int64_t opp0 = side == 0 ? b0 : a0, opp1 = side == 0 ? b1 : a1;
        for (int64_t ug = own0; ug < own1; ++ug, ++s) {
            int64_t lo = rowptr[ug], hi = rowptr[ug + 1];
            while (lo < hi && col[lo] < opp0) ++lo;
            int64_t e = lo;
            while (e < hi && col[e] < opp1) ++e;
            for (int j = 0; j < B; ++j) {
                if (e == lo) {
                    out[s * B + j] = -1;
                    continue;
                }
                uint64_t w[4];
                uint64_t ctr[4] = {(uint64_t)ug, 0, ((uint64_t)(uint32_t)level << 32) | (uint32_t)(r * B + j), tag};
                orc_philox4x64(ctr, key, w);
                out[s * B + j] = (int32_t)(col[lo + (int64_t)uniform_below(w[0], (uint64_t)(e - lo))] - opp0);
            }
        }
    }
}

void orc_train_large(int64_t n, const int64_t *rowptr, const int32_t *col, double *M, int d, int k, int level,
                     int epochs, double lr, double lr_floor, uint64_t seed, uint64_t graph, int K, int B,
                     int64_t *n_updates, int64_t *n_positives) {
    uint64_t key[2] = {seed, graph};
    const int rounds = (epochs + B - 1) / B;
    const uint64_t cap = (uint64_t)epochs * (uint64_t)n;
    uint64_t count = 0;  /* positives applied */
    int64_t applied = 0;
    int64_t *start = (int64_t *)malloc(sizeof(int64_t) * (size_t)(K + 1));
    for (int i = 0; i <= K; ++i) start[i] = n * i / K;
    for (int r = 0; r < rounds; ++r) {
        for (int a = 0; a < K; ++a) {
            for (int b = 0; b <= a; ++b) {
                const int same = a == b;
                const uint64_t tag = K == 1 ? (uint64_t)TAG_SAMPLE : ((uint64_t)TAG_LARGE | ((uint64_t)(a * K + b) << 8));
                for (int side = 0; side < (same ? 1 : 2); ++side) {
                    /* side 0: sources in V^a against V^b; side 1: V^b against V^a */
                    const int64_t own0 = side == 0 ? start[a] : start[b], own1 = side == 0 ? start[a + 1] : start[b + 1];
                    const int64_t opp0 = side == 0 ? start[b] : start[a], opp1 = side == 0 ? start[b + 1] : start[a + 1];
                    for (int64_t ug = own0; ug < own1; ++ug) {
                        const int64_t u = ug - own0;
                        /* neighbours of ug inside the opposite part: a sorted sub-range of its row */
                        int64_t lo = rowptr[ug], hi = rowptr[ug + 1];
                        while (lo < hi && col[lo] < opp0) ++lo;
                        int64_t e = lo;
                        while (e < hi && col[e] < opp1) ++e;
                        const int64_t cnt = e - lo;
                        for (int j = 0; j < B; ++j) {
                            if (count >= cap) continue;  /* budget spent: the group is dropped */
                            const uint32_t t = (uint32_t)(r * B + j);
                            const double lrt = orc_epoch_lr(lr, lr_floor, (int)t, epochs);
                            uint64_t w[64];
                            for (int blk = 0; blk * 4 < k + 1; ++blk) {
                                uint64_t ctr[4] = {(uint64_t)ug, (uint64_t)blk, ((uint64_t)(uint32_t)level << 32) | t, tag};
                                orc_philox4x64(ctr, key, w + 4 * blk);
                            }
                            if (cnt > 0) {
                                const int64_t v = col[lo + (int64_t)uniform_below(w[0], (uint64_t)cnt)];
                                orc_update_embed(M + ug * d, M + v * d, d, 1, lrt);
                                ++applied;
                                ++count;
                            }
                            for (int m = 1; m <= k; ++m) {
                                const int64_t x = (int64_t)uniform_below(w[m], (uint64_t)(opp1 - opp0));
                                if (same && x == u) continue;
                                orc_update_embed(M + ug * d, M + (opp0 + x) * d, d, 0, lrt);
                                ++applied;
                            }
                        }
                    }
                }
            }
        }
    }
    free(start);
    if (n_updates) *n_updates = applied;
    if (n_positives) *n_positives = (int64_t)count;
}
