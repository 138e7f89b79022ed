/*
 * Multi-core CPU baseline of the per-level training step: Alg. 3 with
 * Alg. 1 (GOSH, arxiv 2110.10049), FP32 tables, lock-free ("Hogwild") over
 * all host threads with OpenMP -- the analogue of the paper's 16-thread CPU
 * comparison (Sec. 7, CPU vs GPU training).  Written for the host on its
 * own; it shares no code with the GPU library or with the FP64 oracle, and
 * serves only as a timed comparison point.
 *
 * Per epoch j every source v draws one positive (a uniform neighbour) and k
 * negatives (uniform over V, the source itself skipped) and applies
 * UPDATEEMBED to its private copy of M[v] and to each sample row in turn
 * (score = (b - sigmoid(x)) * lr', lr' = lr * max(1 - j/e, lr_floor)); the
 * source row is written back once.  Sample rows are updated in place without
 * locks, as in the paper's CPU and GPU designs.  Draws come from a
 * splitmix64 stream per (seed, epoch, source), not from the GPU's Philox:
 * this baseline times the step, it does not reproduce the GPU's samples.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

static inline uint64_t splitmix64(uint64_t *s) {
    uint64_t z = (*s += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* floor(w * n / 2^64) */
static inline uint64_t below(uint64_t w, uint64_t n) {
    return (uint64_t)(((unsigned __int128)w * n) >> 64);
}

int hogwild_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Trains M (n x d FP32, row-major, in place) for `epochs` epochs; returns
 * the number of UPDATEEMBED applications. */
int64_t hogwild_train_level(int64_t n, const int64_t *rowptr, const int32_t *col, float *M, int d, int k,
                            int epochs, double lr, double lr_floor, uint64_t seed) {
    int64_t total = 0;
    for (int j = 0; j < epochs; ++j) {
        const double f = 1.0 - (double)j / (double)epochs;
        const float lrj = (float)(lr * (f > lr_floor ? f : lr_floor));
        int64_t applied = 0;
#pragma omp parallel reduction(+ : applied)
        {
            float *r = (float *)malloc(sizeof(float) * (size_t)d);
#pragma omp for schedule(dynamic, 512)
            for (int64_t v = 0; v < n; ++v) {
                uint64_t st = seed ^ ((uint64_t)j << 40) ^ ((uint64_t)v * 0xd1342543de82ef95ULL);
                float *mv = M + v * (int64_t)d;
                memcpy(r, mv, sizeof(float) * (size_t)d);
                const int64_t deg = rowptr[v + 1] - rowptr[v];
                for (int t = 0; t <= k; ++t) {
                    const uint64_t w = splitmix64(&st);
                    int64_t u;
                    if (t == 0) {
                        if (deg == 0) continue;
                        u = col[rowptr[v] + (int64_t)below(w, (uint64_t)deg)];
                    } else {
                        u = (int64_t)below(w, (uint64_t)n);
                        if (u == v) continue;
                    }
                    float *mu = M + u * (int64_t)d;
                    float x = 0.f;
                    for (int c = 0; c < d; ++c) x += r[c] * mu[c];
                    const float g = ((t == 0 ? 1.f : 0.f) - 1.f / (1.f + expf(-x))) * lrj;
                    for (int c = 0; c < d; ++c) r[c] += g * mu[c];
                    for (int c = 0; c < d; ++c) mu[c] += g * r[c];
                    ++applied;
                }
                memcpy(mv, r, sizeof(float) * (size_t)d);
            }
            free(r);
        }
        total += applied;
    }
    return total;
}
