/*
 * rmatgen.c -- seeded synthetic inputs: R-MAT edge draws (Chakrabarti, Zhan,
 * Faloutsos, SDM 2004), symmetrise / dedup / compact into CSR, and the 80/20
 * link-prediction split of Sec. 6.1.  Input preparation only: nothing here
 * belongs to the embedding method.  Random numbers come from splitmix64
 * (Steele, Lea, Flood, OOPSLA 2014) keyed by (seed, index), so results do not
 * depend on the thread count.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static inline uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ULL;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
    return x ^ (x >> 31);
}

static inline double unit53(uint64_t x) { return (double)(x >> 11) * 0x1.0p-53; }

/* LSD radix sort of 64-bit keys on bits [0, bits), 16-bit digits. */
static void radix_sort_u64(uint64_t *a, uint64_t *tmp, int64_t n, int bits) {
    int64_t *cnt = (int64_t *)malloc(sizeof(int64_t) * 65536);
    uint64_t *src = a, *dst = tmp;
    for (int sh = 0; sh < bits; sh += 16) {
        memset(cnt, 0, sizeof(int64_t) * 65536);
        for (int64_t i = 0; i < n; ++i) cnt[(src[i] >> sh) & 0xffff]++;
        int64_t run = 0;
        for (int d = 0; d < 65536; ++d) { int64_t c = cnt[d]; cnt[d] = run; run += c; }
        for (int64_t i = 0; i < n; ++i) dst[cnt[(src[i] >> sh) & 0xffff]++] = src[i];
        uint64_t *t = src; src = dst; dst = t;
    }
    if (src != a) memcpy(a, src, sizeof(uint64_t) * (size_t)n);
    free(cnt);
}

static int bits_for(uint64_t x) { int b = 0; while (b < 64 && (1ULL << b) <= x) ++b; return b ? b : 1; }

/* m directed draws on 2^scale ids, then a seeded relabelling. */
void rmat_edges(int scale, int64_t m, uint64_t seed, double a, double b, double c,
                uint32_t *src, uint32_t *dst) {
    const double ab = a + b, abc = a + b + c;
    const uint64_t key = splitmix64(seed);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        uint64_t st = splitmix64(key ^ ((uint64_t)i * 0xD1342543DE82EF95ULL));
        uint32_t u = 0, v = 0;
        for (int l = 0; l < scale; ++l) {
            st = splitmix64(st);
            const double r = unit53(st);
            u = (u << 1) | (r >= ab);
            v = (v << 1) | ((r >= a && r < ab) || r >= abc);
        }
        src[i] = u;
        dst[i] = v;
    }
    const uint32_t nv = 1u << scale;
    uint32_t *perm = (uint32_t *)malloc(sizeof(uint32_t) * nv);
    for (uint32_t i = 0; i < nv; ++i) perm[i] = i;
    uint64_t st = splitmix64(key ^ 0x5EEDULL);
    for (uint32_t i = nv - 1; i > 0; --i) {
        st = splitmix64(st);
        const uint32_t j = (uint32_t)(((unsigned __int128)st * (i + 1)) >> 64);
        const uint32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) { src[i] = perm[src[i]]; dst[i] = perm[dst[i]]; }
    free(perm);
}

/*
 * Symmetrise, drop self-loops, dedup, optionally drop isolated vertices, CSR.
 * Pass 1 (rowptr == NULL): returns the compacted vertex count in *n_out and
 * the CSR size in *nnz_out and keeps the sorted keys internally in `work`
 * (caller-provided, 2m uint64 x 2).  Pass 2 fills rowptr/col/oldid.
 */
int64_t csr_build(int64_t n, int64_t m, const uint32_t *src, const uint32_t *dst, int compact,
                  uint64_t *work, int64_t *n_out, int64_t *rowptr, int32_t *col, int32_t *oldid) {
    uint64_t *keys = work, *tmp = work + 2 * m;
    int64_t k = 0;
    if (!rowptr) {
        for (int64_t i = 0; i < m; ++i) {
            if (src[i] == dst[i]) continue;
            keys[k++] = ((uint64_t)src[i] << 32) | dst[i];
            keys[k++] = ((uint64_t)dst[i] << 32) | src[i];
        }
        radix_sort_u64(keys, tmp, k, 32 + bits_for((uint64_t)n));
        int64_t w = 0;
        for (int64_t i = 0; i < k; ++i)
            if (i == 0 || keys[i] != keys[i - 1]) keys[w++] = keys[i];
        /* remember the unique count in tmp[0] */
        tmp[0] = (uint64_t)w;
        int64_t nn = n;
        if (compact) {
            nn = 0;
            for (int64_t i = 0; i < w; ++i)
                if (i == 0 || (keys[i] >> 32) != (keys[i - 1] >> 32)) ++nn;
        }
        *n_out = nn;
        return w;
    }
    const int64_t w = (int64_t)tmp[0];
    int32_t *newid = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int64_t nn = 0;
    if (compact) {
        for (int64_t v = 0; v < n; ++v) newid[v] = -1;
        for (int64_t i = 0; i < w; ++i) {
            const int64_t u = (int64_t)(keys[i] >> 32);
            if (newid[u] < 0) { newid[u] = (int32_t)nn; if (oldid) oldid[nn] = (int32_t)u; ++nn; }
        }
    } else {
        for (int64_t v = 0; v < n; ++v) { newid[v] = (int32_t)v; if (oldid) oldid[v] = (int32_t)v; }
        nn = n;
    }
    memset(rowptr, 0, sizeof(int64_t) * (size_t)(nn + 1));
    for (int64_t i = 0; i < w; ++i) {
        rowptr[newid[keys[i] >> 32] + 1]++;
        col[i] = newid[keys[i] & 0xffffffffu];
    }
    for (int64_t v = 0; v < nn; ++v) rowptr[v + 1] += rowptr[v];
    free(newid);
    *n_out = nn;
    return w;
}

static int has_edge(const int64_t *rowptr, const int32_t *col, int32_t u, int32_t v) {
    int64_t lo = rowptr[u], hi = rowptr[u + 1];
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (col[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo < rowptr[u + 1] && col[lo] == v;
}

/*
 * Link-prediction split of a simple symmetric CSR (n, rowptr, col).
 * Pass 1 (train_rowptr == NULL): chooses the test edges and returns the
 * training CSR size; *n_train and *n_test receive the sizes.  `work` holds
 * nnz/2 uint64 + n int32 + nnz/2 uint8 of scratch kept between the passes.
 * Pass 2 writes the training CSR (compacted ids), the held-out positives and
 * the same number of negatives (uniform pairs, u != v, not an edge of G).
 */
int64_t link_split(int64_t n, const int64_t *rowptr, const int32_t *col, uint64_t seed, double test_frac,
                   uint64_t *work, int64_t *n_train, int64_t *n_test,
                   int64_t *train_rowptr, int32_t *train_col, int32_t *test_pos, int32_t *test_neg) {
    const int64_t nnz = rowptr[n];
    const int64_t ne = nnz / 2;
    uint64_t *und = work;                                   /* undirected keys u<v, sorted */
    int32_t *newid = (int32_t *)(work + ne);                 /* [n] */
    uint8_t *is_test = (uint8_t *)(newid + n);               /* [ne] */
    const uint64_t key = splitmix64(seed ^ 0x11A7ULL);
    if (!train_rowptr) {
        int64_t k = 0;
        for (int64_t u = 0; u < n; ++u)
            for (int64_t p = rowptr[u]; p < rowptr[u + 1]; ++p)
                if (col[p] > u) und[k++] = ((uint64_t)u << 32) | (uint32_t)col[p];
        /* choose floor(test_frac * ne + 0.5) edges by a seeded partial shuffle of indices */
        const int64_t nt = (int64_t)(test_frac * (double)ne + 0.5);
        int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ne > 0 ? ne : 1));
        for (int64_t i = 0; i < ne; ++i) idx[i] = i;
        uint64_t st = key;
        for (int64_t i = 0; i < nt; ++i) {
            st = splitmix64(st);
            const int64_t j = i + (int64_t)(((unsigned __int128)st * (uint64_t)(ne - i)) >> 64);
            const int64_t t = idx[i]; idx[i] = idx[j]; idx[j] = t;
        }
        memset(is_test, 0, (size_t)ne);
        for (int64_t i = 0; i < nt; ++i) is_test[idx[i]] = 1;
        free(idx);
        /* training degrees */
        int64_t *deg = (int64_t *)calloc((size_t)n, sizeof(int64_t));
        for (int64_t i = 0; i < ne; ++i)
            if (!is_test[i]) { deg[und[i] >> 32]++; deg[und[i] & 0xffffffffu]++; }
        int64_t nn = 0, m2 = 0;
        for (int64_t v = 0; v < n; ++v) { newid[v] = deg[v] > 0 ? (int32_t)nn++ : -1; m2 += deg[v]; }
        int64_t ntest = 0;
        for (int64_t i = 0; i < ne; ++i)
            if (is_test[i] && newid[und[i] >> 32] >= 0 && newid[und[i] & 0xffffffffu] >= 0) ++ntest;
        free(deg);
        *n_train = nn;
        *n_test = ntest;
        return m2;
    }
    /* pass 2: training CSR in compacted ids (rows stay sorted: ids are monotone) */
    const int64_t nn = *n_train;
    memset(train_rowptr, 0, sizeof(int64_t) * (size_t)(nn + 1));
    /* walk the full CSR; an entry survives when its undirected edge is not a test edge */
    int64_t w = 0;
    for (int64_t u = 0; u < n; ++u) {
        if (newid[u] < 0) continue;
        for (int64_t p = rowptr[u]; p < rowptr[u + 1]; ++p) {
            const int32_t v = col[p];
            const uint64_t k2 = u < v ? (((uint64_t)u << 32) | (uint32_t)v) : (((uint64_t)v << 32) | (uint32_t)u);
            int64_t lo = 0, hi = ne;
            while (lo < hi) { const int64_t mid = (lo + hi) >> 1; if (und[mid] < k2) lo = mid + 1; else hi = mid; }
            if (is_test[lo]) continue;
            train_col[w++] = newid[v];
            train_rowptr[newid[u] + 1]++;
        }
    }
    for (int64_t v = 0; v < nn; ++v) train_rowptr[v + 1] += train_rowptr[v];
    int64_t t = 0;
    for (int64_t i = 0; i < ne; ++i) {
        if (!is_test[i]) continue;
        const int32_t a = newid[und[i] >> 32], b = newid[und[i] & 0xffffffffu];
        if (a < 0 || b < 0) continue;
        test_pos[2 * t] = a;
        test_pos[2 * t + 1] = b;
        ++t;
    }
    /* negatives over V_train: map back to full ids to test membership in G */
    int32_t *oldid = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nn > 0 ? nn : 1));
    for (int64_t v = 0; v < n; ++v) if (newid[v] >= 0) oldid[newid[v]] = (int32_t)v;
    uint64_t st = splitmix64(key ^ 0xBADULL);
    for (int64_t i = 0; i < t && nn > 1;) {
        st = splitmix64(st);
        const int32_t a = (int32_t)(((unsigned __int128)st * (uint64_t)nn) >> 64);
        st = splitmix64(st);
        const int32_t b = (int32_t)(((unsigned __int128)st * (uint64_t)nn) >> 64);
        if (a == b || has_edge(rowptr, col, oldid[a], oldid[b])) continue;
        test_neg[2 * i] = a;
        test_neg[2 * i + 1] = b;
        ++i;
    }
    free(oldid);
    return w;
}

/*
 * The same CSR as csr_build (symmetrised, self-loops dropped, deduplicated,
 * isolated vertices dropped when `compact`, rows ascending) for graphs of
 * billions of entries, in about a third of csr_build's memory and on all
 * threads: entries are bucketed by row with a counting sort (atomic row
 * cursors), then every row is sorted and deduplicated on its own.
 * csr_large_count: builds the rows in a handle, returns the CSR size and the
 * vertex count (*n_out); csr_large_fill copies them out and frees the handle.
 */
typedef struct {
    int64_t n, nn, nnz;
    int64_t *start;   /* [n+1] bucket starts */
    int64_t *uniq;    /* [n] unique entries per row */
    int32_t *ent;     /* [start[n]] bucketed entries, each row sorted and unique in front */
    int32_t *newid;   /* [n] */
} CsrLarge;

static int cmp_i32(const void *a, const void *b) {
    const int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

void *csr_large_count(int64_t n, int64_t m, const uint32_t *src, const uint32_t *dst, int compact,
                      int64_t *n_out, int64_t *nnz_out) {
    CsrLarge *h = (CsrLarge *)calloc(1, sizeof(CsrLarge));
    h->n = n;
    h->start = (int64_t *)calloc((size_t)(n + 1), sizeof(int64_t));
    h->uniq = (int64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
    h->newid = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        if (src[i] == dst[i]) continue;
        __atomic_fetch_add(&h->start[src[i] + 1], 1, __ATOMIC_RELAXED);
        __atomic_fetch_add(&h->start[dst[i] + 1], 1, __ATOMIC_RELAXED);
    }
    for (int64_t v = 0; v < n; ++v) h->start[v + 1] += h->start[v];
    h->ent = (int32_t *)malloc(sizeof(int32_t) * (size_t)(h->start[n] > 0 ? h->start[n] : 1));
    int64_t *cur = h->uniq; /* cursors (reused as unique counts below) */
#pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < n; ++v) cur[v] = h->start[v];
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        if (src[i] == dst[i]) continue;
        h->ent[__atomic_fetch_add(&cur[src[i]], 1, __ATOMIC_RELAXED)] = (int32_t)dst[i];
        h->ent[__atomic_fetch_add(&cur[dst[i]], 1, __ATOMIC_RELAXED)] = (int32_t)src[i];
    }
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t v = 0; v < n; ++v) {
        int32_t *row = h->ent + h->start[v];
        const int64_t len = h->start[v + 1] - h->start[v];
        qsort(row, (size_t)len, sizeof(int32_t), cmp_i32);
        int64_t w = 0;
        for (int64_t i = 0; i < len; ++i)
            if (i == 0 || row[i] != row[i - 1]) row[w++] = row[i];
        h->uniq[v] = w;
    }
    int64_t nn = 0, nnz = 0;
    for (int64_t v = 0; v < n; ++v) {
        h->newid[v] = (!compact || h->uniq[v] > 0) ? (int32_t)nn++ : -1;
        nnz += h->uniq[v];
    }
    h->nn = nn;
    h->nnz = nnz;
    *n_out = nn;
    *nnz_out = nnz;
    return h;
}

void csr_large_fill(void *handle, int64_t *rowptr, int32_t *col) {
    CsrLarge *h = (CsrLarge *)handle;
    rowptr[0] = 0;
    int64_t r = 0;
    for (int64_t v = 0; v < h->n; ++v)
        if (h->newid[v] >= 0) { rowptr[r + 1] = rowptr[r] + h->uniq[v]; ++r; }
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t v = 0; v < h->n; ++v) {
        if (h->newid[v] < 0) continue;
        const int32_t *row = h->ent + h->start[v];
        int32_t *out = col + rowptr[h->newid[v]];
        for (int64_t i = 0; i < h->uniq[v]; ++i) out[i] = h->newid[row[i]];
    }
    free(h->start);
    free(h->uniq);
    free(h->ent);
    free(h->newid);
    free(h);
}
