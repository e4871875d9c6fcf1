/*
 * Seeded synthetic graph generators.
 *
 * This module produces the input graphs that both the CPU oracle and the CUDA
 * path consume.  It holds none of the BFS arithmetic: it only draws random
 * numbers and assembles compressed sparse column (CSC) arrays.
 *
 * Layout of every result: column j lists the out-neighbours of vertex j
 * (the CSC of A^T, Section 7 and Section 9 of the paper), rows sorted
 * ascending within a column, duplicates and self-loops removed.  colptr has
 * n+1 entries, rowidx has nnz = colptr[n] entries, both uint32.
 *
 * Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014) used as a counter-based
 * generator: draw i of stream s under seed z is mix64(z, s, i).  Every draw is
 * therefore independent of thread count and of the order of evaluation.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    uint32_t n;
    uint64_t nnz;
    uint32_t* colptr; /* n+1 */
    uint32_t* rowidx; /* nnz */
} synth_csc;

enum { SYNTH_OK = 0, SYNTH_ERR_ARG = 1, SYNTH_ERR_OOM = 2 };

/* ---- SplitMix64 --------------------------------------------------------- */

static inline uint64_t sm64_next(uint64_t* state) {
    uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Starting state of stream `s`, element `i`: two SplitMix64 steps over a
 * combination of the three keys so that neighbouring counters decorrelate. */
static inline uint64_t sm64_seed(uint64_t seed, uint64_t s, uint64_t i) {
    uint64_t st = seed ^ (s * 0xD1B54A32D192ED03ull);
    uint64_t a = sm64_next(&st);
    st = a ^ (i * 0x9E3779B97F4A7C15ull);
    return sm64_next(&st);
}

/* 53-bit uniform in [0,1). */
static inline double u01(uint64_t x) { return (double)(x >> 11) * (1.0 / 9007199254740992.0); }

/* ---- edge list -> CSC ---------------------------------------------------- */

/* Builds the CSC from `m` arcs (src[e] -> dst[e]): column src[e] gets row
 * dst[e].  With `symmetrize`, the reverse arc is added too.  Arcs with an
 * endpoint >= n are dropped, as are self-loops and duplicates.  Takes
 * ownership of src and dst (frees them). */
static int csc_from_arcs(uint32_t n, uint64_t m, uint32_t* src, uint32_t* dst, int symmetrize,
                         synth_csc* out) {
    uint64_t m2 = symmetrize ? 2 * m : m;
    uint32_t* a_col = (uint32_t*)malloc((m2 ? m2 : 1) * sizeof(uint32_t));
    uint32_t* a_row = (uint32_t*)malloc((m2 ? m2 : 1) * sizeof(uint32_t));
    uint64_t* cnt = (uint64_t*)calloc((size_t)n + 1, sizeof(uint64_t));
    if (!a_col || !a_row || !cnt) {
        free(a_col); free(a_row); free(cnt); free(src); free(dst);
        return SYNTH_ERR_OOM;
    }
    uint64_t k = 0;
    for (uint64_t e = 0; e < m; ++e) {
        uint32_t u = src[e], v = dst[e];
        if (u >= n || v >= n || u == v) continue;
        a_col[k] = u; a_row[k] = v; ++k;
        if (symmetrize) { a_col[k] = v; a_row[k] = u; ++k; }
    }
    free(src); free(dst);
    m2 = k;

    /* Pass 1: stable counting sort by row. */
    uint32_t* b_col = (uint32_t*)malloc((m2 ? m2 : 1) * sizeof(uint32_t));
    uint32_t* b_row = (uint32_t*)malloc((m2 ? m2 : 1) * sizeof(uint32_t));
    if (!b_col || !b_row) {
        free(a_col); free(a_row); free(b_col); free(b_row); free(cnt);
        return SYNTH_ERR_OOM;
    }
    for (uint64_t e = 0; e < m2; ++e) cnt[a_row[e] + 1]++;
    for (uint32_t v = 0; v < n; ++v) cnt[v + 1] += cnt[v];
    for (uint64_t e = 0; e < m2; ++e) {
        uint64_t p = cnt[a_row[e]]++;
        b_col[p] = a_col[e]; b_row[p] = a_row[e];
    }
    /* Pass 2: stable counting sort by column; rows end up ascending. */
    memset(cnt, 0, ((size_t)n + 1) * sizeof(uint64_t));
    for (uint64_t e = 0; e < m2; ++e) cnt[b_col[e] + 1]++;
    for (uint32_t v = 0; v < n; ++v) cnt[v + 1] += cnt[v];
    for (uint64_t e = 0; e < m2; ++e) {
        uint64_t p = cnt[b_col[e]]++;
        a_row[p] = b_row[e];
        a_col[p] = b_col[e];
    }
    free(b_col); free(b_row);

    /* Dedup (columns are contiguous and rows sorted). */
    uint32_t* colptr = (uint32_t*)malloc(((size_t)n + 1) * sizeof(uint32_t));
    if (!colptr) { free(a_col); free(a_row); free(cnt); return SYNTH_ERR_OOM; }
    uint64_t w = 0, e = 0;
    for (uint32_t j = 0; j < n; ++j) {
        colptr[j] = (uint32_t)w;
        int have = 0;
        uint32_t last = 0;
        while (e < m2 && a_col[e] == j) {
            if (!have || a_row[e] != last) { a_row[w++] = a_row[e]; last = a_row[e]; have = 1; }
            ++e;
        }
    }
    colptr[n] = (uint32_t)w;
    free(a_col); free(cnt);
    if (w > 0xFFFFFFFFull) { free(colptr); free(a_row); return SYNTH_ERR_ARG; }
    uint32_t* rowidx = (uint32_t*)realloc(a_row, (w ? w : 1) * sizeof(uint32_t));
    if (!rowidx) rowidx = a_row;
    out->n = n; out->nnz = w; out->colptr = colptr; out->rowidx = rowidx;
    return SYNTH_OK;
}

/* ---- random permutation (Fisher-Yates on one SplitMix64 stream) ---------- */

static uint32_t* random_perm(uint32_t n, uint64_t seed) {
    uint32_t* p = (uint32_t*)malloc(((size_t)n ? n : 1) * sizeof(uint32_t));
    if (!p) return NULL;
    for (uint32_t i = 0; i < n; ++i) p[i] = i;
    uint64_t st = sm64_seed(seed, 0x5045524Dull /* "PERM" */, 0);
    for (uint32_t i = n; i > 1; --i) {
        /* Lemire's multiply-shift maps a 64-bit draw onto [0, i). */
        uint64_t r = sm64_next(&st);
        uint32_t j = (uint32_t)(((unsigned __int128)r * i) >> 64);
        uint32_t t = p[i - 1]; p[i - 1] = p[j]; p[j] = t;
    }
    return p;
}

/* ---- public generators -------------------------------------------------- */

void synth_free(synth_csc* g) {
    if (!g) return;
    free(g->colptr); free(g->rowidx);
    g->colptr = NULL; g->rowidx = NULL; g->n = 0; g->nnz = 0;
}

/* Undirected R-MAT (Chakrabarti, Zhan, Faloutsos 2004) with fixed quadrant
 * probabilities a,b,c (d = 1-a-b-c) and no per-level noise.
 * m = round(edgefactor * 2^scale) edges are drawn on 2^scale vertices; each
 * edge descends `scale` levels, one 53-bit draw per level.  With `permute`,
 * vertex labels go through a seeded random permutation.  Vertices >= n_keep
 * (after permutation) are dropped, which truncates the graph to n_keep
 * vertices (n_keep = 0 keeps all 2^scale). */
int synth_rmat(uint32_t scale, double edgefactor, double a, double b, double c, uint64_t seed,
               int permute, uint32_t n_keep, synth_csc* out) {
    if (!out || scale == 0 || scale > 30 || a < 0 || b < 0 || c < 0 || a + b + c > 1.0)
        return SYNTH_ERR_ARG;
    uint32_t nfull = 1u << scale;
    uint32_t n = n_keep ? n_keep : nfull;
    if (n > nfull) return SYNTH_ERR_ARG;
    uint64_t m = (uint64_t)llround(edgefactor * (double)nfull);
    uint32_t* src = (uint32_t*)malloc((m ? m : 1) * sizeof(uint32_t));
    uint32_t* dst = (uint32_t*)malloc((m ? m : 1) * sizeof(uint32_t));
    if (!src || !dst) { free(src); free(dst); return SYNTH_ERR_OOM; }
    const double ta = a, tab = a + b, tabc = a + b + c;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < (int64_t)m; ++e) {
        uint64_t st = sm64_seed(seed, 0x524D4154ull /* "RMAT" */, (uint64_t)e);
        uint32_t u = 0, v = 0;
        for (uint32_t l = 0; l < scale; ++l) {
            double r = u01(sm64_next(&st));
            uint32_t bu = r >= tab;                          /* quadrants c, d */
            uint32_t bv = (r >= ta && r < tab) || r >= tabc; /* quadrants b, d */
            u = (u << 1) | bu;
            v = (v << 1) | bv;
        }
        src[e] = u; dst[e] = v;
    }
    if (permute) {
        uint32_t* p = random_perm(nfull, seed);
        if (!p) { free(src); free(dst); return SYNTH_ERR_OOM; }
#pragma omp parallel for schedule(static)
        for (int64_t e = 0; e < (int64_t)m; ++e) { src[e] = p[src[e]]; dst[e] = p[dst[e]]; }
        free(p);
    }
    return csc_from_arcs(n, m, src, dst, 1, out);
}

/* Undirected Erdos-Renyi G(n,p) by geometric skipping over the pairs w < v
 * (Batagelj and Brandes, "Efficient generation of large random networks",
 * Phys. Rev. E 71, 2005).  One SplitMix64 stream supplies the skips. */
int synth_er(uint32_t n, double p, uint64_t seed, synth_csc* out) {
    if (!out || n == 0 || !(p >= 0.0) || p > 1.0) return SYNTH_ERR_ARG;
    uint64_t cap = (uint64_t)(p * 0.5 * (double)n * (double)(n - 1) * 1.2) + 1024;
    uint32_t* src = (uint32_t*)malloc(cap * sizeof(uint32_t));
    uint32_t* dst = (uint32_t*)malloc(cap * sizeof(uint32_t));
    if (!src || !dst) { free(src); free(dst); return SYNTH_ERR_OOM; }
    uint64_t m = 0;
    if (p > 0.0) {
        uint64_t st = sm64_seed(seed, 0x4552ull /* "ER" */, 0);
        double lq = log1p(-p);
        int64_t v = 1, w = -1;
        while (v < (int64_t)n) {
            double r = u01(sm64_next(&st));
            int64_t skip = (p >= 1.0) ? 0 : (int64_t)floor(log1p(-r) / lq);
            w += 1 + skip;
            while (w >= v && v < (int64_t)n) { w -= v; v += 1; }
            if (v < (int64_t)n) {
                if (m == cap) {
                    cap = cap * 2;
                    uint32_t* s2 = (uint32_t*)realloc(src, cap * sizeof(uint32_t));
                    uint32_t* d2 = (uint32_t*)realloc(dst, cap * sizeof(uint32_t));
                    if (!s2 || !d2) { free(s2 ? s2 : src); free(d2 ? d2 : dst); return SYNTH_ERR_OOM; }
                    src = s2; dst = d2;
                }
                src[m] = (uint32_t)v; dst[m] = (uint32_t)w; ++m;
            }
        }
    }
    return csc_from_arcs(n, m, src, dst, 1, out);
}

/* Undirected W x H 4-neighbour grid, row-major labels v = r*W + c. */
int synth_grid(uint32_t W, uint32_t H, synth_csc* out) {
    if (!out || W == 0 || H == 0) return SYNTH_ERR_ARG;
    uint64_t n64 = (uint64_t)W * H;
    if (n64 > 0xFFFFFFFEull) return SYNTH_ERR_ARG;
    uint32_t n = (uint32_t)n64;
    uint64_t nnz = 2ull * ((uint64_t)(W - 1) * H + (uint64_t)W * (H - 1));
    uint32_t* colptr = (uint32_t*)malloc(((size_t)n + 1) * sizeof(uint32_t));
    uint32_t* rowidx = (uint32_t*)malloc((nnz ? nnz : 1) * sizeof(uint32_t));
    if (!colptr || !rowidx) { free(colptr); free(rowidx); return SYNTH_ERR_OOM; }
    uint64_t k = 0;
    for (uint32_t r = 0; r < H; ++r) {
        for (uint32_t c = 0; c < W; ++c) {
            uint32_t v = r * W + c;
            colptr[v] = (uint32_t)k;
            if (r > 0) rowidx[k++] = v - W;
            if (c > 0) rowidx[k++] = v - 1;
            if (c + 1 < W) rowidx[k++] = v + 1;
            if (r + 1 < H) rowidx[k++] = v + W;
        }
    }
    colptr[n] = (uint32_t)k;
    out->n = n; out->nnz = k; out->colptr = colptr; out->rowidx = rowidx;
    return SYNTH_OK;
}

/* Directed k-nearest-neighbour random geometric graph: n points uniform in
 * the unit square (two 53-bit draws each), an arc from every point to its k
 * nearest other points by exact squared Euclidean distance, ties broken by
 * the smaller index.  Column p lists p's k nearest neighbours (its
 * out-arcs).  The search uses a uniform bucket grid with about two points per
 * cell and grows square rings of cells until no unvisited cell can hold a
 * closer point. */
int synth_rgg_knn(uint32_t n, uint32_t k, uint64_t seed, synth_csc* out) {
    if (!out || n < 2 || k == 0 || k >= n || k > 64) return SYNTH_ERR_ARG;
    double* x = (double*)malloc((size_t)n * sizeof(double));
    double* y = (double*)malloc((size_t)n * sizeof(double));
    uint32_t G = (uint32_t)floor(sqrt((double)n / 2.0));
    if (G < 1) G = 1;
    uint64_t ncell = (uint64_t)G * G;
    uint32_t* cstart = (uint32_t*)calloc(ncell + 1, sizeof(uint32_t));
    uint32_t* cidx = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
    uint32_t* pcell = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
    uint32_t* colptr = (uint32_t*)malloc(((size_t)n + 1) * sizeof(uint32_t));
    uint32_t* rowidx = (uint32_t*)malloc((size_t)n * k * sizeof(uint32_t));
    if (!x || !y || !cstart || !cidx || !pcell || !colptr || !rowidx) {
        free(x); free(y); free(cstart); free(cidx); free(pcell); free(colptr); free(rowidx);
        return SYNTH_ERR_OOM;
    }
    for (uint32_t i = 0; i < n; ++i) {
        uint64_t st = sm64_seed(seed, 0x524747ull /* "RGG" */, i);
        x[i] = u01(sm64_next(&st));
        y[i] = u01(sm64_next(&st));
        uint32_t cx = (uint32_t)(x[i] * G), cy = (uint32_t)(y[i] * G);
        if (cx >= G) cx = G - 1;
        if (cy >= G) cy = G - 1;
        pcell[i] = cy * G + cx;
        cstart[pcell[i] + 1]++;
    }
    for (uint64_t c = 0; c < ncell; ++c) cstart[c + 1] += cstart[c];
    {
        uint32_t* fill = (uint32_t*)malloc(ncell * sizeof(uint32_t));
        if (!fill) {
            free(x); free(y); free(cstart); free(cidx); free(pcell); free(colptr); free(rowidx);
            return SYNTH_ERR_OOM;
        }
        memcpy(fill, cstart, ncell * sizeof(uint32_t));
        for (uint32_t i = 0; i < n; ++i) cidx[fill[pcell[i]]++] = i; /* ascending i per cell */
        free(fill);
    }
    const double h = 1.0 / G;
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t ii = 0; ii < (int64_t)n; ++ii) {
        uint32_t i = (uint32_t)ii;
        double bd[64];
        uint32_t bi[64];
        uint32_t have = 0;
        int cx = (int)(pcell[i] % G), cy = (int)(pcell[i] / G);
        for (int r = 0;; ++r) {
            /* ring r: cells with Chebyshev distance r from (cx, cy) */
            for (int dy = -r; dy <= r; ++dy) {
                int yy = cy + dy;
                if (yy < 0 || yy >= (int)G) continue;
                int step = (dy == -r || dy == r) ? 1 : 2 * r;
                for (int dx = -r; dx <= r; dx += step) {
                    int xx = cx + dx;
                    if (xx < 0 || xx >= (int)G) continue;
                    uint32_t c = (uint32_t)yy * G + (uint32_t)xx;
                    for (uint32_t q = cstart[c]; q < cstart[c + 1]; ++q) {
                        uint32_t j = cidx[q];
                        if (j == i) continue;
                        double ddx = x[j] - x[i], ddy = y[j] - y[i];
                        double d = ddx * ddx + ddy * ddy;
                        /* insert into the sorted top-k list (distance, then index) */
                        if (have == k && (d > bd[k - 1] || (d == bd[k - 1] && j > bi[k - 1]))) continue;
                        uint32_t pos = have < k ? have : k - 1;
                        while (pos > 0 && (bd[pos - 1] > d || (bd[pos - 1] == d && bi[pos - 1] > j))) {
                            bd[pos] = bd[pos - 1]; bi[pos] = bi[pos - 1]; --pos;
                        }
                        bd[pos] = d; bi[pos] = j;
                        if (have < k) ++have;
                    }
                }
            }
            if (have == k) {
                /* every point outside rings 0..r lies at least this far away */
                double gx = fmin(x[i] - (cx - r) * h, (cx + r + 1) * h - x[i]);
                double gy = fmin(y[i] - (cy - r) * h, (cy + r + 1) * h - y[i]);
                double g = fmin(gx, gy);
                if (g * g > bd[k - 1]) break;
            }
            if (r > (int)G + 1) break;
        }
        /* column i: its k nearest, sorted ascending by index */
        for (uint32_t a = 1; a < k; ++a) {
            uint32_t t = bi[a];
            uint32_t b2 = a;
            while (b2 > 0 && bi[b2 - 1] > t) { bi[b2] = bi[b2 - 1]; --b2; }
            bi[b2] = t;
        }
        for (uint32_t a = 0; a < k; ++a) rowidx[(uint64_t)i * k + a] = bi[a];
    }
    for (uint32_t i = 0; i <= n; ++i) colptr[i] = i * k;
    free(x); free(y); free(cstart); free(cidx); free(pcell);
    out->n = n; out->nnz = (uint64_t)n * k; out->colptr = colptr; out->rowidx = rowidx;
    return SYNTH_OK;
}

/* CSC from caller-supplied arcs (copied), for hand-made test graphs. */
int synth_from_arcs(uint32_t n, uint64_t m, const uint32_t* src, const uint32_t* dst,
                    int symmetrize, synth_csc* out) {
    if (!out || (m && (!src || !dst))) return SYNTH_ERR_ARG;
    uint32_t* s = (uint32_t*)malloc((m ? m : 1) * sizeof(uint32_t));
    uint32_t* d = (uint32_t*)malloc((m ? m : 1) * sizeof(uint32_t));
    if (!s || !d) { free(s); free(d); return SYNTH_ERR_OOM; }
    if (m) { memcpy(s, src, m * sizeof(uint32_t)); memcpy(d, dst, m * sizeof(uint32_t)); }
    return csc_from_arcs(n, m, s, d, symmetrize, out);
}

/* Uniform draws for callers that need seeded choices (sources, batch
 * parameters): out[i] = 53-bit uniform in [0,1) of stream `stream`. */
void synth_uniform(uint64_t seed, uint64_t stream, uint64_t count, double* out) {
    for (uint64_t i = 0; i < count; ++i) {
        uint64_t st = sm64_seed(seed, stream, i);
        out[i] = u01(sm64_next(&st));
    }
}
