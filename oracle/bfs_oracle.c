/*
 * CPU oracle for the algebraic BFS -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * call this code.  It shares nothing with the CUDA path.  It is plain,
 * sequential and written for obvious correctness, not speed.
 *
 * Input layout: CSC with column j = out-neighbours of j (the CSC of A^T;
 * Section 7 uses A^T for directed graphs), colptr[n+1], rowidx[nnz].
 *
 * Result definition (the textbook BFS that Theorem 1 shows the submatrix
 * recurrence reaches):
 *   level[v]  = hop distance from src along arcs j -> i, or -1 if unreachable;
 *   parent[v] = min{ j : i = v in column j, level[j] = level[v] - 1 };
 *   parent[src] = src; parent[v] = -1 if v is unreachable.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static int cmp_u32(const void* a, const void* b) {
    uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
    return (x > y) - (x < y);
}

/*
 * Moore's level-by-level queue BFS (Section 4).  Each level's frontier is
 * sorted ascending before it is expanded, so the first frontier vertex that
 * reaches a new vertex is its smallest-index predecessor on the previous
 * level: that first discovery is exactly the min-index parent.
 *
 * fsizes (optional, length >= n+1) receives the size of frontier k at [k].
 * Returns the number of non-empty frontiers (eccentricity of src + 1),
 * or -1 on a bad argument.
 */
int64_t oracle_bfs_queue(uint32_t n, const uint32_t* colptr, const uint32_t* rowidx, uint32_t src,
                         int32_t* level, int32_t* parent, uint32_t* fsizes) {
    if (src >= n) return -1;
    uint32_t* q = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
    if (!q) return -1;
    for (uint32_t v = 0; v < n; ++v) { level[v] = -1; parent[v] = -1; }
    level[src] = 0;
    parent[src] = (int32_t)src;
    q[0] = src;
    uint64_t head = 0, tail = 1;
    int64_t k = 0;
    while (head < tail) {
        uint64_t end = tail;
        qsort(q + head, (size_t)(end - head), sizeof(uint32_t), cmp_u32);
        if (fsizes) fsizes[k] = (uint32_t)(end - head);
        for (uint64_t t = head; t < end; ++t) {
            uint32_t j = q[t];
            for (uint32_t e = colptr[j]; e < colptr[j + 1]; ++e) {
                uint32_t i = rowidx[e];
                if (level[i] == -1) {
                    level[i] = (int32_t)(k + 1);
                    parent[i] = (int32_t)j;
                    q[tail++] = i;
                }
            }
        }
        head = end;
        ++k;
    }
    free(q);
    return k;
}

/*
 * Parents recomputed from the levels by scanning every stored entry:
 * for each entry j -> i with level[i] = level[j] + 1, parent[i] = min j.
 * A cross-check of the queue BFS that does not depend on visiting order.
 */
void oracle_parent_by_scan(uint32_t n, const uint32_t* colptr, const uint32_t* rowidx,
                           const int32_t* level, int32_t* parent) {
    for (uint32_t v = 0; v < n; ++v) parent[v] = (level[v] == 0) ? (int32_t)v : -1;
    for (uint32_t j = 0; j < n; ++j) {
        if (level[j] < 0) continue;
        for (uint32_t e = colptr[j]; e < colptr[j + 1]; ++e) {
            uint32_t i = rowidx[e];
            if (level[i] == level[j] + 1 && (parent[i] < 0 || (uint32_t)parent[i] > j))
                parent[i] = (int32_t)j;
        }
    }
}

/*
 * Algebraic operation counts of Section 11 (Table 2), measured by running
 * each method's loop and counting two operations per semiring (+,x) pair.
 *
 * out[0] Algorithm 2 (sequential CSR submatrix BFS): a row is multiplied only
 *        while it is unvisited and is marked visited at once, so one nonzero
 *        per reached row is used.  Reading of the garbled loop bound
 *        "j = L[start] .. L[end]": each j in L[start .. end-1].
 * out[1] the all-nonzero variant of Algorithm 2 (Section 9): test T[j] before
 *        scanning column j and do not mark rows during the scan, so every
 *        nonzero of the shrinking submatrix is multiplied once.
 * out[2] masked SpMSpV BFS: every nonzero of every frontier column is
 *        multiplied, and the visited test comes after the multiply.
 * out[3] SpMV BFS: every stored nonzero is multiplied at every step, until a
 *        step finds no new vertex.
 * out[4] number of reached vertices n_c; out[5] nnz_c = sum of the reached
 *        columns' lengths; out[6] number of non-empty frontiers.
 * Returns 0, or -1 on a bad argument / allocation failure.
 */
int oracle_op_counts(uint32_t n, const uint32_t* colptr, const uint32_t* rowidx, uint32_t src,
                     uint64_t* out) {
    if (src >= n) return -1;
    uint8_t* T = (uint8_t*)calloc(n, 1);
    uint32_t* L = (uint32_t*)malloc(((size_t)n + 1) * sizeof(uint32_t));
    uint64_t nnz = colptr[n];
    if (!T || !L) { free(T); free(L); return -1; }

    /* Algorithm 2.  x values are implicit (Boolean), so only the counting of
     * the multiply-add on line "y(col[i]) <- y(col[i]) + nz[i] * x(j)"
     * remains. */
    uint64_t ops = 0;
    uint64_t start = 0, end = 1, z = 1;
    L[0] = src;
    T[src] = 1; /* Algorithm 1 removes the source before the first step */
    while (start < end) {
        for (uint64_t t = start; t < end; ++t) {
            uint32_t j = L[t];
            for (uint32_t e = colptr[j]; e < colptr[j + 1]; ++e) {
                uint32_t i = rowidx[e];
                if (T[i] == 0) {
                    ops += 2;
                    L[z++] = i;
                    T[i] = 1;
                }
            }
            T[j] = 1;
        }
        start = end;
        end = z;
    }
    out[0] = ops;
    uint64_t n_c = z;

    /* nnz_c and the frontier count from a plain level pass. */
    int32_t* lev = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    uint32_t* q = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
    if (!lev || !q) { free(T); free(L); free(lev); free(q); return -1; }
    for (uint32_t v = 0; v < n; ++v) lev[v] = -1;
    lev[src] = 0;
    q[0] = src;
    uint64_t head = 0, tail = 1, nnz_c = 0, levels = 0, spmm = 0;
    while (head < tail) {
        uint64_t stop = tail;
        for (uint64_t t = head; t < stop; ++t) {
            uint32_t j = q[t];
            nnz_c += colptr[j + 1] - colptr[j];
            for (uint32_t e = colptr[j]; e < colptr[j + 1]; ++e) {
                uint32_t i = rowidx[e];
                spmm += 2; /* multiply first ... */
                if (lev[i] == -1) { /* ... then apply the visited mask */
                    lev[i] = lev[j] + 1;
                    q[tail++] = i;
                }
            }
        }
        head = stop;
        ++levels;
    }
    out[2] = spmm;
    out[3] = 2 * nnz * levels;
    out[4] = n_c;
    out[5] = nnz_c;
    out[6] = levels;

    /* All-nonzero variant of Algorithm 2. */
    memset(T, 0, n);
    uint32_t* L2 = (uint32_t*)malloc((nnz + 1) * sizeof(uint32_t));
    if (!L2) { free(T); free(L); free(lev); free(q); return -1; }
    uint64_t ops2 = 0;
    start = 0; end = 1; z = 1;
    L2[0] = src;
    while (start < end) {
        for (uint64_t t = start; t < end; ++t) {
            uint32_t j = L2[t];
            if (T[j]) continue;
            for (uint32_t e = colptr[j]; e < colptr[j + 1]; ++e) {
                uint32_t i = rowidx[e];
                if (T[i] == 0) {
                    ops2 += 2;
                    L2[z++] = i;
                }
            }
            T[j] = 1;
        }
        start = end;
        end = z;
    }
    out[1] = ops2;
    free(T); free(L); free(L2); free(lev); free(q);
    return 0;
}
