/*
 * CPU baselines of the algebraic BFS (Burkhardt, "Optimal algebraic
 * Breadth-First Search for sparse graphs"): the paper's own two CPU methods,
 * timed beside the GPU library on the host cores.  They share no code with
 * the CUDA path or with the oracle.
 *
 *   alg2_bfs  -- Algorithm 2 (Section 9): the CSR product restricted to the
 *                rows not yet visited.  An array T marks visited vertices and a
 *                list L holds the nonzeros of x in discovery order; a row is
 *                marked as soon as its first nonzero is used, so only n - 1
 *                products are made (Theorem 2).  One thread.
 *   alg3_bfs  -- Algorithm 3 (Section 10) as the paper's OpenMP version
 *                describes it: each thread scans its share of the frontier
 *                into a list of its own (testing T, writing the parent P of
 *                each candidate with any write resolution), then removes the
 *                candidates other threads also found with an atomic
 *                test-and-set on T; each thread publishes its count, and a
 *                prefix sum of the counts up to its own id gives it a gap-free
 *                block of L to write.
 *
 * The CSC of A^T that the library takes is the paper's CSR of A read by rows:
 * column j (rowidx[colptr[j] .. colptr[j+1]-1]) lists the out-neighbours of j.
 *
 * Outputs: level[v] (0 at the source, -1 unreached) and parent[v] (the
 * frontier vertex whose product reached v first, parent[source] = source, -1
 * unreached).  Levels are the BFS distances; the parent is a valid
 * predecessor but, unlike the GPU library's least-index rule, depends on the
 * discovery order (Algorithm 2) or on thread timing (Algorithm 3), as the
 * paper allows (Section 10).
 *
 * Each call returns its wall time in nanoseconds (CLOCK_MONOTONIC), taken
 * around the whole search including the clearing of T, or a negative value
 * on a bad argument or a failed allocation.
 */
#define _POSIX_C_SOURCE 200809L
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int64_t now_ns(void) {
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (int64_t)ts.tv_sec * 1000000000ll + ts.tv_nsec;
}

/* Algorithm 2, one thread.  T and L are caller scratch of n bytes and n
 * words. */
int64_t alg2_bfs(uint32_t n, const uint32_t* colptr, const uint32_t* rowidx, uint32_t src,
                 int32_t* level, int32_t* parent, uint8_t* T, uint32_t* L) {
    if (!colptr || !rowidx || !level || !parent || !T || !L || src >= n) return -1;
    const int64_t t0 = now_ns();
    memset(T, 0, n);
    for (uint32_t v = 0; v < n; ++v) {
        level[v] = -1;
        parent[v] = -1;
    }
    /* x = e_src: the source starts the list and is removed from the rows still
     * to be multiplied (Algorithm 1's V_2 = V_1 minus the source) */
    uint64_t start = 0, end = 1, z = 1;
    L[0] = src;
    T[src] = 1;
    level[src] = 0;
    parent[src] = (int32_t)src;
    for (int32_t k = 1; start < end; ++k) {
        for (uint64_t t = start; t < end; ++t) {
            const uint32_t j = L[t];
            for (uint32_t e = colptr[j]; e < colptr[j + 1]; ++e) {
                const uint32_t i = rowidx[e];
                if (T[i] == 0) {
                    /* y(i) <- x(j): the product over the selection semiring */
                    level[i] = k;
                    parent[i] = (int32_t)j;
                    L[z++] = i;
                    T[i] = 1;
                }
            }
        }
        start = end;
        end = z;
    }
    return now_ns() - t0;
}

/* Per-thread candidate list, grown on demand. */
typedef struct {
    uint32_t* v;
    uint64_t len, cap;
    uint64_t pad[5]; /* one cache line per thread */
} Local;

static int local_push(Local* b, uint32_t x) {
    if (b->len == b->cap) {
        const uint64_t cap = b->cap ? 2 * b->cap : 1024;
        uint32_t* p = (uint32_t*)realloc(b->v, cap * sizeof(uint32_t));
        if (!p) return -1;
        b->v = p;
        b->cap = cap;
    }
    b->v[b->len++] = x;
    return 0;
}

/* Algorithm 3 with OpenMP on `threads` threads (<= 0: the runtime's
 * default).  T and L as for alg2_bfs.  *threads_used (may be NULL) receives
 * the team size. */
int64_t alg3_bfs(uint32_t n, const uint32_t* colptr, const uint32_t* rowidx, uint32_t src,
                 int32_t* level, int32_t* parent, uint8_t* T, uint32_t* L, int threads,
                 int* threads_used) {
    if (!colptr || !rowidx || !level || !parent || !T || !L || src >= n) return -1;
    int nt = 1;
#ifdef _OPENMP
    nt = threads > 0 ? threads : omp_get_max_threads();
#endif
    Local* loc = (Local*)calloc((size_t)nt, sizeof(Local));
    uint64_t* count = (uint64_t*)calloc((size_t)nt + 1, sizeof(uint64_t));
    if (!loc || !count) {
        free(loc);
        free(count);
        return -2;
    }
    int failed = 0, team = 1;
    const int64_t t0 = now_ns();
    uint64_t start = 0, end = 1;
#pragma omp parallel num_threads(nt)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#pragma omp single
        team = omp_get_num_threads();
#endif
#pragma omp for schedule(static)
        for (int64_t v = 0; v < (int64_t)n; ++v) {
            T[v] = 0;
            level[v] = -1;
            parent[v] = -1;
        }
#pragma omp single
        {
            L[0] = src;
            T[src] = 1;
            level[src] = 0;
            parent[src] = (int32_t)src;
        }
        for (int32_t k = 1;; ++k) {
            const uint64_t s0 = start, e0 = end;
            if (s0 >= e0) break;
            Local* me = &loc[tid];
            me->len = 0;
            /* for all frontier vertices j and all nonzeros of column j: rows not
             * yet visited are candidates; P gets j (any writer may win) */
#pragma omp for schedule(dynamic, 64)
            for (int64_t t = (int64_t)s0; t < (int64_t)e0; ++t) {
                const uint32_t j = L[t];
                for (uint32_t e = colptr[j]; e < colptr[j + 1]; ++e) {
                    const uint32_t i = rowidx[e];
                    if (__atomic_load_n(&T[i], __ATOMIC_RELAXED) == 0) {
                        __atomic_store_n(&parent[i], (int32_t)j, __ATOMIC_RELAXED);
                        if (local_push(me, i)) {
                            __atomic_store_n(&failed, 1, __ATOMIC_RELAXED);
                        }
                    }
                }
            }
            /* implicit barrier: T is unchanged during the scan above.  Each
             * thread keeps the candidates it wins the test-and-set of T for. */
            uint64_t kept = 0;
            for (uint64_t q = 0; q < me->len; ++q) {
                const uint32_t i = me->v[q];
                if (__atomic_exchange_n(&T[i], (uint8_t)1, __ATOMIC_RELAXED) == 0) {
                    me->v[kept++] = i;
                    level[i] = k;
                }
            }
            me->len = kept;
            count[tid] = kept;
#pragma omp barrier
            /* the sum of the counts below this thread's id is its offset in L */
            uint64_t off = e0;
            for (int q = 0; q < tid; ++q) off += count[q];
            memcpy(L + off, me->v, kept * sizeof(uint32_t));
#pragma omp barrier
#pragma omp single
            {
                uint64_t tot = 0;
                for (int q = 0; q < nt; ++q) tot += count[q];
                start = e0;
                end = e0 + tot;
                if (__atomic_load_n(&failed, __ATOMIC_RELAXED)) start = end;
            }
        }
    }
    const int64_t dt = now_ns() - t0;
    for (int q = 0; q < nt; ++q) free(loc[q].v);
    free(loc);
    free(count);
    if (threads_used) *threads_used = team;
    return failed ? -2 : dt;
}

/* 1 when built with OpenMP, else 0. */
int alg3_has_openmp(void) {
#ifdef _OPENMP
    return 1;
#else
    return 0;
#endif
}
