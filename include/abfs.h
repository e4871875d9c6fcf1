/*
 * abfs -- algebraic breadth-first search by submatrix multiplication on GB300.
 *
 * The method (Burkhardt, "Optimal algebraic Breadth-First Search for sparse
 * graphs"): BFS is the recurrence x_{k+1} = A[V_{k+1}, V_k] x_k (Theorem 1),
 * where V_k holds the vertices not yet reached before step k (Definition 1).
 * Each frontier column is multiplied once (Claim 1), and the rows of visited
 * vertices are masked out before the multiply, so the matrix shrinks as the
 * search advances (Section 6, Section 7).  Algorithm 1 (Section 8) gives the
 * general loop; Algorithm 3 (Section 10) the parallel form.
 *
 * Graph layout.  A graph is given in compressed sparse column form of A^T:
 * column j (rowidx[colptr[j] .. colptr[j+1]-1]) lists the out-neighbours of
 * vertex j.  For undirected graphs A = A^T and column j lists j's
 * neighbours; Section 7 uses A^T for directed graphs.  Vertices are 0..n-1.
 * colptr is uint32[n+1] with colptr[0] = 0, non-decreasing, colptr[n] = nnz;
 * rowidx is uint32[nnz] with every entry < n.  Duplicates and self-loops are
 * allowed and do not change any result.
 *
 * Results.  level[v] is the hop distance from the source (0 at the source),
 * -1 if v is unreachable.  parent[v] is the least-index predecessor of v on
 * the previous level (min{ j : v in column j, level[j] = level[v] - 1 }),
 * parent[source] = source, -1 if unreachable.  The paper allows any write
 * resolution among concurrent parents (Theorem 4, Section 10); this library
 * always takes the minimum index, so results are a pure function of the graph
 * and are identical across runs, modes and batch mixes.
 *
 * Errors.  Every call returns an int status (abfs_status).  No C++ exception
 * crosses this boundary.  abfs_strerror() turns a status into text.
 *
 * Streams.  abfs_stream_t is a cudaStream_t passed as an opaque pointer (NULL
 * is the legacy default stream).  Device work is enqueued on that stream and
 * runs asynchronously unless a call says it synchronises.
 *
 * Device.  Objects belong to the CUDA device that was current when they were
 * created; calls on them must be made with that device current.
 */
#ifndef ABFS_H
#define ABFS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef void* abfs_stream_t;
typedef struct abfs_graph_s* abfs_graph_t;
typedef struct abfs_batch_s* abfs_batch_t;
typedef struct abfs_server_s* abfs_server_t;

typedef enum {
    ABFS_OK = 0,
    ABFS_ERR_INVALID_ARG = 1,   /* null pointer, source >= n, malformed CSC, bad parameter */
    ABFS_ERR_NOT_SYMMETRIC = 2, /* directed = 0 with ABFS_VALIDATE, but A != A^T */
    ABFS_ERR_OOM = 3,           /* a device or host allocation failed */
    ABFS_ERR_CUDA = 4,          /* a CUDA runtime call failed */
    ABFS_ERR_TIMEOUT = 5,       /* a bounded device-side wait ran out; the kernel returned */
    ABFS_ERR_BUSY = 6,          /* serving: the request was not admitted (no slot / memory) */
    ABFS_ERR_DEVICE = 7,        /* a device-side consistency check failed (capacity, bounds) */
    ABFS_ERR_UNSUPPORTED = 8,   /* size beyond the library's limits, or a feature the mode lacks */
    ABFS_ERR_NOT_FOUND = 9      /* serving: unknown ticket */
} abfs_status;

/* abfs_graph_create flags */
#define ABFS_VALIDATE 1u        /* check colptr/rowidx (and symmetry when directed = 0) */
#define ABFS_INPUT_ON_DEVICE 2u /* colptr/rowidx are device pointers (else host pointers) */

/* Execution modes (abfs_params.mode). */
#define ABFS_MODE_SUBMATRIX 0u  /* the paper's method: mask rows, then multiply */
#define ABFS_MODE_PLAIN 1u      /* comparator: masked SpMSpV, multiply every entry, mask after */

/* Tunable launch parameters.  abfs_default_params() fills sound values;
 * abfs_tune() measures and picks them for a graph. */
typedef struct {
    uint32_t mode;            /* ABFS_MODE_SUBMATRIX or ABFS_MODE_PLAIN */
    uint32_t tile;            /* frontier vertices staged per step, 32..1024, multiple of 32 */
    uint32_t unit_entries;    /* granule of work units in entry slots: a power of two,
                                 256..65536; a level's units are 1..65536/unit_entries granules,
                                 chosen per level for about two units per CTA of the grid */
    uint32_t narrow_max;      /* frontiers of <= this many vertices ... */
    uint32_t narrow_edges;    /* ... and <= this many column entries run on one CTA */
    uint32_t ctas_per_sm;     /* persistent grid = ctas_per_sm x SM count (capped by occupancy) */
    float shrink_theta;       /* physical shrink once the reached fraction of n crosses theta;
                                 <= 0 or >= 1 disables it */
    uint32_t shrink_max;      /* at most this many shrinks per search */
    uint32_t timeout_ms;      /* bound on any device-side wait without progress */
    uint32_t narrow_resident; /* 1: consecutive narrow levels run back to back on one CTA with
                                 the frontier kept as a plain list (no per-level hand-off);
                                 0: every narrow level goes through the block bookkeeping */
    uint32_t claim_scan;      /* submatrix mode: a wide level with at least this many entry
                                 slots multiplies and claims by reductions (no returned
                                 values), and a scan of the visited bitmaps then collects the
                                 vertices it reached; 0: never */
    uint32_t bottom_up_alpha; /* hybrid (direction optimisation, not the paper's method): 0 =
                                 off.  Otherwise a level runs bottom-up -- each unvisited
                                 vertex scans its column for the least frontier index and
                                 stops at the first hit -- once the frontier's edges m_f
                                 satisfy m_f * alpha > m_u (edges of vertices not reached
                                 yet), until the frontier's size n_f satisfies
                                 n_f * beta < n.  Results are identical.  Applies to
                                 undirected graphs whose columns ascend (checked at
                                 abfs_graph_create) in abfs_run, abfs_run_host and
                                 batches; path counts and serving stay top-down.  Submatrix mode without physical
                                 shrink only (else ABFS_ERR_INVALID_ARG). */
    uint32_t bottom_up_beta;  /* see bottom_up_alpha */
    uint32_t cluster_ctas;    /* CTAs per thread-block cluster of the persistent launch, 1..16
                                 (1: none).  With clusters, a level small enough for a
                                 resident narrow run runs instead on the advancing CTA and
                                 the idle CTAs of its cluster together (a cluster run): the
                                 frontier list stays in global memory, its counters and the
                                 per-level barrier live in the leading CTA's shared memory
                                 (distributed shared memory).  Results are identical. */
    uint32_t cluster_min;     /* a level of >= this many entry slots starts a cluster run
                                 (smaller ones run on one CTA; a search's first level and a
                                 level too large for one CTA may start one too).  A run
                                 starts only while at least half of the cluster's other
                                 CTAs are idle. */
    uint32_t cluster_max;     /* a cluster run continues while a level has <= this many
                                 frontier vertices ... */
    uint32_t cluster_edges;   /* ... and <= this many entry slots (column entries plus
                                 up to 6 per vertex, so that each vertex starts on a group
                                 of four) */
    uint32_t multi_source;    /* batches (submatrix mode, no path counts): when at least
                                 this many queries search one undirected graph, they run as
                                 multi-source searches of up to 64 sources each -- one
                                 64-bit mask per vertex, so a column of the union frontier
                                 is read once per level for all its sources.  0: never.
                                 Results are identical to single searches. */
} abfs_params;

/* Per-search counters, filled when a stats pointer is passed. */
typedef struct {
    uint32_t levels;              /* non-empty frontiers (eccentricity of the source + 1) */
    uint32_t reached;             /* n_c: vertices reached, source included */
    uint64_t nnz_reached;         /* nnz_c: sum of the reached columns' lengths in the input */
    uint64_t entries_read;        /* stored entries read by the expansion (shrunk matrix after a shrink) */
    uint64_t entries_unmasked;    /* entries whose row passed the visited mask (multiplied) */
    uint64_t claims;              /* atomic claim attempts (parent updates issued) */
    uint32_t shrinks;             /* physical shrink events */
    uint32_t wide_levels;         /* levels run across the whole grid */
    uint64_t shrink_entries_read; /* entries read by shrink kernels */
    uint64_t shrink_entries_kept; /* entries written by shrink kernels */
    uint32_t status;              /* abfs_status of the device side */
    uint32_t reserved;
} abfs_stats;

/* Returns a static string for a status code. */
const char* abfs_strerror(int status);

/* Library version as major*10000 + minor*100 + patch. */
int abfs_version(void);

/* Fills *p with defaults (submatrix mode, no shrink). */
int abfs_default_params(abfs_params* p);

/* ABFS_OK if *p is a valid parameter set, else ABFS_ERR_INVALID_ARG (the same
 * check every call that takes parameters makes).  Needs no device. */
int abfs_check_params(const abfs_params* p);

/*
 * Creates a device-resident graph from CSC arrays (Section 9's compressed
 * format, applied to A^T).  The arrays are copied: the caller keeps ownership
 * of colptr/rowidx, and the library owns the result until
 * abfs_graph_destroy().  With ABFS_INPUT_ON_DEVICE the pointers are device
 * pointers; otherwise host pointers.  With ABFS_VALIDATE the CSC invariants
 * (and, for directed = 0, symmetry of the pattern) are checked on the host
 * (for device input, after a copy back).  `directed` does not change the
 * traversal; it selects validation and the edge convention of reports.
 * Synchronises `stream` before returning.
 * Limits: n < 2^31, nnz + n < 2^32.
 */
int abfs_graph_create(const uint32_t* colptr, const uint32_t* rowidx, uint32_t n, uint64_t nnz,
                      int directed, uint32_t flags, abfs_stream_t stream, abfs_graph_t* out);

int abfs_graph_destroy(abfs_graph_t g);

/* n, nnz and the directed flag of a graph (any pointer may be NULL). */
int abfs_graph_info(abfs_graph_t g, uint32_t* n, uint64_t* nnz, int* directed);

/*
 * Adds to the graph a copy whose vertices are renumbered by column-length
 * class (a layout choice; the paper's method is unchanged): first the longest
 * columns, whole length groups of at most n/64 vertices; then the next
 * longest, up to n/8 with the first class; then the other non-empty columns;
 * the empty ones last; input order inside each class.  On graphs with a
 * skewed degree distribution the mask tests and claims of the high-degree
 * rows then fall on few cache lines.  Graphs whose input order carries
 * locality (grids, geometric graphs) gain nothing from it.  Single searches
 * in submatrix mode without path counts (abfs_run, abfs_run_host,
 * abfs_run_host_many, abfs_run_trace, and the autotuner's trials) run on the
 * copy; a last pass writes level[] and parent[] in the input's labels, with
 * the same least-index parents (Theorem 1).  Path counts, the hybrid (when
 * the graph allows its bottom-up levels: undirected, ascending columns), the
 * comparator, batches and serving keep the input numbering.
 * Costs a second copy of colptr/rowidx plus 8n bytes of label maps, and 8n
 * bytes more per workspace.  Builds on the host (the CSC is copied out and
 * back); synchronises; calling it again does nothing.  Returns ABFS_ERR_OOM or
 * ABFS_ERR_CUDA on failure, leaving the graph as it was.
 */
int abfs_graph_relabel(abfs_graph_t g);

/*
 * The numbering abfs_graph_relabel uses, computed on the host from a CSC
 * column pointer array alone (no GPU, no allocation visible to the caller):
 * lab[i] = the input label of internal vertex i, pos[v] = the internal label
 * of input vertex v (inverse permutations), both caller-owned host arrays of
 * n entries.  Classes in internal order: (0) the longest columns, whole groups
 * of equal length taken from the longest down while they hold at most n/64
 * vertices in all; (1) further whole groups while classes 0-1 hold at most
 * n/8; (2) the other non-empty columns; (3) the empty columns.  Input order
 * inside each class.  colptr: host, n + 1 non-decreasing entries.  Returns
 * ABFS_ERR_INVALID_ARG for a NULL pointer (n > 0) or a decreasing colptr;
 * n = 0 does nothing.
 */
int abfs_relabel_order(const uint32_t* colptr, uint32_t n, uint32_t* lab, uint32_t* pos);

/* Device bytes one search on this graph needs beyond the graph itself
 * (bitmaps, frontier queues, control), for the given parameters
 * (NULL = defaults).  Serving admission uses this figure. */
int abfs_graph_footprint(abfs_graph_t g, const abfs_params* params, size_t* bytes_per_query);

/*
 * One BFS from `source` (Algorithm 1 / Theorem 1): writes level[0..n-1] and
 * parent[0..n-1], caller-owned DEVICE buffers of n int32 each.  Asynchronous
 * on `stream` unless `stats` is non-NULL, in which case it synchronises and
 * fills *stats.  params = NULL uses the graph's tuned parameters if
 * abfs_tune() ran, else defaults.  The graph keeps one search workspace;
 * calls on the same graph are ordered on the GPU (a later call on another
 * stream waits for the earlier one).
 */
int abfs_run(abfs_graph_t g, uint32_t source, int32_t* level, int32_t* parent,
             abfs_stream_t stream, const abfs_params* params, abfs_stats* stats);

/*
 * One search that also counts shortest paths: the all-nonzero variant of
 * Algorithm 2 (Section 8) over the arithmetic semiring, which Proposition 1
 * requires to be used at every step.  With x_1 = e_source, every entry (i, j)
 * of A[V_{k+1}, V_k] (j on level k, row i not yet visited) adds x_k(j) into
 * x_{k+1}(i), so x_{k+1}(i) = sigma[i] is the number of shortest paths from
 * the source to i.  sigma is a caller-owned DEVICE buffer of n uint64, written
 * modulo 2^64; sigma[source] = 1, unreached vertices 0.  A column that stores
 * row i twice counts as the integer entry 2.  level/parent as in abfs_run
 * (same values).  Submatrix mode only (ABFS_ERR_UNSUPPORTED for the
 * comparator); a NULL sigma is ABFS_ERR_INVALID_ARG.  Cost over abfs_run: one
 * 64-bit load and one 64-bit atomic add per multiplied entry (E_adj of them).
 */
int abfs_run_counts(abfs_graph_t g, uint32_t source, int32_t* level, int32_t* parent,
                    uint64_t* sigma, abfs_stream_t stream, const abfs_params* params,
                    abfs_stats* stats);

/*
 * Same search, end to end through host memory: copies the source in, runs,
 * and copies level/parent back into HOST buffers of n int32 each (pinned
 * memory gives full copy bandwidth).  Synchronises `stream` and returns the
 * search's own status (ABFS_ERR_TIMEOUT or ABFS_ERR_DEVICE if the device side
 * failed).
 */
int abfs_run_host(abfs_graph_t g, uint32_t source, int32_t* level_host, int32_t* parent_host,
                  abfs_stream_t stream, const abfs_params* params, abfs_stats* stats);

/*
 * `count` searches of Algorithm 1 from sources[0..count), end to end through
 * host memory: search i writes level_host[i*n .. i*n+n) and
 * parent_host[i*n .. i*n+n) (HOST buffers of count*n int32 each; pinned
 * memory lets the copies overlap the searches).  The searches run one after
 * another on `stream` into two alternating device buffers; while search i+1
 * runs, the outputs of search i travel to the host on a copy stream of the
 * graph's own, so the copies cost no search time when they take less time
 * than a search.  status (host, count entries; may be NULL) receives each
 * search's own status.  Synchronises; returns the first non-zero status,
 * ABFS_ERR_INVALID_ARG (checked before anything runs) if a source is >= n.
 */
int abfs_run_host_many(abfs_graph_t g, const uint32_t* sources, uint32_t count,
                       int32_t* level_host, int32_t* parent_host, abfs_stream_t stream,
                       const abfs_params* params, int32_t* status);

/*
 * abfs_run plus a per-phase trace of the search, for profiling: trace_host
 * receives up to `cap` entries of 8 uint32 each --
 *   [0..1] %globaltimer (ns, low/high), [2] phase kind << 24 | BFS level
 *   (kind 0 level, 1 comparator multiply, 2 comparator mask, 3 shrink,
 *   5 level claimed by reductions, 6 extraction of its new vertices,
 *   7 frontier bitmap of a bottom-up level, 8 bottom-up level,
 *   0xFE start, 0xFF end), [3] 0 if the phase was published to the whole
 *   grid, 1 if it ran on one CTA (or started a cluster run), 2 if it is a
 *   further level of a resident narrow run, 3 if it is a further level of a
 *   cluster run ([4] then holds the run's CTAs), [4] units or touched rows of
 *   the phase, [5] frontier
 *   vertices, [6] entry slots of that frontier (column entries plus up to 6
 *   per vertex, low 32 bits), [7] 0.  For a level, [4] is its number of work
 *   units (comparator mask: touched rows).
 * *count receives the number written.  Synchronises `stream`.
 */
int abfs_run_trace(abfs_graph_t g, uint32_t source, int32_t* level, int32_t* parent,
                   abfs_stream_t stream, const abfs_params* params, uint32_t* trace_host,
                   uint32_t cap, uint32_t* count);

/*
 * Batched search: `count` independent searches (graph g[i], source
 * sources[i]) in ONE persistent launch with per-instance frontier queues;
 * each CTA takes work units from any instance that has them.  level[i] and
 * parent[i] are caller-owned DEVICE buffers of g[i]'s n int32 each.
 * status_per_query (host, count entries, may be NULL) receives each search's
 * abfs_status.  Synchronises `stream`.  Results equal abfs_run's, bit for
 * bit.
 */
int abfs_run_batch(const abfs_graph_t* g, const uint32_t* sources, uint32_t count,
                   int32_t* const* level, int32_t* const* parent, abfs_stream_t stream,
                   const abfs_params* params, int32_t* status_per_query);

/*
 * Reusable batch plan: allocates the per-instance workspaces once and
 * captures the initialisation and the persistent launch in a CUDA graph
 * (captured on `stream` at creation).  abfs_batch_launch() replays it; the
 * output pointers given here are written on every replay.  The plan keeps
 * references to the graphs, which must outlive it.
 */
int abfs_batch_create(const abfs_graph_t* g, const uint32_t* sources, uint32_t count,
                      int32_t* const* level, int32_t* const* parent, const abfs_params* params,
                      abfs_stream_t stream, abfs_batch_t* out);
/*
 * The same plan with shortest-path counts (as abfs_run_counts): sigma[i] is a
 * caller-owned DEVICE buffer of g[i]'s n uint64, written modulo 2^64 on every
 * replay.  Submatrix mode only (ABFS_ERR_UNSUPPORTED otherwise); a NULL sigma
 * array or entry is ABFS_ERR_INVALID_ARG.  Searches with counts stay top-down.
 */
int abfs_batch_create_counts(const abfs_graph_t* g, const uint32_t* sources, uint32_t count,
                             int32_t* const* level, int32_t* const* parent,
                             uint64_t* const* sigma, const abfs_params* params,
                             abfs_stream_t stream, abfs_batch_t* out);
int abfs_batch_launch(abfs_batch_t b, abfs_stream_t stream);
/* Copies per-instance statuses (host array of count) after a launch; synchronises. */
int abfs_batch_status(abfs_batch_t b, abfs_stream_t stream, int32_t* status_per_query);
int abfs_batch_destroy(abfs_batch_t b);

/*
 * Autotuner: times candidate parameter sets on `count` searches from
 * `sources`.  `mode` selects which method is tuned; for the submatrix method
 * the fastest set is also stored in the graph and used when params = NULL (a
 * tuned comparator set is only returned, so NULL params keep meaning the
 * submatrix method).  *best (may be NULL) receives the
 * choice and *best_ms its mean device time per search.  With `cache_path`
 * non-NULL the result is read from / appended to that JSON-lines file, keyed
 * by GPU name, SM count, mode and the graph's size class.  Synchronises.
 */
int abfs_tune(abfs_graph_t g, const uint32_t* sources, uint32_t count, uint32_t mode,
              const char* cache_path, abfs_stream_t stream, abfs_params* best, float* best_ms);

/*
 * Batch autotuner: for each candidate parameter set (work granule, narrow
 * bounds, reduction claims, shrink threshold) builds a batch plan over the
 * `count` searches (graph g[i], source sources[i]), replays it after one
 * warm-up and keeps the fastest whole-batch time; *best receives that set
 * and *best_ms its mean ms per launch.  Device memory for the trial plans and
 * their outputs is allocated and freed inside.  With `cache_path` (JSON
 * lines), an earlier choice for the same GPU, SM count, mode and batch size
 * class is returned without measuring, and a new choice is appended.
 * Synchronises `stream`.
 */
int abfs_batch_tune(const abfs_graph_t* g, const uint32_t* sources, uint32_t count, uint32_t mode,
                    const char* cache_path, abfs_stream_t stream, abfs_params* best,
                    float* best_ms);

/*
 * Serving: a long-lived device loop answers BFS queries on resident graphs
 * (continuous batching).  Requests are queued by abfs_serve_submit; a host
 * admission thread moves them into free device slots as soon as a slot and
 * enough workspace memory (abfs_graph_footprint of the query's graph, carved
 * from a memory budget) are free, while other queries are running; their
 * work overlaps on the device in one persistent launch, which any CTA serves
 * unit by unit.  The launch ends after idle_exit_ms without work and is
 * relaunched on demand.  Each query's result equals abfs_run's, bit for bit.
 * The paper has no counterpart (it evaluates single searches).
 */
typedef struct {
    uint32_t max_slots;       /* queries on the device at once (1..4096) */
    uint32_t queue_capacity;  /* queued requests beyond which submit returns ABFS_ERR_BUSY */
    uint64_t memory_budget;   /* device bytes for query workspaces */
    uint32_t idle_exit_ms;    /* the device loop ends after this long without work */
    abfs_params params;       /* engine parameters of every query */
} abfs_serve_cfg;

typedef struct {
    uint64_t submitted;       /* requests accepted by abfs_serve_submit */
    uint64_t completed;       /* queries finished (any status) */
    uint64_t failed;          /* queries that finished with a non-OK status */
    uint64_t launches;        /* device loop launches */
    double p50_ms, p99_ms, mean_ms, max_ms;  /* submit -> done latency */
    double wall_s;            /* abfs_serve_start -> abfs_serve_stop */
    double qps;               /* completed / wall_s */
} abfs_serve_report;

/* Fills *cfg with defaults (256 slots, 16 GiB budget, 1M queue, 50 ms idle exit). */
int abfs_serve_default_cfg(abfs_serve_cfg* cfg);

/* Starts a server over ngraphs device-resident graphs (abfs_graph_create);
 * the graphs must outlive it.  Allocates the slot table and the workspace
 * budget up front.  cfg = NULL uses defaults. */
int abfs_serve_start(const abfs_graph_t* g, uint32_t ngraphs, const abfs_serve_cfg* cfg,
                     abfs_server_t* out);

/* Queues one query: BFS on graph g[graph_idx] from `source`, results into the
 * caller's DEVICE buffers level/parent (n int32 each), which must stay valid
 * until the query is done.  Non-blocking; *ticket identifies the query.
 * ABFS_ERR_BUSY when the queue is full, ABFS_ERR_INVALID_ARG on a bad graph
 * index, source or buffer. */
int abfs_serve_submit(abfs_server_t s, uint32_t graph_idx, uint32_t source, int32_t* level,
                      int32_t* parent, uint64_t* ticket);

/* *done = 1 and *status = the query's abfs_status once it finished, else
 * *done = 0.  ABFS_ERR_NOT_FOUND for an unknown ticket. */
int abfs_serve_poll(abfs_server_t s, uint64_t ticket, int* done, int32_t* status);

/* Blocks until the query finished or timeout_ms passed (ABFS_ERR_TIMEOUT). */
int abfs_serve_wait(abfs_server_t s, uint64_t ticket, uint32_t timeout_ms, int32_t* status);

/* Finishes every queued and running query, ends the device loop, fills
 * *report (may be NULL) and frees the server. */
int abfs_serve_stop(abfs_server_t s, abfs_serve_report* report);

/*
 * One search, like abfs_run with default parameters, that allocates nothing.
 * The paper has no counterpart: this entry point serves callers that cannot
 * call cudaMalloc -- for example code that runs while an allocator is locked
 * or disallowed (inside a memory pool's callback, a real-time serving thread
 * that must not block on allocation, or a process whose device memory is
 * budgeted up front) and so cannot use abfs_graph_create/abfs_run, which
 * allocate a graph copy and a workspace.
 *
 * The caller passes device pointers: colptr[n+1] and rowidx[nnz] (CSC of A^T
 * as for abfs_graph_create, used in place, not copied or validated) and the
 * outputs level[n] and parent[n].  The scratch memory is a fixed 72 MiB
 * device array inside this library (held on every GPU that loads it until the
 * process exits), enough for graphs up to about 1.1 million vertices; larger
 * inputs are rejected with ABFS_ERR_UNSUPPORTED before any device work.
 *
 * The first call on a device looks up that array's device address (once,
 * with the device current); make that first call before any stream capture.
 * With lazy module loading (CUDA's default) the array takes its device memory
 * at that first lookup, so the first call on a device can fail with
 * ABFS_ERR_CUDA when the device is out of memory: make it at start-up, before
 * the memory is budgeted or an allocator is locked.  Later calls allocate
 * nothing.  The scratch a search needs is about 65 bytes per vertex plus 16
 * bytes per 1024 entry slots (column entries + at most 6 per vertex); graphs
 * whose scratch exceeds the array (72 MiB - 256 bytes), e.g. beyond about 1.1
 * million vertices at average degree 16, are rejected.
 * Every call uses the same array, which keeps the previous call's contents;
 * the call clears everything a search needs at zero.  Calls whose device work
 * overlaps (on different streams or host threads) race on the array and give
 * wrong results: order them on one stream.  Synchronises `stream`; returns the
 * search's status (ABFS_ERR_TIMEOUT or ABFS_ERR_DEVICE if the device side
 * failed).
 */
int abfs_run_static(const uint32_t* colptr, const uint32_t* rowidx, uint32_t n, uint64_t nnz,
                    uint32_t source, int32_t* level, int32_t* parent, abfs_stream_t stream);

/*
 * Device-memory hook: alloc(bytes, ctx) returns device memory or NULL;
 * free_fn(ptr, ctx) releases it.  Both NULL restores cudaMalloc/cudaFree.
 * Memory must be 16-byte aligned (cudaMalloc's is 256-byte aligned): a block
 * that is not goes straight back to free_fn and the call that asked for it
 * fails with ABFS_ERR_INVALID_ARG.
 * Applies to allocations made after the call (graphs, workspaces, plans);
 * memory must be freed by the hook that allocated it.
 */
int abfs_set_allocator(void* (*alloc)(size_t bytes, void* ctx), void (*free_fn)(void* ptr, void* ctx),
                       void* ctx);

/*
 * Test control for the bounded device waits; the paper has no counterpart.
 * While extra_units is non-zero, every search started afterwards (abfs_run,
 * abfs_run_counts, abfs_run_host, abfs_run_trace, abfs_run_batch, and batch
 * plans created afterwards) publishes its first phase as waiting for
 * extra_units more work units than it has.  That phase never completes, the
 * engine's CTAs find no work, their idle wait -- bounded by
 * abfs_params.timeout_ms without progress -- runs out, and the search ends
 * with ABFS_ERR_TIMEOUT while the launch returns normally: no fault, no hang.
 * 0 restores normal operation.  Process-wide; needs no device.
 */
int abfs_test_hold_first_phase(uint32_t extra_units);

/* On-chip ceilings of the expand step, measured on the current device. */
typedef struct {
    uint32_t words;     /* array size in 32-bit words (2^words_log2) */
    uint32_t reserved;
    uint64_t ops;       /* operations per measurement */
    double red_gops;    /* random 32-bit red.min into the array, 10^9 per second */
    double load_gops;   /* random 32-bit loads from the array through L2, 10^9 per second */
} abfs_calibration;

/*
 * Times random 32-bit reductions and random 32-bit L2 loads over an array of
 * 2^words_log2 words (10..26), the two accesses each column entry costs (the
 * visited-bitmap test and the (min, index) claim) when their targets sit in
 * L2.  Allocates and frees 4 * 2^words_log2 bytes; synchronises `stream`.
 * Diagnostics only: no search uses it.
 */
int abfs_calibrate(uint32_t words_log2, abfs_calibration* out, abfs_stream_t stream);

/* Text of the last CUDA runtime error seen by this thread ("" if none). */
const char* abfs_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* ABFS_H */
