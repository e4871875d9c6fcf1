// Persistent BFS engine for sm_103a.
//
// One launch runs one or many searches to completion.  Every search advances
// level by level (Algorithm 1, Section 8).  The frontier x_k is kept as a list
// of vertices in blocks; every vertex carries a weight (the 4-slot chunks that
// hold its column, each chunk one aligned 16-byte group of row indices), and
// the level's column entries form one "entry space" of sum(weights) slots.
// Work units are ranges of that space, sized per level to about two per CTA,
// so a unit holds the same number of entries whether it covers one hub column
// or thousands of short ones (the PRAM "one processor per nonzero" of
// Theorem 4, with load balance instead of a processor per entry).  Any CTA may take any
// unit of any search; the CTA that completes the last unit of a level advances
// the search and publishes the next level.  Small levels run on the advancing
// CTA alone ("narrow" levels), so long, thin searches do not pay a grid-wide
// hand-off per level.
//
// Submatrix mode (the paper's method, Theorem 1): for frontier column j and
// row i in column j, the row is first tested against the visited mask V_{k+1};
// only unmasked rows are multiplied.  The product in the (min, index)
// semiring is an atomicMin of j into parent[i]; the thread that moves parent[i]
// off "unset" claims i for level k+1 (Algorithm 3's P-array dedup with the
// minimum as the write resolution, Theorem 4 / Section 10).
//
// The visited mask is two bitmaps used in turn: at level k the test bitmap holds
// the vertices of levels <= k and stays frozen, so every edge into a vertex of
// level k+1 still reaches the atomicMin and the least parent wins; the other
// bitmap collects the level-k frontier and the level-(k+1) claims and becomes
// the test bitmap of level k+1.
//
// Newly reached vertices gather in a CTA staging buffer and leave it as one
// block (Section 10's per-thread counts and prefix offsets, at CTA scope): a
// single 64-bit atomicAdd reserves the block's number and its entry range at
// once, so blocks are ordered by entry range; each vertex records the unit
// boundaries that fall inside its own range, so every unit of the next level
// finds its first vertex with one load.
//
// Comparator mode (masked SpMSpV, Section 5/Section 11): the multiply runs over
// every entry of the frontier columns into a stamped (min, index) accumulator,
// and the visited mask is applied to the touched rows afterwards.
//
// Shrink phases (Appendix A, A_k = S_k A S_k): when the reached fraction of the
// graph crosses a threshold, every still-unvisited column is stream-compacted
// to its unvisited rows; later levels read the compacted copy.
//
// Waits: a CTA without work polls the searches' published phases; every poll
// loop is bounded by a time limit measured on %globaltimer and reset by
// progress.  On expiry the CTA marks the searches failed (ABFS_ERR_TIMEOUT) and
// returns.
//
// The engine's code is split by topic into engine_*.cuh (included below, each
// building on the previous one); this file holds the initialisation kernels
// and the host-side launch helpers.
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "engine_sched.cuh"
#include "internal.h"

namespace abfs {

// ---------------------------------------------------------------------------
// initialisation: outputs, bitmaps, control blocks, the source (Algorithm 1's
// V_2 := V_1 \ supp(x_1)).
// ---------------------------------------------------------------------------

__global__ void init_fill_kernel(const Inst* insts, uint32_t ninst, uint32_t mode) {
    const Inst& I = insts[blockIdx.y];
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t t0 = blockIdx.x * blockDim.x + threadIdx.x;
    if (I.ms) {
        // multi-source search: every source's outputs, the bit masks, the control block
        for (uint32_t s = 0; s < I.ms; ++s) {
            int32_t* lv = I.ms_level[s];
            int32_t* pv = I.ms_parent[s];
            for (uint32_t v = t0; v < I.n; v += stride) {
                lv[v] = -1;
                pv[v] = -1;
            }
        }
        for (uint32_t v = t0; v < I.n; v += stride) {
            I.ms_vis[v] = 0ull;
            I.ms_fr[0][v] = 0ull;
            I.ms_fr[1][v] = 0ull;
            I.ms_nx[v] = 0ull;
        }
        if (blockIdx.x == 0) {
            uint32_t* c = reinterpret_cast<uint32_t*>(I.ctl);
            for (uint32_t w = threadIdx.x; w < sizeof(InstCtl) / 4; w += blockDim.x) c[w] = 0u;
        }
        return;
    }
    for (uint32_t v = t0; v < I.n; v += stride) {
        I.level[v] = -1;
        I.parent[v] = kUnset;
        if (mode == kModePlain) I.y[v] = ~0ull;
        if (I.sigma) I.sigma[v] = 0ull;
    }
    if (mode == kModeSub) {
        // vertices that no column contains cannot be reached: they start out in
        // both visited bitmaps, so no later pass (extraction, bottom-up levels)
        // looks at them again
        for (uint32_t w = t0; w < I.nwords; w += stride) {
            uint32_t m = 0u;
            if (I.inb) {
                m = ~I.inb[w];
                if (w == I.nwords - 1 && (I.n & 31)) m &= (1u << (I.n & 31)) - 1u;
            }
            I.bm[0][w] = m;
            I.bm[1][w] = m;
        }
    }
    if (blockIdx.x == 0) {
        uint32_t* c = reinterpret_cast<uint32_t*>(I.ctl);
        for (uint32_t w = threadIdx.x; w < sizeof(InstCtl) / 4; w += blockDim.x) c[w] = 0u;
    }
}

// The control block's start state (zeroed before) for a search whose frontier
// of level 0 (w0 entry slots) is set up: the first CTA to arrive advances into
// level 0, which then starts a resident run when it is small (the usual case)
// instead of a grid phase.  One thread.
__device__ void start_ctl(const Inst& I, InstCtl* ctl, uint32_t hold_units, unsigned long long w0) {
    ctl->mat_cur = 0;
    ctl->mat_prev = 0;
    ctl->mat_switch = 0;
    ctl->kind[0] = kPhStart;
    ctl->plevel[0] = 0;
    ctl->nitems[0] = 0;
    ctl->pending[0] = 1 + hold_units;
    ctl->epoch = 0;
    ctl->desc[0] = (0ull << 32) | 1ull;
    ctl->desc[1] = ~0ull;
    ctl->grab = 0ull;
    ctl->status = kRunning;
    if (I.trace && I.trace_cap) {
        const uint64_t now = globaltimer();
        I.trace[0] = make_uint4((uint32_t)now, (uint32_t)(now >> 32), (0xFEu << 24), 0u);
        I.trace[1] = make_uint4(0u, ctl->fcnt[0], (uint32_t)w0, 0u);
        ctl->trace_n = 1;
    }
}

// Level 0 of a single search from source s, input label s_label (outputs
// cleared before): the source's outputs and visited bit, its frontier block
// and unit starts, and the control block's start state.  One thread.
__device__ void start_single(const Inst& I, InstCtl* ctl, const EngineParams& P, uint32_t hold_units,
                             uint32_t s, uint32_t s_label) {
    I.level[s] = 0;
    I.parent[s] = s_label;
    if (I.sigma) I.sigma[s] = 1ull;  // x_1 = e_src over the arithmetic semiring
    if (P.mode == kModeSub) I.bm[0][s >> 5] |= 1u << (s & 31);  // V_2 = V_1 \ {source}
    // frontier of level 0: one block holding the source
    const uint32_t len = I.colptr[s + 1] - I.colptr[s];
    const uint32_t w = col_slots(I, 0, I.colptr[s], len);
    I.fq[0][0] = s;
    I.fbeg[0][0] = I.colptr[s];
    I.fpre[0][0] = 0;
    I.flen[0][0] = len;
    I.blk[0][0].vb = 0;
    I.blk[0][0].nv = 1;
    I.blk[0][0].eb = 0;
    for (unsigned long long x = 0; x < w; x += P.unit) I.ustart[0][x / P.unit] = make_uint2(0, 0);
    ctl->bctr[0] = ((unsigned long long)w << kBlockBits) | 1ull;
    ctl->fent[0] = len;
    ctl->fcnt[0] = 1;
    ctl->reached = 1;
    start_ctl(I, ctl, hold_units, w);
}

__global__ void init_source_kernel(EngineArgs a) {
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q == 0) {
        *a.done_count = 0u;
        *a.heartbeat = 0ull;
    }
    if (q >= a.ninst) return;
    const Inst& I = a.insts[q];
    const EngineParams& P = a.p;
    InstCtl* ctl = I.ctl;
    if (I.ms) {
        // multi-source search: x_1 = e_src for every source bit; the frontier of
        // level 0 is the distinct sources, one block
        uint32_t nv = 0;
        unsigned long long w = 0;  // entry slots so far
        unsigned long long ent = 0;  // column entries so far
        for (uint32_t b = 0; b < I.ms; ++b) {
            const uint32_t v = I.ms_src[b];
            I.ms_level[b][v] = 0;
            I.ms_parent[b][v] = (int32_t)v;
            const unsigned long long bit = 1ull << b;
            if (I.ms_fr[0][v] == 0ull) {
                // first source at v: v joins the frontier list
                const uint32_t len = I.colptr[v + 1] - I.colptr[v];
                I.fq[0][nv] = v;
                I.fbeg[0][nv] = I.colptr[v];
                I.fpre[0][nv] = (uint32_t)w;
                I.flen[0][nv] = len;
                ent += len;
                const unsigned long long w1 = w + col_slots(I, 0, I.colptr[v], len);
                for (unsigned long long x = (w + P.unit - 1) / P.unit * P.unit; x < w1; x += P.unit)
                    I.ustart[0][x / P.unit] = make_uint2(0, nv);
                w = w1;
                ++nv;
            }
            I.ms_fr[0][v] |= bit;
            I.ms_vis[v] |= bit;
        }
        I.blk[0][0].vb = 0;
        I.blk[0][0].nv = nv;
        I.blk[0][0].eb = 0;
        ctl->bctr[0] = (w << kBlockBits) | 1ull;
        ctl->fent[0] = ent;
        ctl->fcnt[0] = nv;
        ctl->reached = nv;
        start_ctl(I, ctl, a.hold_units, w);
    } else {
        start_single(I, ctl, P, a.hold_units, I.src, I.lab ? I.lab[I.src] : I.src);
    }
}

// One search on instance 0 of a workspace (abfs_run and friends): writes the
// call's fields into the descriptor, clears the outputs and bitmaps (as
// init_fill_kernel), and the last block to finish sets up the control block
// and level 0 (as init_source_kernel) -- one launch instead of three.  The
// last block takes the call's fields from the arguments: its cached view of
// the descriptor may predate block 0's update.
__global__ void init_single_kernel(Inst* inst, uint32_t src, uint32_t src_label, int32_t* level,
                                   uint32_t* parent, unsigned long long* sigma, uint32_t bu_ok,
                                   uint4* trace, uint32_t trace_cap, EngineArgs a) {
    Inst& D = *inst;
    const uint32_t n = D.n, nwords = D.nwords;
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t t0 = blockIdx.x * blockDim.x + threadIdx.x;
    for (uint32_t v = t0; v < n; v += stride) {
        level[v] = -1;
        parent[v] = kUnset;
        if (a.p.mode == kModePlain) D.y[v] = ~0ull;
        if (sigma) sigma[v] = 0ull;
    }
    if (a.p.mode == kModeSub) {
        // vertices that no column contains start out in both visited bitmaps
        const uint32_t* inb = D.inb;
        uint32_t* bm0 = D.bm[0];
        uint32_t* bm1 = D.bm[1];
        for (uint32_t w = t0; w < nwords; w += stride) {
            uint32_t m = 0u;
            if (inb) {
                m = ~inb[w];
                if (w == nwords - 1 && (n & 31)) m &= (1u << (n & 31)) - 1u;
            }
            bm0[w] = m;
            bm1[w] = m;
        }
    }
    InstCtl* ctl = D.ctl;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        D.src = src;
        D.level = level;
        D.parent = parent;
        D.sigma = sigma;
        D.bu_ok = bu_ok;
        D.trace = trace;
        D.trace_cap = trace_cap;
    }
    // the last block to get here sees every block's writes
    __shared__ uint32_t last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicInc(&ctl->init_ticket, gridDim.x - 1) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    uint32_t* c = reinterpret_cast<uint32_t*>(ctl);
    for (uint32_t w = threadIdx.x; w < sizeof(InstCtl) / 4; w += blockDim.x) c[w] = 0u;
    __syncthreads();
    if (threadIdx.x == 0) {
        *a.done_count = 0u;
        *a.heartbeat = 0ull;
        Inst I = D;
        I.src = src;
        I.level = level;
        I.parent = parent;
        I.sigma = sigma;
        I.bu_ok = bu_ok;
        I.trace = trace;
        I.trace_cap = trace_cap;
        start_single(I, ctl, a.p, a.hold_units, src, src_label);
    }
}

// Writes the per-call fields of instance 0 (single searches reuse one
// descriptor; kernel arguments avoid a host staging buffer).
__global__ void set_query_kernel(Inst* inst, uint32_t src, int32_t* level, uint32_t* parent,
                                 unsigned long long* sigma, uint32_t bu_ok, uint4* trace,
                                 uint32_t trace_cap) {
    inst->src = src;
    inst->level = level;
    inst->parent = parent;
    inst->sigma = sigma;
    inst->bu_ok = bu_ok;
    inst->trace = trace;
    inst->trace_cap = trace_cap;
}

cudaError_t launch_init_single(const EngineArgs& a, uint32_t src, uint32_t src_label, int32_t* level,
                               uint32_t* parent, unsigned long long* sigma, uint32_t bu_ok,
                               uint4* trace, uint32_t trace_cap, uint32_t n, cudaStream_t s) {
    uint32_t blocks = (n + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    if (blocks == 0) blocks = 1;
    // the descriptor is the workspace's own (writable) copy
    init_single_kernel<<<blocks, 256, 0, s>>>(const_cast<Inst*>(a.insts), src, src_label, level,
                                             parent, sigma, bu_ok, trace, trace_cap, a);
    return cudaGetLastError();
}

// A search on a relabelled graph ran on internal outputs: the caller's level[o]
// and parent[o] are those of internal vertex pos[o] (parents already hold
// input labels).  Internal vertices from n_keep on other than the source s_i
// are known to be unreached (columns without entries of an undirected graph)
// and are not looked up.  Reads pos in order and the internal outputs where
// it points.
__global__ void relabel_out_kernel(const uint32_t* __restrict__ pos, const int32_t* __restrict__ lev_i,
                                   const uint32_t* __restrict__ par_i, int32_t* level, int32_t* parent,
                                   uint32_t n, uint32_t n_keep, uint32_t s_i) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t o = blockIdx.x * blockDim.x + threadIdx.x; o < n; o += stride) {
        const uint32_t i = pos[o];
        int32_t lv = -1, pr = -1;
        if (i < n_keep || i == s_i) {
            lv = __ldg(lev_i + i);
            pr = (int32_t)__ldg(par_i + i);
        }
        level[o] = lv;
        parent[o] = pr;
    }
}

cudaError_t launch_relabel_out(const uint32_t* pos, const int32_t* lev_i, const uint32_t* par_i,
                               int32_t* level, int32_t* parent, uint32_t n, uint32_t n_keep,
                               uint32_t s_i, cudaStream_t s) {
    uint32_t blocks = (n + 255) / 256;
    if (blocks > 2048) blocks = 2048;
    if (blocks == 0) blocks = 1;
    relabel_out_kernel<<<blocks, 256, 0, s>>>(pos, lev_i, par_i, level, parent, n, n_keep, s_i);
    return cudaGetLastError();
}

cudaError_t launch_set_query(Inst* inst, uint32_t src, int32_t* level, uint32_t* parent,
                             unsigned long long* sigma, uint32_t bu_ok, uint4* trace,
                             uint32_t trace_cap, cudaStream_t s) {
    set_query_kernel<<<1, 1, 0, s>>>(inst, src, level, parent, sigma, bu_ok, trace, trace_cap);
    return cudaGetLastError();
}

// Sets *unsorted to 1 if some column's row indices descend (one warp per
// column, 32 neighbouring pairs at a time).
__global__ void sorted_check_kernel(const uint32_t* colptr, const uint32_t* rowidx, uint32_t n,
                                    uint32_t* unsorted) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t warps = gridDim.x * (blockDim.x / 32);
    for (uint32_t v = (blockIdx.x * blockDim.x + threadIdx.x) / 32; v < n; v += warps) {
        const uint32_t b = colptr[v], e = colptr[v + 1];
        bool bad = false;
        for (uint32_t x = b + 1 + lane; x < e; x += 32) bad |= rowidx[x] < rowidx[x - 1];
        if (__any_sync(0xFFFFFFFFu, bad)) {
            if (lane == 0) *unsorted = 1u;
            return;
        }
    }
}

cudaError_t launch_sorted_check(const uint32_t* colptr, const uint32_t* rowidx, uint32_t n,
                                uint32_t* unsorted, cudaStream_t s) {
    uint32_t blocks = (n + 7) / 8;
    if (blocks > 2048) blocks = 2048;
    if (blocks == 0) blocks = 1;
    sorted_check_kernel<<<blocks, 256, 0, s>>>(colptr, rowidx, n, unsorted);
    return cudaGetLastError();
}

// Sets bit r of `bits` for every row index r stored in the matrix (bits must be
// zero on entry).  Once per graph.
__global__ void row_bitmap_kernel(const uint32_t* rowidx, uint64_t nnz, uint32_t* bits) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < nnz; e += stride) {
        const uint32_t r = rowidx[e];
        const uint32_t bit = 1u << (r & 31);
        // most rows repeat: skip the atomic when the bit is already visible
        if (!(__ldcg(bits + (r >> 5)) & bit)) atomicOr(bits + (r >> 5), bit);
    }
}

cudaError_t launch_row_bitmap(const uint32_t* rowidx, uint64_t nnz, uint32_t* bits, uint32_t nwords,
                              cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(bits, 0, (size_t)nwords * 4, s);
    if (e != cudaSuccess || nnz == 0) return e;
    uint64_t blocks = (nnz + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    row_bitmap_kernel<<<(unsigned)blocks, 256, 0, s>>>(rowidx, nnz, bits);
    return cudaGetLastError();
}

// Writes a whole search descriptor (passed by value) into device memory.
__global__ void put_inst_kernel(Inst inst, Inst* dst) { *dst = inst; }

cudaError_t launch_put_inst(const Inst& inst, Inst* dst, cudaStream_t s) {
    put_inst_kernel<<<1, 1, 0, s>>>(inst, dst);
    return cudaGetLastError();
}

cudaError_t launch_init(const EngineArgs& a, uint32_t max_n, cudaStream_t s) {
    uint32_t blocks = (max_n + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    if (blocks == 0) blocks = 1;
    dim3 g1(blocks, a.ninst);
    init_fill_kernel<<<g1, 256, 0, s>>>(a.insts, a.ninst, a.p.mode);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    init_source_kernel<<<(a.ninst + 127) / 128, 128, 0, s>>>(a);
    return cudaGetLastError();
}

template <int MODE>
static cudaError_t set_smem_attr() {
    static bool done = false;  // one attribute call per process and template instance
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(engine_kernel<MODE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(Smem));
#if ABFS_CARVEOUT
    // the smallest shared-memory split that still holds kMinCtas CTAs leaves
    // the rest of the SM's on-chip memory to L1, where the visited-bitmap
    // words are cached
    if (e == cudaSuccess) {
        const int pct = (int)((kMinCtas * (sizeof(Smem) + 1024) * 100 + 228 * 1024 - 1) / (228 * 1024));
        e = cudaFuncSetAttribute(engine_kernel<MODE>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 pct > 100 ? 100 : pct);
    }
#endif
    // clusters of up to 16 CTAs (more than the portable 8)
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(engine_kernel<MODE>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess) done = true;
    return e;
}

// Launch configuration of the persistent engine: `grid` CTAs in clusters of
// a.p.cluster CTAs (grid is a multiple of it).
static cudaLaunchConfig_t engine_config(const EngineArgs& a, int grid, cudaStream_t s,
                                        cudaLaunchAttribute* at) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = sizeof(Smem);
    cfg.stream = s;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = a.p.cluster < 1 ? 1u : a.p.cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cfg;
}

cudaError_t launch_engine(const EngineArgs& a, int grid, cudaStream_t s) {
    cudaLaunchAttribute at[1];
    const cudaLaunchConfig_t cfg = engine_config(a, grid, s, at);
    cudaError_t e;
    if (a.p.mode == kModePlain) {
        e = set_smem_attr<kModePlain>();
        if (e != cudaSuccess) return e;
        e = cudaLaunchKernelEx(&cfg, engine_kernel<kModePlain>, a);
    } else {
        e = set_smem_attr<kModeSub>();
        if (e != cudaSuccess) return e;
        e = cudaLaunchKernelEx(&cfg, engine_kernel<kModeSub>, a);
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t engine_occupancy(uint32_t mode, int* blocks_per_sm) {
    cudaError_t e = (mode == kModePlain) ? set_smem_attr<kModePlain>() : set_smem_attr<kModeSub>();
    if (e != cudaSuccess) return e;
    if (mode == kModePlain)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, engine_kernel<kModePlain>,
                                                             kThreads, sizeof(Smem));
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, engine_kernel<kModeSub>,
                                                         kThreads, sizeof(Smem));
}

cudaError_t engine_max_clusters(uint32_t mode, uint32_t cluster, int* clusters) {
    cudaError_t e = (mode == kModePlain) ? set_smem_attr<kModePlain>() : set_smem_attr<kModeSub>();
    if (e != cudaSuccess) return e;
    EngineArgs a{};
    a.p.cluster = cluster;
    cudaLaunchAttribute at[1];
    const cudaLaunchConfig_t cfg = engine_config(a, (int)cluster * 64, nullptr, at);
    if (mode == kModePlain) return cudaOccupancyMaxActiveClusters(clusters, engine_kernel<kModePlain>, &cfg);
    return cudaOccupancyMaxActiveClusters(clusters, engine_kernel<kModeSub>, &cfg);
}

}  // namespace abfs
