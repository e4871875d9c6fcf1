// Persistent BFS engine for sm_103a.
//
// One launch runs one or many searches to completion.  Every search advances
// level by level (Algorithm 1, Section 8).  The frontier x_k is kept as a list
// of vertices in blocks; every vertex carries a weight (its column length, at
// least 1), and the level's column entries form one "entry space" of
// sum(weights) slots.  Work units are fixed-size ranges of that space, so a
// unit holds the same number of entries whether it covers one hub column or
// thousands of short ones (the PRAM "one processor per nonzero" of Theorem 4,
// with load balance instead of a processor per entry).  Any CTA may take any
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
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "internal.h"

namespace abfs {

// The phases and the expand loop are separate functions: each gets its own
// register allocation, so the cold paths' state does not push the hot loop
// into spills.  -DABFS_INLINE_ALL inlines them instead.
// Longest sleep of an idle CTA between polls for work.
#ifndef ABFS_UNIT_CEIL
#define ABFS_UNIT_CEIL 1
#endif
#ifndef ABFS_IDLE_BACKOFF_NS
#define ABFS_IDLE_BACKOFF_NS 2048
#endif
constexpr uint32_t kIdleBackoffMaxNs = ABFS_IDLE_BACKOFF_NS;

#ifdef ABFS_INLINE_ALL
#define ABFS_NOINLINE
#else
#define ABFS_NOINLINE __noinline__
#endif

// ---------------------------------------------------------------------------
// memory-ordering helpers
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Read of data written earlier in this launch by other CTAs (L2, not L1).
__device__ __forceinline__ uint32_t ld_l2(const uint32_t* p) { return __ldcg(p); }
__device__ __forceinline__ uint2 ld_l2(const uint2* p) { return __ldcg(p); }
__device__ __forceinline__ unsigned long long ld_l2(const unsigned long long* p) { return __ldcg(p); }
// Read of data that no CTA writes during the launch.
__device__ __forceinline__ uint32_t ld_ro(const uint32_t* p) { return __ldg(p); }
// Read of data that no CTA writes during the current phase (the frozen test
// bitmap): a plain load that may hit L1.  Every unit starts after an acquire
// fence, which orders it after the writes of earlier phases.
__device__ __forceinline__ uint32_t ld_frozen(const uint32_t* p) { return *p; }

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// ---------------------------------------------------------------------------
// shared state of one CTA
// ---------------------------------------------------------------------------

struct Cmd {
    uint32_t has;      // 1 = a unit was taken
    uint32_t q;        // instance
    uint32_t epoch;
    uint32_t unit;
    uint32_t kind;
    uint32_t level;
    uint32_t nitems;
    uint32_t last;     // this CTA completed the last unit of the phase
    uint32_t quit;
    uint32_t start;    // serving: this CTA claimed a newly submitted search
};

struct Smem {
    // staged frontier vertices of the unit being expanded: id, column begin
    // minus slot offset (row index of slot s is b[t] + s), slot offset, and
    // end of the vertex's entry slots
    uint32_t v[kTileMax + 1];
    uint32_t b[kTileMax + 1];
    uint32_t off[kTileMax + 1];
    uint32_t end[kTileMax];
    // bit (s - lo) set when slot s starts a staged vertex
    uint32_t sbits[kStartWords];
    // newly reached vertices staged per warp before a global append
    uint32_t wv[kWarps][kWarpBuf];
    uint32_t wcnt[kWarps];
    uint32_t wvoff[kWarps + 1];
    uint32_t wwoff[kWarps + 1];
    uint32_t gbase;
    uint32_t gblk;
    unsigned long long geb;
    uint32_t warp_sums[kWarps + 1];
    // walk state of the current unit
    uint32_t cur_b, cur_i, abort_unit, sub_cnt, sub_nseg;
    // first staged vertex of each warp's slots (the expand loop's vb), kNoVb: none
    uint32_t wvb[kWarps];
    unsigned long long sub_g0, sub_end;
    uint32_t seg_idx[32], seg_pos[32];
    unsigned long long seg_eb[32];
    unsigned long long st_read, st_unmasked, st_claims, st_nnz;
    // resident narrow run: list counters and the search's state between levels
    uint32_t nq_cnt, nt_cnt, nr_f, nr_reached, nr_shrinks, nr_stop, nr_sw, nr_mcur, nr_mprev;
    unsigned long long nq_slots;
    Cmd cmd;
    Inst I;
    uint32_t cur_q;
    uint32_t prof_on;
    uint32_t idle_exit;
    unsigned long long prof[kProfSlots];
};

// Profiling runs: thread 0 adds the cycles since t0 to slot `slot`.
__device__ __forceinline__ long long prof_now(const Smem& sm) {
    return sm.prof_on ? clock64() : 0ll;
}
__device__ __forceinline__ void prof_add(Smem& sm, int slot, long long t0) {
    if (sm.prof_on && threadIdx.x == 0) sm.prof[slot] += (unsigned long long)(clock64() - t0);
}

size_t engine_smem_bytes() { return sizeof(Smem); }

// ---------------------------------------------------------------------------
// block-level building blocks
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x) {
    const uint32_t lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
        if (lane >= (uint32_t)d) x += y;
    }
    return x;
}

// Exclusive scan of a[0..cnt) in place; a[cnt] = total.  cnt <= kThreads*ITEMS.
template <int ITEMS>
__device__ void block_exclusive_scan(uint32_t* a, uint32_t cnt, Smem& sm) {
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t x[ITEMS];
    uint32_t sum = 0;
#pragma unroll
    for (int q = 0; q < ITEMS; ++q) {
        uint32_t idx = tid * ITEMS + q;
        x[q] = idx < cnt ? a[idx] : 0u;
        sum += x[q];
    }
    uint32_t incl = warp_incl_scan(sum);
    if (lane == 31) sm.warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t s = lane < (uint32_t)kWarps ? sm.warp_sums[lane] : 0u;
        uint32_t si = warp_incl_scan(s);
        if (lane < (uint32_t)kWarps) sm.warp_sums[lane] = si - s;
        if (lane == kWarps - 1) sm.warp_sums[kWarps] = si;
    }
    __syncthreads();
    uint32_t run = sm.warp_sums[warp] + incl - sum;
#pragma unroll
    for (int q = 0; q < ITEMS; ++q) {
        uint32_t idx = tid * ITEMS + q;
        if (idx < cnt) a[idx] = run;
        run += x[q];
    }
    if (tid == 0) a[cnt] = sm.warp_sums[kWarps];
    __syncthreads();
}
constexpr int kTileItems = (kTileMax + kThreads - 1) / kThreads;

// Column of vertex v in matrix `mat` (0 = input, 1/2 = shrunk copies).
struct ColRef {
    uint32_t beg;
    uint32_t len;
};

__device__ __forceinline__ ColRef col_of(const Inst& I, uint32_t mat, uint32_t v) {
    ColRef c;
    if (mat == 0) {
        const uint32_t b = ld_ro(I.colptr + v);
        const uint32_t e = ld_ro(I.colptr + v + 1);
        c.beg = b;
        c.len = e - b;
    } else {
        c.beg = ld_l2(I.sbeg[mat - 1] + v);
        c.len = ld_l2(I.slen[mat - 1] + v);
    }
    return c;
}

__device__ __forceinline__ const uint32_t* rows_of(const Inst& I, uint32_t mat) {
    return mat == 0 ? I.rowidx : I.srows[mat - 1];
}

__device__ __forceinline__ uint32_t mat_for_level(const InstCtl* ctl, uint32_t lvl) {
    // mat_cur/mat_prev/mat_switch change only between phases; the acquire at
    // the start of a unit orders these reads.
    const uint32_t sw = ld_relaxed(&ctl->mat_switch);
    return lvl >= sw ? ld_relaxed(&ctl->mat_cur) : ld_relaxed(&ctl->mat_prev);
}

// Matrices read by levels k and k+1, from one round of independent loads.
__device__ __forceinline__ void level_mats(const InstCtl* ctl, uint32_t k, uint32_t& mat,
                                           uint32_t& mat_next) {
    const uint32_t sw = ld_relaxed(&ctl->mat_switch);
    const uint32_t cur = ld_relaxed(&ctl->mat_cur);
    const uint32_t prev = ld_relaxed(&ctl->mat_prev);
    mat = k >= sw ? cur : prev;
    mat_next = k + 1 >= sw ? cur : prev;
}

__device__ __forceinline__ void fail(InstCtl* ctl, uint32_t code) { atomicCAS(&ctl->err, 0u, code); }

// L2 policy for the streamed row indices: evict first, so the search's hot
// state (bitmaps, parents, column pointers, queues) stays resident.
__device__ __forceinline__ uint64_t evict_first_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// Row index load: the input matrix never changes during a launch (read-only
// path); shrunk copies are written by earlier phases of the same launch.
__device__ __forceinline__ uint32_t ld_row(const uint32_t* rows, uint32_t idx, uint32_t mat,
                                           uint64_t pol) {
    uint32_t v;
    if (mat == 0)
        asm("ld.global.nc.L1::no_allocate.L2::cache_hint.u32 %0, [%1], %2;"
            : "=r"(v)
            : "l"(rows + idx), "l"(pol));
    else
        asm volatile("ld.global.cg.L2::cache_hint.u32 %0, [%1], %2;"
                     : "=r"(v)
                     : "l"(rows + idx), "l"(pol)
                     : "memory");
    return v;
}

// ---------------------------------------------------------------------------
// appending newly reached vertices as frontier blocks
// ---------------------------------------------------------------------------

// Each lane's vertex i of block blk (entry range [g0, g0 + w); w = 0: no
// vertex) owns the unit starts (multiples of P.unit) inside its range; the
// warp writes them together, 32 starts per round, so one long column does not
// serialise its lane.  Whole warp.
__device__ __forceinline__ void warp_unit_starts(const Inst& I, InstCtl* ctl, const EngineParams& P,
                                                 uint32_t pn, uint32_t blk, uint32_t i,
                                                 unsigned long long g0, uint32_t w) {
    const uint32_t lane = threadIdx.x & 31;
    const unsigned long long U1 = P.unit - 1;  // a power of two
    unsigned long long uf = 0;
    uint32_t c = 0;
    if (w) {
        uf = (g0 + U1) >> P.unit_shift;
        c = (uint32_t)(((g0 + w + U1) >> P.unit_shift) - uf);
    }
    const uint32_t incl = warp_incl_scan(c);
    const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    for (uint32_t t0 = 0; t0 < total; t0 += 32) {
        const uint32_t t = t0 + lane;
        // owner: the first lane whose inclusive count exceeds t
        uint32_t owner = 0;
#pragma unroll
        for (uint32_t d = 16; d > 0; d >>= 1) {
            const uint32_t probe = __shfl_sync(0xFFFFFFFFu, incl, owner + d - 1);
            if (t >= probe) owner += d;
        }
        const unsigned long long o_uf = __shfl_sync(0xFFFFFFFFu, uf, owner);
        const uint32_t o_excl = __shfl_sync(0xFFFFFFFFu, incl - c, owner);
        const uint32_t o_i = __shfl_sync(0xFFFFFFFFu, i, owner);
        if (t < total) {
            const unsigned long long u = o_uf + (t - o_excl);
            if (u < I.ucap) I.ustart[pn][u] = make_uint2(blk, o_i);
            else fail(ctl, 7 /* ABFS_ERR_DEVICE */);
        }
    }
}

// Reserves a block of `cnt` vertices with `wsum` entries in the frontier of
// parity pn: returns (block number, entry base, vertex base) or fails.
__device__ __forceinline__ bool reserve_block(const Inst& I, InstCtl* ctl, uint32_t pn, uint32_t cnt,
                                              uint32_t wsum, uint32_t& blk,
                                              unsigned long long& eb, uint32_t& vb) {
    const unsigned long long old =
        atomicAdd(&ctl->bctr[pn], ((unsigned long long)wsum << kBlockBits) | 1ull);
    blk = (uint32_t)(old & kBlockMask);
    eb = old >> kBlockBits;
    vb = atomicAdd(&ctl->fcnt[pn], cnt);
    if (blk >= I.bcap || blk >= kBlockMask || (unsigned long long)vb + cnt > I.n) {
        fail(ctl, 7);
        return false;
    }
    Block* B = I.blk[pn] + blk;
    B->vb = vb;
    B->nv = cnt;
    B->eb = eb;
    return true;
}

// Warp-aggregated append of newly reached vertex v (where `want`) to this
// warp's staging buffer; wc is the warp's (uniform) staged count.
__device__ __forceinline__ void stage_warp(bool want, uint32_t v, Smem& sm, uint32_t& wc) {
    const uint32_t mask = __ballot_sync(0xFFFFFFFFu, want);
    if (!mask) return;
    if (want) sm.wv[threadIdx.x >> 5][wc + __popc(mask & lanemask_lt())] = v;
    wc += __popc(mask);
}

// Columns (matrix mat_next) of this warp's n staged vertices, lane-strided:
// entry it of a lane is staged vertex it*32 + lane.
constexpr int kWarpSpans = kWarpBuf / 32;
struct WarpCols {
    uint32_t beg[kWarpSpans];
    uint32_t len[kWarpSpans];
};

// Looks the columns up once; returns the staged vertices' total weight
// (column length + kVertexSlots each).  Whole warp.
__device__ __forceinline__ uint32_t warp_cols(Smem& sm, const Inst& I, uint32_t mat_next, uint32_t n,
                                              WarpCols& c) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t* wv = sm.wv[threadIdx.x >> 5];
    uint32_t sum = 0;
#pragma unroll
    for (int it = 0; it < kWarpSpans; ++it) {
        const uint32_t i = it * 32 + lane;
        c.beg[it] = 0;
        c.len[it] = 0;
        if (i < n) {
            const ColRef r = col_of(I, mat_next, wv[i]);
            c.beg[it] = r.beg;
            c.len[it] = r.len;
            sum += r.len + kVertexSlots;
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) sum += __shfl_xor_sync(0xFFFFFFFFu, sum, d);
    return sum;
}

// Writes this warp's n staged vertices (columns c) at fq[vb + voff ..] of
// block blk (entry base eb), the group starting at weight offset woff within
// the block.  Whole warp.
__device__ __forceinline__ void warp_emit(Smem& sm, const Inst& I, InstCtl* ctl,
                                          const EngineParams& P, uint32_t pn, const WarpCols& c,
                                          uint32_t n, uint32_t blk, unsigned long long eb,
                                          uint32_t vb, uint32_t voff, uint32_t woff) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t* wv = sm.wv[threadIdx.x >> 5];
    uint32_t carry = woff;
#pragma unroll
    for (int it = 0; it < kWarpSpans; ++it) {
        if ((uint32_t)it * 32 >= n) break;
        const uint32_t i = it * 32 + lane;
        const uint32_t w = i < n ? c.len[it] + kVertexSlots : 0u;
        const uint32_t incl = warp_incl_scan(w);
        const uint32_t pre = carry + incl - w;
        if (i < n) {
            const uint32_t at = vb + voff + i;
            I.fq[pn][at] = wv[i];
            I.fbeg[pn][at] = c.beg[it];
            I.fpre[pn][at] = pre;
        }
        warp_unit_starts(I, ctl, P, pn, blk, voff + i, eb + pre, w);
        carry += __shfl_sync(0xFFFFFFFFu, incl, 31);
    }
    __syncwarp();
}

// A warp writes its staging buffer out as a frontier block of its own.  It is
// called from inside the expand loop, so it keeps little state: the columns are
// looked up once for the block's weight and again while writing (a cached copy
// would cost the loop registers).
#ifdef ABFS_FLUSH_INLINE
__device__ __forceinline__ void warp_flush(
#else
__device__ ABFS_NOINLINE void warp_flush(
#endif
    Smem& sm, const Inst& I, InstCtl* ctl, const EngineParams& P, uint32_t pn, uint32_t mat_next,
    uint32_t& wc) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t n = wc;
    const uint32_t* wv = sm.wv[threadIdx.x >> 5];
    uint32_t wtot = 0;
    for (uint32_t i = lane; i < n; i += 32) wtot += col_of(I, mat_next, wv[i]).len + kVertexSlots;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) wtot += __shfl_xor_sync(0xFFFFFFFFu, wtot, d);
    uint32_t blk = 0, vb = 0, ok = 0;
    unsigned long long eb = 0;
    if (lane == 0) ok = reserve_block(I, ctl, pn, n, wtot, blk, eb, vb);
    ok = __shfl_sync(0xFFFFFFFFu, ok, 0);
    blk = __shfl_sync(0xFFFFFFFFu, blk, 0);
    vb = __shfl_sync(0xFFFFFFFFu, vb, 0);
    eb = __shfl_sync(0xFFFFFFFFu, eb, 0);
    if (ok) {
        uint32_t carry = 0;
        for (uint32_t base = 0; base < n; base += 32) {
            const uint32_t i = base + lane;
            ColRef c;
            c.beg = 0;
            c.len = 0;
            uint32_t v = 0;
            if (i < n) {
                v = wv[i];
                c = col_of(I, mat_next, v);
            }
            const uint32_t w = i < n ? c.len + kVertexSlots : 0u;
            const uint32_t incl = warp_incl_scan(w);
            const uint32_t pre = carry + incl - w;
            if (i < n) {
                I.fq[pn][vb + i] = v;
                I.fbeg[pn][vb + i] = c.beg;
                I.fpre[pn][vb + i] = pre;
            }
            warp_unit_starts(I, ctl, P, pn, blk, i, eb + pre, w);
            carry += __shfl_sync(0xFFFFFFFFu, incl, 31);
        }
    }
    __syncwarp();
    wc = 0;
}

// End of a unit: the leftovers of all warps (counts in sm.wcnt) leave as one
// frontier block.  Whole CTA.
__device__ ABFS_NOINLINE void cta_flush(Smem& sm, const Inst& I, InstCtl* ctl,
                                        const EngineParams& P, uint32_t pn, uint32_t mat_next) {
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    const uint32_t n = sm.wcnt[warp];
    WarpCols c;
    const uint32_t wtot = warp_cols(sm, I, mat_next, n, c);
    if (lane == 0) {
        sm.wvoff[warp] = n;
        sm.wwoff[warp] = wtot;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t v = 0, w = 0;
        for (int q = 0; q < kWarps; ++q) {
            const uint32_t a = sm.wvoff[q], b = sm.wwoff[q];
            sm.wvoff[q] = v;
            sm.wwoff[q] = w;
            v += a;
            w += b;
        }
        sm.wvoff[kWarps] = v;
        sm.wwoff[kWarps] = w;
        uint32_t blk = 0, vb = 0;
        unsigned long long eb = 0;
        const bool ok = v ? reserve_block(I, ctl, pn, v, w, blk, eb, vb) : false;
        sm.gblk = ok ? blk : kUnset;
        sm.geb = eb;
        sm.gbase = vb;
    }
    __syncthreads();
    if (sm.gblk != kUnset && n)
        warp_emit(sm, I, ctl, P, pn, c, n, sm.gblk, sm.geb, sm.gbase, sm.wvoff[warp],
                  sm.wwoff[warp]);
    if (lane == 0) sm.wcnt[warp] = 0;
    __syncthreads();
}

// Resident narrow runs: a warp appends its n staged vertices to the frontier
// list of parity pn (vertex, column begin, column length in matrix mat_next),
// at a position taken from a shared-memory counter.  Whole warp.
__device__ __forceinline__ void narrow_append(Smem& sm, const Inst& I, InstCtl* ctl, uint32_t pn, uint32_t mat_next,
                              uint32_t& wc) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t n = wc;
    const uint32_t* wv = sm.wv[threadIdx.x >> 5];
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(&sm.nq_cnt, n);
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    uint32_t wsum = 0;
    for (uint32_t i0 = 0; i0 < n; i0 += 32 * kIlp) {
        uint32_t v[kIlp];
        ColRef c[kIlp];
#pragma unroll
        for (int q = 0; q < kIlp; ++q) {
            const uint32_t i = i0 + 32 * q + lane;
            v[q] = 0;
            c[q].beg = 0;
            c[q].len = 0;
            if (i < n) {
                v[q] = wv[i];
                c[q] = col_of(I, mat_next, v[q]);
            }
        }
#pragma unroll
        for (int q = 0; q < kIlp; ++q) {
            const uint32_t i = i0 + 32 * q + lane;
            if (i < n) {
                const uint32_t at = base + i;
                if (at < I.n) {
                    I.fq[pn][at] = v[q];
                    I.fbeg[pn][at] = c[q].beg;
                    I.fpre[pn][at] = c[q].len;
                } else {
                    fail(ctl, 7);
                }
                wsum += c[q].len + kVertexSlots;
            }
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) wsum += __shfl_xor_sync(0xFFFFFFFFu, wsum, d);
    if (lane == 0 && n) atomicAdd(&sm.nq_slots, (unsigned long long)wsum);
    __syncwarp();
    wc = 0;
}

// Resident narrow runs of the comparator: a warp appends its n staged
// first-touched rows to the touched list.  Whole warp.
__device__ __forceinline__ void narrow_touch(Smem& sm, const Inst& I, InstCtl* ctl, uint32_t& wc) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t n = wc;
    const uint32_t* wv = sm.wv[threadIdx.x >> 5];
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(&sm.nt_cnt, n);
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    for (uint32_t i = lane; i < n; i += 32) {
        const uint32_t at = base + i;
        if (at < I.n) I.touched[at] = wv[i];
        else fail(ctl, 7);
    }
    __syncwarp();
    wc = 0;
}

// Comparator accumulator key of frontier column j at level k: the high word is
// a stamp that decreases with k (and stays below the all-ones initial value),
// so one atomicMin both overwrites stale keys and keeps the least j.
__device__ __forceinline__ uint32_t plain_stamp(uint32_t k) { return kUnset - 1u - k; }
__device__ __forceinline__ unsigned long long plain_key(uint32_t k, uint32_t j) {
    return ((unsigned long long)plain_stamp(k) << 32) | (unsigned long long)j;
}

// Per-thread counters of one work unit.
struct Tally {
    uint32_t read = 0;
    uint32_t unmasked = 0;
    uint32_t claims = 0;
};

// ---------------------------------------------------------------------------
// the per-entry step: mask, multiply, claim -- kIlp entries per thread at once
// ---------------------------------------------------------------------------

// How a level claims the vertices it reaches.
enum ClaimVar : int {
    kVarWide = 0,    // atomicMin with return; the winner stages the vertex (frontier blocks)
    kVarNarrow = 1,  // the same inside a resident narrow run (plain frontier list)
    kVarScan = 2,    // reductions only: atomicMin and the bit in the write bitmap without
                     // return; an extraction phase collects the new vertices afterwards
};

// Groups of 32 entries each thread keeps in flight, per claim variant.
__host__ __device__ constexpr int ilp_of(int var) { return var == kVarScan ? kIlpScan : kIlp; }

// Entries (r[u] in column j[u]; r[u] == kUnset: none) at level k.  Each stage issues
// kIlp independent memory operations before consuming any.  Submatrix mode
// appends the vertices of level k+1 to the next frontier; comparator mode
// appends first-touched rows to the touched list.  All 32 lanes must call.
template <int MODE, int VAR>
__device__ __forceinline__ void process_group(const Inst& I, InstCtl* ctl, const EngineParams& P,
                                              Smem& sm, uint32_t k, const uint32_t (&r)[ilp_of(VAR)],
                                              const uint32_t (&j)[ilp_of(VAR)], Tally& t,
                                              uint32_t& wc) {
    constexpr int L = ilp_of(VAR);
    const uint32_t p = k & 1;
    if (MODE == kModeSub) {
        const uint32_t* test_bm = I.bm[p];
        uint32_t* write_bm = I.bm[p ^ 1];
        // all-nonzero variant over the arithmetic semiring (shortest-path
        // counts): every entry that passes the mask adds x_k(j) = sigma[j],
        // final since level k-1 completed, into sigma[r]
        unsigned long long* const sigma = I.sigma;
        uint32_t w[L];
#pragma unroll
        for (int u = 0; u < L; ++u)
            w[u] = r[u] != kUnset
                       ? (VAR == kVarNarrow ? ld_l2(test_bm + (r[u] >> 5))
                                            : ld_frozen(test_bm + (r[u] >> 5)))
                       : 0xFFFFFFFFu;
        if (VAR == kVarScan) {
            // the (min, index) product as a reduction: the least column still
            // wins, and once the level is complete the new vertices are the
            // unvisited ones whose parent is set
#pragma unroll
            for (int u = 0; u < L; ++u) {
                if (!((w[u] >> (r[u] & 31)) & 1u)) {
                    ++t.unmasked;
                    ++t.claims;
                    atomicMin(I.parent + r[u], j[u]);
                    if (sigma) atomicAdd(sigma + r[u], ld_l2(sigma + j[u]));
                }
            }
            return;
        }
        // rows outside V_{k+1} are masked before the multiply; the (min, index)
        // product is an atomicMin of j into parent[r], and moving parent[r]
        // off "unset" claims r for level k+1
        bool win[L];
#pragma unroll
        for (int u = 0; u < L; ++u) {
            win[u] = false;
            if (!((w[u] >> (r[u] & 31)) & 1u)) {
                ++t.unmasked;
                ++t.claims;
                win[u] = atomicMin(I.parent + r[u], j[u]) == kUnset;
                if (sigma) atomicAdd(sigma + r[u], ld_l2(sigma + j[u]));
            }
        }
#pragma unroll
        for (int u = 0; u < L; ++u) {
            if (win[u]) {
                I.level[r[u]] = (int32_t)(k + 1);
                atomicOr(write_bm + (r[u] >> 5), 1u << (r[u] & 31));
            }
            stage_warp(win[u], r[u], sm, wc);
        }
    } else {
        // multiply first: every entry reaches the accumulator
        unsigned long long old[L];
#pragma unroll
        for (int u = 0; u < L; ++u) {
            old[u] = 0ull;
            if (r[u] != kUnset) {
                ++t.unmasked;
                ++t.claims;
                old[u] = atomicMin(I.y + r[u], plain_key(k, j[u]));
            }
        }
        // first touch of row r at this level: it goes to the touched list
        // (narrow runs stage it with the warp's other appends)
        if (VAR == kVarNarrow) {
#pragma unroll
            for (int u = 0; u < L; ++u)
                stage_warp(r[u] != kUnset && (uint32_t)(old[u] >> 32) != plain_stamp(k), r[u], sm, wc);
            return;
        }
#pragma unroll
        for (int u = 0; u < L; ++u) {
            const bool first = r[u] != kUnset && (uint32_t)(old[u] >> 32) != plain_stamp(k);
            const uint32_t mask = __ballot_sync(0xFFFFFFFFu, first);
            if (mask) {
                const uint32_t lane = threadIdx.x & 31, leader = __ffs(mask) - 1;
                uint32_t base = 0;
                if (lane == leader) base = atomicAdd(&ctl->tcnt, (uint32_t)__popc(mask));
                base = __shfl_sync(0xFFFFFFFFu, base, leader);
                if (first) {
                    const uint32_t at = base + __popc(mask & lanemask_lt());
                    if (at < I.n) I.touched[at] = r[u];
                    else fail(ctl, 7);
                }
            }
        }
    }
}

__device__ __forceinline__ void tally_flush(Smem& sm, Tally t) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        t.read += __shfl_xor_sync(0xFFFFFFFFu, t.read, d);
        t.unmasked += __shfl_xor_sync(0xFFFFFFFFu, t.unmasked, d);
        t.claims += __shfl_xor_sync(0xFFFFFFFFu, t.claims, d);
    }
    if ((threadIdx.x & 31) == 0) {
        if (t.read) atomicAdd(&sm.st_read, (unsigned long long)t.read);
        if (t.unmasked) atomicAdd(&sm.st_unmasked, (unsigned long long)t.unmasked);
        if (t.claims) atomicAdd(&sm.st_claims, (unsigned long long)t.claims);
    }
}

__device__ __forceinline__ void stats_flush(Smem& sm, InstCtl* ctl) {
    __syncthreads();
    if (threadIdx.x == 0) {
        if (sm.st_read) atomicAdd(&ctl->entries_read, sm.st_read);
        if (sm.st_unmasked) atomicAdd(&ctl->entries_unmasked, sm.st_unmasked);
        if (sm.st_claims) atomicAdd(&ctl->claims, sm.st_claims);
        if (sm.st_nnz) atomicAdd(&ctl->nnz_reached, sm.st_nnz);
        sm.st_read = sm.st_unmasked = sm.st_claims = sm.st_nnz = 0;
    }
}

// ---------------------------------------------------------------------------
// work units
// ---------------------------------------------------------------------------

// Slots [lo, hi) are split evenly over the warps: warp w starts at
// lo + w * per, per = ceil((hi - lo) / kWarps).  Staged vertex s, whose slots
// are [st, en), records itself for every warp that starts inside its range (as
// s - 1 when the warp starts on s's first slot, since that start bit counts
// again in the expand loop).  Called for every staged vertex before the loop.
constexpr uint32_t kNoVb = 0xFFFFFFFEu;  // real values are -1 .. kTileMax - 1
__device__ __forceinline__ uint32_t warp_share(uint32_t lo, uint32_t hi) {
    return (hi - lo + kWarps - 1) / kWarps;
}
__device__ __forceinline__ void mark_warp_starts(Smem& sm, uint32_t s, uint32_t st, uint32_t en,
                                                 uint32_t lo, uint32_t hi) {
    if (hi <= lo || en <= lo || st >= hi) return;
    const uint32_t per = warp_share(lo, hi);
    for (uint32_t w = st > lo ? (st - lo + per - 1) / per : 0u; w < (uint32_t)kWarps; ++w) {
        const uint32_t e0 = lo + w * per;
        if (e0 >= en || e0 >= hi) break;
        sm.wvb[w] = e0 == st ? s - 1u : s;
    }
}

// Expands the slots [l0, l1) of the staged vertices (cnt of them; sm.off holds
// their first slots, sm.off[cnt] the end; sm.sbits marks the first slots that
// fall in [l0, l1)).  Slot s of vertex t is the column entry with row index
// b[t] + s if s < end[t]; the kVertexSlots slots after its entries are empty.
// The slots are split evenly over the warps; a warp takes 32 consecutive
// slots per group (coalesced row loads) and kIlp groups per step.  The vertex
// of slot s is a prefix count of vertex starts, read from sm.sbits with one
// popcount.  The row loads of step s+1 are issued before step s is processed.
template <int MODE, int VAR>
__device__ __forceinline__ void expand_core(const Inst& I, InstCtl* ctl, const EngineParams& P, Smem& sm,
                             uint32_t cnt, uint32_t l0, uint32_t l1, uint32_t mat,
                             uint32_t mat_next, uint32_t k, Tally& t) {
    constexpr int L = ilp_of(VAR);
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#ifdef ABFS_EXPAND_PROFILE
    const long long xt0 = sm.prof_on ? clock64() : 0ll;
#endif
    const uint32_t span = l1 - l0;
    const uint32_t per = (span + kWarps - 1) / kWarps;
    const uint32_t e0 = l0 + min(span, warp * per);
    const uint32_t e1 = l0 + min(span, warp * per + per);
    const uint32_t* rows = rows_of(I, mat);
    const uint64_t pol = evict_first_policy();
    const uint32_t le_mask = (2u << lane) - 1u;  // lanes 0..lane
    // vertex(s) = vb + (number of vertex starts in [e0, s])
    uint32_t vb = 0;
    if (e0 < e1) {
        vb = sm.wvb[warp];
        // recorded while staging; searched for only if the record is missing
        if (vb == kNoVb || (vb != kUnset && vb >= cnt)) {
            uint32_t lo = 0, hi = cnt;  // off[lo] <= e0 < off[hi]
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (sm.off[mid] <= e0) lo = mid;
                else hi = mid;
            }
            vb = lo - (sm.off[lo] == e0 ? 1u : 0u);
        }
    }
    uint32_t starts = 0;  // vertex starts in [e0, current group base)
    // row index (kUnset: no entry in this slot) and frontier column of each group
    uint32_t r[L], j[L];
    auto load_step = [&](uint32_t base, uint32_t (&rr)[L], uint32_t (&jj)[L]) {
#pragma unroll
        for (int u = 0; u < L; ++u) {
            const uint32_t gb = base + 32 * u;
            const uint32_t rel = gb - l0;
            const uint32_t sh = rel & 31;
            uint32_t w = sm.sbits[rel >> 5] >> sh;
            if (sh) w |= sm.sbits[(rel >> 5) + 1] << (32 - sh);
            const uint32_t s = gb + lane;
            const uint32_t v = vb + starts + __popc(w & le_mask);
            starts += __popc(w);
            rr[u] = kUnset;
            jj[u] = 0;
            if (s < e1 && s < sm.end[v]) {
                jj[u] = sm.v[v];
                rr[u] = ld_row(rows, sm.b[v] + s, mat, pol);
            }
        }
    };
    uint32_t wc = sm.wcnt[warp];
    if (e0 < e1) load_step(e0, r, j);
#ifdef ABFS_EXPAND_PROFILE
    long long xt1 = 0, xflush = 0, xproc = 0;
    if (sm.prof_on) xt1 = clock64();
#endif
    for (uint32_t base = e0; base < e1; base += 32 * L) {
        uint32_t r2[L], j2[L];
        if (base + 32 * L < e1) {
            load_step(base + 32 * L, r2, j2);
        } else {
#pragma unroll
            for (int u = 0; u < L; ++u) {
                r2[u] = kUnset;
                j2[u] = 0;
            }
        }
#pragma unroll
        for (int u = 0; u < L; ++u) t.read += (r[u] != kUnset);
#ifdef ABFS_EXPAND_PROFILE
        const long long xp0 = sm.prof_on ? clock64() : 0ll;
#endif
        process_group<MODE, VAR>(I, ctl, P, sm, k, r, j, t, wc);
#ifdef ABFS_EXPAND_PROFILE
        const long long xp1 = sm.prof_on ? clock64() : 0ll;
        xproc += xp1 - xp0;
#endif
        if (VAR == kVarScan) {
            // nothing staged
        } else if (VAR == kVarNarrow) {
            if (wc > (uint32_t)kWarpFlushAt) {
                if (MODE == kModeSub) narrow_append(sm, I, ctl, (k + 1) & 1, mat_next, wc);
                else narrow_touch(sm, I, ctl, wc);
            }
        } else if (MODE == kModeSub && wc > (uint32_t)kWarpFlushAt) {
            warp_flush(sm, I, ctl, P, (k + 1) & 1, mat_next, wc);
        }
#ifdef ABFS_EXPAND_PROFILE
        if (sm.prof_on) xflush += clock64() - xp1;
#endif
#pragma unroll
        for (int u = 0; u < L; ++u) {
            r[u] = r2[u];
            j[u] = j2[u];
        }
    }
    if (lane == 0) sm.wcnt[warp] = wc;
#ifdef ABFS_EXPAND_PROFILE
    // per-warp accounting, in builds made for profiling the expand loop
    if (sm.prof_on && lane == 0) {
        const long long xt2 = clock64();
        atomicAdd(&sm.prof[kProfXSetup], (unsigned long long)(xt1 - xt0));
        atomicAdd(&sm.prof[kProfXProcess], (unsigned long long)xproc);
        atomicAdd(&sm.prof[kProfXFlush], (unsigned long long)xflush);
        atomicAdd(&sm.prof[kProfXLoop], (unsigned long long)(xt2 - xt1));
        atomicAdd(&sm.prof[kProfXCalls], 1ull);
    }
#endif
    __syncwarp();
}

// The expand loop of wide units, compiled as a function of its own.
template <int MODE, int VAR>
__device__ ABFS_NOINLINE void expand_slots(const Inst& I, InstCtl* ctl, const EngineParams& P,
                                           Smem& sm, uint32_t cnt, uint32_t l0, uint32_t l1,
                                           uint32_t mat, uint32_t mat_next, uint32_t k, Tally& t) {
    expand_core<MODE, VAR>(I, ctl, P, sm, cnt, l0, l1, mat, mat_next, k, t);
}

// Unit u of the level-k frontier: entry slots [u*U, min((u+1)*U, total)) with
// U = m granules of P.unit slots (m is chosen per level).  The unit walks the
// frontier blocks in entry order from the vertex recorded in the unit start of
// its first granule, staging up to `tile` vertices from up to 32 blocks at a
// time.
template <int MODE, int VAR>
__device__ ABFS_NOINLINE void unit_level(const Inst& I, InstCtl* ctl, const EngineParams& P, Smem& sm,
                           uint32_t k, uint32_t u, uint32_t m) {
    const uint32_t p = k & 1;
    const unsigned long long bc = ld_relaxed64(&ctl->bctr[p]);
    uint32_t mat, mat_next;
    level_mats(ctl, k, mat, mat_next);
    const unsigned long long total = bc >> kBlockBits;
    const uint32_t nb = (uint32_t)(bc & kBlockMask);
    const unsigned long long U = (unsigned long long)P.unit * m;
    const unsigned long long u_lo = (unsigned long long)u * U;
    const unsigned long long u_hi = min(total, u_lo + U);
    const Block* blk = I.blk[p];
    if (threadIdx.x == 0) {
        const uint2 st = ld_l2(I.ustart[p] + (unsigned long long)u * m);
        sm.cur_b = st.x;
        sm.cur_i = st.y;
    }
    __syncthreads();
    Tally t;
    unsigned long long e = u_lo;
    uint32_t nnz_local = 0;
    while (e < u_hi) {
        const long long pt0 = prof_now(sm);
        // warp 0: the next up-to-32 blocks, as segments of this sub-tile
        if (threadIdx.x < 32) {
            const uint32_t lane = threadIdx.x;
            const uint32_t b = sm.cur_b + lane;
            uint32_t vb = 0, nv = 0;
            unsigned long long eb = total;
            if (b < nb && b < I.bcap) {
                vb = ld_l2(&blk[b].vb);
                nv = ld_l2(&blk[b].nv);
                eb = ld_l2(&blk[b].eb);
            }
            const uint32_t i0 = lane == 0 ? sm.cur_i : 0u;
            const uint32_t avail = (b < nb && nv > i0) ? nv - i0 : 0u;
            // entry position of the segment's first vertex
            unsigned long long start = eb;
            if (lane == 0 && avail) start = eb + ld_l2(I.fpre[p] + vb + i0);
            const uint32_t incl = warp_incl_scan(avail);
            const uint32_t excl = incl - avail;
            uint32_t take = 0;
            if (avail && start < u_hi && excl < P.tile) take = min(avail, P.tile - excl);
            const uint32_t tmask = __ballot_sync(0xFFFFFFFFu, take > 0);
            const uint32_t nseg = __popc(tmask);  // a prefix of the lanes
            const uint32_t ntake = __shfl_sync(0xFFFFFFFFu, excl + take, nseg ? nseg - 1 : 0);
            if (take) {
                sm.seg_idx[lane] = vb + i0;
                sm.seg_pos[lane] = excl;
                sm.seg_eb[lane] = eb;
            }
            const unsigned long long eb_next = __shfl_down_sync(0xFFFFFFFFu, eb, 1);
            if (nseg && lane == nseg - 1) {
                // end slot of the last staged vertex, and where the next sub-tile starts
                const uint32_t last_i = i0 + take;  // one past the last staged vertex
                unsigned long long end;
                if (last_i < nv) {
                    end = eb + ld_l2(I.fpre[p] + vb + last_i);
                    sm.cur_b = b;
                    sm.cur_i = last_i;
                } else {
                    end = (b + 1 >= nb) ? total : (lane < 31 ? eb_next : ld_l2(&blk[b + 1].eb));
                    sm.cur_b = b + 1;
                    sm.cur_i = 0;
                }
                sm.sub_end = end;
            }
            if (lane == 0) {
                sm.sub_cnt = nseg ? ntake : 0u;
                sm.sub_nseg = nseg;
                sm.sub_g0 = start;
                // the first segment must contain slot e: otherwise an invariant broke
                sm.abort_unit = (!(tmask & 1u) || start > e) ? 1u : 0u;
            }
        }
        __syncthreads();
        if (sm.abort_unit) {
            if (threadIdx.x == 0) fail(ctl, 7);
            break;
        }
        const uint32_t cnt = sm.sub_cnt, nseg = sm.sub_nseg;
        const unsigned long long g0 = sm.sub_g0;
        for (uint32_t s = threadIdx.x; s < cnt; s += kThreads) {
            uint32_t q = 0, hi = nseg;  // seg_pos[q] <= s < seg_pos[hi]
            while (hi - q > 1) {
                const uint32_t mid = (q + hi) >> 1;
                if (sm.seg_pos[mid] <= s) q = mid;
                else hi = mid;
            }
            const uint32_t idx = sm.seg_idx[q] + (s - sm.seg_pos[q]);
            sm.v[s] = ld_l2(I.fq[p] + idx);
            sm.b[s] = ld_l2(I.fbeg[p] + idx);
            sm.off[s] = (uint32_t)(sm.seg_eb[q] + ld_l2(I.fpre[p] + idx) - g0);
        }
        if (threadIdx.x == 0) sm.off[cnt] = (uint32_t)(sm.sub_end - g0);
        if (threadIdx.x < (uint32_t)kWarps) sm.wvb[threadIdx.x] = kNoVb;
        // slots [lo, hi) of this sub-tile belong to the unit
        const uint32_t lo = (uint32_t)(e - g0);
        const uint32_t hi_s = (uint32_t)(min(u_hi, (unsigned long long)sm.sub_end) - g0);
        const uint32_t nwords = (hi_s - lo + 31) / 32 + 1;
        for (uint32_t w = threadIdx.x; w < nwords; w += kThreads) sm.sbits[w] = 0u;
        __syncthreads();
        for (uint32_t s = threadIdx.x; s < cnt; s += kThreads) {
            const uint32_t st = sm.off[s];
            const uint32_t len = sm.off[s + 1] - st - kVertexSlots;
            sm.end[s] = st + len;
            sm.b[s] -= st;  // row index of slot x is b + x
            mark_warp_starts(sm, s, st, st + len + kVertexSlots, lo, hi_s);
            if (st >= lo && st < hi_s) {
                // the vertex's first slot lies in this unit: it joins the visited
                // set of the next level's test (once), and starts a run of slots
                atomicOr(&sm.sbits[(st - lo) >> 5], 1u << ((st - lo) & 31));
                const uint32_t v = sm.v[s];
                if (MODE == kModeSub) atomicOr(I.bm[p ^ 1] + (v >> 5), 1u << (v & 31));
                nnz_local += (mat == 0) ? len : (ld_ro(I.colptr + v + 1) - ld_ro(I.colptr + v));
            }
        }
        __syncthreads();
        const unsigned long long s_hi = min(u_hi, (unsigned long long)sm.sub_end);
        const long long pt1 = prof_now(sm);
        prof_add(sm, kProfGather, pt0);
        expand_slots<MODE, VAR>(I, ctl, P, sm, cnt, (uint32_t)(e - g0), (uint32_t)(s_hi - g0), mat,
                                mat_next, k, t);
        const long long pt2 = prof_now(sm);
        prof_add(sm, kProfExpand, pt1);
        e = s_hi;
        __syncthreads();
        prof_add(sm, kProfWait, pt2);
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) nnz_local += __shfl_xor_sync(0xFFFFFFFFu, nnz_local, d);
    if ((threadIdx.x & 31) == 0 && nnz_local) atomicAdd(&sm.st_nnz, (unsigned long long)nnz_local);
    tally_flush(sm, t);
    const long long pt3 = prof_now(sm);
    if (MODE == kModeSub && VAR != kVarScan) cta_flush(sm, I, ctl, P, p ^ 1, mat_next);
    prof_add(sm, kProfFlush, pt3);
}

// Comparator: apply the visited mask to a tile of touched rows of level k.
__device__ ABFS_NOINLINE void unit_plain_mask(const Inst& I, InstCtl* ctl, const EngineParams& P, Smem& sm,
                                uint32_t k, uint32_t tile_idx, uint32_t ntouched) {
    const uint32_t pn = (k + 1) & 1;
    const uint32_t base = tile_idx * P.tile;
    const uint32_t cnt = min(P.tile, ntouched - base);
    uint32_t mat, mat_next;
    level_mats(ctl, k, mat, mat_next);
    uint32_t wc = sm.wcnt[threadIdx.x >> 5];
    for (uint32_t b0 = 0; b0 < cnt; b0 += kThreads) {
        const uint32_t t = b0 + threadIdx.x;
        bool want = false;
        uint32_t r = 0;
        if (t < cnt) {
            r = ld_l2(I.touched + base + t);
            if ((int32_t)ld_relaxed((const uint32_t*)I.level + r) == -1) {
                const unsigned long long y = ld_relaxed64(I.y + r);
                I.level[r] = (int32_t)(k + 1);
                I.parent[r] = (uint32_t)(y & 0xFFFFFFFFull);
                want = true;
            }
        }
        stage_warp(want, r, sm, wc);
        if (wc > (uint32_t)(kWarpBuf - 32)) warp_flush(sm, I, ctl, P, pn, mat_next, wc);
    }
    if ((threadIdx.x & 31) == 0) sm.wcnt[threadIdx.x >> 5] = wc;
    cta_flush(sm, I, ctl, P, pn, mat_next);
}

// Vertices per extraction unit: one bitmap word per thread.
// Bitmap-word phases (extraction, frontier bitmap, bottom-up levels) work in
// chunks of 8 words, one chunk per warp at a time; a unit is a run of chunks
// (nitems per unit, chosen by the advancing CTA so a phase makes about two
// units per CTA), which keeps the per-unit costs (take, flush, count-down) to
// two per CTA whatever the size of the graph.
constexpr uint32_t kChunkWords = 8;

// Extraction after a level k whose claims were reductions: the vertices of
// level k+1 (V_{k+1} minus V_{k+2} in the paper's terms) are those outside the
// test bitmap (not reached by level k) whose parent the level set.  A warp
// loads the parents of all candidates of its chunk first (coalesced, one word
// per load, all eight in flight), then hands the new vertices to the frontier
// blocks of level k+1 and adds them to the write bitmap (one store per word;
// the level's frontier marks are already there).
__device__ __forceinline__ void extract_chunk(const Inst& I, InstCtl* ctl, const EngineParams& P,
                                              Smem& sm, uint32_t k, uint32_t w0, uint32_t mat_next,
                                              uint32_t& wc) {
    const uint32_t p = k & 1, pn = p ^ 1;
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t wi = w0 + lane;
    const bool own = lane < kChunkWords && wi < I.nwords;
    uint32_t cand = 0, wb = 0;
    if (own) {
        cand = ~ld_l2(I.bm[p] + wi);
        wb = ld_l2(I.bm[pn] + wi);
        // no vertices past n in the last word
        if (wi == I.nwords - 1 && (I.n & 31)) cand &= (1u << (I.n & 31)) - 1u;
    }
    uint32_t par[kChunkWords];
#pragma unroll
    for (uint32_t q = 0; q < kChunkWords; ++q) {
        const uint32_t c = __shfl_sync(0xFFFFFFFFu, cand, q);
        par[q] = ((c >> lane) & 1u) ? ld_l2(I.parent + (w0 + q) * 32 + lane) : kUnset;
    }
    uint32_t fresh = 0;  // lane q: the new vertices of word w0 + q
#pragma unroll
    for (uint32_t q = 0; q < kChunkWords; ++q) {
        const bool want = par[q] != kUnset;
        const uint32_t bits = __ballot_sync(0xFFFFFFFFu, want);
        if (!bits) continue;
        if (lane == q) fresh = bits;
        const uint32_t v = (w0 + q) * 32 + lane;
        if (want) I.level[v] = (int32_t)(k + 1);
        stage_warp(want, v, sm, wc);
        if (wc > (uint32_t)(kWarpBuf - 32)) warp_flush(sm, I, ctl, P, pn, mat_next, wc);
    }
    if (own) {
        if (fresh) I.bm[pn][wi] = wb | fresh;
        // hybrid: the frontier bitmap of level k+1, in case it runs bottom-up
        if (P.bu_alpha && I.bu_ok) I.fbm[pn][wi] = fresh;
    }
}

// Unit u of an extraction: chunks [u*per, (u+1)*per).
__device__ ABFS_NOINLINE void unit_extract(const Inst& I, InstCtl* ctl, const EngineParams& P, Smem& sm,
                             uint32_t k, uint32_t u, uint32_t per) {
    const uint32_t warp = threadIdx.x >> 5;
    uint32_t mat, mat_next;
    level_mats(ctl, k, mat, mat_next);
    const uint32_t chunks = (I.nwords + kChunkWords - 1) / kChunkWords;
    const uint32_t c1 = min(chunks, (u + 1) * per);
    uint32_t wc = sm.wcnt[warp];
    for (uint32_t c = u * per + warp; c < c1; c += kWarps)
        extract_chunk(I, ctl, P, sm, k, c * kChunkWords, mat_next, wc);
    if ((threadIdx.x & 31) == 0) sm.wcnt[warp] = wc;
    __syncwarp();
    cta_flush(sm, I, ctl, P, (k & 1) ^ 1, mat_next);
}

// ---------------------------------------------------------------------------
// hybrid: bottom-up levels (direction optimisation; not the paper's method)
// ---------------------------------------------------------------------------
//
// For an undirected graph whose columns are sorted, the product of a level can
// also be evaluated row by row: x_{k+1}(i) for an unvisited row i is the least
// frontier index j in column i (= row i, A symmetric), and with the column
// ascending the first frontier entry is that least index, so the scan stops
// there.  The result (levels and min-index parents) is the submatrix method's;
// only the order of evaluation changes.  The frontier of level k is read from
// a bitmap (fbm[k & 1]).

constexpr uint32_t kBuLaneBatches = 4;  // lane-serial scan: 4 batches of 4 entries

// Frontier bitmap of level k after a top-down level: at the start of level k
// the test bitmap holds the levels <= k and the write bitmap the levels < k.
// Unit u: chunks [u*per, (u+1)*per).
__device__ ABFS_NOINLINE void unit_bu_prep(const Inst& I, uint32_t k, uint32_t u, uint32_t per) {
    const uint32_t p = k & 1;
    const uint32_t w1 = min(I.nwords, (u + 1) * per * kChunkWords);
    for (uint32_t w = u * per * kChunkWords + threadIdx.x; w < w1; w += kThreads)
        I.fbm[p][w] = ld_l2(I.bm[p] + w) & ~ld_l2(I.bm[p ^ 1] + w);
}

// Bottom-up level k over the chunk at word w0: each lane takes one unvisited
// vertex of a word and scans the first entries of its column itself, four at
// a time; columns still unresolved after that are scanned by the whole warp,
// 32 entries at a time.  Found vertices get level k+1 and their parent, go to
// the frontier blocks of level k+1, the write bitmap (one store per word:
// test | new = the levels <= k+1) and the next frontier bitmap.
__device__ __forceinline__ void bu_chunk(const Inst& I, InstCtl* ctl, const EngineParams& P,
                                         Smem& sm, uint32_t k, uint32_t w0, uint32_t mat_next,
                                         uint32_t& wc, Tally& t) {
    const uint32_t p = k & 1, pn = p ^ 1;
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t* fbm = I.fbm[p];
    const uint32_t wi = w0 + lane;
    const bool own = lane < kChunkWords && wi < I.nwords;
    uint32_t tb = 0, cand = 0;
    if (own) {
        tb = ld_frozen(I.bm[p] + wi);
        cand = ~tb;
        if (wi == I.nwords - 1 && (I.n & 31)) cand &= (1u << (I.n & 31)) - 1u;
    }
    uint32_t fresh = 0;  // lane q: the new vertices of word w0 + q
    for (uint32_t q = 0; q < kChunkWords; ++q) {
        const uint32_t c = __shfl_sync(0xFFFFFFFFu, cand, q);
        if (!c) continue;
        const uint32_t v = (w0 + q) * 32 + lane;
        uint32_t e = 0, end = 0, par = kUnset;
        if ((c >> lane) & 1u) {
            e = ld_ro(I.colptr + v);
            end = ld_ro(I.colptr + v + 1);
        }
        for (uint32_t b = 0; b < kBuLaneBatches && e < end; ++b) {
            uint32_t jj[4], fw[4];
#pragma unroll
            for (int x = 0; x < 4; ++x) jj[x] = e + x < end ? ld_ro(I.rowidx + e + x) : kUnset;
#pragma unroll
            for (int x = 0; x < 4; ++x) fw[x] = jj[x] != kUnset ? ld_frozen(fbm + (jj[x] >> 5)) : 0u;
            t.read += min(4u, end - e);
#pragma unroll
            for (int x = 3; x >= 0; --x)
                if ((fw[x] >> (jj[x] & 31)) & 1u) par = jj[x];
            e = par != kUnset ? end : e + 4;
        }
        bool defer = par == kUnset && e < end;
        uint32_t dm;
        while ((dm = __ballot_sync(0xFFFFFFFFu, defer)) != 0u) {
            const uint32_t ldr = __ffs(dm) - 1;
            const uint32_t le = __shfl_sync(0xFFFFFFFFu, e, ldr);
            const uint32_t lend = __shfl_sync(0xFFFFFFFFu, end, ldr);
            uint32_t found = kUnset;
            for (uint32_t x = le; x < lend; x += 32) {
                const uint32_t idx = x + lane;
                const uint32_t j = idx < lend ? ld_ro(I.rowidx + idx) : kUnset;
                const bool hit = j != kUnset && ((ld_frozen(fbm + (j >> 5)) >> (j & 31)) & 1u);
                const uint32_t hb = __ballot_sync(0xFFFFFFFFu, hit);
                if (lane == 0) t.read += min(32u, lend - x);
                if (hb) {
                    found = __shfl_sync(0xFFFFFFFFu, j, __ffs(hb) - 1);
                    break;
                }
            }
            if (lane == ldr) {
                par = found;
                defer = false;
            }
        }
        const bool got = par != kUnset;
        if (got) {
            I.parent[v] = par;
            I.level[v] = (int32_t)(k + 1);
            ++t.unmasked;
            ++t.claims;
        }
        const uint32_t bits = __ballot_sync(0xFFFFFFFFu, got);
        if (lane == q) fresh = bits;
        stage_warp(got, v, sm, wc);
        if (wc > (uint32_t)(kWarpBuf - 32)) warp_flush(sm, I, ctl, P, pn, mat_next, wc);
    }
    if (own) {
        I.bm[pn][wi] = tb | fresh;
        I.fbm[pn][wi] = fresh;
    }
}

// Unit u of a bottom-up level: chunks [u*per, (u+1)*per).
__device__ ABFS_NOINLINE void unit_bottom_up(const Inst& I, InstCtl* ctl, const EngineParams& P,
                                             Smem& sm, uint32_t k, uint32_t u, uint32_t per) {
    const uint32_t warp = threadIdx.x >> 5;
    uint32_t mat, mat_next;
    level_mats(ctl, k, mat, mat_next);
    const uint32_t chunks = (I.nwords + kChunkWords - 1) / kChunkWords;
    const uint32_t c1 = min(chunks, (u + 1) * per);
    Tally t;
    uint32_t wc = sm.wcnt[warp];
    for (uint32_t c = u * per + warp; c < c1; c += kWarps)
        bu_chunk(I, ctl, P, sm, k, c * kChunkWords, mat_next, wc, t);
    if ((threadIdx.x & 31) == 0) sm.wcnt[warp] = wc;
    __syncwarp();
    tally_flush(sm, t);
    cta_flush(sm, I, ctl, P, (k & 1) ^ 1, mat_next);
}

// Shrink: compacts the unvisited columns among vertices
// [u*shrink_tile, (u+1)*shrink_tile) to their unvisited rows (A_k = S_k A S_k
// restricted to the columns still to be multiplied).  `vis` holds the
// vertices reached so far; src_mat is the matrix those columns are read from
// and dst (1 or 2) the shrunk copy being written.
__device__ ABFS_NOINLINE void unit_shrink(const Inst& I, InstCtl* ctl, const EngineParams& P, Smem& sm,
                            uint32_t u, const uint32_t* vis, uint32_t src_mat, uint32_t dst) {
    const uint32_t v0 = u * P.shrink_tile;
    const uint32_t cnt = min(P.shrink_tile, I.n - v0);
    const uint32_t s = dst - 1;
    uint32_t* cnt_arr = sm.v;  // survivors per column, then running write cursor
    for (uint32_t t = threadIdx.x; t < cnt; t += kThreads) {
        const uint32_t v = v0 + t;
        const bool unvisited = !((ld_l2(vis + (v >> 5)) >> (v & 31)) & 1u);
        uint32_t beg = 0, len = 0;
        if (unvisited) {
            const ColRef c = col_of(I, src_mat, v);
            beg = c.beg;
            len = c.len;
        }
        sm.b[t] = beg;
        sm.off[t] = len;
        cnt_arr[t] = 0;
    }
    __syncthreads();
    block_exclusive_scan<kTileItems>(sm.off, cnt, sm);
    const uint32_t E = sm.off[cnt];
    const uint32_t* rows = rows_of(I, src_mat);
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t per = (E + kWarps - 1) / kWarps;
    const uint32_t e0 = min(E, warp * per), e1 = min(E, e0 + per);
    // pass 0 counts the surviving rows of each column, pass 1 writes them
    for (int pass = 0; pass < 2; ++pass) {
        uint32_t e = e0 + lane;
        uint32_t i = 0;
        if (e < e1) {
            uint32_t lo = 0, hi = cnt;
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (sm.off[mid] <= e) lo = mid;
                else hi = mid;
            }
            i = lo;
        }
        for (; e < e1; e += 32) {
            while (sm.off[i + 1] <= e) ++i;
            const uint32_t r = ld_l2(rows + sm.b[i] + (e - sm.off[i]));
            const bool keep = !((ld_l2(vis + (r >> 5)) >> (r & 31)) & 1u);
            if (keep) {
                const uint32_t pos = atomicAdd(&cnt_arr[i], 1u);
                if (pass == 1) {
                    const unsigned long long dpos = (unsigned long long)sm.gbase + pos;
                    if (dpos < I.scap) I.srows[s][dpos] = r;
                }
            }
        }
        __syncthreads();
        if (pass == 0) {
            // lengths of the new columns, then their begins
            for (uint32_t t = threadIdx.x; t < cnt; t += kThreads) I.slen[s][v0 + t] = cnt_arr[t];
            __syncthreads();
            block_exclusive_scan<kTileItems>(cnt_arr, cnt, sm);
            if (threadIdx.x == 0) {
                const uint32_t S = cnt_arr[cnt];
                const uint32_t g = atomicAdd(&ctl->shrink_out, S);
                if ((unsigned long long)g + S > I.scap) fail(ctl, 7);
                sm.gbase = g;
                atomicAdd(&ctl->shrink_kept, (unsigned long long)S);
            }
            __syncthreads();
            // cnt_arr[t] now holds column t's offset and serves as its write cursor
            for (uint32_t t = threadIdx.x; t < cnt; t += kThreads)
                I.sbeg[s][v0 + t] = sm.gbase + cnt_arr[t];
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) atomicAdd(&ctl->shrink_read, (unsigned long long)E);
    __syncthreads();
}

// Serving: clears the outputs (and bitmaps) of vertices [u*init_tile, ...) of
// a newly started search -- the work the initialisation kernels do for
// abfs_run, done inside the long-lived launch.
__device__ ABFS_NOINLINE void unit_init(const Inst& I, const EngineParams& P, uint32_t u) {
    const uint32_t v0 = u * P.init_tile;
    const uint32_t v1 = min(I.n, v0 + P.init_tile);
    for (uint32_t v = v0 + threadIdx.x; v < v1; v += kThreads) {
        I.level[v] = -1;
        I.parent[v] = kUnset;
        if (P.mode == kModePlain) I.y[v] = ~0ull;
        if (I.sigma) I.sigma[v] = 0ull;
    }
    if (P.mode == kModeSub) {
        const uint32_t w0 = v0 >> 5, w1 = (v1 + 31) >> 5;  // init_tile is a multiple of 32
        for (uint32_t w = w0 + threadIdx.x; w < w1; w += kThreads) {
            I.bm[0][w] = 0u;
            I.bm[1][w] = 0u;
        }
    }
}

// ---------------------------------------------------------------------------
// phase control
// ---------------------------------------------------------------------------

// Runs one unit of phase (kind, k).
template <int MODE>
__device__ void run_unit(const Inst& I, InstCtl* ctl, const EngineParams& P, Smem& sm,
                         uint32_t kind, uint32_t k, uint32_t unit, uint32_t nitems) {
    if (kind == kPhInit) {
        unit_init(I, P, unit);
    } else if (kind == kPhStart) {
        // nothing: the CTA that completes it advances into level 0
    } else if (kind == kPhShrink) {
        // k = level just completed; its write bitmap holds every vertex reached so far
        const uint32_t src_mat = ld_relaxed(&ctl->mat_cur);
        unit_shrink(I, ctl, P, sm, unit, I.bm[(k + 1) & 1], src_mat, /*dst=*/nitems);
    } else if (kind == kPhPlainMask) {
        unit_plain_mask(I, ctl, P, sm, k, unit, nitems);
    } else if (kind == kPhExtract) {
        unit_extract(I, ctl, P, sm, k, unit, nitems);
    } else if (kind == kPhBuPrep) {
        unit_bu_prep(I, k, unit, nitems);
    } else if (MODE == kModeSub && kind == kPhBottomUp) {
        unit_bottom_up(I, ctl, P, sm, k, unit, nitems);
    } else if (MODE == kModeSub && kind == kPhLevelScan) {
        unit_level<MODE, kVarScan>(I, ctl, P, sm, k, unit, nitems);
    } else {
        unit_level<MODE, kVarWide>(I, ctl, P, sm, k, unit, nitems);
    }
    stats_flush(sm, ctl);
}

// Optional per-phase trace entry: [time lo, time hi, kind<<24 | level, alone]
// and [items, vertices, entries (low 32 bits), 0].
__device__ ABFS_NOINLINE void trace_put(const Inst& I, InstCtl* ctl, uint32_t kind, uint32_t level,
                          uint32_t alone, uint32_t ni, uint32_t nf, unsigned long long ne) {
    const uint32_t tn = ld_relaxed(&ctl->trace_n);
    if (tn >= I.trace_cap) return;
    const uint64_t now = globaltimer();
    I.trace[2 * tn] = make_uint4((uint32_t)now, (uint32_t)(now >> 32),
                                 (kind << 24) | (level & 0xFFFFFFu), alone);
    I.trace[2 * tn + 1] = make_uint4(ni, nf, (uint32_t)min(ne, 0xFFFFFFFFull), 0u);
    st_relaxed(&ctl->trace_n, tn + 1);
}

// Whether the i-th physical shrink (i = shrinks + 1) is due once `reached`
// vertices are reached: it waits until a fraction 1-(1-theta)^i of n is reached.
__device__ __forceinline__ bool shrink_due(const EngineParams& P, uint32_t reached, uint32_t n,
                                           uint32_t shrinks) {
    if (!(P.shrink_theta > 0.f && P.shrink_theta < 1.f) || shrinks >= P.shrink_max) return false;
    const float frac = (float)reached / (float)n;
    const float need = 1.f - powf(1.f - P.shrink_theta, (float)(shrinks + 1));
    return frac >= need;
}

// ---------------------------------------------------------------------------
// resident narrow runs
// ---------------------------------------------------------------------------
// While a search's frontier stays within narrow_max vertices and narrow_edges
// slots, one CTA runs its levels back to back without the block bookkeeping of
// wide levels.  The frontier of level k is a plain list at fq/fbeg/fpre[k&1]:
// vertex, column begin and column length.  Claims gather in the warp staging
// buffers and are appended with a shared-memory counter; the reached count
// and the level stay in shared memory until the run ends.  The run ends when
// the frontier empties, outgrows the narrow bounds, or a shrink is due; the
// last frontier is then rewritten as blocks and the general path decides what
// follows.

// Expands the f vertices of the level-k list (lens: fbeg/fpre hold column
// begins and lengths in matrix mat; otherwise only the ids are valid and the
// columns are looked up) in chunks of up to `tile` vertices and windows of up
// to kUnitMax slots.  Whole CTA.
template <int MODE>
__device__ __forceinline__ void narrow_expand(const Inst& I, InstCtl* ctl, const EngineParams& P, Smem& sm,
                              uint32_t k, uint32_t f, bool lens, uint32_t mat, uint32_t mat_next,
                              Tally& t, uint32_t& nnz_local) {
    const uint32_t p = k & 1;
    for (uint32_t c0 = 0; c0 < f; c0 += P.tile) {
        const long long pt0 = prof_now(sm);
        const uint32_t cnt = min(P.tile, f - c0);
        for (uint32_t s = threadIdx.x; s < cnt; s += kThreads) {
            const uint32_t v = ld_l2(I.fq[p] + c0 + s);
            uint32_t beg, len;
            if (lens) {
                beg = ld_l2(I.fbeg[p] + c0 + s);
                len = ld_l2(I.fpre[p] + c0 + s);
            } else {
                const ColRef c = col_of(I, mat, v);
                beg = c.beg;
                len = c.len;
            }
            sm.v[s] = v;
            sm.b[s] = beg;
            sm.off[s] = len + kVertexSlots;
            // the frontier joins the visited set of the next level's test
            if (MODE == kModeSub) atomicOr(I.bm[p ^ 1] + (v >> 5), 1u << (v & 31));
            nnz_local += (mat == 0) ? len : (ld_ro(I.colptr + v + 1) - ld_ro(I.colptr + v));
        }
        for (uint32_t w = threadIdx.x; w < (uint32_t)kStartWords; w += kThreads) sm.sbits[w] = 0u;
        if (threadIdx.x < (uint32_t)kWarps) sm.wvb[threadIdx.x] = kNoVb;
        __syncthreads();
        block_exclusive_scan<kTileItems>(sm.off, cnt, sm);
        const uint32_t S = sm.off[cnt];
        // window [l0, l1) of at most kUnitMax slots; its vertex starts in sbits
        uint32_t l0 = 0, l1 = min(S, kUnitMax);
        for (uint32_t s = threadIdx.x; s < cnt; s += kThreads) {
            const uint32_t st = sm.off[s], en = sm.off[s + 1];
            sm.end[s] = en - kVertexSlots;
            sm.b[s] -= st;  // row index of slot x is b + x
            if (st < l1) atomicOr(&sm.sbits[st >> 5], 1u << (st & 31));
            mark_warp_starts(sm, s, st, en, l0, l1);
        }
        __syncthreads();
        prof_add(sm, kProfNLoad, pt0);
        for (;;) {
            const long long pt1 = prof_now(sm);
            expand_core<MODE, kVarNarrow>(I, ctl, P, sm, cnt, l0, l1, mat, mat_next, k, t);
            __syncthreads();
            prof_add(sm, kProfNExpand, pt1);
            if (l1 >= S) break;
            l0 = l1;
            l1 = min(S, l0 + kUnitMax);
            for (uint32_t w = threadIdx.x; w < (uint32_t)kStartWords; w += kThreads) sm.sbits[w] = 0u;
            if (threadIdx.x < (uint32_t)kWarps) sm.wvb[threadIdx.x] = kNoVb;
            __syncthreads();
            for (uint32_t s = threadIdx.x; s < cnt; s += kThreads) {
                const uint32_t st = sm.off[s];
                if (st >= l0 && st < l1) atomicOr(&sm.sbits[(st - l0) >> 5], 1u << ((st - l0) & 31));
                mark_warp_starts(sm, s, st, sm.off[s + 1], l0, l1);
            }
            __syncthreads();
        }
    }
}

// Rewrites the list of parity pn (fn vertices; fpre holds column lengths) as
// frontier blocks of up to kWarps*kWarpBuf vertices: slot offsets within the
// block, unit starts, and the parity's counters.  The warp staging buffers
// (empty here) stage each chunk so global reads and writes stay coalesced.
// Whole CTA.
__device__ ABFS_NOINLINE void narrow_to_blocks(const Inst& I, InstCtl* ctl, const EngineParams& P,
                                               Smem& sm, uint32_t pn, uint32_t fn) {
    constexpr uint32_t kChunk = kWarps * kWarpBuf;
    constexpr uint32_t kItems = kChunk / kThreads;
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t* buf = &sm.wv[0][0];
    unsigned long long eb = 0;
    uint32_t nb = 0;
    for (uint32_t c0 = 0; c0 < fn; c0 += kChunk, ++nb) {
        const uint32_t cnt = min(kChunk, fn - c0);
        for (uint32_t i = tid; i < cnt; i += kThreads) buf[i] = ld_l2(I.fpre[pn] + c0 + i);
        __syncthreads();
        uint32_t x[kItems];
        uint32_t sum = 0;
#pragma unroll
        for (uint32_t q = 0; q < kItems; ++q) {
            const uint32_t idx = tid * kItems + q;
            x[q] = idx < cnt ? buf[idx] + kVertexSlots : 0u;
            sum += x[q];
        }
        const uint32_t incl = warp_incl_scan(sum);
        if (lane == 31) sm.warp_sums[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const uint32_t w = lane < (uint32_t)kWarps ? sm.warp_sums[lane] : 0u;
            const uint32_t wi = warp_incl_scan(w);
            if (lane < (uint32_t)kWarps) sm.warp_sums[lane] = wi - w;
            if (lane == kWarps - 1) sm.warp_sums[kWarps] = wi;
        }
        __syncthreads();
        uint32_t run = sm.warp_sums[warp] + incl - sum;
        const uint32_t total = sm.warp_sums[kWarps];
        const bool ok = nb < I.bcap && nb < kBlockMask;
        for (uint32_t q = 0; q < kItems; ++q) {
            const uint32_t idx = tid * kItems + q;
            if (idx < cnt) buf[idx] = run;
            warp_unit_starts(I, ctl, P, pn, nb, idx, eb + run, (idx < cnt && ok) ? x[q] : 0u);
            run += x[q];
        }
        __syncthreads();
        if (ok)
            for (uint32_t i = tid; i < cnt; i += kThreads) I.fpre[pn][c0 + i] = buf[i];
        if (tid == 0) {
            if (ok) {
                Block* B = I.blk[pn] + nb;
                B->vb = c0;
                B->nv = cnt;
                B->eb = eb;
            } else {
                fail(ctl, 7);
            }
        }
        eb += total;
        __syncthreads();  // buf and warp_sums are reused
    }
    if (tid == 0) {
        st_relaxed64(&ctl->bctr[pn], (eb << kBlockBits) | (unsigned long long)nb);
        st_relaxed(&ctl->fcnt[pn], fn);
    }
}

// Runs levels k, k+1, ... of the current search on this CTA (the frontier of
// level k is in the parity's blocks, its ids contiguous at fq[k&1]).  Returns
// the last level run; its successor frontier is left in block form with the
// search's counters set as the general path expects.  Whole CTA.
template <int MODE>
__device__ ABFS_NOINLINE uint32_t narrow_run(const Inst& I, InstCtl* ctl, const EngineParams& P, Smem& sm,
                               uint32_t k, unsigned long long* heartbeat) {
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        // the matrices change only at shrinks, which end a run
        sm.nr_f = ld_relaxed(&ctl->fcnt[k & 1]);
        sm.nr_reached = ld_relaxed(&ctl->reached);
        sm.nr_shrinks = ld_relaxed(&ctl->shrinks);
        sm.nr_sw = ld_relaxed(&ctl->mat_switch);
        sm.nr_mcur = ld_relaxed(&ctl->mat_cur);
        sm.nr_mprev = ld_relaxed(&ctl->mat_prev);
        sm.nq_cnt = 0;
        sm.nt_cnt = 0;
        sm.nq_slots = 0;
    }
    __syncthreads();
    const uint32_t sw = sm.nr_sw, mat_cur = sm.nr_mcur, mat_prev = sm.nr_mprev;
    bool lens = false;
    // counters stay in registers until the run ends
    Tally t;
    uint32_t nnz_local = 0;
    // a search has at most n levels: a broken invariant ends the run instead
    // of looping
    for (uint32_t guard = I.n + 1;; --guard) {
        const uint32_t pn = (k + 1) & 1;
        const uint32_t f = sm.nr_f;
        const uint32_t mat = k >= sw ? mat_cur : mat_prev;
        const uint32_t mat_next = k + 1 >= sw ? mat_cur : mat_prev;
        // issued now, read when the level ends
        const uint32_t err = threadIdx.x == 0 ? ld_relaxed(&ctl->err) : 0u;
        narrow_expand<MODE>(I, ctl, P, sm, k, f, lens, mat, mat_next, t, nnz_local);
        const long long pt2 = prof_now(sm);
        {
            // the warps' leftovers
            uint32_t wc = sm.wcnt[warp];
            if (wc) {
                if (MODE == kModeSub) narrow_append(sm, I, ctl, pn, mat_next, wc);
                else narrow_touch(sm, I, ctl, wc);
            }
            if (lane == 0) sm.wcnt[warp] = 0;
        }
        __syncthreads();
        if (MODE == kModePlain) {
            // comparator mask: touched rows not yet reached join level k+1 with
            // the least column of the accumulator
            const uint32_t T = sm.nt_cnt;
            uint32_t wc = 0;
            for (uint32_t b0 = 0; b0 < T; b0 += kThreads) {
                const uint32_t i = b0 + threadIdx.x;
                bool want = false;
                uint32_t r = 0;
                if (i < T) {
                    r = ld_l2(I.touched + i);
                    if ((int32_t)ld_l2((const uint32_t*)I.level + r) == -1) {
                        const unsigned long long y = ld_l2(I.y + r);
                        I.level[r] = (int32_t)(k + 1);
                        I.parent[r] = (uint32_t)(y & 0xFFFFFFFFull);
                        want = true;
                    }
                }
                stage_warp(want, r, sm, wc);
                if (wc > (uint32_t)(kWarpBuf - 32)) narrow_append(sm, I, ctl, pn, mat_next, wc);
            }
            if (wc) narrow_append(sm, I, ctl, pn, mat_next, wc);
            __syncthreads();
        }
        const long long pt3 = prof_now(sm);
        prof_add(sm, kProfNAppend, pt2);
        if (threadIdx.x == 0) {
            const uint32_t fn = sm.nq_cnt;
            const unsigned long long slots = sm.nq_slots;
            sm.nq_cnt = 0;
            sm.nt_cnt = 0;
            sm.nq_slots = 0;
            uint32_t stop = 0;
            if (fn == 0 || err != 0 || fn > P.narrow_max || slots > P.narrow_edges || guard <= 1)
                stop = 1;
            else if (MODE == kModeSub && shrink_due(P, sm.nr_reached + fn, I.n, sm.nr_shrinks))
                stop = 1;
            if (!stop) {
                sm.nr_reached += fn;
                if (I.trace)
                    trace_put(I, ctl, MODE == kModePlain ? kPhPlainMult : kPhLevel, k + 1, 2u, 0u, fn,
                              slots);
            }
            sm.nr_stop = stop;
            sm.nr_f = fn;
            atomicAdd(heartbeat, 1ull);
            if (sm.prof_on) sm.prof[kProfNLevels] += 1;
        }
        __syncthreads();
        prof_add(sm, kProfNDecide, pt3);
        if (sm.nr_stop) break;
        lens = true;
        ++k;
    }
    const long long pt4 = prof_now(sm);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) nnz_local += __shfl_xor_sync(0xFFFFFFFFu, nnz_local, d);
    if (lane == 0 && nnz_local) atomicAdd(&sm.st_nnz, (unsigned long long)nnz_local);
    tally_flush(sm, t);
    narrow_to_blocks(I, ctl, P, sm, (k + 1) & 1, sm.nr_f);
    if (threadIdx.x == 0) st_relaxed(&ctl->reached, sm.nr_reached);
    stats_flush(sm, ctl);
    prof_add(sm, kProfNBlocks, pt4);
    return k;
}

// Thread 0 of the advancing CTA: the phase that follows (kind, k), written to
// sm.cmd; sm.cmd.quit = 1 when the search is over.
template <int MODE>
__device__ ABFS_NOINLINE void decide_next(const Inst& I, InstCtl* ctl, const EngineParams& P, Smem& sm,
                            uint32_t kind, uint32_t k, uint32_t* done_count) {
    uint32_t nkind = 0, nk = 0, ni = 0, finish = 0;
    if (kind == kPhInit) {
        // the outputs are clear: the source forms the frontier of level 0
        // (Algorithm 1's V_2 := V_1 \ supp(x_1))
        const uint32_t s = I.src;
        I.level[s] = 0;
        I.parent[s] = s;
        if (I.sigma) I.sigma[s] = 1ull;
        if (MODE == kModeSub) atomicOr(I.bm[0] + (s >> 5), 1u << (s & 31));
        const uint32_t b0 = ld_ro(I.colptr + s);
        const uint32_t w = ld_ro(I.colptr + s + 1) - b0 + kVertexSlots;
        I.fq[0][0] = s;
        I.fbeg[0][0] = b0;
        I.fpre[0][0] = 0;
        I.blk[0][0].vb = 0;
        I.blk[0][0].nv = 1;
        I.blk[0][0].eb = 0;
        for (unsigned long long x = 0; x < w; x += P.unit) I.ustart[0][x / P.unit] = make_uint2(0, 0);
        st_relaxed64(&ctl->bctr[0], ((unsigned long long)w << kBlockBits) | 1ull);
        st_relaxed(&ctl->fcnt[0], 1u);
        st_relaxed(&ctl->reached, 1u);
        nkind = (MODE == kModePlain) ? kPhPlainMult : kPhLevel;
        nk = 0;
    } else if (kind == kPhStart) {
        // the frontier of level 0 (the source) was set up before the launch
        nkind = (MODE == kModePlain) ? kPhPlainMult : kPhLevel;
        nk = 0;
    } else if (kind == kPhLevelScan) {
        // the new vertices of a level claimed by reductions are read off the bitmaps
        nkind = kPhExtract;
        nk = k;
    } else if (kind == kPhBuPrep) {
        nkind = kPhBottomUp;
        nk = k;
    } else if (kind == kPhPlainMult) {
        // comparator: the mask phase of the same level follows the multiply
        const uint32_t t = ld_relaxed(&ctl->tcnt);
        nkind = kPhPlainMask;
        nk = k;
        ni = t;
        if (t == 0) {
            finish = 1;
            st_relaxed(&ctl->levels, k + 1);
        }
    } else {
        // the frontier of level k+1 is complete (after a level, or after a shrink)
        const uint32_t pn = (k + 1) & 1, pc = k & 1;
        const uint32_t nf = ld_relaxed(&ctl->fcnt[pn]);
        uint32_t reached = ld_relaxed(&ctl->reached);
        uint32_t shrinks = ld_relaxed(&ctl->shrinks);
        if (kind != kPhShrink) {
            st_relaxed(&ctl->levels, k + 1);
            if (nf == 0) {
                finish = 1;
            } else {
                reached += nf;
                st_relaxed(&ctl->reached, reached);
                // the buffers of level k become the "next" buffers of level k+1
                st_relaxed(&ctl->fcnt[pc], 0u);
                st_relaxed64(&ctl->bctr[pc], 0ull);
                if (MODE == kModePlain) st_relaxed(&ctl->tcnt, 0u);
            }
        } else {
            // the copy just written serves the levels from k+2 on
            const uint32_t dst = sm.cmd.nitems;
            st_relaxed(&ctl->mat_prev, ld_relaxed(&ctl->mat_cur));
            st_relaxed(&ctl->mat_cur, dst);
            st_relaxed(&ctl->mat_switch, k + 2);
            shrinks += 1;
            st_relaxed(&ctl->shrinks, shrinks);
        }
        if (!finish) {
            const bool do_shrink =
                MODE == kModeSub && kind != kPhShrink && shrink_due(P, reached, I.n, shrinks);
            if (do_shrink) {
                // alternate copies so the frontier of level k+1 keeps its matrix
                const uint32_t cur = ld_relaxed(&ctl->mat_cur);
                nkind = kPhShrink;
                nk = k;
                ni = (cur == 1) ? 2u : 1u;
                st_relaxed(&ctl->shrink_out, 0u);
            } else {
                nkind = (MODE == kModePlain) ? kPhPlainMult : kPhLevel;
                nk = k + 1;
                if (MODE == kModeSub && P.bu_alpha && I.bu_ok && kind != kPhShrink) {
                    // hybrid direction choice from the frontier's edges m_f and the
                    // edges of vertices not reached yet m_u: bottom-up once
                    // m_f * alpha > m_u, back to top-down once n_f * beta < n
                    const unsigned long long ne1 = ld_relaxed64(&ctl->bctr[pn]) >> kBlockBits;
                    const unsigned long long mf = ne1 - (unsigned long long)kVertexSlots * nf;
                    const unsigned long long seen = ld_relaxed64(&ctl->nnz_reached) + mf;
                    const unsigned long long nnz = ld_ro(I.colptr + I.n);
                    const unsigned long long mu = nnz > seen ? nnz - seen : 0ull;
                    uint32_t bu = ld_relaxed(&ctl->bu_on);
                    bu = bu ? ((unsigned long long)nf * P.bu_beta >= I.n)
                            : (mf * (unsigned long long)P.bu_alpha > mu);
                    st_relaxed(&ctl->bu_on, bu);
                    if (bu) {
                        // the frontier's columns are never expanded: count them here
                        atomicAdd(&ctl->nnz_reached, mf);
                        nkind = (kind == kPhExtract || kind == kPhBottomUp) ? kPhBottomUp : kPhBuPrep;
                    }
                }
            }
        }
    }
    if (ld_relaxed(&ctl->err) != 0) finish = 1;
    sm.cmd.kind = nkind;
    sm.cmd.level = nk;
    sm.cmd.nitems = ni;
    sm.cmd.quit = finish;
    if (finish) {
        const uint32_t e = ld_relaxed(&ctl->err);
        __threadfence();
        if (atomicCAS(&ctl->status, (uint32_t)kRunning, e ? (uint32_t)kFailed : (uint32_t)kDone) ==
            kRunning) {
            atomicAdd(done_count, 1u);
            if (I.notify) {
                // serving: the ticket and status reach the host's mapped word after
                // every write of the search
                __threadfence_system();
                const unsigned long long word = (I.ticket << 8) | (unsigned long long)(e & 0xFFu);
                asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(I.notify), "l"(word)
                             : "memory");
            }
        }
    }
}

// Called by the whole CTA that completed the last unit of phase (kind, k).
// Runs small follow-up phases alone ("narrow") and publishes large ones.
template <int MODE>
__device__ void advance(const Inst& I, InstCtl* ctl, const EngineParams& P, Smem& sm,
                        uint32_t kind, uint32_t k, uint32_t* done_count,
                        unsigned long long* heartbeat) {
    for (;;) {
        if (threadIdx.x == 0) {
            __threadfence();
            decide_next<MODE>(I, ctl, P, sm, kind, k, done_count);
            atomicAdd(heartbeat, 1ull);
        }
        __syncthreads();
        if (sm.cmd.quit) {
            if (I.trace && threadIdx.x == 0) trace_put(I, ctl, 0xFFu, k, 0u, 0u, 0u, 0ull);
            return;
        }
        const uint32_t nk = sm.cmd.level;
        uint32_t nkind = sm.cmd.kind;
        uint32_t ni = sm.cmd.nitems;
        uint32_t units, nf = 0;
        unsigned long long ne = 0;
        bool alone;
        if (nkind == kPhShrink) {
            units = (I.n + P.shrink_tile - 1) / P.shrink_tile;
            alone = units <= 1;
        } else if (nkind == kPhPlainMask) {
            units = (ni + P.tile - 1) / P.tile;
            alone = ni <= P.narrow_max;
        } else if (nkind == kPhExtract || nkind == kPhBuPrep || nkind == kPhBottomUp) {
            // runs of 8-word chunks, about two units per CTA (ni = chunks per unit)
            const uint32_t chunks = (I.nwords + kChunkWords - 1) / kChunkWords;
            const uint32_t two = 2u * gridDim.x;
            ni = max((chunks + two - 1) / two, (uint32_t)kWarps);
            units = (chunks + ni - 1) / ni;
            alone = units <= 1;
        } else {
            // a level (or the comparator's multiply) over the frontier of level nk;
            // its units are m granules, about two per CTA of the grid (ni = m)
            ne = ld_relaxed64(&ctl->bctr[nk & 1]) >> kBlockBits;
            nf = ld_relaxed(&ctl->fcnt[nk & 1]);
            const unsigned long long mmax = kUnitMax / P.unit;
#if ABFS_UNIT_CEIL
            // at most two units per CTA: a third round for a few CTAs would
            // stretch the level by half
            const unsigned long long per2 = (unsigned long long)P.unit * 2ull * gridDim.x;
            unsigned long long m = (ne + per2 - 1) / per2;
#else
            unsigned long long m = ne / ((unsigned long long)P.unit * 2ull * gridDim.x);
#endif
            m = m < 1ull ? 1ull : (m > mmax ? mmax : m);
            ni = (uint32_t)m;
            units = (uint32_t)((ne + P.unit * m - 1) / (P.unit * m));
            alone = nf <= P.narrow_max && ne <= P.narrow_edges;
            // a large level claims by reductions and a bitmap scan
            if (MODE == kModeSub && nkind == kPhLevel && !alone && P.scan_min && ne >= P.scan_min)
                nkind = kPhLevelScan;
        }
        if (I.trace && threadIdx.x == 0)
            trace_put(I, ctl, nkind, nk, alone, nkind == kPhPlainMask ? ni : units, nf, ne);
        if (!alone) {
            if (threadIdx.x == 0) {
                const uint32_t e = ld_relaxed(&ctl->epoch) + 1;
                const uint32_t q = e & 1;
                st_relaxed(&ctl->kind[q], nkind);
                st_relaxed(&ctl->plevel[q], nk);
                st_relaxed(&ctl->nitems[q], ni);
                st_relaxed(&ctl->pending[q], units);
                st_relaxed(&ctl->epoch, e);
                st_relaxed(&ctl->wide_levels, ld_relaxed(&ctl->wide_levels) + 1);
                __threadfence();
                atomicExch(&ctl->desc[q], ((unsigned long long)e << 32) | units);
                __threadfence();
                atomicExch(&ctl->grab, (unsigned long long)e << 32);
            }
            __syncthreads();
            return;
        }
        if (P.narrow_loop && (nkind == kPhLevel || nkind == kPhPlainMult)) {
            // a resident run of narrow levels on this CTA
            k = narrow_run<MODE>(I, ctl, P, sm, nk, heartbeat);
            kind = kPhLevel;
            __threadfence();
            __syncthreads();
            continue;
        }
        // narrow: this CTA runs every unit of the phase, then decides again
        for (uint32_t u = 0; u < units; ++u) run_unit<MODE>(I, ctl, P, sm, nkind, nk, u, ni);
        __threadfence();
        __syncthreads();
        kind = nkind;
        k = nk;
    }
}

// Control block of instance q (fixed for the launch, also per serving slot,
// but a serving slot's other descriptor fields change while the launch runs,
// so those launches read it without the read-only path).
__device__ __forceinline__ InstCtl* ctl_of(const EngineArgs& a, uint32_t q) {
    const unsigned long long* p = reinterpret_cast<const unsigned long long*>(&a.insts[q].ctl);
    return reinterpret_cast<InstCtl*>(a.serve ? ld_relaxed64(p) : __ldg(p));
}

// Whether instance q has an untaken unit in its published phase (or, when
// serving, is a newly submitted search waiting to start).  The published
// phase's grab epoch and descriptor are returned in e and d.
__device__ __forceinline__ bool has_work(const EngineArgs& a, uint32_t q, uint32_t& e,
                                         unsigned long long& d) {
    if (a.serve) {
        // a slot that never held a search has no control block yet
        const uint32_t st = ld_relaxed(a.slot_state + q);
        if (st == kSlotSubmitted) return true;
        if (st != kSlotRunning) return false;
    }
    const InstCtl* ctl = ctl_of(a, q);
    // one round of independent loads
    const uint32_t status = ld_relaxed(&ctl->status);
    const unsigned long long g = ld_relaxed64(&ctl->grab);
    const unsigned long long d0 = ld_relaxed64(&ctl->desc[0]);
    const unsigned long long d1 = ld_relaxed64(&ctl->desc[1]);
    e = (uint32_t)(g >> 32);
    d = (e & 1) ? d1 : d0;
    const uint32_t taken = (uint32_t)g;
    return status == kRunning && (uint32_t)(d >> 32) == e && taken < (uint32_t)d;
}

// One lane: takes a unit of instance q if one is left (or claims the start
// of a submitted search); fills sm.cmd.  (e_seen, d_seen) is what has_work
// saw: the descriptor of epoch e_seen, reused when the grab lands in that
// epoch.
__device__ __forceinline__ bool take_unit(const EngineArgs& a, uint32_t q, Smem& sm, uint32_t e_seen,
                                          unsigned long long d_seen) {
    if (a.serve && ld_relaxed(a.slot_state + q) == kSlotSubmitted) {
        if (atomicCAS(a.slot_state + q, (uint32_t)kSlotSubmitted, (uint32_t)kSlotRunning) !=
            kSlotSubmitted)
            return false;
        __threadfence();  // acquire: the descriptor the host wrote before the state
        sm.cmd.q = q;
        sm.cmd.start = 1;
        return true;
    }
    InstCtl* ctl = ctl_of(a, q);
    const unsigned long long old = atomicAdd(&ctl->grab, 1ull);
    const uint32_t e = (uint32_t)(old >> 32), t = (uint32_t)old;
    // the descriptor of epoch e is written before grab moves to e
    const unsigned long long d =
        (e == e_seen && (uint32_t)(d_seen >> 32) == e) ? d_seen : ld_relaxed64(&ctl->desc[e & 1]);
    if ((uint32_t)(d >> 32) != e || t >= (uint32_t)d) return false;
    __threadfence();  // acquire: the phase fields and the data of earlier phases
    const uint32_t qq = e & 1;
    sm.cmd.q = q;
    sm.cmd.start = 0;
    sm.cmd.epoch = e;
    sm.cmd.unit = t;
    sm.cmd.kind = ld_relaxed(&ctl->kind[qq]);
    sm.cmd.level = ld_relaxed(&ctl->plevel[qq]);
    sm.cmd.nitems = ld_relaxed(&ctl->nitems[qq]);
    return true;
}

// Serving: the CTA that claimed a submitted search resets its control block
// and publishes the initialisation phase.  The slot's epoch sequence goes on
// from the previous search instead of restarting: a CTA that looked at the
// slot during the previous search may still add to `grab` late, and with a
// fresh epoch that stale grab can never match the new phase's descriptor.
// Whole CTA.
__device__ ABFS_NOINLINE void start_search(const EngineArgs& a, Smem& sm) {
    const Inst& I = sm.I;
    InstCtl* ctl = I.ctl;
    uint32_t* c = reinterpret_cast<uint32_t*>(ctl);
    // everything but grab, desc[] and epoch is cleared (status: idle)
    const uint32_t keep_lo = offsetof(InstCtl, grab) / 4, keep_hi = offsetof(InstCtl, bctr) / 4;
    const uint32_t keep_ep = offsetof(InstCtl, epoch) / 4;
    for (uint32_t w = threadIdx.x; w < sizeof(InstCtl) / 4; w += kThreads)
        if ((w < keep_lo || w >= keep_hi) && w != keep_ep) c[w] = 0u;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t units = (I.n + a.p.init_tile - 1) / a.p.init_tile;
        const uint32_t e = ld_relaxed(&ctl->epoch) + 1;
        const uint32_t q = e & 1;
        st_relaxed(&ctl->kind[q], kPhInit);
        st_relaxed(&ctl->plevel[q], 0u);
        st_relaxed(&ctl->nitems[q], 0u);
        st_relaxed(&ctl->pending[q], units);
        st_relaxed(&ctl->epoch, e);
        __threadfence();
        atomicExch(&ctl->desc[q], ((unsigned long long)e << 32) | units);
        __threadfence();
        atomicExch(&ctl->grab, (unsigned long long)e << 32);
        __threadfence();
        st_relaxed(&ctl->status, kRunning);
        atomicAdd(a.heartbeat, 1ull);
    }
    __syncthreads();
}

// Warp 0 scans the instances 32 at a time from `cursor` and takes the first
// unit it can; the whole CTA then runs it.  Returns true if a unit was run.
template <int MODE>
__device__ bool find_and_run(const EngineArgs& a, Smem& sm, uint32_t& cursor) {
    const long long pt0 = prof_now(sm);
    if (threadIdx.x < 32) {
        const uint32_t lane = threadIdx.x;
        bool got = false;
        for (uint32_t base = 0; base < a.ninst && !got; base += 32) {
            const uint32_t idx = base + lane;
            const uint32_t q = (cursor + idx) % a.ninst;
            uint32_t e_seen = 0;
            unsigned long long d_seen = 0;
            const bool avail = idx < a.ninst && has_work(a, q, e_seen, d_seen);
            uint32_t mask = __ballot_sync(0xFFFFFFFFu, avail);
            while (mask && !got) {
                const uint32_t l = __ffs(mask) - 1;
                bool ok = false;
                if (lane == l) ok = take_unit(a, q, sm, e_seen, d_seen);
                got = __shfl_sync(0xFFFFFFFFu, ok, l);
                mask &= mask - 1;
            }
        }
        __syncwarp();
        if (lane == 0) sm.cmd.has = got;
        __syncwarp();
        // serving slots are reused by new searches: always reload their descriptor
        if (got && (a.serve || sm.cur_q != sm.cmd.q)) {
            const uint32_t* src = reinterpret_cast<const uint32_t*>(a.insts + sm.cmd.q);
            uint32_t* dst = reinterpret_cast<uint32_t*>(&sm.I);
            for (uint32_t w = lane; w < sizeof(Inst) / 4; w += 32) dst[w] = src[w];
            if (lane == 0) sm.cur_q = sm.cmd.q;
        }
    }
    __syncthreads();
    if (!sm.cmd.has) return false;
    if (sm.cmd.start) {
        start_search(a, sm);
        return true;
    }
    prof_add(sm, kProfTake, pt0);
    if (sm.prof_on && threadIdx.x == 0) sm.prof[kProfUnits] += 1;
    cursor = sm.cmd.q;
    const Inst& I = sm.I;
    InstCtl* ctl = I.ctl;
    const uint32_t kind = sm.cmd.kind, k = sm.cmd.level, epoch = sm.cmd.epoch;
    run_unit<MODE>(I, ctl, a.p, sm, kind, k, sm.cmd.unit, sm.cmd.nitems);
    // completion: release this CTA's writes, then count the unit down
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t left = atomicSub(&ctl->pending[epoch & 1], 1u);
        sm.cmd.last = (left == 1);
        atomicAdd(a.heartbeat, 1ull);
    }
    __syncthreads();
    if (sm.cmd.last) {
        const long long pt1 = prof_now(sm);
        advance<MODE>(I, ctl, a.p, sm, kind, k, a.done_count, a.heartbeat);
        prof_add(sm, kProfAdvance, pt1);
    }
    return true;
}

template <int MODE>
__global__ void __launch_bounds__(kThreads, kMinCtas) engine_kernel(EngineArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem& sm = *reinterpret_cast<Smem*>(smem_raw);
    if (threadIdx.x == 0) {
        for (int q = 0; q < kWarps; ++q) sm.wcnt[q] = 0;
        sm.prof_on = a.prof != nullptr;
        sm.idle_exit = 0;
        sm.cmd.start = 0;
        for (int q = 0; q < kProfSlots; ++q) sm.prof[q] = 0;
        sm.st_read = sm.st_unmasked = sm.st_claims = sm.st_nnz = 0;
        sm.cur_q = kUnset;
    }
    __syncthreads();
    uint32_t cursor = blockIdx.x % a.ninst;
    uint64_t idle_since = globaltimer();
    unsigned long long last_beat = ~0ull;
    uint32_t backoff = 64;
    for (;;) {
        if (threadIdx.x == 0)
            sm.cmd.quit = a.serve ? (ld_relaxed(a.stop_flag) != 0 || sm.idle_exit)
                                  : (ld_relaxed(a.done_count) >= a.ninst);
        __syncthreads();
        if (sm.cmd.quit) break;
        const long long pti = prof_now(sm);
        if (find_and_run<MODE>(a, sm, cursor)) {
            backoff = 64;
            continue;
        }
        // nothing to take: wait, bounded by the time limit without progress
        if (threadIdx.x == 0) {
            const unsigned long long beat = ld_relaxed64(a.heartbeat);
            const uint64_t now = globaltimer();
            if (beat != last_beat) {
                last_beat = beat;
                idle_since = now;
            } else if (a.serve) {
                // serving: a launch without work for idle_exit_ns ends (bounded
                // wait); the host relaunches it when requests arrive
                if (now - idle_since > a.idle_exit_ns) sm.idle_exit = 1;
            } else if (now - idle_since > a.p.timeout_ns) {
                for (uint32_t q = 0; q < a.ninst; ++q) {
                    InstCtl* ctl = a.insts[q].ctl;
                    if (atomicCAS(&ctl->status, (uint32_t)kRunning, (uint32_t)kFailed) == kRunning) {
                        atomicCAS(&ctl->err, 0u, 5u /* ABFS_ERR_TIMEOUT */);
                        atomicAdd(a.done_count, 1u);
                    }
                }
            }
            __nanosleep(backoff);
            if (backoff < kIdleBackoffMaxNs) backoff <<= 1;
        }
        __syncthreads();
        prof_add(sm, kProfIdle, pti);
    }
    if (a.prof && threadIdx.x == 0)
        for (int q = 0; q < kProfSlots; ++q) atomicAdd(a.prof + q, sm.prof[q]);
}

// ---------------------------------------------------------------------------
// initialisation: outputs, bitmaps, control blocks, the source (Algorithm 1's
// V_2 := V_1 \ supp(x_1)).
// ---------------------------------------------------------------------------

__global__ void init_fill_kernel(const Inst* insts, uint32_t ninst, uint32_t mode) {
    const Inst& I = insts[blockIdx.y];
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t t0 = blockIdx.x * blockDim.x + threadIdx.x;
    for (uint32_t v = t0; v < I.n; v += stride) {
        I.level[v] = -1;
        I.parent[v] = kUnset;
        if (mode == kModePlain) I.y[v] = ~0ull;
        if (I.sigma) I.sigma[v] = 0ull;
    }
    if (mode == kModeSub) {
        for (uint32_t w = t0; w < I.nwords; w += stride) {
            I.bm[0][w] = 0u;
            I.bm[1][w] = 0u;
        }
    }
    if (blockIdx.x == 0) {
        uint32_t* c = reinterpret_cast<uint32_t*>(I.ctl);
        for (uint32_t w = threadIdx.x; w < sizeof(InstCtl) / 4; w += blockDim.x) c[w] = 0u;
    }
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
    const uint32_t s = I.src;
    I.level[s] = 0;
    I.parent[s] = s;
    if (I.sigma) I.sigma[s] = 1ull;  // x_1 = e_src over the arithmetic semiring
    if (P.mode == kModeSub) I.bm[0][s >> 5] |= 1u << (s & 31);  // V_2 = V_1 \ {source}
    // frontier of level 0: one block holding the source
    const uint32_t len = I.colptr[s + 1] - I.colptr[s];
    const uint32_t w = len + kVertexSlots;
    I.fq[0][0] = s;
    I.fbeg[0][0] = I.colptr[s];
    I.fpre[0][0] = 0;
    I.blk[0][0].vb = 0;
    I.blk[0][0].nv = 1;
    I.blk[0][0].eb = 0;
    for (unsigned long long x = 0; x < w; x += P.unit) I.ustart[0][x / P.unit] = make_uint2(0, 0);
    ctl->bctr[0] = ((unsigned long long)w << kBlockBits) | 1ull;
    ctl->fcnt[0] = 1;
    ctl->reached = 1;
    ctl->mat_cur = 0;
    ctl->mat_prev = 0;
    ctl->mat_switch = 0;
    // the first CTA to arrive advances into level 0, which then starts a
    // resident run when it is small (the usual case) instead of a grid phase
    ctl->kind[0] = kPhStart;
    ctl->plevel[0] = 0;
    ctl->nitems[0] = 0;
    ctl->pending[0] = 1;
    ctl->epoch = 0;
    ctl->desc[0] = (0ull << 32) | 1ull;
    ctl->desc[1] = ~0ull;
    ctl->grab = 0ull;
    ctl->status = kRunning;
    if (I.trace && I.trace_cap) {
        const uint64_t now = globaltimer();
        I.trace[0] = make_uint4((uint32_t)now, (uint32_t)(now >> 32), (0xFEu << 24), 0u);
        I.trace[1] = make_uint4(0u, 1u, w, 0u);
        ctl->trace_n = 1;
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
    if (e == cudaSuccess) done = true;
    return e;
}

cudaError_t launch_engine(const EngineArgs& a, int grid, cudaStream_t s) {
    cudaError_t e;
    if (a.p.mode == kModePlain) {
        e = set_smem_attr<kModePlain>();
        if (e != cudaSuccess) return e;
        engine_kernel<kModePlain><<<grid, kThreads, sizeof(Smem), s>>>(a);
    } else {
        e = set_smem_attr<kModeSub>();
        if (e != cudaSuccess) return e;
        engine_kernel<kModeSub><<<grid, kThreads, sizeof(Smem), s>>>(a);
    }
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

}  // namespace abfs
