// Persistent BFS engine for sm_103a.
//
// One launch runs one or many searches to completion.  Every search advances
// level by level (Algorithm 1, Section 8): the frontier x_k is split into work
// units (tiles of frontier vertices, and fixed-size chunks of heavy columns);
// any CTA may take any unit of any search; the CTA that completes the last unit
// of a level advances that search to the next level and publishes the next
// level's units.  Small levels run on the advancing CTA alone ("narrow"
// levels), so long, thin searches do not pay a grid-wide hand-off per level.
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
// Comparator mode (masked SpMSpV, Section 5/Section 11): the multiply runs over
// every entry of the frontier columns into a stamped (min, index) accumulator,
// and the visited mask is applied to the touched rows afterwards.
//
// Shrink phases (Appendix A, A_k = S_k A S_k): when the reached fraction of the
// graph crosses a threshold, every still-unvisited column is stream-compacted
// to its unvisited rows; later levels read the compacted copy.
//
// Waits: a CTA without work polls a search's published phase; every poll loop
// is bounded by a time limit measured on %globaltimer and reset by progress.
// On expiry the CTA marks the searches failed (ABFS_ERR_TIMEOUT) and returns.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace abfs {

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
__device__ __forceinline__ unsigned long long ld_acquire64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Read of data written earlier in this launch by other CTAs (L2, not L1).
__device__ __forceinline__ uint32_t ld_l2(const uint32_t* p) { return __ldcg(p); }
__device__ __forceinline__ uint2 ld_l2(const uint2* p) { return __ldcg(p); }
// Read of data that no CTA writes during the launch.
__device__ __forceinline__ uint32_t ld_ro(const uint32_t* p) { return __ldg(p); }

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
    uint32_t nheavy;
    uint32_t nitems;
    uint32_t last;     // this CTA completed the last unit of the phase
    uint32_t quit;
};

struct Smem {
    uint32_t v[kTileMax + 1];
    uint32_t b[kTileMax];
    uint32_t off[kTileMax + 1];
    uint32_t out[kOutBuf];
    uint32_t out_cnt;
    uint32_t out_valid;
    uint32_t gbase;
    uint32_t warp_sums[kWarps + 1];
    unsigned long long st_read, st_unmasked, st_claims, st_nnz;
    Cmd cmd;
    Inst I;
    uint32_t cur_q;
};

// ---------------------------------------------------------------------------
// small block-level building blocks
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

// Exclusive scan of a[0..cnt) in place; a[cnt] = total.  cnt <= kThreads*4.
__device__ void block_exclusive_scan(uint32_t* a, uint32_t cnt, Smem& sm) {
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int kItems = kTileMax / kThreads;
    uint32_t x[kItems];
    uint32_t sum = 0;
#pragma unroll
    for (int q = 0; q < kItems; ++q) {
        uint32_t idx = tid * kItems + q;
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
    for (int q = 0; q < kItems; ++q) {
        uint32_t idx = tid * kItems + q;
        if (idx < cnt) a[idx] = run;
        run += x[q];
    }
    if (tid == 0) a[cnt] = sm.warp_sums[kWarps];
    __syncthreads();
}

// Column location of vertex v for a search at BFS level `lvl`: which matrix
// (input or a shrunk copy) holds its current column.
struct ColRef {
    uint32_t beg;
    uint32_t len;
    const uint32_t* rows;
};

__device__ __forceinline__ ColRef col_of(const Inst& I, uint32_t mat, uint32_t v) {
    ColRef c;
    if (mat == 0) {
        uint32_t b = ld_ro(I.colptr + v);
        uint32_t e = ld_ro(I.colptr + v + 1);
        c.beg = b;
        c.len = e - b;
        c.rows = I.rowidx;
    } else {
        const uint32_t s = mat - 1;
        c.beg = ld_l2(I.sbeg[s] + v);
        c.len = ld_l2(I.slen[s] + v);
        c.rows = I.srows[s];
    }
    return c;
}

__device__ __forceinline__ uint32_t mat_for_level(const InstCtl* ctl, uint32_t lvl) {
    // mat_cur/mat_prev/mat_switch change only at a level boundary, between
    // phases; the acquire at the start of a unit orders these reads.
    uint32_t sw = ld_relaxed(&ctl->mat_switch);
    return lvl >= sw ? ld_relaxed(&ctl->mat_cur) : ld_relaxed(&ctl->mat_prev);
}

__device__ __forceinline__ void fail(InstCtl* ctl, uint32_t code) {
    atomicCAS(&ctl->err, 0u, code);
}

// ---------------------------------------------------------------------------
// appending newly reached vertices
// ---------------------------------------------------------------------------

// Warp-aggregated append of `val` (where `want`) into the CTA staging buffer;
// overflow goes straight to the global queue.  All 32 lanes must call.
__device__ __forceinline__ void append_warp(bool want, uint32_t val, Smem& sm, uint32_t* gq,
                                            uint32_t* gcnt, uint32_t gcap, InstCtl* ctl) {
    const uint32_t mask = __ballot_sync(0xFFFFFFFFu, want);
    if (!mask) return;
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t leader = __ffs(mask) - 1;
    const uint32_t cnt = __popc(mask);
    const uint32_t rank = __popc(mask & lanemask_lt());
    uint32_t pos = 0;
    if (lane == leader) pos = atomicAdd(&sm.out_cnt, cnt);
    pos = __shfl_sync(0xFFFFFFFFu, pos, leader);
    if (pos + cnt <= (uint32_t)kOutBuf) {
        if (want) sm.out[pos + rank] = val;
    } else {
        uint32_t g = 0;
        if (lane == leader) {
            atomicMin(&sm.out_valid, pos);
            g = atomicAdd(gcnt, cnt);
        }
        g = __shfl_sync(0xFFFFFFFFu, g, leader);
        if (want) {
            if (g + rank < gcap) gq[g + rank] = val;
            else fail(ctl, 7 /* ABFS_ERR_DEVICE */);
        }
    }
}

// Block-wide flush of the staging buffer to the global queue.
__device__ void flush_out(Smem& sm, uint32_t* gq, uint32_t* gcnt, uint32_t gcap, InstCtl* ctl) {
    __syncthreads();
    const uint32_t n = min(sm.out_cnt, sm.out_valid);
    if (threadIdx.x == 0) {
        uint32_t base = n ? atomicAdd(gcnt, n) : 0u;
        if (base + n > gcap) {
            fail(ctl, 7);
            base = kUnset;
        }
        sm.gbase = base;
    }
    __syncthreads();
    const uint32_t base = sm.gbase;
    if (base != kUnset)
        for (uint32_t i = threadIdx.x; i < n; i += kThreads) gq[base + i] = sm.out[i];
    __syncthreads();
    if (threadIdx.x == 0) {
        sm.out_cnt = 0;
        sm.out_valid = kOutBuf;
    }
    __syncthreads();
}

// A vertex r has just joined the frontier of level lvl+1.  Heavy columns go to
// the heavy-chunk queue here (one thread writes its chunk descriptors); the
// return value says whether r belongs in the light frontier.
__device__ __forceinline__ bool route_new(const Inst& I, InstCtl* ctl, const EngineParams& P,
                                          uint32_t r, uint32_t lvl_next) {
    const uint32_t mat = mat_for_level(ctl, lvl_next);
    const ColRef c = col_of(I, mat, r);
    if (c.len < P.heavy) return true;
    const uint32_t pn = lvl_next & 1;
    const uint32_t nch = (c.len + P.chunk - 1) / P.chunk;
    const uint32_t base = atomicAdd(&ctl->hcnt[pn], nch);
    atomicAdd(&ctl->hvert[pn], 1u);
    if (base + nch > I.hcap) {
        fail(ctl, 7);
        return false;
    }
    for (uint32_t q = 0; q < nch; ++q) I.hq[pn][base + q] = make_uint2(r, q);
    return false;
}

// Comparator accumulator key of frontier column j at level k: the high word is
// a stamp that decreases with k (and stays below the all-ones initial value),
// so one atomicMin both overwrites stale keys and keeps the least j.
__device__ __forceinline__ uint32_t plain_stamp(uint32_t k) { return kUnset - 1u - k; }
__device__ __forceinline__ unsigned long long plain_key(uint32_t k, uint32_t j) {
    return ((unsigned long long)plain_stamp(k) << 32) | (unsigned long long)j;
}

// Row index load: the input matrix never changes during a launch (read-only
// path); shrunk copies are written by earlier phases of the same launch.
__device__ __forceinline__ uint32_t ld_row(const uint32_t* rows, uint32_t idx, uint32_t mat) {
    return mat == 0 ? ld_ro(rows + idx) : ld_l2(rows + idx);
}

// ---------------------------------------------------------------------------
// the per-entry step: mask, multiply, claim
// ---------------------------------------------------------------------------

// Submatrix mode: row r of frontier column j at level k.
__device__ __forceinline__ bool claim_sub(const Inst& I, InstCtl* ctl, const EngineParams& P,
                                          const uint32_t* test_bm, uint32_t* write_bm, uint32_t r,
                                          uint32_t j, uint32_t k, uint32_t& unmasked,
                                          uint32_t& claims, bool& light) {
    light = false;
    const uint32_t w = ld_l2(test_bm + (r >> 5));
    if ((w >> (r & 31)) & 1u) return false;  // row outside V_{k+1}: masked before the multiply
    ++unmasked;
    const uint32_t cur = ld_relaxed(I.parent + r);
    if (cur <= j) return false;  // a smaller parent is already in place; product cannot win
    ++claims;
    const uint32_t old = atomicMin(I.parent + r, j);
    if (old != kUnset) return false;
    // first product into row r: r joins x_{k+1}
    I.level[r] = (int32_t)(k + 1);
    atomicOr(write_bm + (r >> 5), 1u << (r & 31));
    light = route_new(I, ctl, P, r, k + 1);
    return true;
}

// ---------------------------------------------------------------------------
// work units
// ---------------------------------------------------------------------------

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

__device__ __forceinline__ void warp_stats(Smem& sm, uint32_t unmasked, uint32_t claims) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        unmasked += __shfl_xor_sync(0xFFFFFFFFu, unmasked, d);
        claims += __shfl_xor_sync(0xFFFFFFFFu, claims, d);
    }
    if ((threadIdx.x & 31) == 0) {
        if (unmasked) atomicAdd(&sm.st_unmasked, (unsigned long long)unmasked);
        if (claims) atomicAdd(&sm.st_claims, (unsigned long long)claims);
    }
}

// Expands the entries e in [e0, e1) of the tile described by sm.v/sm.b/sm.off
// (cnt columns).  Each lane walks its own column cursor forward.
template <int MODE>
__device__ void expand_entries(const Inst& I, InstCtl* ctl, const EngineParams& P, Smem& sm,
                               uint32_t cnt, uint32_t e0, uint32_t e1, const uint32_t* rows,
                               uint32_t mat, uint32_t k) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t p = k & 1;
    const uint32_t* test_bm = I.bm[p];
    uint32_t* write_bm = I.bm[p ^ 1];
    uint32_t unmasked = 0, claims = 0;
    // initial column of this lane: last i with off[i] <= e
    uint32_t e = e0 + lane;
    uint32_t i = 0;
    if (e < e1) {
        uint32_t lo = 0, hi = cnt;  // off[lo] <= e < off[hi]
        while (hi - lo > 1) {
            uint32_t mid = (lo + hi) >> 1;
            if (sm.off[mid] <= e) lo = mid;
            else hi = mid;
        }
        i = lo;
    }
    for (uint32_t base = e0; base < e1; base += 32, e += 32) {
        bool active = e < e1;
        bool want = false;
        uint32_t r = 0;
        if (active) {
            while (sm.off[i + 1] <= e) ++i;
            const uint32_t j = sm.v[i];
            r = ld_row(rows, sm.b[i] + (e - sm.off[i]), mat);
            if (MODE == kModeSub) {
                bool light;
                claim_sub(I, ctl, P, test_bm, write_bm, r, j, k, unmasked, claims, light);
                want = light;
            } else {
                // multiply first: every entry reaches the accumulator
                ++unmasked;
                ++claims;
                const unsigned long long old = atomicMin(I.y + r, plain_key(k, j));
                want = (uint32_t)(old >> 32) != plain_stamp(k);  // first touch of row r this level
            }
        }
        if (MODE == kModeSub)
            append_warp(want, r, sm, I.fq[p ^ 1], &ctl->fcnt[p ^ 1], I.n, ctl);
        else
            append_warp(want, r, sm, I.touched, &ctl->tcnt, I.n, ctl);
    }
    warp_stats(sm, unmasked, claims);
}

// A tile of light frontier vertices at level k.
template <int MODE>
__device__ void unit_light(const Inst& I, InstCtl* ctl, const EngineParams& P, Smem& sm,
                           uint32_t k, uint32_t tile_idx, uint32_t nf) {
    const uint32_t p = k & 1;
    const uint32_t base = tile_idx * P.tile;
    const uint32_t cnt = min(P.tile, nf - base);
    const uint32_t mat = mat_for_level(ctl, k);
    const uint32_t* fq = I.fq[p];
    uint32_t nnz_local = 0;
    for (uint32_t t = threadIdx.x; t < cnt; t += kThreads) {
        const uint32_t v = ld_l2(fq + base + t);
        const ColRef c = col_of(I, mat, v);
        sm.v[t] = v;
        sm.b[t] = c.beg;
        sm.off[t] = c.len;
        if (MODE == kModeSub) atomicOr(I.bm[p ^ 1] + (v >> 5), 1u << (v & 31));
        nnz_local += (mat == 0) ? c.len : (ld_ro(I.colptr + v + 1) - ld_ro(I.colptr + v));
    }
    // reached-column nonzeros (input matrix), for reports
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) nnz_local += __shfl_xor_sync(0xFFFFFFFFu, nnz_local, d);
    if ((threadIdx.x & 31) == 0 && nnz_local) atomicAdd(&sm.st_nnz, (unsigned long long)nnz_local);
    __syncthreads();
    block_exclusive_scan(sm.off, cnt, sm);
    const uint32_t E = sm.off[cnt];
    const uint32_t warp = threadIdx.x >> 5;
    const uint32_t per = (E + kWarps - 1) / kWarps;
    const uint32_t e0 = min(E, warp * per), e1 = min(E, e0 + per);
    const uint32_t* rows = (mat == 0) ? I.rowidx : I.srows[mat - 1];
    expand_entries<MODE>(I, ctl, P, sm, cnt, e0, e1, rows, mat, k);
    if (threadIdx.x == 0) sm.st_read += E;
    if (MODE == kModeSub)
        flush_out(sm, I.fq[p ^ 1], &ctl->fcnt[p ^ 1], I.n, ctl);
    else
        flush_out(sm, I.touched, &ctl->tcnt, I.n, ctl);
}

// One chunk of a heavy column at level k.
template <int MODE>
__device__ void unit_heavy(const Inst& I, InstCtl* ctl, const EngineParams& P, Smem& sm,
                           uint32_t k, uint32_t h) {
    const uint32_t p = k & 1;
    const uint2 d = ld_l2(I.hq[p] + h);
    const uint32_t v = d.x, q = d.y;
    const uint32_t mat = mat_for_level(ctl, k);
    const ColRef c = col_of(I, mat, v);
    const uint32_t lo = c.beg + q * P.chunk;
    const uint32_t hi = c.beg + min(c.len, (q + 1) * P.chunk);
    if (q == 0 && threadIdx.x == 0) {
        if (MODE == kModeSub) atomicOr(I.bm[p ^ 1] + (v >> 5), 1u << (v & 31));
        sm.st_nnz += (mat == 0) ? c.len : (ld_ro(I.colptr + v + 1) - ld_ro(I.colptr + v));
    }
    const uint32_t* test_bm = I.bm[p];
    uint32_t* write_bm = I.bm[p ^ 1];
    uint32_t unmasked = 0, claims = 0;
    for (uint32_t base = lo; base < hi; base += kThreads) {
        const uint32_t e = base + threadIdx.x;
        bool want = false;
        uint32_t r = 0;
        if (e < hi) {
            r = ld_row(c.rows, e, mat);
            if (MODE == kModeSub) {
                bool light;
                claim_sub(I, ctl, P, test_bm, write_bm, r, v, k, unmasked, claims, light);
                want = light;
            } else {
                ++unmasked;
                ++claims;
                const unsigned long long old = atomicMin(I.y + r, plain_key(k, v));
                want = (uint32_t)(old >> 32) != plain_stamp(k);
            }
        }
        if (MODE == kModeSub)
            append_warp(want, r, sm, I.fq[p ^ 1], &ctl->fcnt[p ^ 1], I.n, ctl);
        else
            append_warp(want, r, sm, I.touched, &ctl->tcnt, I.n, ctl);
    }
    warp_stats(sm, unmasked, claims);
    if (threadIdx.x == 0) sm.st_read += (hi > lo ? hi - lo : 0u);
    if (MODE == kModeSub)
        flush_out(sm, I.fq[p ^ 1], &ctl->fcnt[p ^ 1], I.n, ctl);
    else
        flush_out(sm, I.touched, &ctl->tcnt, I.n, ctl);
}

// Comparator: apply the visited mask to a tile of touched rows of level k.
__device__ void unit_plain_mask(const Inst& I, InstCtl* ctl, const EngineParams& P, Smem& sm,
                                uint32_t k, uint32_t tile_idx, uint32_t ntouched) {
    const uint32_t pn = (k + 1) & 1;
    const uint32_t base = tile_idx * P.tile;
    const uint32_t cnt = min(P.tile, ntouched - base);
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
                want = route_new(I, ctl, P, r, k + 1);
            }
        }
        append_warp(want, r, sm, I.fq[pn], &ctl->fcnt[pn], I.n, ctl);
    }
    flush_out(sm, I.fq[pn], &ctl->fcnt[pn], I.n, ctl);
}

// Shrink: compacts the unvisited columns among vertices
// [u*shrink_tile, (u+1)*shrink_tile) to their unvisited rows (A_k = S_k A S_k
// restricted to the columns still to be multiplied).  `vis` holds the
// vertices reached so far; src_mat is the matrix those columns are read from
// and dst (1 or 2) the shrunk copy being written.
__device__ void unit_shrink(const Inst& I, InstCtl* ctl, const EngineParams& P, Smem& sm,
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
    block_exclusive_scan(sm.off, cnt, sm);
    const uint32_t E = sm.off[cnt];
    const uint32_t* rows = (src_mat == 0) ? I.rowidx : I.srows[src_mat - 1];
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t per = (E + kWarps - 1) / kWarps;
    const uint32_t e0 = min(E, warp * per), e1 = min(E, e0 + per);
    // pass 1: count surviving rows per column
    for (int pass = 0; pass < 2; ++pass) {
        uint32_t e = e0 + lane;
        uint32_t i = 0;
        if (e < e1) {
            uint32_t lo = 0, hi = cnt;
            while (hi - lo > 1) {
                uint32_t mid = (lo + hi) >> 1;
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
                    const unsigned long long dst_pos = (unsigned long long)sm.gbase + pos;
                    if (dst_pos < I.scap) I.srows[s][dst_pos] = r;
                }
            }
        }
        __syncthreads();
        if (pass == 0) {
            // lengths of the new columns, then their begins
            for (uint32_t t = threadIdx.x; t < cnt; t += kThreads) I.slen[s][v0 + t] = cnt_arr[t];
            __syncthreads();
            block_exclusive_scan(cnt_arr, cnt, sm);
            if (threadIdx.x == 0) {
                const uint32_t S = cnt_arr[cnt];
                const uint32_t g = atomicAdd(&ctl->shrink_out, S);
                if ((unsigned long long)g + S > I.scap) fail(ctl, 7);
                sm.gbase = g;
                atomicAdd(&ctl->shrink_kept, (unsigned long long)S);
            }
            __syncthreads();
            for (uint32_t t = threadIdx.x; t < cnt; t += kThreads) I.sbeg[s][v0 + t] = sm.gbase + cnt_arr[t];
            // cnt_arr[t] now serves as the write cursor of column t, starting at its offset
            __syncthreads();
        }
    }
    // rows of column t occupy [gbase + off_t, ...): cursors advanced from the
    // exclusive offsets, so pass 2 wrote at gbase + offset + rank.
    if (threadIdx.x == 0) atomicAdd(&ctl->shrink_read, (unsigned long long)E);
    __syncthreads();
}

// ---------------------------------------------------------------------------
// phase control
// ---------------------------------------------------------------------------

// Runs one unit of phase (kind, k).
template <int MODE>
__device__ void run_unit(const Inst& I, InstCtl* ctl, const EngineParams& P, Smem& sm,
                         uint32_t kind, uint32_t k, uint32_t unit, uint32_t nheavy,
                         uint32_t nitems) {
    if (kind == kPhShrink) {
        // k = level just completed; its write bitmap holds every vertex reached so far
        const uint32_t src_mat = ld_relaxed(&ctl->mat_cur);
        unit_shrink(I, ctl, P, sm, unit, I.bm[(k + 1) & 1], src_mat, /*dst=*/nitems);
    } else if (kind == kPhPlainMask) {
        unit_plain_mask(I, ctl, P, sm, k, unit, nitems);
    } else if (unit < nheavy) {
        unit_heavy<MODE>(I, ctl, P, sm, k, unit);
    } else {
        unit_light<MODE>(I, ctl, P, sm, k, unit - nheavy, nitems);
    }
    stats_flush(sm, ctl);
}

__device__ __forceinline__ uint32_t units_of(const EngineParams& P, uint32_t kind, uint32_t nheavy,
                                             uint32_t nitems, uint32_t n) {
    if (kind == kPhShrink) return (n + P.shrink_tile - 1) / P.shrink_tile;
    return nheavy + (nitems + P.tile - 1) / P.tile;
}

// Thread 0 of the advancing CTA: the phase that follows (kind, k), written to
// sm.cmd; sm.cmd.quit = 1 when the search is over.
template <int MODE>
__device__ void decide_next(const Inst& I, InstCtl* ctl, const EngineParams& P, Smem& sm,
                            uint32_t kind, uint32_t k, uint32_t* done_count) {
    uint32_t nkind = 0, nk = 0, nh = 0, ni = 0, finish = 0;
    if (kind == kPhPlainMult) {
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
        const uint32_t nhc = ld_relaxed(&ctl->hcnt[pn]);
        const uint32_t nhv = ld_relaxed(&ctl->hvert[pn]);
        uint32_t reached = ld_relaxed(&ctl->reached);
        uint32_t shrinks = ld_relaxed(&ctl->shrinks);
        if (kind != kPhShrink) {
            st_relaxed(&ctl->levels, k + 1);
            if (nf == 0 && nhc == 0) {
                finish = 1;
            } else {
                reached += nf + nhv;
                st_relaxed(&ctl->reached, reached);
                // the buffers of level k become the "next" buffers of level k+1
                st_relaxed(&ctl->fcnt[pc], 0u);
                st_relaxed(&ctl->hcnt[pc], 0u);
                st_relaxed(&ctl->hvert[pc], 0u);
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
            bool do_shrink = false;
            if (MODE == kModeSub && kind != kPhShrink && P.shrink_theta > 0.f &&
                P.shrink_theta < 1.f && shrinks < P.shrink_max) {
                // the i-th shrink waits until a fraction 1-(1-theta)^i of n is reached
                const float frac = (float)reached / (float)I.n;
                const float need = 1.f - powf(1.f - P.shrink_theta, (float)(shrinks + 1));
                do_shrink = frac >= need;
            }
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
                nh = nhc;
                ni = nf;
            }
        }
    }
    if (ld_relaxed(&ctl->err) != 0) finish = 1;
    sm.cmd.kind = nkind;
    sm.cmd.level = nk;
    sm.cmd.nheavy = nh;
    sm.cmd.nitems = ni;
    sm.cmd.quit = finish;
    if (finish) {
        const uint32_t e = ld_relaxed(&ctl->err);
        __threadfence();
        if (atomicCAS(&ctl->status, (uint32_t)kRunning, e ? (uint32_t)kFailed : (uint32_t)kDone) ==
            kRunning)
            atomicAdd(done_count, 1u);
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
        if (sm.cmd.quit) return;
        const uint32_t nkind = sm.cmd.kind, nk = sm.cmd.level;
        const uint32_t nh = sm.cmd.nheavy, ni = sm.cmd.nitems;
        const uint32_t units = units_of(P, nkind, nh, ni, I.n);
        const bool alone = (nkind == kPhShrink) ? (units <= 1) : (nh == 0 && ni <= P.narrow_max);
        if (!alone) {
            if (threadIdx.x == 0) {
                const uint32_t e = ld_relaxed(&ctl->epoch) + 1;
                const uint32_t q = e & 1;
                st_relaxed(&ctl->kind[q], nkind);
                st_relaxed(&ctl->plevel[q], nk);
                st_relaxed(&ctl->nheavy[q], nh);
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
        // narrow: this CTA runs every unit of the phase, then decides again
        for (uint32_t u = 0; u < units; ++u) run_unit<MODE>(I, ctl, P, sm, nkind, nk, u, nh, ni);
        __threadfence();
        __syncthreads();
        kind = nkind;
        k = nk;
    }
}

// Thread 0: whether instance q has an untaken unit in its published phase.
__device__ __forceinline__ bool has_work(const Inst* insts, uint32_t q) {
    InstCtl* ctl = insts[q].ctl;
    if (ld_relaxed(&ctl->status) != kRunning) return false;
    const unsigned long long g = ld_relaxed64(&ctl->grab);
    const uint32_t e = (uint32_t)(g >> 32), taken = (uint32_t)g;
    const unsigned long long d = ld_relaxed64(&ctl->desc[e & 1]);
    return (uint32_t)(d >> 32) == e && taken < (uint32_t)d;
}

// Thread 0: takes a unit of instance q if one is left; fills sm.cmd.
__device__ __forceinline__ bool take_unit(const Inst* insts, uint32_t q, Smem& sm) {
    InstCtl* ctl = insts[q].ctl;
    const unsigned long long old = atomicAdd(&ctl->grab, 1ull);
    const uint32_t e = (uint32_t)(old >> 32), t = (uint32_t)old;
    const unsigned long long d = ld_relaxed64(&ctl->desc[e & 1]);
    if ((uint32_t)(d >> 32) != e || t >= (uint32_t)d) return false;
    __threadfence();  // acquire: the phase fields and the data of earlier phases
    const uint32_t qq = e & 1;
    sm.cmd.q = q;
    sm.cmd.epoch = e;
    sm.cmd.unit = t;
    sm.cmd.kind = ld_relaxed(&ctl->kind[qq]);
    sm.cmd.level = ld_relaxed(&ctl->plevel[qq]);
    sm.cmd.nheavy = ld_relaxed(&ctl->nheavy[qq]);
    sm.cmd.nitems = ld_relaxed(&ctl->nitems[qq]);
    return true;
}

// Warp 0 scans the instances 32 at a time from `cursor` and takes the first
// unit it can; the whole CTA then runs it.  Returns true if a unit was run.
template <int MODE>
__device__ bool find_and_run(const EngineArgs& a, Smem& sm, uint32_t& cursor) {
    if (threadIdx.x < 32) {
        const uint32_t lane = threadIdx.x;
        bool got = false;
        for (uint32_t base = 0; base < a.ninst && !got; base += 32) {
            const uint32_t idx = base + lane;
            const uint32_t q = (cursor + idx) % a.ninst;
            const bool avail = idx < a.ninst && has_work(a.insts, q);
            uint32_t mask = __ballot_sync(0xFFFFFFFFu, avail);
            while (mask && !got) {
                const uint32_t l = __ffs(mask) - 1;
                bool ok = false;
                if (lane == l) ok = take_unit(a.insts, q, sm);
                got = __shfl_sync(0xFFFFFFFFu, ok, l);
                mask &= mask - 1;
            }
        }
        __syncwarp();
        if (lane == 0) {
            sm.cmd.has = got;
            if (got && sm.cur_q != sm.cmd.q) {
                sm.I = a.insts[sm.cmd.q];
                sm.cur_q = sm.cmd.q;
            }
        }
    }
    __syncthreads();
    if (!sm.cmd.has) return false;
    cursor = sm.cmd.q;
    const Inst& I = sm.I;
    InstCtl* ctl = I.ctl;
    const uint32_t kind = sm.cmd.kind, k = sm.cmd.level, epoch = sm.cmd.epoch;
    run_unit<MODE>(I, ctl, a.p, sm, kind, k, sm.cmd.unit, sm.cmd.nheavy, sm.cmd.nitems);
    // completion: release this CTA's writes, then count the unit down
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t left = atomicSub(&ctl->pending[epoch & 1], 1u);
        sm.cmd.last = (left == 1);
        atomicAdd(a.heartbeat, 1ull);
    }
    __syncthreads();
    if (sm.cmd.last) advance<MODE>(I, ctl, a.p, sm, kind, k, a.done_count, a.heartbeat);
    return true;
}

template <int MODE>
__global__ void __launch_bounds__(kThreads, 2) engine_kernel(EngineArgs a) {
    __shared__ Smem sm;
    if (threadIdx.x == 0) {
        sm.out_cnt = 0;
        sm.out_valid = kOutBuf;
        sm.st_read = sm.st_unmasked = sm.st_claims = sm.st_nnz = 0;
        sm.cur_q = kUnset;
    }
    __syncthreads();
    uint32_t cursor = blockIdx.x % a.ninst;
    uint64_t idle_since = globaltimer();
    unsigned long long last_beat = ~0ull;
    uint32_t backoff = 64;
    for (;;) {
        if (threadIdx.x == 0) sm.cmd.quit = (ld_relaxed(a.done_count) >= a.ninst);
        __syncthreads();
        if (sm.cmd.quit) break;
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
            if (backoff < 2048) backoff <<= 1;
        }
        __syncthreads();
    }
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
    const Inst* insts = a.insts;
    const EngineParams& P = a.p;
    const Inst& I = insts[q];
    InstCtl* ctl = I.ctl;
    const uint32_t s = I.src;
    I.level[s] = 0;
    I.parent[s] = s;
    if (P.mode == kModeSub) I.bm[0][s >> 5] |= 1u << (s & 31);  // V_2 = V_1 \ {source}
    const uint32_t len = I.colptr[s + 1] - I.colptr[s];
    uint32_t nh = 0, nf = 0;
    if (len >= P.heavy) {
        nh = (len + P.chunk - 1) / P.chunk;
        for (uint32_t c = 0; c < nh; ++c) I.hq[0][c] = make_uint2(s, c);
        ctl->hcnt[0] = nh;
        ctl->hvert[0] = 1;
    } else {
        I.fq[0][0] = s;
        nf = 1;
        ctl->fcnt[0] = 1;
    }
    ctl->reached = 1;
    ctl->mat_cur = 0;
    ctl->mat_prev = 0;
    ctl->mat_switch = 0;
    const uint32_t units = nh + (nf ? 1u : 0u);
    ctl->kind[0] = (P.mode == kModePlain) ? kPhPlainMult : kPhLevel;
    ctl->plevel[0] = 0;
    ctl->nheavy[0] = nh;
    ctl->nitems[0] = nf;
    ctl->pending[0] = units;
    ctl->epoch = 0;
    ctl->desc[0] = (0ull << 32) | units;
    ctl->desc[1] = ~0ull;
    ctl->grab = 0ull;
    ctl->status = kRunning;
}

// Writes the per-call fields of instance 0 (single searches reuse one
// descriptor; kernel arguments avoid a host staging buffer).
__global__ void set_query_kernel(Inst* inst, uint32_t src, int32_t* level, uint32_t* parent) {
    inst->src = src;
    inst->level = level;
    inst->parent = parent;
}

cudaError_t launch_set_query(Inst* inst, uint32_t src, int32_t* level, uint32_t* parent,
                             cudaStream_t s) {
    set_query_kernel<<<1, 1, 0, s>>>(inst, src, level, parent);
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

cudaError_t launch_engine(const EngineArgs& a, int grid, cudaStream_t s) {
    if (a.p.mode == kModePlain)
        engine_kernel<kModePlain><<<grid, kThreads, 0, s>>>(a);
    else
        engine_kernel<kModeSub><<<grid, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t engine_occupancy(uint32_t mode, int* blocks_per_sm) {
    if (mode == kModePlain)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, engine_kernel<kModePlain>,
                                                             kThreads, 0);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, engine_kernel<kModeSub>,
                                                         kThreads, 0);
}

}  // namespace abfs
