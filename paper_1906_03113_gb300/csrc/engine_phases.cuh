// Bitmap-word phases of the direction-optimising hybrid, the physical shrink
// (Appendix A) and the in-launch initialisation used by serving.
// Part of the persistent engine (engine.cu), split by topic; included in order.
#pragma once

#include "engine_expand.cuh"

namespace abfs {

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

// ---------------------------------------------------------------------------
// multi-source searches: the update phase of a level
// ---------------------------------------------------------------------------
//
// After the expand phase of level k, ms_nx[v] holds the sources (bits) that
// reach v first at level k+1.  For each such source s, v's parent is the least
// frontier vertex j of level k, for s, that has v in its column; on an
// undirected graph that is the least j in v's own column with bit s in
// ms_fr[k&1][j], and with the column ascending the first such entry.  A lane
// scans its vertex's column itself for the first entries, four at a time;
// longer scans run on the whole warp, 32 entries at a time, where each lane
// keeps the bits no lower lane has (a prefix OR across the warp).

// Parent output of vertex v for the sources in `bits`: j.  (Levels are written
// source by source for a warp's 32 vertices at once, in unit_ms_update.)
__device__ __forceinline__ void ms_write(const Inst& I, uint32_t v, uint32_t j, unsigned long long bits) {
    while (bits) {
        const uint32_t s = (uint32_t)(__ffsll((long long)bits) - 1);
        bits &= bits - 1;
        I.ms_parent[s][v] = (int32_t)j;
    }
}

// Inclusive prefix OR of a 64-bit value across the warp's lanes.
__device__ __forceinline__ unsigned long long warp_prefix_or(unsigned long long x) {
    const uint32_t lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, x, d);
        if (lane >= (uint32_t)d) x |= y;
    }
    return x;
}

// Unit u of the update of level k: chunks [u*per, (u+1)*per) of 8 x 32 vertices.
__device__ ABFS_NOINLINE void unit_ms_update(const Inst& I, InstCtl* ctl, const EngineParams& P,
                                             Smem& sm, uint32_t k, uint32_t u, uint32_t per) {
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t p = k & 1, pn = p ^ 1;
    const unsigned long long* fr = I.ms_fr[p];
    const uint32_t chunks = (I.nwords + kChunkWords - 1) / kChunkWords;
    const uint32_t c1 = min(chunks, (u + 1) * per);
    uint32_t wc = sm.wcnt[warp];
    Tally t;
    for (uint32_t c = u * per + warp; c < c1; c += kWarps) {
        for (uint32_t q = 0; q < kChunkWords; ++q) {
            const uint32_t v = (c * kChunkWords + q) * 32 + lane;
            unsigned long long nb = 0;
            uint32_t e = 0, end = 0;
            if (v < I.n) {
                nb = ld_l2(I.ms_nx + v);
                // every vertex gets its bits of the next frontier (0: none)
                I.ms_fr[pn][v] = nb;
                if (nb) {
                    I.ms_nx[v] = 0ull;
                    I.ms_vis[v] = ld_l2(I.ms_vis + v) | nb;
                    e = ld_ro(I.colptr + v);
                    end = ld_ro(I.colptr + v + 1);
                }
            }
            unsigned long long rem = nb;
            for (uint32_t b = 0; b < kBuLaneBatches && rem && e < end; ++b) {
                uint32_t jj[4];
                unsigned long long fm[4];
#pragma unroll
                for (int x = 0; x < 4; ++x) jj[x] = e + x < end ? ld_ro(I.rowidx + e + x) : kUnset;
#pragma unroll
                for (int x = 0; x < 4; ++x) fm[x] = jj[x] != kUnset ? ld_l2(fr + jj[x]) : 0ull;
                t.read += min(4u, end - e);
#pragma unroll
                for (int x = 0; x < 4; ++x) {
                    const unsigned long long hit = fm[x] & rem;
                    if (hit) {
                        ms_write(I, v, jj[x], hit);
                        rem &= ~hit;
                    }
                }
                e += 4;
            }
            bool defer = rem != 0 && e < end;
            uint32_t dm;
            while ((dm = __ballot_sync(0xFFFFFFFFu, defer)) != 0u) {
                const uint32_t ldr = __ffs(dm) - 1;
                const uint32_t lv = __shfl_sync(0xFFFFFFFFu, v, ldr);
                const uint32_t le = __shfl_sync(0xFFFFFFFFu, e, ldr);
                const uint32_t lend = __shfl_sync(0xFFFFFFFFu, end, ldr);
                unsigned long long lrem = __shfl_sync(0xFFFFFFFFu, rem, ldr);
                for (uint32_t x = le; x < lend && lrem; x += 32) {
                    const uint32_t idx = x + lane;
                    const uint32_t j = idx < lend ? ld_ro(I.rowidx + idx) : kUnset;
                    const unsigned long long h = j != kUnset ? (ld_l2(fr + j) & lrem) : 0ull;
                    const unsigned long long incl = warp_prefix_or(h);
                    // the bits this lane's entry is the first (least) to hold
                    const unsigned long long prev = __shfl_up_sync(0xFFFFFFFFu, incl, 1);
                    const unsigned long long first = lane ? (h & ~prev) : h;
                    if (first) ms_write(I, lv, j, first);
                    if (lane == 0) t.read += min(32u, lend - x);
                    lrem &= ~__shfl_sync(0xFFFFFFFFu, incl, 31);
                }
                if (lane == ldr) defer = false;
            }
            {
                // levels source by source: the lanes that hold a source's bit
                // write consecutive vertices of that source's level array
                unsigned long long un = nb;
#pragma unroll
                for (int d = 16; d > 0; d >>= 1) un |= __shfl_xor_sync(0xFFFFFFFFu, un, d);
                while (un) {
                    const uint32_t s = (uint32_t)(__ffsll((long long)un) - 1);
                    un &= un - 1;
                    if ((nb >> s) & 1ull) I.ms_level[s][v] = (int32_t)(k + 1);
                }
            }
            stage_warp(nb != 0ull, v, sm, wc);
            if (wc > (uint32_t)(kWarpBuf - 32)) warp_flush(sm, I, ctl, P, pn, 0u, wc);
        }
    }
    if (lane == 0) sm.wcnt[warp] = wc;
    __syncwarp();
    tally_flush(sm, t);
    cta_flush(sm, I, ctl, P, pn, 0u);
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

}  // namespace abfs
