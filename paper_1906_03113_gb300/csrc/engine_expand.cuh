// The per-entry step (mask, multiply, claim; Theorem 1) and the work units of
// a level, including the extraction after a level claimed by reductions.
// Part of the persistent engine (engine.cu), split by topic; included in order.
#pragma once

#include "engine_frontier.cuh"

namespace abfs {

// ---------------------------------------------------------------------------
// the per-entry step: mask, multiply, claim -- kIlp entries per thread at once
// ---------------------------------------------------------------------------

// How a level claims the vertices it reaches.
enum ClaimVar : int {
    kVarWide = 0,    // atomicMin with return; the winner stages the vertex (frontier blocks)
    kVarNarrow = 1,  // the same inside a resident narrow run (plain frontier list)
    kVarScan = 2,    // reductions only: atomicMin and the bit in the write bitmap without
                     // return; an extraction phase collects the new vertices afterwards
    kVarMs = 3,      // multi-source search: the next-bit mask of row r gets the frontier
                     // bits of column j that r has not reached (a 64-bit reduction); an
                     // update phase turns them into levels, parents and the next frontier
};

// Groups of 32 entries each thread keeps in flight, per claim variant.
__host__ __device__ constexpr int ilp_of(int var) {
    return (var == kVarScan || var == kVarMs) ? kIlpScan : kIlp;
}

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
    if (VAR == kVarMs) {
        // x_{k+1}(r) gets, for every source s, the product of frontier column j
        // with row r masked by r's reached set: one bit per source.  fr and vis
        // change only between phases (plain loads after the unit's acquire).
        const unsigned long long* fr = I.ms_fr[p];
        unsigned long long fm[L], vv[L];
#pragma unroll
        for (int u = 0; u < L; ++u) {
            fm[u] = r[u] != kUnset ? fr[j[u]] : 0ull;
            vv[u] = r[u] != kUnset ? I.ms_vis[r[u]] : ~0ull;
        }
#pragma unroll
        for (int u = 0; u < L; ++u) {
            const unsigned long long nb = fm[u] & ~vv[u];
            if (nb) {
                ++t.unmasked;
                ++t.claims;
                atomicOr(I.ms_nx + r[u], nb);
            }
        }
        return;
    }
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

// Chunks [lo, hi) are split evenly over the warps: warp w starts at
// lo + w * per, per = ceil((hi - lo) / kWarps).  Staged vertex s, whose chunks
// are [st, en), records itself for every warp that starts inside its range (as
// s - 1 when the warp starts on s's first chunk, since that start bit counts
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

// Staged vertex s, whose slots start at st (a multiple of kChunk), with
// sm.b[s] holding its column begin and sm.end[s] its length on entry: sm.b[s]
// becomes beg - st and sm.end[s] the end of its entry slots.  The column's
// entries occupy slots [st + h, st + h + len), h = col_head(beg), so slot x
// holds the row index at position b + x - h and each chunk of four slots is one
// aligned 16-byte group of the column.
__device__ __forceinline__ void set_slot_map(Smem& sm, const Inst& I, uint32_t mat, uint32_t s,
                                             uint32_t st) {
    const uint32_t beg = sm.b[s], len = sm.end[s];
    sm.b[s] = beg - st;
    sm.end[s] = st + col_head(I, mat, beg) + len;
}

// Expands the slots [l0, l1) (multiples of kChunk) of the staged vertices (cnt
// of them; sm.off holds their first slots, sm.off[cnt] the end; sm.sbits has a
// bit per chunk of [l0, l1) that starts a vertex; sm.b and sm.end as
// set_slot_map leaves them).  The chunks are split evenly over the warps; a
// lane takes one chunk per step, 32 consecutive chunks per warp, and reads its
// four row indices with one 16-byte load (coalesced across the warp).  The
// vertex of a chunk is a prefix count of vertex starts, read from sm.sbits
// with one popcount.  The row loads of step s+1 are issued before step s is
// processed.
template <int MODE, int VAR>
__device__ __forceinline__ void expand_core(const Inst& I, InstCtl* ctl, const EngineParams& P, Smem& sm,
                             uint32_t cnt, uint32_t l0, uint32_t l1, uint32_t mat,
                             uint32_t mat_next, uint32_t k, Tally& t) {
    constexpr int L = ilp_of(VAR);
    static_assert(L == (int)kChunk, "one chunk of row indices per lane and step");
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#ifdef ABFS_EXPAND_PROFILE
    const long long xt0 = sm.prof_on ? clock64() : 0ll;
#endif
    const uint32_t c0 = l0 / kChunk, span = (l1 - l0) / kChunk;
    const uint32_t per = (span + kWarps - 1) / kWarps;
    const uint32_t e0 = c0 + min(span, warp * per);
    const uint32_t e1 = c0 + min(span, warp * per + per);
    const uint32_t* rows = rows_of(I, mat);
    const uint32_t* const rows_hi = rows_end(I, mat);
    const uint32_t rs = row_shift(rows);
    const uint64_t pol = evict_first_policy();
    const uint32_t le_mask = (2u << lane) - 1u;  // lanes 0..lane
    // vertex(c) = vb + (number of vertex starts in [e0, c])
    uint32_t vb = 0;
    if (e0 < e1) {
        vb = sm.wvb[warp];
        // recorded while staging; searched for only if the record is missing
        if (vb == kNoVb || (vb != kUnset && vb >= cnt)) {
            uint32_t lo = 0, hi = cnt;  // chunk of off[lo] <= e0 < chunk of off[hi]
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (sm.off[mid] / kChunk <= e0) lo = mid;
                else hi = mid;
            }
            vb = lo - (sm.off[lo] / kChunk == e0 ? 1u : 0u);
        }
    }
    uint32_t starts = 0;  // vertex starts in [e0, current group base)
    // row indices (kUnset: no entry in this slot) and frontier column of a lane's chunk
    uint32_t r[L], j[L];
    auto load_step = [&](uint32_t base, uint32_t (&rr)[L], uint32_t (&jj)[L]) {
        const uint32_t rel = base - c0;
        const uint32_t sh = rel & 31;
        uint32_t w = sm.sbits[rel >> 5] >> sh;
        if (sh) w |= sm.sbits[(rel >> 5) + 1] << (32 - sh);
        const uint32_t c = base + lane;
        const uint32_t v = vb + starts + __popc(w & le_mask);
        starts += __popc(w);
#pragma unroll
        for (int q = 0; q < L; ++q) {
            rr[q] = kUnset;
            jj[q] = 0;
        }
        if (c < e1) {
            const uint32_t s = c * kChunk;
            const uint32_t pb = sm.b[v], hi = sm.end[v];
            const uint32_t h = (pb + rs) & (kChunk - 1);
            // the vertex's first chunk starts with h empty slots
            const uint32_t lo = ((w >> lane) & 1u) ? h : 0u;
            if (s + lo < hi) {
                const uint32_t jv = sm.v[v];
                // pb + s is the position of the chunk's slot h (never negative);
                // the group may start up to three indices before the row array
                const uint32_t* cp = rows + (pb + s) - h;
                if (cp >= rows && cp + kChunk <= rows_hi) {
                    const uint4 x = ld_row4(cp, mat, pol);
                    rr[0] = x.x;
                    rr[1] = x.y;
                    rr[2] = x.z;
                    rr[3] = x.w;
#pragma unroll
                    for (int q = 0; q < L; ++q)
                        if ((uint32_t)q < lo || s + q >= hi) rr[q] = kUnset;
                } else {
                    // the group reaches past either end of the row array
#pragma unroll
                    for (int q = 0; q < L; ++q)
                        if ((uint32_t)q >= lo && s + q < hi) rr[q] = ld_row(cp, q, mat, pol);
                }
#pragma unroll
                for (int q = 0; q < L; ++q) jj[q] = jv;
            }
        }
    };
    uint32_t wc = sm.wcnt[warp];
    if (e0 < e1) load_step(e0, r, j);
#ifdef ABFS_EXPAND_PROFILE
    long long xt1 = 0, xflush = 0, xproc = 0;
    if (sm.prof_on) xt1 = clock64();
#endif
    for (uint32_t base = e0; base < e1; base += 32) {
        uint32_t r2[L], j2[L];
        if (base + 32 < e1) {
            load_step(base + 32, r2, j2);
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
        if (VAR == kVarScan || VAR == kVarMs) {
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
        // slots [lo, hi) of this sub-tile belong to the unit
        const uint32_t lo = (uint32_t)(e - g0);
        const uint32_t hi_s = (uint32_t)(min(u_hi, (unsigned long long)sm.sub_end) - g0);
        for (uint32_t s = threadIdx.x; s < cnt; s += kThreads) {
            uint32_t q = 0, hi = nseg;  // seg_pos[q] <= s < seg_pos[hi]
            while (hi - q > 1) {
                const uint32_t mid = (q + hi) >> 1;
                if (sm.seg_pos[mid] <= s) q = mid;
                else hi = mid;
            }
            const uint32_t idx = sm.seg_idx[q] + (s - sm.seg_pos[q]);
            const uint32_t v = ld_l2(I.fq[p] + idx);
            const uint32_t len = ld_l2(I.flen[p] + idx);
            const uint32_t st = (uint32_t)(sm.seg_eb[q] + ld_l2(I.fpre[p] + idx) - g0);
            // the column index its products carry: the input label on a relabelled graph
            sm.v[s] = I.lab ? ld_ro(I.lab + v) : v;
            sm.b[s] = ld_l2(I.fbeg[p] + idx);
            sm.end[s] = len;
            sm.off[s] = st;
            if (st >= lo && st < hi_s) {
                // the vertex's first slot lies in this unit: it joins the visited
                // set of the next level's test (once)
                if (MODE == kModeSub && VAR != kVarMs) atomicOr(I.bm[p ^ 1] + (v >> 5), 1u << (v & 31));
                nnz_local += (mat == 0) ? len : (ld_ro(I.colptr + v + 1) - ld_ro(I.colptr + v));
            }
        }
        if (threadIdx.x == 0) sm.off[cnt] = (uint32_t)(sm.sub_end - g0);
        if (threadIdx.x < (uint32_t)kWarps) sm.wvb[threadIdx.x] = kNoVb;
        const uint32_t nwords = ((hi_s - lo) / kChunk + 31) / 32 + 1;
        for (uint32_t w = threadIdx.x; w < nwords; w += kThreads) sm.sbits[w] = 0u;
        __syncthreads();
        for (uint32_t s = threadIdx.x; s < cnt; s += kThreads) {
            const uint32_t st = sm.off[s];
            set_slot_map(sm, I, mat, s, st);
            mark_warp_starts(sm, s, st / kChunk, sm.off[s + 1] / kChunk, lo / kChunk, hi_s / kChunk);
            if (st >= lo && st < hi_s) {
                // the vertex's first slot lies in this unit: it starts a run of chunks
                const uint32_t c = (st - lo) / kChunk;
                atomicOr(&sm.sbits[c >> 5], 1u << (c & 31));
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
    if (MODE == kModeSub && VAR != kVarScan && VAR != kVarMs) cta_flush(sm, I, ctl, P, p ^ 1, mat_next);
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

}  // namespace abfs
