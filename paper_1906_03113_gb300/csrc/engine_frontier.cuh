// Appending newly reached vertices as frontier blocks (Section 10's counts
// and prefix offsets at warp and CTA scope) and as resident-run lists.
// Part of the persistent engine (engine.cu), split by topic; included in order.
#pragma once

#include "engine_common.cuh"

namespace abfs {

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
// (col_slots each) and, in ent, their column entries.  Whole warp.
__device__ __forceinline__ uint32_t warp_cols(Smem& sm, const Inst& I, uint32_t mat_next, uint32_t n,
                                              WarpCols& c, uint32_t& ent) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t* wv = sm.wv[threadIdx.x >> 5];
    uint32_t sum = 0;
    ent = 0;
#pragma unroll
    for (int it = 0; it < kWarpSpans; ++it) {
        const uint32_t i = it * 32 + lane;
        c.beg[it] = 0;
        c.len[it] = 0;
        if (i < n) {
            const ColRef r = col_of(I, mat_next, wv[i]);
            c.beg[it] = r.beg;
            c.len[it] = r.len;
            sum += col_slots(I, mat_next, r.beg, r.len);
            ent += r.len;
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        sum += __shfl_xor_sync(0xFFFFFFFFu, sum, d);
        ent += __shfl_xor_sync(0xFFFFFFFFu, ent, d);
    }
    return sum;
}

// Writes this warp's n staged vertices (columns c) at fq[vb + voff ..] of
// block blk (entry base eb), the group starting at weight offset woff within
// the block.  Whole warp.
__device__ __forceinline__ void warp_emit(Smem& sm, const Inst& I, InstCtl* ctl,
                                          const EngineParams& P, uint32_t pn, uint32_t mat_next,
                                          const WarpCols& c,
                                          uint32_t n, uint32_t blk, unsigned long long eb,
                                          uint32_t vb, uint32_t voff, uint32_t woff) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t* wv = sm.wv[threadIdx.x >> 5];
    uint32_t carry = woff;
#pragma unroll
    for (int it = 0; it < kWarpSpans; ++it) {
        if ((uint32_t)it * 32 >= n) break;
        const uint32_t i = it * 32 + lane;
        const uint32_t w = i < n ? col_slots(I, mat_next, c.beg[it], c.len[it]) : 0u;
        const uint32_t incl = warp_incl_scan(w);
        const uint32_t pre = carry + incl - w;
        if (i < n) {
            const uint32_t at = vb + voff + i;
            I.fq[pn][at] = wv[i];
            I.fbeg[pn][at] = c.beg[it];
            I.fpre[pn][at] = pre;
            I.flen[pn][at] = c.len[it];
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
    uint32_t wtot = 0, ent = 0;
    for (uint32_t i = lane; i < n; i += 32) {
        const ColRef c = col_of(I, mat_next, wv[i]);
        wtot += col_slots(I, mat_next, c.beg, c.len);
        ent += c.len;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) wtot += __shfl_xor_sync(0xFFFFFFFFu, wtot, d);
    if (P.bu_alpha) {
        // the hybrid's direction choice needs the frontier's exact entries
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) ent += __shfl_xor_sync(0xFFFFFFFFu, ent, d);
        if (lane == 0 && ent) atomicAdd(&ctl->fent[pn], (unsigned long long)ent);
    }
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
            const uint32_t w = i < n ? col_slots(I, mat_next, c.beg, c.len) : 0u;
            const uint32_t incl = warp_incl_scan(w);
            const uint32_t pre = carry + incl - w;
            if (i < n) {
                I.fq[pn][vb + i] = v;
                I.fbeg[pn][vb + i] = c.beg;
                I.fpre[pn][vb + i] = pre;
                I.flen[pn][vb + i] = c.len;
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
    uint32_t ent = 0;
    const uint32_t wtot = warp_cols(sm, I, mat_next, n, c, ent);
    if (P.bu_alpha && lane == 0 && ent) atomicAdd(&ctl->fent[pn], (unsigned long long)ent);
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
        warp_emit(sm, I, ctl, P, pn, mat_next, c, n, sm.gblk, sm.geb, sm.gbase, sm.wvoff[warp],
                  sm.wwoff[warp]);
    if (lane == 0) sm.wcnt[warp] = 0;
    __syncthreads();
}

// Resident narrow runs: a warp appends its n staged vertices to the frontier
// list of parity pn (vertex, column begin, column length in matrix mat_next),
// at a position taken from a shared-memory counter (in a cluster run, the
// leader CTA's counter, reached through DSMEM).  Whole warp.
__device__ __forceinline__ void narrow_append(Smem& sm, const Inst& I, InstCtl* ctl, uint32_t pn, uint32_t mat_next,
                              uint32_t& wc) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t n = wc;
    const uint32_t* wv = sm.wv[threadIdx.x >> 5];
    uint32_t base = 0;
    // positions: this CTA's own counter, or in a cluster run the leader's
    // (DSMEM); the CTA's own counter always counts its appends
    if (lane == 0) {
        base = atomicAdd(&sm.nq_cnt, n);
        if (sm.ds_ctr) base = ds_add(sm.ds_ctr, n);
    }
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
                    I.flen[pn][at] = c[q].len;
                } else {
                    fail(ctl, 7);
                }
                wsum += col_slots(I, mat_next, c[q].beg, c[q].len);
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
// first-touched rows to the touched list (counter as in narrow_append).
// Whole warp.
__device__ __forceinline__ void narrow_touch(Smem& sm, const Inst& I, InstCtl* ctl, uint32_t& wc) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t n = wc;
    const uint32_t* wv = sm.wv[threadIdx.x >> 5];
    uint32_t base = 0;
    if (lane == 0) {
        base = atomicAdd(&sm.nt_cnt, n);
        if (sm.ds_ctr) base = ds_add(sm.ds_ctr, n);
    }
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

}  // namespace abfs
