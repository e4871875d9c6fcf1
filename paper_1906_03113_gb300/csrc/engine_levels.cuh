// Phase control: running a unit, resident narrow runs, choosing and publishing
// the next phase of a search.
// Part of the persistent engine (engine.cu), split by topic; included in order.
#pragma once

#include "engine_phases.cuh"

namespace abfs {

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
    // the search's phase counter: written only by the advancing CTA, visible
    // here since this CTA took a unit of the current phase
    const uint32_t epoch0 = threadIdx.x == 0 ? ld_relaxed(&ctl->epoch) : 0u;
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
            // at most two units per CTA: a third round for a few CTAs would
            // stretch the level by half
            const unsigned long long per2 = (unsigned long long)P.unit * 2ull * gridDim.x;
            unsigned long long m = (ne + per2 - 1) / per2;
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
                const uint32_t e = epoch0 + 1;
                const uint32_t q = e & 1;
                const unsigned long long d = ((unsigned long long)e << 32) | units;
                st_relaxed(&ctl->kind[q], nkind);
                st_relaxed(&ctl->plevel[q], nk);
                st_relaxed(&ctl->nitems[q], ni);
                st_relaxed(&ctl->pending[q], units);
                st_relaxed(&ctl->epoch, e);
                atomicAdd(&ctl->wide_levels, 1u);
                st_relaxed64(&ctl->desc[q], d);
                // the phase becomes takeable only after all of the above
                st_release64(&ctl->grab, (unsigned long long)e << 32);
                // this CTA knows the phase it published: its first take needs
                // neither a poll nor a second acquire
                sm.ran.valid = 1;
                sm.ran.fresh = 1;
                sm.ran.q = sm.cmd.q;
                sm.ran.epoch = e;
                sm.ran.kind = nkind;
                sm.ran.level = nk;
                sm.ran.nitems = ni;
                sm.ran.desc = d;
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

}  // namespace abfs
