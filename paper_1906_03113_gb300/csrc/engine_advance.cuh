// Choosing and publishing the next phase of a search; the advancing CTA runs
// small follow-up levels itself (resident narrow runs) or with the idle CTAs
// of its thread-block cluster (cluster runs).
// Part of the persistent engine (engine.cu), split by topic; included in order.
#pragma once

#include "engine_cluster.cuh"

namespace abfs {

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
        const uint32_t len = ld_ro(I.colptr + s + 1) - b0;
        const uint32_t w = col_slots(I, 0, b0, len);
        I.fq[0][0] = s;
        I.fbeg[0][0] = b0;
        I.fpre[0][0] = 0;
        I.flen[0][0] = len;
        I.blk[0][0].vb = 0;
        I.blk[0][0].nv = 1;
        I.blk[0][0].eb = 0;
        for (unsigned long long x = 0; x < w; x += P.unit) I.ustart[0][x / P.unit] = make_uint2(0, 0);
        st_relaxed64(&ctl->bctr[0], ((unsigned long long)w << kBlockBits) | 1ull);
        st_relaxed64(&ctl->fent[0], (unsigned long long)len);
        st_relaxed(&ctl->fcnt[0], 1u);
        st_relaxed(&ctl->reached, 1u);
        nkind = (MODE == kModePlain) ? kPhPlainMult : kPhLevel;
        nk = 0;
    } else if (kind == kPhStart) {
        // the frontier of level 0 (the source) was set up before the launch
        nkind = (MODE == kModePlain) ? kPhPlainMult : (I.ms ? kPhMsLevel : kPhLevel);
        nk = 0;
    } else if (kind == kPhMsLevel) {
        // the new bits of a multi-source level become levels, parents, frontier
        nkind = kPhMsUpdate;
        nk = k;
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
                st_relaxed64(&ctl->fent[pc], 0ull);
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
            const bool do_shrink = MODE == kModeSub && !I.ms && kind != kPhShrink &&
                                   shrink_due(P, reached, I.n, shrinks);
            if (do_shrink) {
                // alternate copies so the frontier of level k+1 keeps its matrix
                const uint32_t cur = ld_relaxed(&ctl->mat_cur);
                nkind = kPhShrink;
                nk = k;
                ni = (cur == 1) ? 2u : 1u;
                st_relaxed(&ctl->shrink_out, 0u);
            } else {
                nkind = (MODE == kModePlain) ? kPhPlainMult : (I.ms ? kPhMsLevel : kPhLevel);
                nk = k + 1;
                if (MODE == kModeSub && P.bu_alpha && I.bu_ok && kind != kPhShrink) {
                    // hybrid direction choice from the frontier's edges m_f and the
                    // edges of vertices not reached yet m_u: bottom-up once
                    // m_f * alpha > m_u, back to top-down once n_f * beta < n
                    const unsigned long long mf = ld_relaxed64(&ctl->fent[pn]);
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
        } else if (nkind == kPhExtract || nkind == kPhBuPrep || nkind == kPhBottomUp ||
                   nkind == kPhMsUpdate) {
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
        // a small level runs on this CTA and the idle CTAs of its cluster
        if (P.cluster > 1 && P.narrow_loop && (nkind == kPhLevel || nkind == kPhPlainMult) &&
            (nk == 0 || ne >= P.cluster_min || !alone) && nf <= P.cluster_max &&
            ne <= P.cluster_edges) {
            if (threadIdx.x < 32) {
                const uint32_t mem = cluster_try_lead(sm, sm.cmd.q, nk);
                if (threadIdx.x == 0) sm.cr_join = mem;
            }
            __syncthreads();
            if (sm.cr_join) {
                k = cluster_lead_run<MODE>(I, ctl, P, sm, nk, heartbeat);
                kind = kPhLevel;
                __threadfence();
                __syncthreads();
                continue;
            }
        }
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
