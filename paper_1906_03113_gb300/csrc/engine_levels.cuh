// Phase control: running a unit, and resident narrow runs of small levels on
// one CTA.
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
    } else if (MODE == kModeSub && kind == kPhMsLevel) {
        unit_level<MODE, kVarMs>(I, ctl, P, sm, k, unit, nitems);
    } else if (MODE == kModeSub && kind == kPhMsUpdate) {
        unit_ms_update(I, ctl, P, sm, k, unit, nitems);
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
// wide levels.  The frontier of level k is a plain list at fq/fbeg/flen[k&1]:
// vertex, column begin and column length.  Claims gather in the warp staging
// buffers and are appended with a shared-memory counter; the reached count
// and the level stay in shared memory until the run ends.  The run ends when
// the frontier empties, outgrows the narrow bounds, or a shrink is due; the
// last frontier is then rewritten as blocks and the general path decides what
// follows.  (fpre is unused until the blocks are written.)

// Expands the f vertices at [base, base + f) of the level-k list (lens:
// fbeg/flen hold column begins and lengths in matrix mat; otherwise only the
// ids are valid and the columns are looked up) in chunks of up to `tile`
// vertices and windows of up to kUnitMax slots.  Whole CTA.
template <int MODE>
__device__ __forceinline__ void narrow_expand(const Inst& I, InstCtl* ctl, const EngineParams& P, Smem& sm,
                              uint32_t k, uint32_t base, uint32_t f, bool lens, uint32_t mat,
                              uint32_t mat_next, Tally& t, uint32_t& nnz_local) {
    const uint32_t p = k & 1;
    for (uint32_t c0 = 0; c0 < f; c0 += P.tile) {
        const long long pt0 = prof_now(sm);
        const uint32_t cnt = min(P.tile, f - c0);
        for (uint32_t s = threadIdx.x; s < cnt; s += kThreads) {
            const uint32_t at = base + c0 + s;
            const uint32_t v = ld_l2(I.fq[p] + at);
            uint32_t beg, len;
            if (lens) {
                beg = ld_l2(I.fbeg[p] + at);
                len = ld_l2(I.flen[p] + at);
            } else {
                const ColRef c = col_of(I, mat, v);
                beg = c.beg;
                len = c.len;
            }
            sm.v[s] = I.lab ? ld_ro(I.lab + v) : v;  // the column index of its products
            sm.b[s] = beg;
            sm.end[s] = len;
            sm.off[s] = col_slots(I, mat, beg, len);
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
            set_slot_map(sm, I, mat, s, st);
            if (st < l1) {
                const uint32_t c = st / kChunk;
                atomicOr(&sm.sbits[c >> 5], 1u << (c & 31));
            }
            mark_warp_starts(sm, s, st / kChunk, en / kChunk, l0 / kChunk, l1 / kChunk);
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
                if (st >= l0 && st < l1) {
                    const uint32_t c = (st - l0) / kChunk;
                    atomicOr(&sm.sbits[c >> 5], 1u << (c & 31));
                }
                mark_warp_starts(sm, s, st / kChunk, sm.off[s + 1] / kChunk, l0 / kChunk, l1 / kChunk);
            }
            __syncthreads();
        }
    }
}

// Short columns: a list slice of at most kThreads vertices whose columns all
// hold at most kShortCol entries is expanded one vertex per thread, with all
// of a vertex's row loads, mask tests and claims in flight together and no CTA
// barrier inside; the column of a row that passes the mask is looked up while
// its claim is in flight, so a claimed vertex is appended without a further
// round trip.  Submatrix mode appends the vertices of level k+1 to the next
// list; the comparator multiplies every entry into the stamped accumulator and
// appends first-touched rows to the touched list.  Returns false, having
// changed nothing, when the slice does not qualify (the caller then uses
// narrow_expand).  Whole CTA.
constexpr uint32_t kShortCol = 4;

template <int MODE>
__device__ ABFS_NOINLINE bool narrow_expand_short(const Inst& I, InstCtl* ctl, const EngineParams& P,
                                                  Smem& sm, uint32_t k, uint32_t base, uint32_t f,
                                                  bool lens, uint32_t mat, uint32_t mat_next,
                                                  Tally& t, uint32_t& nnz_local) {
    if (f > (uint32_t)kThreads) return false;
    const uint32_t p = k & 1, pn = p ^ 1;
    const uint32_t tid = threadIdx.x, lane = tid & 31;
    const bool have = tid < f;
    uint32_t v = 0, vo = 0, beg = 0, len = 0;  // vo: the claims' column index (v's input label)
    if (have) {
        const uint32_t at = base + tid;
        v = ld_l2(I.fq[p] + at);
        if (lens) {
            beg = ld_l2(I.fbeg[p] + at);
            len = ld_l2(I.flen[p] + at);
        } else {
            const ColRef c = col_of(I, mat, v);
            beg = c.beg;
            len = c.len;
        }
    }
    if (__syncthreads_or(have && len > kShortCol)) return false;
    const uint32_t* rows = rows_of(I, mat);
    const uint64_t pol = evict_first_policy();
    uint32_t r[kShortCol];
#pragma unroll
    for (uint32_t j = 0; j < kShortCol; ++j)
        r[j] = (have && j < len) ? ld_row(rows, beg + j, mat, pol) : kUnset;
    if (have) {
        vo = I.lab ? ld_ro(I.lab + v) : v;  // issued beside the row loads
        // the frontier joins the visited set of the next level's test
        if (MODE == kModeSub) atomicOr(I.bm[pn] + (v >> 5), 1u << (v & 31));
        nnz_local += (mat == 0) ? len : (ld_ro(I.colptr + v + 1) - ld_ro(I.colptr + v));
        t.read += len;
    }
    uint32_t won = 0;  // bit j: entry j claimed (submatrix) / first touch (comparator)
    uint32_t nb[kShortCol], nl[kShortCol];
    if (MODE == kModeSub) {
        const uint32_t* test_bm = I.bm[p];
        unsigned long long* const sigma = I.sigma;
        const unsigned long long sv = (sigma && have) ? ld_l2(sigma + v) : 0ull;
        uint32_t w[kShortCol];
#pragma unroll
        for (uint32_t j = 0; j < kShortCol; ++j)
            w[j] = r[j] != kUnset ? ld_l2(test_bm + (r[j] >> 5)) : 0xFFFFFFFFu;
        uint32_t old[kShortCol];
#pragma unroll
        for (uint32_t j = 0; j < kShortCol; ++j) {
            old[j] = 0;
            nb[j] = 0;
            nl[j] = 0;
            if (!((w[j] >> (r[j] & 31)) & 1u)) {
                ++t.unmasked;
                ++t.claims;
                old[j] = atomicMin(I.parent + r[j], vo);
                const ColRef c = col_of(I, mat_next, r[j]);
                nb[j] = c.beg;
                nl[j] = c.len;
                if (sigma) atomicAdd(sigma + r[j], sv);
            }
        }
#pragma unroll
        for (uint32_t j = 0; j < kShortCol; ++j) {
            if (!((w[j] >> (r[j] & 31)) & 1u) && old[j] == kUnset) {
                won |= 1u << j;
                I.level[r[j]] = (int32_t)(k + 1);
                atomicOr(I.bm[pn] + (r[j] >> 5), 1u << (r[j] & 31));
            }
        }
    } else {
#pragma unroll
        for (uint32_t j = 0; j < kShortCol; ++j) {
            nb[j] = 0;
            nl[j] = 0;
            if (r[j] != kUnset) {
                ++t.unmasked;
                ++t.claims;
                const unsigned long long o = atomicMin(I.y + r[j], plain_key(k, v));
                if ((uint32_t)(o >> 32) != plain_stamp(k)) won |= 1u << j;
            }
        }
    }
    // positions: each warp reserves its entries in this CTA's counter; in a
    // cluster run the CTA then reserves its total in the leader's counter with
    // one DSMEM atomic (not one per warp: they would queue at one address)
    const uint32_t cnt = __popc(won);
    const uint32_t incl = warp_incl_scan(cnt);
    const uint32_t wtot = __shfl_sync(0xFFFFFFFFu, incl, 31);
    uint32_t woff = 0;
    if (lane == 31 && wtot) woff = atomicAdd(MODE == kModeSub ? &sm.nq_cnt : &sm.nt_cnt, wtot);
    woff = __shfl_sync(0xFFFFFFFFu, woff, 31);
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t tot = MODE == kModeSub ? sm.nq_cnt : sm.nt_cnt;
        sm.cr_base = (sm.ds_ctr && tot) ? ds_add(sm.ds_ctr, tot) : 0u;
    }
    __syncthreads();
    if (wtot) {
        uint32_t at = sm.cr_base + woff + incl - cnt;
        uint32_t slots = 0;
#pragma unroll
        for (uint32_t j = 0; j < kShortCol; ++j) {
            if ((won >> j) & 1u) {
                if (at < I.n) {
                    if (MODE == kModeSub) {
                        I.fq[pn][at] = r[j];
                        I.fbeg[pn][at] = nb[j];
                        I.flen[pn][at] = nl[j];
                        slots += col_slots(I, mat_next, nb[j], nl[j]);
                        // the next level reads this column: start bringing it to L2
                        if (nl[j]) {
                            const uint32_t* c = rows_of(I, mat_next) + nb[j];
                            asm volatile("prefetch.global.L2 [%0];" ::"l"(c));
                            asm volatile("prefetch.global.L2 [%0];" ::"l"(c + nl[j] - 1));
                        }
                    } else {
                        I.touched[at] = r[j];
                    }
                } else {
                    fail(ctl, 7 /* ABFS_ERR_DEVICE */);
                }
                ++at;
            }
        }
        if (MODE == kModeSub) {
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) slots += __shfl_xor_sync(0xFFFFFFFFu, slots, d);
            if (lane == 0 && slots) atomicAdd(&sm.nq_slots, (unsigned long long)slots);
        }
    }
    __syncthreads();
    return true;
}

// Rewrites the list of level kl (fn vertices; columns in matrix mat) as
// frontier blocks of up to kWarps*kWarpBuf vertices: slot offsets within the
// block, unit starts, and the parity's counters.  The warp staging buffers
// (empty here) stage each chunk so global reads and writes stay coalesced.
// Whole CTA.
__device__ ABFS_NOINLINE void narrow_to_blocks(const Inst& I, InstCtl* ctl, const EngineParams& P,
                                               Smem& sm, uint32_t kl, uint32_t mat, uint32_t fn) {
    const uint32_t pn = kl & 1;
    // the hybrid's direction choice needs the list's exact entries
    if (P.bu_alpha) {
        if (threadIdx.x == 0) st_relaxed64(&ctl->fent[pn], 0ull);
        __syncthreads();
    }
    uint32_t ent = 0;
    constexpr uint32_t kListChunk = kWarps * kWarpBuf;
    constexpr uint32_t kItems = kListChunk / kThreads;
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t* buf = &sm.wv[0][0];
    unsigned long long eb = 0;
    uint32_t nb = 0;
    for (uint32_t c0 = 0; c0 < fn; c0 += kListChunk, ++nb) {
        const uint32_t cnt = min(kListChunk, fn - c0);
        for (uint32_t i = tid; i < cnt; i += kThreads) {
            const uint32_t len = ld_l2(I.flen[pn] + c0 + i);
            buf[i] = col_slots(I, mat, ld_l2(I.fbeg[pn] + c0 + i), len);
            ent += len;
        }
        __syncthreads();
        uint32_t x[kItems];
        uint32_t sum = 0;
#pragma unroll
        for (uint32_t q = 0; q < kItems; ++q) {
            const uint32_t idx = tid * kItems + q;
            x[q] = idx < cnt ? buf[idx] : 0u;
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
    if (P.bu_alpha) {
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) ent += __shfl_xor_sync(0xFFFFFFFFu, ent, d);
        if (lane == 0 && ent) atomicAdd(&ctl->fent[pn], (unsigned long long)ent);
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
        if (!narrow_expand_short<MODE>(I, ctl, P, sm, k, 0u, f, lens, mat, mat_next, t, nnz_local))
            narrow_expand<MODE>(I, ctl, P, sm, k, 0u, f, lens, mat, mat_next, t, nnz_local);
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
        if (P.cluster > 1 && threadIdx.x < 32) {
            // a level big enough for a cluster run ends this run when idle CTAs
            // of the cluster could take it together
            const unsigned long long sl = sm.nq_slots;
            const uint32_t fn = sm.nq_cnt;
            uint32_t idle = 0;
            if (sl >= P.cluster_min && sl <= P.cluster_edges && fn <= P.cluster_max)
                idle = cluster_idle_peers(sm);
            // as for starting a run: at least half of the other CTAs idle
            if (threadIdx.x == 0) sm.cr_idle = 2u * __popc(idle) >= cluster_size() - 1u ? idle : 0u;
        }
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
            else if (P.cluster > 1 && sm.cr_idle)
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
    narrow_to_blocks(I, ctl, P, sm, k + 1, k + 1 >= sw ? mat_cur : mat_prev, sm.nr_f);
    if (threadIdx.x == 0) st_relaxed(&ctl->reached, sm.nr_reached);
    stats_flush(sm, ctl);
    prof_add(sm, kProfNBlocks, pt4);
    return k;
}

}  // namespace abfs
