// Cluster runs: small levels of one search run on the advancing CTA and the
// idle CTAs of its thread-block cluster, back to back, with the level barrier
// in distributed shared memory.
// Part of the persistent engine (engine.cu), split by topic; included in order.
//
// A resident narrow run (engine_levels.cuh) keeps long, thin searches off the
// grid-wide hand-off, but one CTA then issues all of a level's scattered
// accesses through one SM.  A cluster run spreads each level over the members
// of a cluster.  The frontier list stays in global memory in the narrow-run
// format (vertex, column begin, column length); member i expands the i-th of m
// equal slices of it and appends the vertices it claims at positions taken
// from a counter in the leader CTA's shared memory (DSMEM atomics).  At the
// end of a step every member releases its writes and sends one message -- the
// step, its appends and their entry slots, its error flag -- into its slot of
// every member's mailbox, then waits on its own mailbox for the others'.
// Every member takes the same decision (next step, or stop) from the same
// messages, so a level costs one DSMEM hop of synchronisation.  The semantics
// of a level are those of a narrow run -- frozen test bitmap, atomicMin claim,
// ping-pong bitmaps -- so results are unchanged.
//
// Joining.  A leader invites only peers that report themselves idle, takes
// the cluster's run lock (rank 0's mailbox), writes an invitation into each
// invited peer's mailbox and waits a few microseconds; a peer that finds an
// invitation between work units adds its bit to the leader's join word if the
// word still carries the invitation's sequence number and is not closed.  The
// leader then closes the word; the bits set at that moment are the members.
//
// Every wait is bounded: by the join window, or by timeout_ns without the
// awaited message (the search then fails with ABFS_ERR_TIMEOUT and every CTA
// returns).  DSMEM stays valid because every CTA of the cluster waits at a
// cluster barrier before it exits the kernel.
#pragma once

#include "engine_levels.cuh"

namespace abfs {

constexpr uint32_t kJoinClosed = 1u << 16;
constexpr uint32_t kJoinSeqShift = 17;
constexpr uint32_t kJoinSeqMask = 0x7FFFu;
// How long a leader waits for the invited CTAs: an idle CTA looks at its box
// every 128 ns while it sleeps, and between sleeps scans the searches for
// work (about a microsecond).
constexpr uint64_t kJoinWindowNs = 8000;
constexpr unsigned long long kMsgErr = 1ull << 63;

__device__ __forceinline__ void fence_cluster() { asm volatile("fence.acq_rel.cluster;" ::: "memory"); }

__device__ __forceinline__ void ds_st_relaxed(uint32_t a, uint32_t v) {
    asm volatile("st.relaxed.cluster.shared::cluster.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void ds_st_relaxed64(uint32_t a, unsigned long long v) {
    asm volatile("st.relaxed.cluster.shared::cluster.u64 [%0], %1;" ::"r"(a), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ds_cas64(uint32_t a, unsigned long long cmp,
                                                       unsigned long long v) {
    unsigned long long old;
    asm volatile("atom.relaxed.cluster.shared::cluster.cas.b64 %0, [%1], %2, %3;"
                 : "=l"(old) : "r"(a), "l"(cmp), "l"(v) : "memory");
    return old;
}

// Warp 0 of the advancing CTA: tries to start a cluster run of instance q at
// level k.  Returns the member bits (this CTA's included) to every lane, or 0
// when no run starts (no idle peer, another run holds the cluster, or no peer
// joined in time).
__device__ ABFS_NOINLINE uint32_t cluster_try_lead(Smem& sm, uint32_t q, uint32_t k) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t C = cluster_size(), me = cluster_rank();
    const uint32_t invited = cluster_idle_peers(sm);
    uint32_t result = 0;
    // a run with few members helps little and keeps busy CTAs waiting: at
    // least half of the other CTAs must be idle
    if (lane == 0 && 2u * __popc(invited) >= C - 1u && invited) {
        const uint32_t lock_a = ds_addr(&sm.cbox.lock, 0);
        if (ds_cas(lock_a, 0u, me + 1u) == 0u) {
            // run numbers are unique in the cluster (the leader's rank in the low
            // bits): messages of an earlier run, led by any CTA, never match
            const uint32_t seq = (((sm.cbox.seq >> 4) + 1u) << 4) | me;
            sm.cbox.seq = seq;
            sm.cbox.ctr[0] = 0;
            sm.cbox.ctr[1] = 0;
            sm.cbox.start = 0;
            sm.cbox.members = 0;
            sm.cbox.run_q = q;
            sm.cbox.run_k = k;
            const uint32_t ja = ds_addr(&sm.cbox.join, me);
            ds_st_relaxed(ja, ((seq & kJoinSeqMask) << kJoinSeqShift) | (1u << me));
            // the box is ready before any invitation can be seen
            fence_cluster();
            const unsigned long long inv = ((unsigned long long)seq << 32) | (me + 1u);
            for (uint32_t r = 0; r < C; ++r)
                if ((invited >> r) & 1u) ds_st_relaxed64(ds_addr(&sm.cbox.inv, r), inv);
            const uint32_t want = invited | (1u << me);
            const uint64_t t0 = globaltimer();
            while ((ds_ld_relaxed(ja) & 0xFFFFu) != want && globaltimer() - t0 < kJoinWindowNs) {
            }
            const uint32_t mem = ds_or(ja, kJoinClosed) & 0xFFFFu;
            if (__popc(mem) >= 2) {
                sm.cbox.members = mem;
                result = mem;
            } else {
                ds_st_release(lock_a, 0u);  // nobody came: the cluster is free again
            }
        }
    }
    return __shfl_sync(0xFFFFFFFFu, result, 0);
}

// Lane 0 of warp 0, between work units: takes an invitation found in this
// CTA's box and tries to join that run.  Returns 1 when joined (sm.cr_leader
// and sm.cr_seq then name the run).
__device__ __forceinline__ uint32_t cluster_take_invitation(Smem& sm) {
    // a plain read of this CTA's own box first: it is on every unit take
    const unsigned long long inv = *(volatile const unsigned long long*)&sm.cbox.inv;
    if (!inv) return 0;
    fence_cluster();  // acquire: the leader's box was ready before the invitation
    const uint32_t me = cluster_rank();
    ds_cas64(ds_addr(&sm.cbox.inv, me), inv, 0ull);  // a newer invitation stays
    const uint32_t L = (uint32_t)inv - 1u, seq = (uint32_t)(inv >> 32);
    if (L >= cluster_size() || L == me) return 0;
    const uint32_t ja = ds_addr(&sm.cbox.join, L);
    for (int tries = 0; tries < 64; ++tries) {
        const uint32_t j = ds_ld_relaxed(ja);
        if ((j >> kJoinSeqShift) != (seq & kJoinSeqMask) || (j & kJoinClosed)) return 0;
        if (ds_cas(ja, j, j | (1u << me)) == j) {
            sm.cr_leader = L;
            sm.cr_seq = seq;
            return 1;
        }
    }
    return 0;
}

// Sums of one step's messages over the members of a run.
struct StepSums {
    unsigned long long cnt;    // vertices (or comparator rows) appended
    unsigned long long slots;  // their entry slots
    bool err;                  // a member reported an error, or a message did not come
};

// Tag of the messages of step `step`.
__device__ __forceinline__ uint32_t msg_tag(uint32_t step) { return (step + 1u) & 0x7FFFu; }

// Warp 0 at the end of step `step` (after a CTA barrier): releases this CTA's
// writes, sends its message into its slot of every member's box (lane r
// writes to member r), and waits for every member's message in its own box
// (lane r waits for member r).  Messages alternate between two slots by step
// parity: a member can be at most one step ahead of any other.  The summed
// slots are counted in units of 256 (every member sums the same values).
__device__ __forceinline__ StepSums cluster_exchange(Smem& sm, InstCtl* ctl, const EngineParams& P,
                                                     uint32_t mem, uint32_t step,
                                                     unsigned long long cnt,
                                                     unsigned long long slots, bool err) {
    const uint32_t lane = threadIdx.x & 31, me = cluster_rank();
    const uint32_t par = step & 1u;
    const unsigned long long tag = (unsigned long long)msg_tag(step);
    const bool member = lane < (uint32_t)kClusterMax && ((mem >> lane) & 1u);
    // release this CTA's writes (made before the CTA barrier) to the members
    fence_cluster();
    if (member) {
        const unsigned long long s16 = (slots >> 8) > 0xFFFFull ? 0xFFFFull : (slots >> 8);
        const unsigned long long word = (tag << 49) | ((err ? 1ull : 0ull) << 48) | (s16 << 32) |
                                        (cnt > 0xFFFFFFFFull ? 0xFFFFFFFFull : cnt);
        ds_st_relaxed64(ds_addr(&sm.cbox.msg[par][me], lane), word);
    }
    // the warp polls in step (lane r: member r's slot) and fences once: a
    // fence inside diverged lanes would run once per lane, one after another.
    // Reading %globaltimer is slow: the clock starts only after 1024 polls.
    const volatile ClusterMsg* in = &sm.cbox.msg[par][lane & (kClusterMax - 1)];
    unsigned long long w = 0;
    bool bad = false;
    uint64_t t0 = 0;
    for (uint32_t spin = 0;; ++spin) {
        bool ok = true;
        if (member) {
            w = *in;
            ok = (w >> 49) == tag;
        }
        if (__all_sync(0xFFFFFFFFu, ok)) break;
        if ((spin & 1023u) == 1023u) {
            uint64_t now = lane == 0 ? globaltimer() : 0ull;
            now = __shfl_sync(0xFFFFFFFFu, now, 0);
            if (t0 == 0) {
                t0 = now;
            } else if (now - t0 > P.timeout_ns) {
                bad = !ok;
                if (lane == 0) fail(ctl, 5 /* ABFS_ERR_TIMEOUT */);
                break;
            }
        }
    }
    fence_cluster();  // acquire: the members' writes before their messages
    unsigned long long c = 0, s = 0;
    if (member && !bad) {
        bad = ((w >> 48) & 1ull) != 0;
        c = w & 0xFFFFFFFFull;
        s = ((w >> 32) & 0xFFFFull) << 8;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        c += __shfl_xor_sync(0xFFFFFFFFu, c, d);
        s += __shfl_xor_sync(0xFFFFFFFFu, s, d);
    }
    StepSums r;
    r.cnt = c;
    r.slots = s;
    r.err = __any_sync(0xFFFFFFFFu, bad) != 0;
    return r;
}

// Every member, as its run ends: clears the message slots of its own box, so
// no message of this run can be taken for one of a later run.  Whole CTA.
__device__ __forceinline__ void cluster_clear_box(Smem& sm) {
    unsigned long long* w = reinterpret_cast<unsigned long long*>(&sm.cbox.msg[0][0]);
    for (uint32_t i = threadIdx.x; i < sizeof(sm.cbox.msg) / 8; i += kThreads)
        *(volatile unsigned long long*)&w[i] = 0ull;
}

// The steps of a cluster run, for every member (leader included).  The first
// step expands level k from the list at fq[k & 1] (sm.cr_f vertices, ids
// only; later levels carry column begins and lengths).  Submatrix mode: one
// step per level.  Comparator: an expand step (multiply into the accumulator,
// append touched rows) and a mask step (claim the touched rows not yet
// reached) per level.  Returns the last level run; sm.cr_f then holds the
// size of the list that follows it, sm.nr_reached the vertices reached.
// Whole CTA.
template <int MODE>
__device__ ABFS_NOINLINE uint32_t cluster_loop(const Inst& I, InstCtl* ctl, const EngineParams& P,
                                               Smem& sm, uint32_t k, bool leader,
                                               unsigned long long* heartbeat) {
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t L = sm.cr_leader, me = cluster_rank();
    const uint32_t mem = sm.cr_join;
    const uint32_t m = __popc(mem), mi = __popc(mem & ((1u << me) - 1u));
    const uint32_t sw = sm.nr_sw, mcur = sm.nr_mcur, mprev = sm.nr_mprev;
    const uint32_t ctr_a0 = ds_addr(&sm.cbox.ctr[0], L), ctr_a1 = ds_addr(&sm.cbox.ctr[1], L);
    uint32_t f = sm.cr_f;
    bool lens = false;
    uint32_t guard = I.n + 1;
    Tally t;
    uint32_t nnz_local = 0;
    for (uint32_t step = 0;; ++step) {
        const bool mask_step = MODE == kModePlain && (step & 1u);
        const long long pt0 = prof_now(sm);
        uint32_t err0 = 0;
        if (threadIdx.x == 0) {
            // the counter of step - 1 is free again; step + 1 uses it
            if (leader && step > 0) sm.cbox.ctr[(step + 1) & 1] = 0;
            sm.ds_ctr = (step & 1) ? ctr_a1 : ctr_a0;
            sm.nq_cnt = 0;
            sm.nt_cnt = 0;
            sm.nq_slots = 0;
            // the search's error word and the launch's heartbeat share lines that
            // every idle CTA polls: touched every few steps only, at the start of
            // a step, so their latency hides behind the expansion (the heartbeat
            // only has to move well within timeout_ns)
            if ((step & 15u) == 0) err0 = ld_relaxed(&ctl->err);
            if (leader && (step & 31u) == 31u) atomicAdd(heartbeat, 32ull);
        }
        __syncthreads();
        const uint32_t mat = k >= sw ? mcur : mprev;
        const uint32_t mat_next = k + 1 >= sw ? mcur : mprev;
        const uint32_t pn = (k + 1) & 1;
        // this member's slice of the list (or of the touched rows)
        const uint32_t lo = (uint32_t)((unsigned long long)f * mi / m);
        const uint32_t hi = (uint32_t)((unsigned long long)f * (mi + 1) / m);
        if (!mask_step) {
            if (!narrow_expand_short<MODE>(I, ctl, P, sm, k, lo, hi - lo, lens, mat, mat_next, t,
                                           nnz_local))
                narrow_expand<MODE>(I, ctl, P, sm, k, lo, hi - lo, lens, mat, mat_next, t,
                                    nnz_local);
            uint32_t wc = sm.wcnt[warp];
            if (wc) {
                if (MODE == kModeSub) narrow_append(sm, I, ctl, pn, mat_next, wc);
                else narrow_touch(sm, I, ctl, wc);
            }
            if (lane == 0) sm.wcnt[warp] = 0;
        } else {
            // comparator mask: touched rows not yet reached join level k+1 with
            // the least column of the accumulator (each row is touched once)
            uint32_t wc = 0;
            for (uint32_t b0 = lo; b0 < hi; b0 += kThreads) {
                const uint32_t i = b0 + threadIdx.x;
                bool want = false;
                uint32_t r = 0;
                if (i < hi) {
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
        }
        __syncthreads();
        const long long pt1 = prof_now(sm);
        prof_add(sm, kProfNExpand, pt0);
        if (warp == 0) {
            const unsigned long long cnt =
                (MODE == kModePlain && !mask_step) ? sm.nt_cnt : sm.nq_cnt;
            const bool e0 = __shfl_sync(0xFFFFFFFFu, err0, 0) != 0;
            const StepSums sums = cluster_exchange(sm, ctl, P, mem, step, cnt, sm.nq_slots, e0);
            if (lane == 0) {
                const unsigned long long tot = sums.cnt;
                uint32_t stop;
                if (MODE == kModePlain && !mask_step) {
                    stop = sums.err;  // the mask step of this level follows
                } else {
                    stop = sums.err || tot == 0 || tot > P.cluster_max ||
                           sums.slots > P.cluster_edges || guard <= 1;
                    if (!stop && MODE == kModeSub &&
                        shrink_due(P, sm.nr_reached + (uint32_t)tot, I.n, sm.nr_shrinks))
                        stop = 1;
                    if (!stop) {
                        sm.nr_reached += (uint32_t)tot;
                        if (leader) {
                            if (I.trace)
                                trace_put(I, ctl, MODE == kModePlain ? kPhPlainMult : kPhLevel,
                                          k + 1, 3u, m, (uint32_t)tot, sums.slots);
                            if (sm.prof_on) sm.prof[kProfNLevels] += 1;
                        }
                    }
                    --guard;
                }
                sm.cr_stop = stop;
                sm.cr_f = (uint32_t)tot;
            }
        }
        __syncthreads();
        prof_add(sm, kProfNDecide, pt1);
        f = sm.cr_f;
        if (!(MODE == kModePlain && !mask_step)) {
            ++k;
            lens = true;
        }
        if (sm.cr_stop) break;
    }
    // the run's counters reach the search
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) nnz_local += __shfl_xor_sync(0xFFFFFFFFu, nnz_local, d);
    if (lane == 0 && nnz_local) atomicAdd(&sm.st_nnz, (unsigned long long)nnz_local);
    tally_flush(sm, t);
    stats_flush(sm, ctl);
    cluster_clear_box(sm);
    if (threadIdx.x == 0) sm.ds_ctr = 0;
    __syncthreads();
    return k - 1;
}

// The advancing CTA leads a run that starts at level k (members already
// joined: sm.cr_join).  Returns the last level run; its successor frontier is
// left in block form with the search's counters set as the general path
// expects (as narrow_run does).  Whole CTA.
template <int MODE>
__device__ ABFS_NOINLINE uint32_t cluster_lead_run(const Inst& I, InstCtl* ctl,
                                                   const EngineParams& P, Smem& sm, uint32_t k,
                                                   unsigned long long* heartbeat) {
    const uint32_t me = cluster_rank();
    if (threadIdx.x == 0) {
        const uint32_t f = ld_relaxed(&ctl->fcnt[k & 1]);
        sm.nr_reached = ld_relaxed(&ctl->reached);
        sm.nr_shrinks = ld_relaxed(&ctl->shrinks);
        sm.nr_sw = ld_relaxed(&ctl->mat_switch);
        sm.nr_mcur = ld_relaxed(&ctl->mat_cur);
        sm.nr_mprev = ld_relaxed(&ctl->mat_prev);
        sm.cbox.run_f = f;
        sm.cbox.run_reached = sm.nr_reached;
        sm.cbox.run_shrinks = sm.nr_shrinks;
        sm.cbox.run_sw = sm.nr_sw;
        sm.cbox.run_mcur = sm.nr_mcur;
        sm.cbox.run_mprev = sm.nr_mprev;
        sm.cr_leader = me;
        sm.cr_seq = sm.cbox.seq;
        sm.cr_f = f;
        // the members read the run's fields once they see the start word
        ds_st_release64(ds_addr(&sm.cbox.start, me), ((unsigned long long)sm.cr_seq << 32) | 1ull);
    }
    __syncthreads();
    const uint32_t last = cluster_loop<MODE>(I, ctl, P, sm, k, true, heartbeat);
    narrow_to_blocks(I, ctl, P, sm, last + 1, last + 1 >= sm.nr_sw ? sm.nr_mcur : sm.nr_mprev, sm.cr_f);
    if (threadIdx.x == 0) {
        st_relaxed(&ctl->reached, sm.nr_reached);
        ds_st_release(ds_addr(&sm.cbox.lock, 0), 0u);  // the cluster is free for the next run
    }
    __syncthreads();
    return last;
}

// A CTA that joined a run (sm.cr_leader, sm.cr_seq) takes part in it to the
// end.  Whole CTA.
template <int MODE>
__device__ ABFS_NOINLINE void cluster_member_run(const EngineArgs& a, Smem& sm) {
    const uint32_t L = sm.cr_leader;
    if (threadIdx.x == 0) {
        const uint32_t sa = ds_addr(&sm.cbox.start, L);
        const unsigned long long want = ((unsigned long long)sm.cr_seq << 32) | 1ull;
        const uint64_t t0 = globaltimer();
        uint32_t ok = 0;
        for (;;) {
            if (ds_ld_acquire64(sa) == want) {
                ok = 1;
                break;
            }
            if (globaltimer() - t0 > a.p.timeout_ns) break;
        }
        sm.cur_q = kUnset;
        sm.ran.valid = 0;
        sm.cmd.q = kUnset;
        if (ok) {
            sm.cr_join = ds_ld_relaxed(ds_addr(&sm.cbox.members, L));
            sm.cmd.q = ds_ld_relaxed(ds_addr(&sm.cbox.run_q, L));
            sm.cmd.level = ds_ld_relaxed(ds_addr(&sm.cbox.run_k, L));
            sm.cr_f = ds_ld_relaxed(ds_addr(&sm.cbox.run_f, L));
            sm.nr_reached = ds_ld_relaxed(ds_addr(&sm.cbox.run_reached, L));
            sm.nr_shrinks = ds_ld_relaxed(ds_addr(&sm.cbox.run_shrinks, L));
            sm.nr_sw = ds_ld_relaxed(ds_addr(&sm.cbox.run_sw, L));
            sm.nr_mcur = ds_ld_relaxed(ds_addr(&sm.cbox.run_mcur, L));
            sm.nr_mprev = ds_ld_relaxed(ds_addr(&sm.cbox.run_mprev, L));
        }
    }
    __syncthreads();
    const uint32_t q = sm.cmd.q;
    if (q >= a.ninst) return;  // the run never started (cannot happen once joined)
    if (threadIdx.x < 32) {
        const uint32_t* src = reinterpret_cast<const uint32_t*>(a.insts + q);
        uint32_t* dst = reinterpret_cast<uint32_t*>(&sm.I);
        for (uint32_t w = threadIdx.x; w < sizeof(Inst) / 4; w += 32) dst[w] = src[w];
        if (threadIdx.x == 0) sm.cur_q = q;
    }
    __syncthreads();
    cluster_loop<MODE>(sm.I, sm.I.ctl, a.p, sm, sm.cmd.level, false, a.heartbeat);
}

}  // namespace abfs
