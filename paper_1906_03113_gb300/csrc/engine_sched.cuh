// Work distribution of the persistent launch: finding, taking and running
// units of any search, bounded idle waits, and the engine kernel itself.
// Part of the persistent engine (engine.cu), split by topic; included in order.
#pragma once

#include "engine_advance.cuh"

namespace abfs {

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
        sm.ran.valid = 0;
        return true;
    }
    InstCtl* ctl = ctl_of(a, q);
    const unsigned long long old = atomicAdd(&ctl->grab, 1ull);
    const uint32_t e = (uint32_t)(old >> 32), t = (uint32_t)old;
    // the descriptor of epoch e is written before grab moves to e
    const unsigned long long d =
        (e == e_seen && (uint32_t)(d_seen >> 32) == e) ? d_seen : ld_relaxed64(&ctl->desc[e & 1]);
    if ((uint32_t)(d >> 32) != e || t >= (uint32_t)d) return false;
    sm.cmd.q = q;
    sm.cmd.start = 0;
    sm.cmd.epoch = e;
    sm.cmd.unit = t;
    if (sm.ran.valid && sm.ran.q == q && sm.ran.epoch == e) {
        // a further unit of the phase this CTA took a unit of before: that
        // take's acquire and the phase's fields still hold
        sm.cmd.kind = sm.ran.kind;
        sm.cmd.level = sm.ran.level;
        sm.cmd.nitems = sm.ran.nitems;
        return true;
    }
    __threadfence();  // acquire: the phase fields and the data of earlier phases
    const uint32_t qq = e & 1;
    sm.cmd.kind = ld_relaxed(&ctl->kind[qq]);
    sm.cmd.level = ld_relaxed(&ctl->plevel[qq]);
    sm.cmd.nitems = ld_relaxed(&ctl->nitems[qq]);
    sm.ran.valid = 1;
    sm.ran.q = q;
    sm.ran.epoch = e;
    sm.ran.kind = sm.cmd.kind;
    sm.ran.level = sm.cmd.level;
    sm.ran.nitems = sm.cmd.nitems;
    sm.ran.desc = d;
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
        // an invitation to a cluster run comes before any unit
        uint32_t joined = 0;
        if (a.p.cluster > 1 && lane == 0) joined = cluster_take_invitation(sm);
        joined = __shfl_sync(0xFFFFFFFFu, joined, 0);
        if (joined) {
            if (lane == 0) sm.cmd.has = 2;
            __syncwarp();
        } else if (sm.ran.valid && sm.ran.fresh) {
            // right after a unit that did not end its phase, first try that
            // phase again without polling (an idle CTA polls instead)
            bool ok = false;
            if (lane == 0) {
                ok = take_unit(a, sm.ran.q, sm, sm.ran.epoch, sm.ran.desc);
                sm.ran.fresh = 0;
            }
            got = __shfl_sync(0xFFFFFFFFu, ok, 0);
        }
        for (uint32_t base = 0; base < a.ninst && !got && !joined; base += 32) {
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
        if (lane == 0 && !joined) sm.cmd.has = got;
        // busy from now on: leaders of cluster runs do not wait for this CTA
        if (lane == 0 && (got || joined) && a.p.cluster > 1) *(volatile uint32_t*)&sm.cbox.idle = 0u;
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
    if (sm.cmd.has == 2) {
        cluster_member_run<MODE>(a, sm);
        return true;
    }
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
        sm.ran.fresh = left != 1;
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
        sm.ran.valid = 0;
        sm.ran.fresh = 0;
        sm.ds_ctr = 0;
        sm.cr_join = 0;
        uint32_t* cb = reinterpret_cast<uint32_t*>(&sm.cbox);
        for (uint32_t w = 0; w < sizeof(ClusterBox) / 4; ++w) cb[w] = 0u;
    }
    __syncthreads();
    // peers reach this CTA's box only after every CTA of the cluster has
    // cleared its own
    const bool clustered = cluster_size() > 1;
    if (clustered) cluster_barrier_all();
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
            if (clustered && threadIdx.x == 0) *(volatile uint32_t*)&sm.cbox.idle = 0u;
            backoff = 64;
            continue;
        }
        // leaders of cluster runs invite CTAs that find no work
        if (clustered && threadIdx.x == 0) *(volatile uint32_t*)&sm.cbox.idle = 1u;
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
            if (clustered) {
                // short naps that end as soon as a cluster run invites this CTA
                for (uint32_t slept = 0; slept < backoff; slept += 128) {
                    if (*(volatile const unsigned long long*)&sm.cbox.inv) break;
                    __nanosleep(128);
                }
            } else {
                __nanosleep(backoff);
            }
            if (backoff < kIdleBackoffMaxNs) backoff <<= 1;
        }
        __syncthreads();
        prof_add(sm, kProfIdle, pti);
    }
    if (a.prof && threadIdx.x == 0)
        for (int q = 0; q < kProfSlots; ++q) atomicAdd(a.prof + q, sm.prof[q]);
    // no CTA leaves while a peer may still reach its shared memory
    if (clustered) {
        if (threadIdx.x == 0) *(volatile uint32_t*)&sm.cbox.idle = 0u;
        cluster_barrier_all();
    }
}

}  // namespace abfs
