// Engine building blocks: build options, memory-ordering helpers, the CTA's
// shared state, scans and column lookups.
// Part of the persistent engine (engine.cu), split by topic; included in order.
#pragma once

#include "internal.h"

namespace abfs {

// Longest sleep of an idle CTA between polls for work.
#ifndef ABFS_IDLE_BACKOFF_NS
#define ABFS_IDLE_BACKOFF_NS 2048
#endif
constexpr uint32_t kIdleBackoffMaxNs = ABFS_IDLE_BACKOFF_NS;

// The phases and the expand loop are separate functions: each gets its own
// register allocation, so the cold paths' state does not push the hot loop
// into spills.  -DABFS_INLINE_ALL inlines them instead.
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
// Store that orders every earlier write of the thread before it (release).
__device__ __forceinline__ void st_release64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
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

// ---------------------------------------------------------------------------
// thread-block cluster: distributed shared memory (DSMEM)
// ---------------------------------------------------------------------------
// Addresses below are shared::cluster addresses: mapa turns this CTA's
// shared-memory address of a variable into the address of the same variable
// in the CTA of rank `rank` of the cluster.  Every launch is a cluster launch
// (a plain launch is a cluster of one CTA), so these are valid with rank 0 in
// a launch without clusters.

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_size() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t ds_addr(const void* p, uint32_t rank) {
    const uint32_t la = (uint32_t)__cvta_generic_to_shared(p);
    uint32_t ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(la), "r"(rank));
    return ra;
}
__device__ __forceinline__ uint32_t ds_ld_acquire(uint32_t a) {
    uint32_t v;
    asm volatile("ld.acquire.cluster.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ds_ld_acquire64(uint32_t a) {
    unsigned long long v;
    asm volatile("ld.acquire.cluster.shared::cluster.u64 %0, [%1];" : "=l"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t ds_ld_relaxed(uint32_t a) {
    uint32_t v;
    asm volatile("ld.relaxed.cluster.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ void ds_st_release(uint32_t a, uint32_t v) {
    asm volatile("st.release.cluster.shared::cluster.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void ds_st_release64(uint32_t a, unsigned long long v) {
    asm volatile("st.release.cluster.shared::cluster.u64 [%0], %1;" ::"r"(a), "l"(v) : "memory");
}
__device__ __forceinline__ uint32_t ds_add(uint32_t a, uint32_t v) {
    uint32_t old;
    asm volatile("atom.relaxed.cluster.shared::cluster.add.u32 %0, [%1], %2;"
                 : "=r"(old) : "r"(a), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ void ds_add64(uint32_t a, unsigned long long v) {
    asm volatile("red.relaxed.cluster.shared::cluster.add.u64 [%0], %1;" ::"r"(a), "l"(v) : "memory");
}
__device__ __forceinline__ void ds_add_release(uint32_t a, uint32_t v) {
    asm volatile("red.release.cluster.shared::cluster.add.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ds_cas(uint32_t a, uint32_t cmp, uint32_t v) {
    uint32_t old;
    asm volatile("atom.relaxed.cluster.shared::cluster.cas.b32 %0, [%1], %2, %3;"
                 : "=r"(old) : "r"(a), "r"(cmp), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ uint32_t ds_or(uint32_t a, uint32_t v) {
    uint32_t old;
    asm volatile("atom.relaxed.cluster.shared::cluster.or.b32 %0, [%1], %2;"
                 : "=r"(old) : "r"(a), "r"(v) : "memory");
    return old;
}
// Every thread of every CTA of the cluster (hardware barrier).  Used only at
// the start and the end of the kernel, which every CTA reaches.
__device__ __forceinline__ void cluster_barrier_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;"
                 ::: "memory");
}

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

// The phase of the last unit this CTA took: a further unit of the same phase
// needs neither the acquire fence nor the phase's fields again.
struct RanPhase {
    uint32_t valid;
    uint32_t fresh;   // a unit of the phase just completed (not the last one)
    uint32_t q;
    uint32_t epoch;
    uint32_t kind;
    uint32_t level;
    uint32_t nitems;
    unsigned long long desc;  // [epoch:32][units:32] of the phase
};

// The cluster mailbox of a CTA.  Peers reach it through DSMEM.
//
// A cluster run (engine_cluster.cuh) has no per-level leader step: at the end
// of every step each member writes a message -- its step tag, the vertices it
// appended, their entry slots, its error flag -- into its slot of every
// member's box, then waits on its own box for the others' messages; every
// member takes the same decision from the same messages.  The leader's box
// also holds the run's fields and the append counters the members share.
constexpr int kClusterMax = 16;
static_assert(kClusterMax <= 16, "a run number keeps the leader's rank in 4 bits");
// A message is one 64-bit word (one remote store per member):
// [step + 1 : 15][error : 1][entry slots / 256, saturated : 16][vertices or
// rows appended : 32].  Members clear their own slots when a run ends, so a
// tag can only match a message of the current run.
typedef unsigned long long ClusterMsg;
struct ClusterBox {
    uint32_t lock;       // rank 0's copy: 0 = no run in the cluster, else leader rank + 1
    uint32_t idle;       // 1 while this CTA finds no work (leaders invite idle CTAs only)
    unsigned long long inv;    // invitation to this CTA: [seq : 32][leader rank + 1 : 32]
    uint32_t join;       // leader: [seq : 15][closed : 1][member bits : 16]
    uint32_t ctr[2];     // leader: append positions of the members, by step parity
    uint32_t seq;        // leader: number of its last run: [count : 28][leader rank : 4]
    unsigned long long start;  // leader: [seq : 32][1 : 32] once the run's fields are set
    uint32_t members;    // leader: member bits of the current run
    uint32_t run_q;      // leader: instance of the run
    uint32_t run_k;      // leader: first level of the run
    uint32_t run_f;      // leader: vertices of the first level's list
    uint32_t run_reached, run_shrinks;     // leader: search counters at the start
    uint32_t run_sw, run_mcur, run_mprev;  // leader: matrices of the run
    ClusterMsg msg[2][kClusterMax];        // every box: [step parity][member r]
};

struct Smem {
    // staged frontier vertices of the unit being expanded: the column index
    // their products carry (the vertex, or its input label on a relabelled
    // graph), column begin minus slot offset (row index of slot s is b[t] + s), slot offset, and
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
    // cluster run: shared::cluster address of the leader's append counter of
    // the current step (positions in the list / touched rows); 0 outside runs.
    // The member's own appends are still counted in nq_cnt / nt_cnt / nq_slots.
    uint32_t ds_ctr;
    // cluster run state of this CTA: leader rank, run sequence, members, step
    // decision (stop flag and the next step's items), idle peers seen
    uint32_t cr_leader, cr_seq, cr_join, cr_stop, cr_f, cr_idle, cr_base;
    unsigned long long cr_slots;
    ClusterBox cbox;
    Cmd cmd;
    RanPhase ran;
    Inst I;
    uint32_t cur_q;
    uint32_t prof_on;
    uint32_t idle_exit;
    unsigned long long prof[kProfSlots];
};

// Warp 0: the other CTAs of the cluster that report themselves idle (a hint:
// they may take work before they see an invitation), as bits, to every lane.
__device__ __forceinline__ uint32_t cluster_idle_peers(Smem& sm) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t C = cluster_size(), me = cluster_rank();
    bool idle = false;
    if (lane < C && lane != me) idle = ds_ld_relaxed(ds_addr(&sm.cbox.idle, lane)) != 0u;
    return __ballot_sync(0xFFFFFFFFu, idle);
}

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
// One past the last row index of matrix mat that may be read.
__device__ __forceinline__ const uint32_t* rows_end(const Inst& I, uint32_t mat) {
    return mat == 0 ? I.rowidx + I.nnz : I.srows[mat - 1] + I.scap;
}
// Position of row index beg of matrix mat within its aligned 16-byte group
// (the row arrays need only be 4-byte aligned).
__device__ __forceinline__ uint32_t row_shift(const uint32_t* rows) {
    return (uint32_t)(reinterpret_cast<uintptr_t>(rows) >> 2);
}
__device__ __forceinline__ uint32_t col_head(const Inst& I, uint32_t mat, uint32_t beg) {
    return (row_shift(rows_of(I, mat)) + beg) & (kChunk - 1);
}
// Entry slots of a frontier vertex whose column (matrix mat) starts at beg.
__device__ __forceinline__ uint32_t col_slots(const Inst& I, uint32_t mat, uint32_t beg, uint32_t len) {
    return vslots(col_head(I, mat, beg), len);
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

// Four row indices from a 16-byte aligned address p, as ld_row.
__device__ __forceinline__ uint4 ld_row4(const uint32_t* p, uint32_t mat, uint64_t pol) {
    uint4 v;
    if (mat == 0)
        asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
            : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
            : "l"(p), "l"(pol));
    else
        asm volatile("ld.global.cg.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
                     : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                     : "l"(p), "l"(pol)
                     : "memory");
    return v;
}

}  // namespace abfs
