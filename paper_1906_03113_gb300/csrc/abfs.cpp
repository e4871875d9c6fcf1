// Host runtime behind the C-ABI declared in include/abfs.h: graph storage and
// validation, search workspaces, single and batched searches, the autotuner.
// Every step of a search runs in the device engine (engine.cu); this file only
// allocates, initialises descriptors and launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstddef>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <functional>
#include <mutex>
#include <sstream>
#include <string>
#include <thread>
#include <vector>

#include "../../include/abfs.h"
#include "internal.h"

using namespace abfs;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------

extern "C" const char* abfs_strerror(int status) {
    switch (status) {
        case ABFS_OK: return "ok";
        case ABFS_ERR_INVALID_ARG: return "invalid argument";
        case ABFS_ERR_NOT_SYMMETRIC: return "graph marked undirected is not symmetric";
        case ABFS_ERR_OOM: return "out of memory";
        case ABFS_ERR_CUDA: return "CUDA runtime error";
        case ABFS_ERR_TIMEOUT: return "bounded device wait expired";
        case ABFS_ERR_BUSY: return "not admitted: no free slot or memory";
        case ABFS_ERR_DEVICE: return "device-side consistency check failed";
        case ABFS_ERR_UNSUPPORTED: return "size beyond the library's limits, or unsupported in this mode";
        case ABFS_ERR_NOT_FOUND: return "unknown ticket";
        default: return "unknown status";
    }
}

extern "C" int abfs_version(void) { return 10100; }

namespace {

thread_local std::string g_last_cuda_error;

int cuda_fail(cudaError_t e) {
    if (e == cudaSuccess) return ABFS_OK;
    g_last_cuda_error = cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return ABFS_ERR_OOM;
    return ABFS_ERR_CUDA;
}

#define CK(call)                                  \
    do {                                          \
        cudaError_t e_ = (call);                  \
        if (e_ != cudaSuccess) return cuda_fail(e_); \
    } while (0)

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// ---------------------------------------------------------------------------
// allocator hook
// ---------------------------------------------------------------------------

struct Allocator {
    void* (*alloc)(size_t, void*) = nullptr;
    void (*free)(void*, void*) = nullptr;
    void* ctx = nullptr;
};
Allocator g_alloc;
std::mutex g_alloc_mu;

int dev_alloc(void** p, size_t bytes) {
    if (bytes == 0) bytes = 256;
    Allocator a;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        a = g_alloc;
    }
    if (a.alloc) {
        *p = a.alloc(bytes, a.ctx);
        if (!*p) return ABFS_ERR_OOM;
        // the kernels read 8- and 16-byte words from every block
        if (reinterpret_cast<uintptr_t>(*p) & 15u) {
            a.free(*p, a.ctx);
            *p = nullptr;
            return ABFS_ERR_INVALID_ARG;
        }
        return ABFS_OK;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? ABFS_ERR_OOM : cuda_fail(e);
    }
    return ABFS_OK;
}

void dev_free(void* p) {
    if (!p) return;
    Allocator a;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        a = g_alloc;
    }
    if (a.free) a.free(p, a.ctx);
    else cudaFree(p);
}

}  // namespace

// ---------------------------------------------------------------------------
// parameters and per-search workspace layout (shared with static_ws.cu)
// ---------------------------------------------------------------------------

namespace abfs {

abfs_params default_params() {
    abfs_params p;
    p.mode = ABFS_MODE_SUBMATRIX;
    p.tile = 1024;
    p.unit_entries = 1024;
    p.narrow_max = 1024;
    p.narrow_edges = 16384;
    p.ctas_per_sm = 2;
    p.shrink_theta = 0.f;
    p.shrink_max = 0;
    p.timeout_ms = 10000;
    p.narrow_resident = 1;
    p.claim_scan = 1u << 22;
    p.bottom_up_alpha = 0;
    p.bottom_up_beta = 24;
    p.cluster_ctas = 8;
    p.cluster_min = 2048;
    p.cluster_max = 16384;
    p.cluster_edges = 1u << 16;
    p.multi_source = 8;
    return p;
}

bool shrink_enabled(const abfs_params& p) {
    return p.mode == ABFS_MODE_SUBMATRIX && p.shrink_theta > 0.f && p.shrink_theta < 1.f &&
           p.shrink_max > 0;
}

int check_params(const abfs_params& p) {
    if (p.mode > ABFS_MODE_PLAIN) return ABFS_ERR_INVALID_ARG;
    if (p.tile < 32 || p.tile > (uint32_t)kTileMax || p.tile % 32) return ABFS_ERR_INVALID_ARG;
    if (p.unit_entries < 256 || p.unit_entries > kUnitMax || (p.unit_entries & (p.unit_entries - 1)))
        return ABFS_ERR_INVALID_ARG;
    if (p.ctas_per_sm < 1 || p.ctas_per_sm > 8) return ABFS_ERR_INVALID_ARG;
    if (!(p.shrink_theta >= 0.f) || p.shrink_theta > 1.f) return ABFS_ERR_INVALID_ARG;
    if (p.timeout_ms < 1 || p.timeout_ms > 600000) return ABFS_ERR_INVALID_ARG;
    if (p.narrow_resident > 1) return ABFS_ERR_INVALID_ARG;
    if (p.cluster_ctas < 1 || p.cluster_ctas > 16) return ABFS_ERR_INVALID_ARG;
    // the hybrid reads the input columns: submatrix mode, no physical shrink
    if (p.bottom_up_alpha && (p.mode != ABFS_MODE_SUBMATRIX || shrink_enabled(p)))
        return ABFS_ERR_INVALID_ARG;
    return ABFS_OK;
}

EngineParams engine_params(const abfs_params& p) {
    EngineParams e;
    e.mode = p.mode;
    e.tile = p.tile;
    e.unit = p.unit_entries;
    e.unit_shift = 0;
    while ((1u << e.unit_shift) < p.unit_entries) ++e.unit_shift;
    e.narrow_max = p.narrow_max;
    e.narrow_edges = p.narrow_edges;
    e.narrow_loop = p.narrow_resident;
    e.scan_min = p.mode == ABFS_MODE_SUBMATRIX ? p.claim_scan : 0u;
    e.bu_alpha = p.mode == ABFS_MODE_SUBMATRIX ? p.bottom_up_alpha : 0u;
    e.bu_beta = p.bottom_up_beta;
    e.shrink_theta = shrink_enabled(p) ? p.shrink_theta : 0.f;
    e.shrink_max = shrink_enabled(p) ? std::min<uint32_t>(p.shrink_max, 64) : 0;
    e.shrink_tile = kTileMax;
    e.init_tile = 65536;
    e.timeout_ns = (unsigned long long)p.timeout_ms * 1000000ull;
    e.cluster = p.cluster_ctas;
    e.cluster_min = p.cluster_min;
    e.cluster_max = p.cluster_max;
    e.cluster_edges = p.cluster_edges;
    return e;
}

bool same_layout(const abfs_params& a, const abfs_params& b) {
    return a.mode == b.mode && a.unit_entries == b.unit_entries && shrink_enabled(a) == shrink_enabled(b) &&
           (!shrink_enabled(a) || std::min(a.shrink_max, 2u) == std::min(b.shrink_max, 2u));
}

// ---------------------------------------------------------------------------
// per-search workspace layout
// ---------------------------------------------------------------------------

Layout layout_for(uint32_t n, uint64_t nnz, const abfs_params& p, uint32_t ms, bool relabel) {
    Layout L;
    std::memset(&L, 0, sizeof(L));
    const size_t A = 256;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = align_up(o + bytes, A);
        return at;
    };
    L.nwords = (n + 31) / 32;
    L.bcap = std::min<uint32_t>(n, kBlockMask);
    // a level's frontier holds at most every vertex: nnz column entries plus
    // at most kVertexSlotsMax slots per vertex
    L.nnz = nnz;
    L.ucap = (nnz + (uint64_t)kVertexSlotsMax * n) / p.unit_entries + 2;
    L.ctl = take(sizeof(InstCtl));
    L.inst = take(sizeof(Inst));
    for (int i = 0; i < 2; ++i) {
        L.fq[i] = take((size_t)n * 4);
        L.fbeg[i] = take((size_t)n * 4);
        L.fpre[i] = take((size_t)n * 4);
        L.flen[i] = take((size_t)n * 4);
        L.blk[i] = take((size_t)L.bcap * sizeof(Block));
        L.ustart[i] = take((size_t)L.ucap * sizeof(uint2));
    }
    if (p.mode == ABFS_MODE_SUBMATRIX)
        for (int i = 0; i < 2; ++i) L.bm[i] = take((size_t)L.nwords * 4);
    if (p.mode == ABFS_MODE_SUBMATRIX)
        for (int i = 0; i < 2; ++i) L.fbm[i] = take((size_t)L.nwords * 4);
    if (p.mode == ABFS_MODE_PLAIN) {
        L.y = take((size_t)n * 8);
        L.touched = take((size_t)n * 4);
    }
    if (ms) {
        // multi-source search: reached / frontier / next bit masks, the sources
        // and the per-source output pointers
        L.ms_vis = take((size_t)n * 8);
        for (int i = 0; i < 2; ++i) L.ms_fr[i] = take((size_t)n * 8);
        L.ms_nx = take((size_t)n * 8);
        L.ms_src = take((size_t)ms * 4);
        L.ms_lev = take((size_t)ms * 8);
        L.ms_par = take((size_t)ms * 8);
    }
    if (shrink_enabled(p) && !ms) {
        L.ncopies = std::min(p.shrink_max, 2u);
        L.scap = nnz;
        for (uint32_t i = 0; i < L.ncopies; ++i) {
            L.sbeg[i] = take((size_t)n * 4);
            L.slen[i] = take((size_t)n * 4);
            L.srows[i] = take((size_t)std::max<uint64_t>(nnz, 1) * 4);
        }
    }
    if (relabel && !ms) {
        // searches on the relabelled copy: a second descriptor and the
        // internal outputs
        L.inst_r = take(sizeof(Inst));
        L.lev_i = take((size_t)n * 4);
        L.par_i = take((size_t)n * 4);
    }
    L.total = o;
    return L;
}

Inst make_inst_raw(const uint32_t* colptr, const uint32_t* rowidx, uint32_t n, char* base,
                   const Layout& L, uint32_t src, int32_t* level, int32_t* parent) {
    Inst I;
    std::memset(&I, 0, sizeof(I));
    I.colptr = colptr;
    I.rowidx = rowidx;
    I.nnz = L.nnz;
    I.n = n;
    I.src = src;
    I.nwords = L.nwords;
    I.bcap = L.bcap;
    I.ucap = L.ucap;
    I.level = level;
    I.parent = reinterpret_cast<uint32_t*>(parent);
    for (int i = 0; i < 2; ++i) {
        I.fq[i] = reinterpret_cast<uint32_t*>(base + L.fq[i]);
        I.fbeg[i] = reinterpret_cast<uint32_t*>(base + L.fbeg[i]);
        I.fpre[i] = reinterpret_cast<uint32_t*>(base + L.fpre[i]);
        I.flen[i] = reinterpret_cast<uint32_t*>(base + L.flen[i]);
        I.blk[i] = reinterpret_cast<Block*>(base + L.blk[i]);
        I.ustart[i] = reinterpret_cast<uint2*>(base + L.ustart[i]);
        I.bm[i] = L.bm[i] ? reinterpret_cast<uint32_t*>(base + L.bm[i]) : nullptr;
        I.fbm[i] = L.fbm[i] ? reinterpret_cast<uint32_t*>(base + L.fbm[i]) : nullptr;
    }
    if (L.y) I.y = reinterpret_cast<unsigned long long*>(base + L.y);
    if (L.touched) I.touched = reinterpret_cast<uint32_t*>(base + L.touched);
    for (uint32_t i = 0; i < L.ncopies; ++i) {
        I.sbeg[i] = reinterpret_cast<uint32_t*>(base + L.sbeg[i]);
        I.slen[i] = reinterpret_cast<uint32_t*>(base + L.slen[i]);
        I.srows[i] = reinterpret_cast<uint32_t*>(base + L.srows[i]);
    }
    I.scap = L.scap;
    I.ctl = reinterpret_cast<InstCtl*>(base + L.ctl);
    return I;
}

int grid_for(int sms, const abfs_params& p) {
    int bps = 0;
    if (engine_occupancy(p.mode, &bps) != cudaSuccess || bps < 1) bps = 1;
    const int per_sm = std::min<int>(bps, (int)p.ctas_per_sm);
    int grid = std::max(per_sm * std::max(sms, 1), 1);
    const int c = (int)p.cluster_ctas;
    if (c > 1) {
        // whole clusters only, and no more than can be resident at once: every
        // CTA of the persistent launch runs from the start
        int nc = 0;
        if (engine_max_clusters(p.mode, (uint32_t)c, &nc) != cudaSuccess || nc < 1) nc = 1;
        grid = std::min(grid / c, nc) * c;
        if (grid < c) grid = c;
    }
    return grid;
}

}  // namespace abfs

// ---------------------------------------------------------------------------
// graph
// ---------------------------------------------------------------------------

struct Workspace {
    char* base = nullptr;
    Layout L{};
    abfs_params p{};
    bool relabel = false;     // laid out for searches on the relabelled copy too
    Inst* d_inst = nullptr;   // device descriptor (instance 0)
    Inst* d_inst_r = nullptr; // the same on the relabelled copy
    uint32_t* d_done = nullptr;
    unsigned long long* d_beat = nullptr;
    InstCtl* h_ctl = nullptr; // pinned copy for stats
};

struct abfs_graph_s {
    uint32_t* d_colptr = nullptr;
    uint32_t* d_rowidx = nullptr;
    uint32_t n = 0;
    uint64_t nnz = 0;
    int directed = 0;
    bool sorted = false;          // every column's row indices ascend (bottom-up levels allowed)
    // abfs_graph_relabel: a copy with vertices numbered by column-length class
    // (internal labels) and the maps between the two numberings
    bool relabeled = false;
    uint32_t* r_colptr = nullptr;
    uint32_t* r_rowidx = nullptr;
    uint32_t* r_inb = nullptr;
    uint32_t* d_lab = nullptr;     // internal label -> input label
    uint32_t* d_pos = nullptr;     // input label -> internal label
    std::vector<uint32_t> h_pos;
    uint32_t r_keep = 0;           // internal vertices that may be reached (all but the
                                   // empty columns of an undirected graph)
    uint32_t* d_inb = nullptr;    // rows that occur in some column, one bit per vertex
    int device = 0;
    int sms = 0;
    bool tuned = false;
    abfs_params tuned_params{};
    std::mutex mu;
    Workspace ws;
    int32_t* d_level = nullptr;   // device outputs of host-output runs (abfs_run_host)
    int32_t* d_parent = nullptr;
    cudaEvent_t last_use = nullptr;
    bool used = false;
    // abfs_run_host_many: a second pair of device outputs, the stream that copies
    // one search's outputs out while the next one runs, and pinned status words
    int32_t* d_level2 = nullptr;
    int32_t* d_parent2 = nullptr;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t computed[2] = {nullptr, nullptr};
    cudaEvent_t copied[2] = {nullptr, nullptr};
    uint32_t* h_status = nullptr;  // two words (status, err) per search
    uint32_t h_status_cap = 0;     // searches h_status holds
};

namespace {

int validate_host(const uint32_t* colptr, const uint32_t* rowidx, uint32_t n, uint64_t nnz,
                  int directed) {
    if (colptr[0] != 0 || colptr[n] != nnz) return ABFS_ERR_INVALID_ARG;
    for (uint32_t v = 0; v < n; ++v)
        if (colptr[v + 1] < colptr[v]) return ABFS_ERR_INVALID_ARG;
    for (uint64_t e = 0; e < nnz; ++e)
        if (rowidx[e] >= n) return ABFS_ERR_INVALID_ARG;
    if (!directed) {
        // symmetric pattern: every entry (i in column j) has its mirror
        std::vector<uint32_t> rows(rowidx, rowidx + nnz);
        for (uint32_t v = 0; v < n; ++v) std::sort(rows.begin() + colptr[v], rows.begin() + colptr[v + 1]);
        for (uint32_t j = 0; j < n; ++j) {
            for (uint32_t e = colptr[j]; e < colptr[j + 1]; ++e) {
                const uint32_t i = rows[e];
                if (!std::binary_search(rows.begin() + colptr[i], rows.begin() + colptr[i + 1], j))
                    return ABFS_ERR_NOT_SYMMETRIC;
            }
        }
    }
    return ABFS_OK;
}

void free_workspace(Workspace& w) {
    dev_free(w.base);
    dev_free(w.d_done);
    dev_free(w.d_beat);
    if (w.h_ctl) cudaFreeHost(w.h_ctl);
    w = Workspace{};
}

Inst make_inst(const abfs_graph_s* g, char* base, const Layout& L, uint32_t src, int32_t* level,
               int32_t* parent) {
    Inst I = make_inst_raw(g->d_colptr, g->d_rowidx, g->n, base, L, src, level, parent);
    // the hybrid's bottom-up levels need a symmetric pattern and ascending columns
    I.bu_ok = (!g->directed && g->sorted) ? 1u : 0u;
    I.inb = g->d_inb;
    return I;
}

// Ensures g->ws fits params p (reallocating after the previous use finished).
int ensure_workspace(abfs_graph_s* g, const abfs_params& p) {
    Workspace& w = g->ws;
    if (w.base && same_layout(w.p, p) && w.relabel == g->relabeled) {
        w.p = p;
        return ABFS_OK;
    }
    if (w.base) {
        if (g->used) CK(cudaEventSynchronize(g->last_use));
        free_workspace(w);
    }
    Layout L = layout_for(g->n, g->nnz, p, 0, g->relabeled);
    int rc = dev_alloc((void**)&w.base, L.total);
    if (rc) return rc;
    rc = dev_alloc((void**)&w.d_done, 64);
    if (!rc) rc = dev_alloc((void**)&w.d_beat, 64);
    if (rc) {
        free_workspace(w);
        return rc;
    }
    if (cudaMallocHost((void**)&w.h_ctl, sizeof(InstCtl)) != cudaSuccess) {
        cudaGetLastError();
        free_workspace(w);
        return ABFS_ERR_OOM;
    }
    w.L = L;
    w.p = p;
    w.d_inst = reinterpret_cast<Inst*>(w.base + L.inst);
    Inst I = make_inst(g, w.base, L, 0, nullptr, nullptr);
    cudaError_t e = cudaMemcpy(w.d_inst, &I, sizeof(Inst), cudaMemcpyHostToDevice);
    w.relabel = g->relabeled;
    w.d_inst_r = nullptr;
    if (e == cudaSuccess && g->relabeled) {
        Inst Ir = make_inst_raw(g->r_colptr, g->r_rowidx, g->n, w.base, L, 0, nullptr, nullptr);
        Ir.inb = g->r_inb;
        Ir.bu_ok = 0;  // the relabelled columns are not in ascending input-label order
        Ir.lab = g->d_lab;
        w.d_inst_r = reinterpret_cast<Inst*>(w.base + L.inst_r);
        e = cudaMemcpy(w.d_inst_r, &Ir, sizeof(Inst), cudaMemcpyHostToDevice);
    }
    // the initialisation kernel of single searches counts its blocks in the
    // control block, which must start at zero
    if (e == cudaSuccess) e = cudaMemset(w.base + L.ctl, 0, sizeof(InstCtl));
    if (e != cudaSuccess) {
        free_workspace(w);
        return cuda_fail(e);
    }
    return ABFS_OK;
}

int grid_size(const abfs_graph_s* g, const abfs_params& p, uint32_t) { return grid_for(g->sms, p); }

void fill_stats(const InstCtl& c, abfs_stats* st) {
    std::memset(st, 0, sizeof(*st));
    st->levels = c.levels;
    st->reached = c.reached;
    st->nnz_reached = c.nnz_reached;
    st->entries_read = c.entries_read;
    st->entries_unmasked = c.entries_unmasked;
    st->claims = c.claims;
    st->shrinks = c.shrinks;
    st->wide_levels = c.wide_levels;
    st->shrink_entries_read = c.shrink_read;
    st->shrink_entries_kept = c.shrink_kept;
    st->status = (c.status == kDone) ? 0u : (c.err ? c.err : (uint32_t)ABFS_ERR_DEVICE);
}

const abfs_params& pick_params(const abfs_graph_s* g, const abfs_params* params,
                               abfs_params& tmp) {
    if (params) return *params;
    tmp = g->tuned ? g->tuned_params : default_params();
    return tmp;
}

// Enqueues one search into g's workspace; caller holds g->mu.
int enqueue_single(abfs_graph_s* g, uint32_t source, int32_t* level, int32_t* parent,
                   cudaStream_t s, const abfs_params& p, uint4* trace = nullptr,
                   uint32_t trace_cap = 0, unsigned long long* prof = nullptr,
                   uint64_t* sigma = nullptr) {
    int rc = ensure_workspace(g, p);
    if (rc) return rc;
    Workspace& w = g->ws;
    if (g->used) CK(cudaStreamWaitEvent(s, g->last_use, 0));
    // submatrix searches without path counts run on the relabelled copy, except
    // those that may take bottom-up levels: their scans need each column in
    // ascending input-label order, which only the input numbering has
    const bool bu_wanted = p.bottom_up_alpha && !g->directed && g->sorted;
    const bool rel = w.relabel && p.mode == ABFS_MODE_SUBMATRIX && !sigma && !bu_wanted;
    const uint32_t bu_ok = (!rel && !g->directed && g->sorted && !sigma) ? 1u : 0u;
    EngineArgs a;
    a.insts = rel ? w.d_inst_r : w.d_inst;
    a.ninst = 1;
    a.done_count = w.d_done;
    a.heartbeat = w.d_beat;
    a.prof = prof;
    a.serve = 0;
    a.slot_state = nullptr;
    a.stop_flag = nullptr;
    a.idle_exit_ns = 0;
    a.p = engine_params(p);
    a.hold_units = test_hold_units();
    if (rel) {
        int32_t* lev_i = reinterpret_cast<int32_t*>(w.base + w.L.lev_i);
        uint32_t* par_i = reinterpret_cast<uint32_t*>(w.base + w.L.par_i);
        CK(launch_init_single(a, g->h_pos[source], source, lev_i, par_i, nullptr, 0u, trace,
                              trace_cap, g->n, s));
        CK(launch_engine(a, grid_size(g, p, 0), s));
        CK(launch_relabel_out(g->d_pos, lev_i, par_i, level, parent, g->n, g->r_keep,
                              g->h_pos[source], s));
        CK(cudaEventRecord(g->last_use, s));
        g->used = true;
        return ABFS_OK;
    }
    CK(launch_init_single(a, source, source, level, reinterpret_cast<uint32_t*>(parent),
                          reinterpret_cast<unsigned long long*>(sigma), bu_ok, trace, trace_cap,
                          g->n, s));
    CK(launch_engine(a, grid_size(g, p, 0), s));
    CK(cudaEventRecord(g->last_use, s));
    g->used = true;
    return ABFS_OK;
}

int finish_stats(abfs_graph_s* g, cudaStream_t s, abfs_stats* stats) {
    Workspace& w = g->ws;
    CK(cudaMemcpyAsync(w.h_ctl, w.base + w.L.ctl, sizeof(InstCtl), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    fill_stats(*w.h_ctl, stats);
    return stats->status;
}

}  // namespace

namespace abfs {
int graph_arrays(abfs_graph_t g, const uint32_t** colptr, const uint32_t** rowidx, uint32_t* n,
                 uint64_t* nnz, int* device, int* sms) {
    if (!g) return ABFS_ERR_INVALID_ARG;
    *colptr = g->d_colptr;
    *rowidx = g->d_rowidx;
    *n = g->n;
    *nnz = g->nnz;
    *device = g->device;
    *sms = g->sms;
    return ABFS_OK;
}
}  // namespace abfs

extern "C" int abfs_default_params(abfs_params* p) {
    if (!p) return ABFS_ERR_INVALID_ARG;
    *p = default_params();
    return ABFS_OK;
}

extern "C" int abfs_check_params(const abfs_params* p) {
    if (!p) return ABFS_ERR_INVALID_ARG;
    return check_params(*p);
}

extern "C" int abfs_graph_create(const uint32_t* colptr, const uint32_t* rowidx, uint32_t n,
                                 uint64_t nnz, int directed, uint32_t flags, abfs_stream_t stream,
                                 abfs_graph_t* out) {
    if (!out || !colptr || (nnz && !rowidx) || n == 0) return ABFS_ERR_INVALID_ARG;
    *out = nullptr;
    if (n >= (1u << 31) || nnz + n >= (1ull << 32)) return ABFS_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    const bool on_dev = flags & ABFS_INPUT_ON_DEVICE;
    std::vector<uint32_t> hc, hr;
    if ((flags & ABFS_VALIDATE) && on_dev) {
        hc.resize((size_t)n + 1);
        hr.resize(nnz);
        CK(cudaMemcpy(hc.data(), colptr, hc.size() * 4, cudaMemcpyDeviceToHost));
        if (nnz) CK(cudaMemcpy(hr.data(), rowidx, nnz * 4, cudaMemcpyDeviceToHost));
    }
    if (flags & ABFS_VALIDATE) {
        int rc = on_dev ? validate_host(hc.data(), hr.data(), n, nnz, directed)
                        : validate_host(colptr, rowidx, n, nnz, directed);
        if (rc) return rc;
    }
    abfs_graph_s* g = new (std::nothrow) abfs_graph_s();
    if (!g) return ABFS_ERR_OOM;
    g->n = n;
    g->nnz = nnz;
    g->directed = directed ? 1 : 0;
    cudaGetDevice(&g->device);
    cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, g->device);
    int rc = dev_alloc((void**)&g->d_colptr, ((size_t)n + 1) * 4);
    if (!rc) rc = dev_alloc((void**)&g->d_rowidx, std::max<uint64_t>(nnz, 1) * 4);
    if (rc) {
        abfs_graph_destroy(g);
        return rc;
    }
    const cudaMemcpyKind kind = on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cudaError_t e = cudaMemcpyAsync(g->d_colptr, colptr, ((size_t)n + 1) * 4, kind, s);
    if (e == cudaSuccess && nnz) e = cudaMemcpyAsync(g->d_rowidx, rowidx, nnz * 4, kind, s);
    // whether every column ascends (the hybrid's bottom-up levels need it)
    uint32_t* d_flag = nullptr;
    if (e == cudaSuccess && dev_alloc((void**)&d_flag, 4) != ABFS_OK) e = cudaErrorMemoryAllocation;
    uint32_t unsorted = 1;
    if (e == cudaSuccess) e = cudaMemsetAsync(d_flag, 0, 4, s);
    if (e == cudaSuccess) e = launch_sorted_check(g->d_colptr, g->d_rowidx, n, d_flag, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&unsorted, d_flag, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dev_free(d_flag);
    g->sorted = unsorted == 0;
    // the rows that occur at all: the others are never reached
    const uint32_t nwords = (n + 31) / 32;
    if (e == cudaSuccess && dev_alloc((void**)&g->d_inb, (size_t)nwords * 4) != ABFS_OK)
        e = cudaErrorMemoryAllocation;
    if (e == cudaSuccess) e = launch_row_bitmap(g->d_rowidx, nnz, g->d_inb, nwords, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->last_use, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        abfs_graph_destroy(g);
        return cuda_fail(e);
    }
    *out = g;
    return ABFS_OK;
}

extern "C" int abfs_graph_destroy(abfs_graph_t g) {
    if (!g) return ABFS_ERR_INVALID_ARG;
    if (g->used && g->last_use) cudaEventSynchronize(g->last_use);
    free_workspace(g->ws);
    if (g->copy_stream) cudaStreamSynchronize(g->copy_stream);
    dev_free(g->d_level);
    dev_free(g->d_parent);
    dev_free(g->d_level2);
    dev_free(g->d_parent2);
    for (int b = 0; b < 2; ++b) {
        if (g->computed[b]) cudaEventDestroy(g->computed[b]);
        if (g->copied[b]) cudaEventDestroy(g->copied[b]);
    }
    if (g->copy_stream) cudaStreamDestroy(g->copy_stream);
    if (g->h_status) cudaFreeHost(g->h_status);
    dev_free(g->d_colptr);
    dev_free(g->d_rowidx);
    dev_free(g->d_inb);
    dev_free(g->r_colptr);
    dev_free(g->r_rowidx);
    dev_free(g->r_inb);
    dev_free(g->d_lab);
    dev_free(g->d_pos);
    if (g->last_use) cudaEventDestroy(g->last_use);
    delete g;
    return ABFS_OK;
}

extern "C" int abfs_relabel_order(const uint32_t* colptr, uint32_t n, uint32_t* lab, uint32_t* pos) {
    if (n == 0) return ABFS_OK;
    if (!colptr || !lab || !pos) return ABFS_ERR_INVALID_ARG;
    const uint32_t* cp = colptr;
    for (uint32_t v = 0; v < n; ++v)
        if (cp[v + 1] < cp[v]) return ABFS_ERR_INVALID_ARG;
    // internal label of each vertex: by class, and in input order inside a
    // class -- (0) the longest columns, whole length groups of at most n/64
    // vertices in all; (1) the next longest, up to n/8 with class 0; (2) the
    // other non-empty columns; (3) the empty ones.  The hubs the first levels
    // reach share cache lines of every per-vertex array; the input order
    // inside a class keeps whatever locality the input numbering had.
    std::vector<uint32_t> len(n);
    for (uint32_t v = 0; v < n; ++v) len[v] = cp[v + 1] - cp[v];
    const uint64_t cap[2] = {(uint64_t)n / 64, (uint64_t)n / 8};
    // the k = n/8 + 1 longest lengths, descending, place both thresholds: a
    // length group that reaches index k - 1 holds more than n/8 vertices
    const size_t k = (size_t)std::min<uint64_t>(n, cap[1] + 1);
    std::vector<uint32_t> top(len);
    std::nth_element(top.begin(), top.begin() + (k - 1), top.end(), std::greater<uint32_t>());
    std::sort(top.begin(), top.begin() + k, std::greater<uint32_t>());
    // thr[c]: the shortest length in classes 0..c (no class: above every length)
    uint64_t thr[2];
    size_t i = 0;  // vertices in the classes so far
    for (int c = 0; c < 2; ++c) {
        while (i < k && top[i] > 0) {
            size_t j = i;
            while (j < k && top[j] == top[i]) ++j;
            if ((j == k && k < n) || j > cap[c]) break;  // the group does not fit
            i = j;
        }
        thr[c] = i > 0 ? top[i - 1] : (uint64_t)UINT32_MAX + 1;
    }
    std::vector<uint8_t> cls(n);
    uint64_t start[5] = {0, 0, 0, 0, 0};
    for (uint32_t v = 0; v < n; ++v) {
        const uint32_t d = len[v];
        cls[v] = d >= thr[0] ? 0 : (d >= thr[1] ? 1 : (d > 0 ? 2 : 3));
        ++start[cls[v] + 1];
    }
    for (int c = 1; c < 5; ++c) start[c] += start[c - 1];
    for (uint32_t v = 0; v < n; ++v) {
        const uint32_t i = (uint32_t)start[cls[v]]++;
        lab[i] = v;
        pos[v] = i;
    }
    return ABFS_OK;
}

extern "C" int abfs_graph_relabel(abfs_graph_t g) {
    if (!g) return ABFS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g->mu);
    if (g->relabeled) return ABFS_OK;
    if (g->used) CK(cudaEventSynchronize(g->last_use));
    const uint32_t n = g->n;
    const uint64_t nnz = g->nnz;
    std::vector<uint32_t> cp((size_t)n + 1), rows(std::max<uint64_t>(nnz, 1));
    CK(cudaMemcpy(cp.data(), g->d_colptr, ((size_t)n + 1) * 4, cudaMemcpyDeviceToHost));
    if (nnz) CK(cudaMemcpy(rows.data(), g->d_rowidx, nnz * 4, cudaMemcpyDeviceToHost));
    std::vector<uint32_t> lab(n), pos(n);
    {
        const int rc0 = abfs_relabel_order(cp.data(), n, lab.data(), pos.data());
        if (rc0) return rc0;
    }
    // the relabelled CSC: column i is column lab[i], its rows renamed (in the
    // input's order; no search on the copy depends on the row order).
    // Columns are filled by several host threads.
    std::vector<uint32_t> rcp((size_t)n + 1), rrows(std::max<uint64_t>(nnz, 1));
    rcp[0] = 0;
    for (uint32_t i = 0; i < n; ++i) rcp[i + 1] = rcp[i] + (cp[lab[i] + 1] - cp[lab[i]]);
    {
        auto fill = [&](uint32_t i0, uint32_t i1) {
            for (uint32_t i = i0; i < i1; ++i) {
                const uint32_t b = cp[lab[i]];
                uint32_t* out = rrows.data() + rcp[i];
                const uint32_t len = rcp[i + 1] - rcp[i];
                for (uint32_t x = 0; x < len; ++x) out[x] = pos[rows[(size_t)b + x]];
            }
        };
        const unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
        std::vector<std::thread> th;
        // column ranges of about nnz / nt entries each
        uint32_t i0 = 0;
        for (unsigned t = 1; t <= nt && i0 < n; ++t) {
            const uint64_t goal = nnz * t / nt;
            uint32_t i1 = (uint32_t)(std::upper_bound(rcp.begin() + i0, rcp.end(), (uint32_t)goal) -
                                     rcp.begin());
            i1 = t == nt ? n : std::min(std::max(i1, i0 + 1), n);
            th.emplace_back(fill, i0, i1);
            i0 = i1;
        }
        for (auto& x : th) x.join();
    }
    const uint32_t nwords = (n + 31) / 32;
    int rc = dev_alloc((void**)&g->r_colptr, ((size_t)n + 1) * 4);
    if (!rc) rc = dev_alloc((void**)&g->r_rowidx, std::max<uint64_t>(nnz, 1) * 4);
    if (!rc) rc = dev_alloc((void**)&g->r_inb, (size_t)nwords * 4);
    if (!rc) rc = dev_alloc((void**)&g->d_lab, (size_t)n * 4);
    if (!rc) rc = dev_alloc((void**)&g->d_pos, (size_t)n * 4);
    cudaError_t e = cudaSuccess;
    if (!rc) {
        e = cudaMemcpy(g->r_colptr, rcp.data(), ((size_t)n + 1) * 4, cudaMemcpyHostToDevice);
        if (e == cudaSuccess && nnz)
            e = cudaMemcpy(g->r_rowidx, rrows.data(), nnz * 4, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(g->d_lab, lab.data(), (size_t)n * 4, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(g->d_pos, pos.data(), (size_t)n * 4, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = launch_row_bitmap(g->r_rowidx, nnz, g->r_inb, nwords, nullptr);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    if (rc || e != cudaSuccess) {
        for (uint32_t** q : {&g->r_colptr, &g->r_rowidx, &g->r_inb, &g->d_lab, &g->d_pos}) {
            dev_free(*q);
            *q = nullptr;
        }
        return rc ? rc : cuda_fail(e);
    }
    // an undirected graph's empty columns (the last internal labels) are
    // vertices without edges: unreachable from any other source
    uint32_t keep = n;
    if (!g->directed)
        while (keep > 0 && rcp[keep] == rcp[keep - 1]) --keep;
    g->h_pos = std::move(pos);
    g->r_keep = keep;
    g->relabeled = true;
    // the next search lays its workspace out for the relabelled copy
    free_workspace(g->ws);
    return ABFS_OK;
}

extern "C" int abfs_graph_info(abfs_graph_t g, uint32_t* n, uint64_t* nnz, int* directed) {
    if (!g) return ABFS_ERR_INVALID_ARG;
    if (n) *n = g->n;
    if (nnz) *nnz = g->nnz;
    if (directed) *directed = g->directed;
    return ABFS_OK;
}

extern "C" int abfs_graph_footprint(abfs_graph_t g, const abfs_params* params, size_t* bytes) {
    if (!g || !bytes) return ABFS_ERR_INVALID_ARG;
    abfs_params tmp;
    const abfs_params& p = pick_params(g, params, tmp);
    int rc = check_params(p);
    if (rc) return rc;
    *bytes = layout_for(g->n, g->nnz, p, 0, g->relabeled).total;
    return ABFS_OK;
}

extern "C" int abfs_run(abfs_graph_t g, uint32_t source, int32_t* level, int32_t* parent,
                        abfs_stream_t stream, const abfs_params* params, abfs_stats* stats) {
    if (!g || !level || !parent || source >= g->n) return ABFS_ERR_INVALID_ARG;
    abfs_params tmp;
    const abfs_params& p = pick_params(g, params, tmp);
    int rc = check_params(p);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g->mu);
    rc = enqueue_single(g, source, level, parent, s, p);
    if (rc) return rc;
    if (stats) return finish_stats(g, s, stats);
    return ABFS_OK;
}

extern "C" int abfs_run_counts(abfs_graph_t g, uint32_t source, int32_t* level, int32_t* parent,
                               uint64_t* sigma, abfs_stream_t stream, const abfs_params* params,
                               abfs_stats* stats) {
    if (!g || !level || !parent || !sigma || source >= g->n) return ABFS_ERR_INVALID_ARG;
    abfs_params tmp;
    const abfs_params& p = pick_params(g, params, tmp);
    int rc = check_params(p);
    if (rc) return rc;
    if (p.mode != ABFS_MODE_SUBMATRIX) return ABFS_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g->mu);
    rc = enqueue_single(g, source, level, parent, s, p, nullptr, 0, nullptr, sigma);
    if (rc) return rc;
    if (stats) return finish_stats(g, s, stats);
    return ABFS_OK;
}

extern "C" int abfs_run_host(abfs_graph_t g, uint32_t source, int32_t* level_host,
                             int32_t* parent_host, abfs_stream_t stream, const abfs_params* params,
                             abfs_stats* stats) {
    if (!g || !level_host || !parent_host || source >= g->n) return ABFS_ERR_INVALID_ARG;
    abfs_params tmp;
    const abfs_params& p = pick_params(g, params, tmp);
    int rc = check_params(p);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g->mu);
    if (!g->d_level) {
        rc = dev_alloc((void**)&g->d_level, (size_t)g->n * 4);
        if (!rc) rc = dev_alloc((void**)&g->d_parent, (size_t)g->n * 4);
        if (rc) return rc;
    }
    rc = enqueue_single(g, source, g->d_level, g->d_parent, s, p);
    if (rc) return rc;
    CK(cudaMemcpyAsync(level_host, g->d_level, (size_t)g->n * 4, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(parent_host, g->d_parent, (size_t)g->n * 4, cudaMemcpyDeviceToHost, s));
    // the call synchronises anyway: it returns the search's own status
    abfs_stats local;
    return finish_stats(g, s, stats ? stats : &local);
}

extern "C" int abfs_run_host_many(abfs_graph_t g, const uint32_t* sources, uint32_t count,
                                  int32_t* level_host, int32_t* parent_host, abfs_stream_t stream,
                                  const abfs_params* params, int32_t* status) {
    if (!g || (count && (!sources || !level_host || !parent_host))) return ABFS_ERR_INVALID_ARG;
    for (uint32_t i = 0; i < count; ++i)
        if (sources[i] >= g->n) return ABFS_ERR_INVALID_ARG;
    if (count == 0) return ABFS_OK;
    abfs_params tmp;
    const abfs_params& p = pick_params(g, params, tmp);
    int rc = check_params(p);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g->mu);
    const size_t nb = (size_t)g->n * 4;
    if (!g->d_level) {
        rc = dev_alloc((void**)&g->d_level, nb);
        if (!rc) rc = dev_alloc((void**)&g->d_parent, nb);
        if (rc) return rc;
    }
    if (!g->d_level2) {
        rc = dev_alloc((void**)&g->d_level2, nb);
        if (!rc) rc = dev_alloc((void**)&g->d_parent2, nb);
        if (rc) return rc;
    }
    if (!g->copy_stream) {
        CK(cudaStreamCreateWithFlags(&g->copy_stream, cudaStreamNonBlocking));
        for (int b = 0; b < 2; ++b) {
            CK(cudaEventCreateWithFlags(&g->computed[b], cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&g->copied[b], cudaEventDisableTiming));
        }
    }
    if (g->h_status_cap < count) {
        if (g->h_status) cudaFreeHost(g->h_status);
        g->h_status = nullptr;
        g->h_status_cap = 0;
        if (cudaMallocHost((void**)&g->h_status, (size_t)count * 8) != cudaSuccess) {
            cudaGetLastError();
            return ABFS_ERR_OOM;
        }
        g->h_status_cap = count;
    }
    int32_t* const dl[2] = {g->d_level, g->d_level2};
    int32_t* const dp[2] = {g->d_parent, g->d_parent2};
    cudaStream_t c = g->copy_stream;
    // search i writes buffer pair i & 1; its outputs leave on the copy stream
    // while search i + 1 runs, and search i + 2 waits until they have left
    for (uint32_t i = 0; i < count; ++i) {
        const int b = (int)(i & 1u);
        if (i >= 2) CK(cudaStreamWaitEvent(s, g->copied[b], 0));
        rc = enqueue_single(g, sources[i], dl[b], dp[b], s, p);
        if (rc) break;
        const char* ctl = g->ws.base + g->ws.L.ctl;
        CK(cudaMemcpyAsync(g->h_status + 2 * (size_t)i, ctl + offsetof(InstCtl, status), 8,
                           cudaMemcpyDeviceToHost, s));
        CK(cudaEventRecord(g->computed[b], s));
        CK(cudaStreamWaitEvent(c, g->computed[b], 0));
        CK(cudaMemcpyAsync(level_host + (size_t)i * g->n, dl[b], nb, cudaMemcpyDeviceToHost, c));
        CK(cudaMemcpyAsync(parent_host + (size_t)i * g->n, dp[b], nb, cudaMemcpyDeviceToHost, c));
        CK(cudaEventRecord(g->copied[b], c));
    }
    CK(cudaStreamSynchronize(c));
    CK(cudaStreamSynchronize(s));
    if (rc) return rc;
    int first = ABFS_OK;
    for (uint32_t i = 0; i < count; ++i) {
        const uint32_t st = g->h_status[2 * (size_t)i], err = g->h_status[2 * (size_t)i + 1];
        const int v = (st == kDone) ? ABFS_OK : (err ? (int)err : ABFS_ERR_DEVICE);
        if (status) status[i] = v;
        if (v && !first) first = v;
    }
    return first;
}

extern "C" int abfs_run_trace(abfs_graph_t g, uint32_t source, int32_t* level, int32_t* parent,
                              abfs_stream_t stream, const abfs_params* params, uint32_t* trace_host,
                              uint32_t cap, uint32_t* count) {
    if (!g || !level || !parent || source >= g->n || !trace_host || !count || cap == 0)
        return ABFS_ERR_INVALID_ARG;
    abfs_params tmp;
    const abfs_params& p = pick_params(g, params, tmp);
    int rc = check_params(p);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    uint4* d_trace = nullptr;
    rc = dev_alloc((void**)&d_trace, (size_t)cap * 2 * sizeof(uint4) + kProfSlots * 8);
    if (rc) return rc;
    unsigned long long* d_prof =
        reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(d_trace) + (size_t)cap * 32);
    std::lock_guard<std::mutex> lk(g->mu);
    if (cudaMemsetAsync(d_prof, 0, kProfSlots * 8, s) != cudaSuccess) {
        dev_free(d_trace);
        return ABFS_ERR_CUDA;
    }
    // the last kProfEntries entries carry the CTA cycle accounting (kind 0xFD):
    // a header of 4 words, then kProfSlots 64-bit totals
    constexpr uint32_t kProfEntries = (4 + 2 * kProfSlots + 7) / 8;
    const uint32_t tcap = cap > kProfEntries ? cap - kProfEntries : 0;
    rc = enqueue_single(g, source, level, parent, s, p, d_trace, tcap, d_prof);
    if (!rc) {
        abfs_stats st;
        rc = finish_stats(g, s, &st);
        const uint32_t n = std::min(g->ws.h_ctl->trace_n, tcap);
        if (cudaMemcpy(trace_host, d_trace, (size_t)n * 2 * sizeof(uint4), cudaMemcpyDeviceToHost) !=
            cudaSuccess)
            rc = ABFS_ERR_CUDA;
        unsigned long long prof[kProfSlots];
        if (cudaMemcpy(prof, d_prof, sizeof(prof), cudaMemcpyDeviceToHost) != cudaSuccess)
            rc = ABFS_ERR_CUDA;
        uint32_t* out = trace_host + (size_t)n * 8;
        if (cap <= kProfEntries) out = nullptr;
        if (out) {
        out[0] = 0;
        out[1] = 0;
        out[2] = 0xFDu << 24;
        out[3] = 0;
        for (int q = 0; q < kProfSlots; ++q) {
            out[4 + 2 * q] = (uint32_t)prof[q];
            out[5 + 2 * q] = (uint32_t)(prof[q] >> 32);
        }
        for (uint32_t q = 4 + 2 * kProfSlots; q < 8 * kProfEntries; ++q) out[q] = 0;
        }
        *count = (cap > kProfEntries) ? n + kProfEntries : n;
        // the workspace descriptor keeps no pointer to the freed trace buffer
        launch_set_query(g->ws.d_inst, 0, nullptr, nullptr, nullptr, 0u, nullptr, 0, s);
        cudaStreamSynchronize(s);
    }
    dev_free(d_trace);
    return rc;
}

// ---------------------------------------------------------------------------
// batches
// ---------------------------------------------------------------------------

struct abfs_batch_s {
    std::vector<abfs_graph_t> graphs;
    uint32_t count = 0;
    abfs_params p{};
    char* ws = nullptr;          // all per-instance workspaces
    Inst* d_insts = nullptr;
    uint32_t* d_done = nullptr;
    unsigned long long* d_beat = nullptr;
    std::vector<size_t> ctl_off; // offset of each search instance's InstCtl in ws
    std::vector<uint32_t> qinst; // query -> the search instance that answers it
    uint32_t ninst = 0;          // search instances (a multi-source search answers several queries)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    InstCtl* h_ctl = nullptr;    // pinned, ninst entries
};

extern "C" int abfs_batch_destroy(abfs_batch_t b) {
    if (!b) return ABFS_ERR_INVALID_ARG;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    dev_free(b->ws);
    dev_free(b->d_insts);
    dev_free(b->d_done);
    dev_free(b->d_beat);
    if (b->h_ctl) cudaFreeHost(b->h_ctl);
    delete b;
    return ABFS_OK;
}

namespace {
// Shared by abfs_batch_create and abfs_batch_create_counts (sigma == NULL: no counts).
int batch_create(const abfs_graph_t* g, const uint32_t* sources, uint32_t count,
                 int32_t* const* level, int32_t* const* parent, uint64_t* const* sigma,
                 const abfs_params* params, abfs_batch_t* out) {
    if (!g || !sources || !level || !parent || !out || count == 0) return ABFS_ERR_INVALID_ARG;
    *out = nullptr;
    abfs_params tmp;
    const abfs_params& p = pick_params(g[0], params, tmp);
    int rc = check_params(p);
    if (rc) return rc;
    if (sigma && p.mode != ABFS_MODE_SUBMATRIX) return ABFS_ERR_UNSUPPORTED;
    for (uint32_t i = 0; i < count; ++i) {
        if (!g[i] || !level[i] || !parent[i] || sources[i] >= g[i]->n) return ABFS_ERR_INVALID_ARG;
        if (sigma && !sigma[i]) return ABFS_ERR_INVALID_ARG;
        if (g[i]->device != g[0]->device) return ABFS_ERR_INVALID_ARG;
    }
    abfs_batch_s* b = new (std::nothrow) abfs_batch_s();
    if (!b) return ABFS_ERR_OOM;
    b->graphs.assign(g, g + count);
    b->count = count;
    b->p = p;
    // search instances: the queries on one undirected graph run as multi-source
    // searches of up to kMsMax sources when there are at least p.multi_source of
    // them (submatrix mode, no path counts); every other query runs alone
    struct Search {
        uint32_t gi;                  // a query on the instance's graph
        std::vector<uint32_t> q;      // its queries (one unless multi-source)
    };
    std::vector<Search> inst;
    b->qinst.assign(count, 0);
    {
        std::vector<char> done(count, 0);
        const bool group = p.multi_source >= 1 && p.mode == ABFS_MODE_SUBMATRIX && !sigma;
        for (uint32_t i = 0; i < count; ++i) {
            if (done[i]) continue;
            std::vector<uint32_t> same;
            // the parent rule of multi-source searches scans a vertex's column
            // (= its in-neighbours) in ascending order: undirected, sorted graphs
            if (group && !g[i]->directed && g[i]->sorted)
                for (uint32_t j = i; j < count; ++j)
                    if (!done[j] && g[j] == g[i]) same.push_back(j);
            if (same.size() >= std::max<uint32_t>(p.multi_source, 2u)) {
                for (size_t c0 = 0; c0 < same.size(); c0 += kMsMax) {
                    Search m;
                    m.gi = i;
                    for (size_t c = c0; c < std::min(same.size(), c0 + kMsMax); ++c) {
                        m.q.push_back(same[c]);
                        done[same[c]] = 1;
                    }
                    inst.push_back(m);
                }
            } else {
                Search one;
                one.gi = i;
                one.q.push_back(i);
                done[i] = 1;
                inst.push_back(one);
            }
        }
    }
    const uint32_t ninst = (uint32_t)inst.size();
    b->ninst = ninst;
    std::vector<Layout> L(ninst);
    std::vector<size_t> base(ninst);
    size_t total = 0;
    uint32_t max_n = 0;
    for (uint32_t t = 0; t < ninst; ++t) {
        const abfs_graph_s* gt = g[inst[t].gi];
        const uint32_t ms = inst[t].q.size() > 1 ? (uint32_t)inst[t].q.size() : 0u;
        L[t] = layout_for(gt->n, gt->nnz, p, ms);
        base[t] = total;
        total = align_up(total + L[t].total, 256);
        max_n = std::max(max_n, gt->n);
    }
    rc = dev_alloc((void**)&b->ws, total);
    if (!rc) rc = dev_alloc((void**)&b->d_insts, sizeof(Inst) * ninst);
    if (!rc) rc = dev_alloc((void**)&b->d_done, 64);
    if (!rc) rc = dev_alloc((void**)&b->d_beat, 64);
    if (rc) {
        abfs_batch_destroy(b);
        return rc;
    }
    if (cudaMallocHost((void**)&b->h_ctl, sizeof(InstCtl) * ninst) != cudaSuccess) {
        cudaGetLastError();
        abfs_batch_destroy(b);
        return ABFS_ERR_OOM;
    }
    std::vector<Inst> hI(ninst);
    b->ctl_off.resize(ninst);
    for (uint32_t t = 0; t < ninst; ++t) {
        const Search& m = inst[t];
        const abfs_graph_s* gt = g[m.gi];
        char* wb = b->ws + base[t];
        for (uint32_t q : m.q) b->qinst[q] = t;
        if (m.q.size() == 1) {
            const uint32_t q = m.q[0];
            hI[t] = make_inst(gt, wb, L[t], sources[q], level[q], parent[q]);
            if (sigma) {
                // path counts: every multiplied entry contributes, so the search stays top-down
                hI[t].sigma = reinterpret_cast<unsigned long long*>(sigma[q]);
                hI[t].bu_ok = 0;
            }
        } else {
            // multi-source: the sources and the outputs' pointers go to the workspace
            const uint32_t ms = (uint32_t)m.q.size();
            std::vector<uint32_t> src(ms);
            std::vector<int32_t*> lv(ms), pv(ms);
            for (uint32_t s2 = 0; s2 < ms; ++s2) {
                src[s2] = sources[m.q[s2]];
                lv[s2] = level[m.q[s2]];
                pv[s2] = parent[m.q[s2]];
            }
            cudaError_t ce = cudaMemcpy(wb + L[t].ms_src, src.data(), 4 * ms, cudaMemcpyHostToDevice);
            if (ce == cudaSuccess)
                ce = cudaMemcpy(wb + L[t].ms_lev, lv.data(), 8 * ms, cudaMemcpyHostToDevice);
            if (ce == cudaSuccess)
                ce = cudaMemcpy(wb + L[t].ms_par, pv.data(), 8 * ms, cudaMemcpyHostToDevice);
            if (ce != cudaSuccess) {
                abfs_batch_destroy(b);
                return cuda_fail(ce);
            }
            hI[t] = make_inst(gt, wb, L[t], src[0], nullptr, nullptr);
            hI[t].bu_ok = 0;
            hI[t].ms = ms;
            hI[t].ms_sorted = gt->sorted ? 1u : 0u;
            hI[t].ms_vis = reinterpret_cast<unsigned long long*>(wb + L[t].ms_vis);
            for (int i2 = 0; i2 < 2; ++i2)
                hI[t].ms_fr[i2] = reinterpret_cast<unsigned long long*>(wb + L[t].ms_fr[i2]);
            hI[t].ms_nx = reinterpret_cast<unsigned long long*>(wb + L[t].ms_nx);
            hI[t].ms_src = reinterpret_cast<const uint32_t*>(wb + L[t].ms_src);
            hI[t].ms_level = reinterpret_cast<int32_t* const*>(wb + L[t].ms_lev);
            hI[t].ms_parent = reinterpret_cast<int32_t* const*>(wb + L[t].ms_par);
        }
        b->ctl_off[t] = base[t] + L[t].ctl;
    }
    cudaError_t e = cudaMemcpy(b->d_insts, hI.data(), sizeof(Inst) * ninst, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        abfs_batch_destroy(b);
        return cuda_fail(e);
    }
    // capture initialisation + the persistent launch in a CUDA graph
    cudaStream_t cap;
    e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        abfs_batch_destroy(b);
        return cuda_fail(e);
    }
    EngineArgs a;
    a.insts = b->d_insts;
    a.ninst = ninst;
    a.done_count = b->d_done;
    a.heartbeat = b->d_beat;
    a.prof = nullptr;
    a.serve = 0;
    a.slot_state = nullptr;
    a.stop_flag = nullptr;
    a.idle_exit_ns = 0;
    a.p = engine_params(p);
    a.hold_units = test_hold_units();
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t e1 = launch_init(a, max_n, cap);
        cudaError_t e2 = launch_engine(a, grid_size(g[0], p, 0), cap);
        e = cudaStreamEndCapture(cap, &b->graph);
        if (e == cudaSuccess) e = (e1 != cudaSuccess) ? e1 : e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) {
        abfs_batch_destroy(b);
        return cuda_fail(e);
    }
    *out = b;
    return ABFS_OK;
}
}  // namespace

extern "C" int abfs_batch_create(const abfs_graph_t* g, const uint32_t* sources, uint32_t count,
                                 int32_t* const* level, int32_t* const* parent,
                                 const abfs_params* params, abfs_stream_t stream,
                                 abfs_batch_t* out) {
    (void)stream;
    return batch_create(g, sources, count, level, parent, nullptr, params, out);
}

extern "C" int abfs_batch_create_counts(const abfs_graph_t* g, const uint32_t* sources,
                                        uint32_t count, int32_t* const* level,
                                        int32_t* const* parent, uint64_t* const* sigma,
                                        const abfs_params* params, abfs_stream_t stream,
                                        abfs_batch_t* out) {
    (void)stream;
    if (!sigma) return ABFS_ERR_INVALID_ARG;
    return batch_create(g, sources, count, level, parent, sigma, params, out);
}

extern "C" int abfs_batch_launch(abfs_batch_t b, abfs_stream_t stream) {
    if (!b) return ABFS_ERR_INVALID_ARG;
    CK(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
    return ABFS_OK;
}

extern "C" int abfs_batch_status(abfs_batch_t b, abfs_stream_t stream, int32_t* status) {
    if (!b || !status) return ABFS_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    for (uint32_t i = 0; i < b->ninst; ++i)
        CK(cudaMemcpyAsync(b->h_ctl + i, b->ws + b->ctl_off[i], sizeof(InstCtl),
                           cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    int worst = ABFS_OK;
    for (uint32_t i = 0; i < b->count; ++i) {
        const InstCtl& c = b->h_ctl[b->qinst[i]];
        status[i] = (c.status == kDone) ? ABFS_OK : (c.err ? (int)c.err : ABFS_ERR_DEVICE);
        if (status[i] && !worst) worst = status[i];
    }
    return worst;
}

extern "C" int abfs_run_batch(const abfs_graph_t* g, const uint32_t* sources, uint32_t count,
                              int32_t* const* level, int32_t* const* parent, abfs_stream_t stream,
                              const abfs_params* params, int32_t* status_per_query) {
    abfs_batch_t b = nullptr;
    int rc = abfs_batch_create(g, sources, count, level, parent, params, stream, &b);
    if (rc) return rc;
    rc = abfs_batch_launch(b, stream);
    std::vector<int32_t> st(count);
    int rc2 = abfs_batch_status(b, stream, st.data());
    if (status_per_query) std::copy(st.begin(), st.end(), status_per_query);
    abfs_batch_destroy(b);
    return rc ? rc : rc2;
}

// ---------------------------------------------------------------------------
// autotuner
// ---------------------------------------------------------------------------

namespace {

std::string size_class(const abfs_graph_s* g) {
    const int lgn = (int)std::ceil(std::log2((double)g->n + 1));
    const double deg = (double)g->nnz / std::max<uint32_t>(g->n, 1);
    const int lgd = (int)std::floor(std::log2(deg + 1.0));
    std::ostringstream o;
    o << "n2^" << lgn << "_d2^" << lgd << (g->directed ? "_dir" : "_und");
    return o.str();
}

std::string gpu_name(int dev) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "unknown";
    std::string s = prop.name;
    for (char& c : s)
        if (c == ' ' || c == '"') c = '_';
    return s;
}

std::string params_json(const abfs_params& p) {
    std::ostringstream o;
    o << "\"mode\":" << p.mode << ",\"tile\":" << p.tile << ",\"unit_entries\":" << p.unit_entries
      << ",\"narrow_max\":" << p.narrow_max
      << ",\"narrow_edges\":" << p.narrow_edges
      << ",\"ctas_per_sm\":" << p.ctas_per_sm << ",\"shrink_theta\":" << p.shrink_theta
      << ",\"shrink_max\":" << p.shrink_max << ",\"narrow_resident\":" << p.narrow_resident
      << ",\"claim_scan\":" << p.claim_scan << ",\"cluster_ctas\":" << p.cluster_ctas;
    return o.str();
}

bool json_num(const std::string& line, const std::string& key, double* v) {
    const std::string k = "\"" + key + "\":";
    size_t at = line.find(k);
    if (at == std::string::npos) return false;
    *v = std::strtod(line.c_str() + at + k.size(), nullptr);
    return true;
}

bool json_str(const std::string& line, const std::string& key, std::string* v) {
    const std::string k = "\"" + key + "\":\"";
    size_t at = line.find(k);
    if (at == std::string::npos) return false;
    size_t end = line.find('"', at + k.size());
    if (end == std::string::npos) return false;
    *v = line.substr(at + k.size(), end - at - k.size());
    return true;
}

}  // namespace

extern "C" int abfs_tune(abfs_graph_t g, const uint32_t* sources, uint32_t count, uint32_t mode,
                         const char* cache_path, abfs_stream_t stream, abfs_params* best,
                         float* best_ms) {
    if (!g || !sources || count == 0 || mode > ABFS_MODE_PLAIN) return ABFS_ERR_INVALID_ARG;
    for (uint32_t i = 0; i < count; ++i)
        if (sources[i] >= g->n) return ABFS_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const std::string key_gpu = gpu_name(g->device);
    const std::string key_cls = size_class(g);
    // cache lookup: JSON lines {"gpu":..,"sms":..,"mode":..,"class":..,<params>,"ms":..}
    if (cache_path) {
        std::ifstream in(cache_path);
        std::string line, found;
        while (std::getline(in, line)) {
            std::string gpu, cls;
            double sms = 0, md = -1;
            if (json_str(line, "gpu", &gpu) && json_str(line, "class", &cls) &&
                json_num(line, "sms", &sms) && json_num(line, "mode", &md) && gpu == key_gpu &&
                cls == key_cls && (int)sms == g->sms && (uint32_t)md == mode)
                found = line;
        }
        if (!found.empty()) {
            abfs_params p = default_params();
            double v;
            if (json_num(found, "tile", &v)) p.tile = (uint32_t)v;
            if (json_num(found, "unit_entries", &v)) p.unit_entries = (uint32_t)v;
            if (json_num(found, "narrow_max", &v)) p.narrow_max = (uint32_t)v;
            if (json_num(found, "narrow_edges", &v)) p.narrow_edges = (uint32_t)v;
            if (json_num(found, "ctas_per_sm", &v)) p.ctas_per_sm = (uint32_t)v;
            if (json_num(found, "shrink_theta", &v)) p.shrink_theta = (float)v;
            if (json_num(found, "shrink_max", &v)) p.shrink_max = (uint32_t)v;
            if (json_num(found, "narrow_resident", &v)) p.narrow_resident = (uint32_t)v;
            if (json_num(found, "claim_scan", &v)) p.claim_scan = (uint32_t)v;
            if (json_num(found, "cluster_ctas", &v)) p.cluster_ctas = (uint32_t)v;
            p.mode = mode;
            if (check_params(p) == ABFS_OK) {
                std::lock_guard<std::mutex> lk(g->mu);
                if (mode == ABFS_MODE_SUBMATRIX) {
                    g->tuned = true;
                    g->tuned_params = p;
                }
                if (best) *best = p;
                if (best_ms && json_num(found, "ms", &v)) *best_ms = (float)v;
                return ABFS_OK;
            }
        }
    }
    // candidate sets
    std::vector<abfs_params> cands;
    const uint32_t units[] = {512, 1024, 4096};
    const uint32_t narrow_e[] = {0, 16384, 65536};
    const uint32_t ctas[] = {1, 2};
    for (uint32_t ue : units)
        for (uint32_t ne : narrow_e)
            for (uint32_t cp : ctas) {
                abfs_params p = default_params();
                p.mode = mode;
                p.unit_entries = ue;
                p.narrow_edges = ne;
                p.narrow_max = ne ? ne / 8 : 0;
                p.ctas_per_sm = cp;
                cands.push_back(p);
            }
    // cluster runs of other sizes, and none; 16-CTA clusters with one CTA per
    // SM, so that a run's CTAs sit on 16 SMs (faster on grids and geometric
    // graphs, whose levels are all cluster runs)
    for (uint32_t cc : {1u, 4u, 16u}) {
        abfs_params p = default_params();
        p.mode = mode;
        p.cluster_ctas = cc;
        if (cc == 16) p.ctas_per_sm = 1;
        cands.push_back(p);
    }
    if (mode == ABFS_MODE_SUBMATRIX) {
        const float thetas[] = {0.5f, 0.8f, 0.95f};
        for (float th : thetas) {
            abfs_params p = default_params();
            p.mode = mode;
            p.shrink_theta = th;
            p.shrink_max = 1;
            cands.push_back(p);
        }
    }
    int32_t *d_level = nullptr, *d_parent = nullptr;
    int rc = dev_alloc((void**)&d_level, (size_t)g->n * 4);
    if (!rc) rc = dev_alloc((void**)&d_parent, (size_t)g->n * 4);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (!rc && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        rc = ABFS_ERR_CUDA;
    float best_time = INFINITY;
    abfs_params best_p = default_params();
    best_p.mode = mode;
    for (size_t ci = 0; ci < cands.size() && !rc; ++ci) {
        const abfs_params& p = cands[ci];
        std::lock_guard<std::mutex> lk(g->mu);
        // warm-up (also allocates the workspace)
        rc = enqueue_single(g, sources[0], d_level, d_parent, s, p);
        if (rc) break;
        if (cudaEventRecord(e0, s) != cudaSuccess) { rc = ABFS_ERR_CUDA; break; }
        for (uint32_t i = 0; i < count && !rc; ++i)
            rc = enqueue_single(g, sources[i], d_level, d_parent, s, p);
        if (rc) break;
        if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
            rc = ABFS_ERR_CUDA;
            break;
        }
        abfs_stats st;
        rc = finish_stats(g, s, &st);
        if (rc) break;
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= count;
        if (ms < best_time) {
            best_time = ms;
            best_p = p;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    dev_free(d_level);
    dev_free(d_parent);
    if (rc) return rc;
    {
        std::lock_guard<std::mutex> lk(g->mu);
        if (mode == ABFS_MODE_SUBMATRIX) {
            g->tuned = true;
            g->tuned_params = best_p;
        }
    }
    if (best) *best = best_p;
    if (best_ms) *best_ms = best_time;
    if (cache_path) {
        std::ofstream o(cache_path, std::ios::app);
        o << "{\"gpu\":\"" << key_gpu << "\",\"sms\":" << g->sms << ",\"class\":\"" << key_cls
          << "\"," << params_json(best_p) << ",\"ms\":" << best_time << "}\n";
    }
    return ABFS_OK;
}

// ---------------------------------------------------------------------------
// allocator hook
// ---------------------------------------------------------------------------

extern "C" int abfs_set_allocator(void* (*alloc)(size_t, void*), void (*free_fn)(void*, void*),
                                  void* ctx) {
    if ((alloc == nullptr) != (free_fn == nullptr)) return ABFS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc.alloc = alloc;
    g_alloc.free = free_fn;
    g_alloc.ctx = ctx;
    return ABFS_OK;
}

extern "C" const char* abfs_last_cuda_error(void) { return g_last_cuda_error.c_str(); }

// ---------------------------------------------------------------------------
// test control: a first phase that never completes
// ---------------------------------------------------------------------------

namespace {
std::atomic<uint32_t> g_hold_units{0};
}  // namespace

namespace abfs {
uint32_t test_hold_units() { return g_hold_units.load(std::memory_order_relaxed); }
}  // namespace abfs

extern "C" int abfs_test_hold_first_phase(uint32_t extra_units) {
    g_hold_units.store(extra_units, std::memory_order_relaxed);
    return ABFS_OK;
}

// ---------------------------------------------------------------------------
// batch autotuner
// ---------------------------------------------------------------------------

namespace {

std::string batch_class(const abfs_graph_t* g, uint32_t count) {
    double n = 0, nnz = 0;
    for (uint32_t i = 0; i < count; ++i) {
        n += g[i]->n;
        nnz += (double)g[i]->nnz;
    }
    std::ostringstream o;
    o << "batch" << count << "_n2^" << (int)std::ceil(std::log2(n + 1)) << "_e2^"
      << (int)std::ceil(std::log2(nnz + 1));
    return o.str();
}

}  // namespace

extern "C" int abfs_batch_tune(const abfs_graph_t* g, const uint32_t* sources, uint32_t count,
                               uint32_t mode, const char* cache_path, abfs_stream_t stream,
                               abfs_params* best, float* best_ms) {
    if (!g || !sources || count == 0 || mode > ABFS_MODE_PLAIN) return ABFS_ERR_INVALID_ARG;
    for (uint32_t i = 0; i < count; ++i)
        if (!g[i] || sources[i] >= g[i]->n) return ABFS_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const std::string key_gpu = gpu_name(g[0]->device);
    const std::string key_cls = batch_class(g, count);
    if (cache_path) {
        std::ifstream in(cache_path);
        std::string line, found;
        while (std::getline(in, line)) {
            std::string gpu, cls;
            double sms = 0, md = -1;
            if (json_str(line, "gpu", &gpu) && json_str(line, "class", &cls) &&
                json_num(line, "sms", &sms) && json_num(line, "mode", &md) && gpu == key_gpu &&
                cls == key_cls && (int)sms == g[0]->sms && (uint32_t)md == mode)
                found = line;
        }
        if (!found.empty()) {
            abfs_params p = default_params();
            double v;
            if (json_num(found, "tile", &v)) p.tile = (uint32_t)v;
            if (json_num(found, "unit_entries", &v)) p.unit_entries = (uint32_t)v;
            if (json_num(found, "narrow_max", &v)) p.narrow_max = (uint32_t)v;
            if (json_num(found, "narrow_edges", &v)) p.narrow_edges = (uint32_t)v;
            if (json_num(found, "ctas_per_sm", &v)) p.ctas_per_sm = (uint32_t)v;
            if (json_num(found, "shrink_theta", &v)) p.shrink_theta = (float)v;
            if (json_num(found, "shrink_max", &v)) p.shrink_max = (uint32_t)v;
            if (json_num(found, "narrow_resident", &v)) p.narrow_resident = (uint32_t)v;
            if (json_num(found, "claim_scan", &v)) p.claim_scan = (uint32_t)v;
            if (json_num(found, "cluster_ctas", &v)) p.cluster_ctas = (uint32_t)v;
            p.mode = mode;
            if (check_params(p) == ABFS_OK) {
                if (best) *best = p;
                if (best_ms && json_num(found, "ms", &v)) *best_ms = (float)v;
                return ABFS_OK;
            }
        }
    }
    // candidates: granule x narrow bounds (x reduction claims), plus shrink thresholds
    std::vector<abfs_params> cands;
    const uint32_t granules[] = {512, 1024, 4096};
    const uint32_t narrow_e[] = {16384, 65536};
    const uint32_t scans[] = {0, 1u << 22};
    // with cluster runs (default cluster size) and without (single-CTA narrow runs)
    const uint32_t clusters[] = {default_params().cluster_ctas, 1u};
    for (uint32_t ue : granules)
        for (uint32_t ne : narrow_e)
            for (uint32_t sc : scans)
                for (uint32_t cc : clusters) {
                    if (mode == ABFS_MODE_PLAIN && sc) continue;
                    abfs_params p = default_params();
                    p.mode = mode;
                    p.unit_entries = ue;
                    p.narrow_edges = ne;
                    p.narrow_max = ne / 16;
                    p.claim_scan = sc;
                    p.cluster_ctas = cc;
                    cands.push_back(p);
                }
    if (mode == ABFS_MODE_SUBMATRIX) {
        const float thetas[] = {0.5f, 0.8f};
        for (float th : thetas) {
            abfs_params p = default_params();
            p.shrink_theta = th;
            p.shrink_max = 1;
            cands.push_back(p);
        }
    }
    // outputs for the trial plans
    std::vector<int32_t*> lv(count, nullptr), pr(count, nullptr);
    int rc = ABFS_OK;
    for (uint32_t i = 0; i < count && !rc; ++i) {
        rc = dev_alloc((void**)&lv[i], (size_t)g[i]->n * 4);
        if (!rc) rc = dev_alloc((void**)&pr[i], (size_t)g[i]->n * 4);
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (!rc && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        rc = ABFS_ERR_CUDA;
    float best_time = INFINITY;
    abfs_params best_p = default_params();
    best_p.mode = mode;
    std::vector<int32_t> st(count);
    for (size_t ci = 0; ci < cands.size() && !rc; ++ci) {
        abfs_batch_t b = nullptr;
        rc = abfs_batch_create(g, sources, count, lv.data(), pr.data(), &cands[ci], stream, &b);
        if (rc) break;
        const int reps = 2;
        rc = abfs_batch_launch(b, stream);  // warm-up
        if (!rc && cudaEventRecord(e0, s) != cudaSuccess) rc = ABFS_ERR_CUDA;
        for (int r = 0; r < reps && !rc; ++r) rc = abfs_batch_launch(b, stream);
        if (!rc && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
            rc = ABFS_ERR_CUDA;
        if (!rc) rc = abfs_batch_status(b, stream, st.data());
        bool ok = !rc;
        for (uint32_t i = 0; i < count && ok; ++i) ok = st[i] == ABFS_OK;
        float ms = 0;
        if (ok) {
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= reps;
            if (ms < best_time) {
                best_time = ms;
                best_p = cands[ci];
            }
        }
        const int rd = abfs_batch_destroy(b);
        if (!rc) rc = rd;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    for (uint32_t i = 0; i < count; ++i) {
        dev_free(lv[i]);
        dev_free(pr[i]);
    }
    if (rc) return rc;
    if (!(best_time < INFINITY)) return ABFS_ERR_DEVICE;
    if (best) *best = best_p;
    if (best_ms) *best_ms = best_time;
    if (cache_path) {
        std::ofstream o(cache_path, std::ios::app);
        o << "{\"gpu\":\"" << key_gpu << "\",\"sms\":" << g[0]->sms << ",\"class\":\"" << key_cls
          << "\"," << params_json(best_p) << ",\"ms\":" << best_time << "}\n";
    }
    return ABFS_OK;
}
