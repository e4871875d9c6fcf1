// Serving: continuous batching of BFS queries over device-resident graphs.
//
// A host admission thread moves queued requests into free device slots as
// soon as a slot and enough workspace memory are free; the long-lived engine
// launch (serve mode) picks up newly submitted slots between work units, so
// requests that arrive while others run are admitted at once and their work
// overlaps on the device.  Completion reaches the host through a host-mapped
// word per slot (ticket << 8 | status); latency is measured submit -> done on
// the host's steady clock.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/abfs.h"
#include "internal.h"

using namespace abfs;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket;
    uint32_t g;
    uint32_t src;
    int32_t* level;
    int32_t* parent;
    Clock::time_point t0;
};

struct Slot {
    bool busy = false;
    Request req{};
    size_t off = 0;
    size_t bytes = 0;
};

// First-fit allocator over the workspace budget [0, size), coalescing on free.
class Arena {
  public:
    void init(size_t size) {
        free_.clear();
        if (size) free_[0] = size;
    }
    bool alloc(size_t bytes, size_t* off) {
        bytes = (bytes + 255) / 256 * 256;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                const size_t o = it->first, rem = it->second - bytes;
                free_.erase(it);
                if (rem) free_[o + bytes] = rem;
                *off = o;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = (bytes + 255) / 256 * 256;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }

  private:
    std::map<size_t, size_t> free_;
};

}  // namespace

struct abfs_server_s {
    std::vector<abfs_graph_t> graphs;
    std::vector<Layout> layouts;
    abfs_serve_cfg cfg{};
    int device = 0, sms = 0;
    // device
    Inst* d_slots = nullptr;
    InstCtl* d_ctl = nullptr;
    uint32_t* d_state = nullptr;
    uint32_t* d_stop = nullptr;
    uint32_t* d_done = nullptr;
    unsigned long long* d_beat = nullptr;
    char* d_arena = nullptr;
    // host (pinned / mapped)
    unsigned long long* h_notify = nullptr;
    unsigned long long* d_notify = nullptr;
    Inst* h_stage = nullptr;
    uint32_t* h_words = nullptr;  // [0] = kSlotSubmitted, [1] = 1 (stop)
    cudaStream_t kstream = nullptr, cstream = nullptr;
    // bookkeeping
    std::mutex mu;
    std::condition_variable cv_done;
    std::deque<Request> pending;
    std::vector<Slot> slots;
    Arena arena;
    std::unordered_map<uint64_t, int32_t> done_status;
    std::vector<double> lat_ms;
    uint64_t next_ticket = 1, submitted = 0, completed = 0, failed = 0, launches = 0;
    std::atomic<bool> stopping{false};
    std::thread th;
    Clock::time_point t_start;
    int fatal = 0;
};

namespace {

void release_server(abfs_server_s* S) {
    if (S->kstream) cudaStreamDestroy(S->kstream);
    if (S->cstream) cudaStreamDestroy(S->cstream);
    cudaFree(S->d_slots);
    cudaFree(S->d_ctl);
    cudaFree(S->d_state);
    cudaFree(S->d_stop);
    cudaFree(S->d_done);
    cudaFree(S->d_beat);
    cudaFree(S->d_arena);
    if (S->h_notify) cudaFreeHost(S->h_notify);
    if (S->h_stage) cudaFreeHost(S->h_stage);
    if (S->h_words) cudaFreeHost(S->h_words);
    delete S;
}

EngineArgs serve_args(abfs_server_s* S) {
    EngineArgs a;
    a.insts = S->d_slots;
    a.ninst = S->cfg.max_slots;
    a.done_count = S->d_done;
    a.heartbeat = S->d_beat;
    a.prof = nullptr;
    a.serve = 1;
    a.slot_state = S->d_state;
    a.stop_flag = S->d_stop;
    a.idle_exit_ns = (unsigned long long)S->cfg.idle_exit_ms * 1000000ull;
    a.p = engine_params(S->cfg.params);
    return a;
}

// The admission thread.
void serve_loop(abfs_server_s* S) {
    cudaSetDevice(S->device);
    const uint32_t nslots = S->cfg.max_slots;
    bool launched = false;
    for (;;) {
        bool progress = false;
        // 1. completions: the mapped word of a busy slot shows its ticket
        for (uint32_t i = 0; i < nslots; ++i) {
            Slot& sl = S->slots[i];
            if (!sl.busy) continue;
            const unsigned long long w = *reinterpret_cast<volatile unsigned long long*>(S->h_notify + i);
            if ((w >> 8) != sl.req.ticket) continue;
            const int32_t status = (int32_t)(w & 0xFFu);
            const double ms =
                std::chrono::duration<double, std::milli>(Clock::now() - sl.req.t0).count();
            std::lock_guard<std::mutex> lk(S->mu);
            S->done_status[sl.req.ticket] = status;
            S->lat_ms.push_back(ms);
            S->completed += 1;
            if (status) S->failed += 1;
            S->arena.release(sl.off, sl.bytes);
            sl.busy = false;
            progress = true;
        }
        if (progress) S->cv_done.notify_all();
        // 2. admissions: free slot + workspace memory -> the request joins the running launch
        bool any_busy = false;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            uint32_t i = 0;
            while (!S->pending.empty()) {
                while (i < nslots && S->slots[i].busy) ++i;
                if (i >= nslots) break;
                const Request& rq = S->pending.front();
                const Layout& L = S->layouts[rq.g];
                size_t off = 0;
                if (!S->arena.alloc(L.total, &off)) break;
                const uint32_t* cp;
                const uint32_t* ri;
                uint32_t n;
                uint64_t nnz;
                int dev, sms;
                graph_arrays(S->graphs[rq.g], &cp, &ri, &n, &nnz, &dev, &sms);
                Inst I = make_inst_raw(cp, ri, n, S->d_arena + off, L, rq.src, rq.level, rq.parent);
                I.ctl = S->d_ctl + i;  // fixed per slot, so a scan of slot i always reads its own block
                I.slot = i;
                I.ticket = rq.ticket;
                I.notify = S->d_notify + i;
                S->h_stage[i] = I;
                // the descriptor first, then the state word: the device reads the
                // state, then (after an acquire) the descriptor
                cudaError_t e = cudaMemcpyAsync(S->d_slots + i, S->h_stage + i, sizeof(Inst),
                                                cudaMemcpyHostToDevice, S->cstream);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(S->d_state + i, S->h_words, 4, cudaMemcpyHostToDevice,
                                        S->cstream);
                if (e != cudaSuccess) {
                    S->fatal = ABFS_ERR_CUDA;
                    S->arena.release(off, L.total);
                    break;
                }
                Slot& sl = S->slots[i];
                sl.busy = true;
                sl.req = rq;
                sl.off = off;
                sl.bytes = L.total;
                S->pending.pop_front();
                progress = true;
            }
            for (uint32_t q = 0; q < nslots && !any_busy; ++q) any_busy = S->slots[q].busy;
        }
        // 3. the device loop: (re)launch it while queries are on the device
        if (any_busy && !S->fatal) {
            const bool running = launched && cudaStreamQuery(S->kstream) == cudaErrorNotReady;
            if (!running) {
                cudaGetLastError();
                const EngineArgs a = serve_args(S);
                if (launch_engine(a, grid_for(S->sms, S->cfg.params), S->kstream) != cudaSuccess) {
                    S->fatal = ABFS_ERR_CUDA;
                } else {
                    launched = true;
                    std::lock_guard<std::mutex> lk(S->mu);
                    S->launches += 1;
                }
            }
        }
        // 4. exit once stopping and everything has finished
        if (S->stopping.load()) {
            std::lock_guard<std::mutex> lk(S->mu);
            if ((S->pending.empty() && !any_busy) || S->fatal) break;
        }
        if (!progress) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    // end the device loop
    cudaMemcpyAsync(S->d_stop, S->h_words + 1, 4, cudaMemcpyHostToDevice, S->cstream);
    cudaStreamSynchronize(S->cstream);
    cudaStreamSynchronize(S->kstream);
}

}  // namespace

extern "C" int abfs_serve_default_cfg(abfs_serve_cfg* cfg) {
    if (!cfg) return ABFS_ERR_INVALID_ARG;
    cfg->max_slots = 256;
    cfg->queue_capacity = 1u << 20;
    cfg->memory_budget = 16ull << 30;
    cfg->idle_exit_ms = 50;
    cfg->params = default_params();
    return ABFS_OK;
}

extern "C" int abfs_serve_start(const abfs_graph_t* g, uint32_t ngraphs, const abfs_serve_cfg* cfg,
                                abfs_server_t* out) {
    if (!g || !ngraphs || !out) return ABFS_ERR_INVALID_ARG;
    *out = nullptr;
    abfs_serve_cfg c;
    if (cfg) c = *cfg;
    else abfs_serve_default_cfg(&c);
    if (c.max_slots < 1 || c.max_slots > 4096 || c.queue_capacity < 1 || c.idle_exit_ms < 1 ||
        c.idle_exit_ms > 600000)
        return ABFS_ERR_INVALID_ARG;
    if (check_params(c.params) != ABFS_OK || shrink_enabled(c.params)) return ABFS_ERR_INVALID_ARG;
    abfs_server_s* S = new (std::nothrow) abfs_server_s();
    if (!S) return ABFS_ERR_OOM;
    S->cfg = c;
    S->graphs.assign(g, g + ngraphs);
    size_t largest = 0;
    for (uint32_t i = 0; i < ngraphs; ++i) {
        const uint32_t* cp;
        const uint32_t* ri;
        uint32_t n;
        uint64_t nnz;
        int dev, sms;
        if (graph_arrays(g[i], &cp, &ri, &n, &nnz, &dev, &sms) != ABFS_OK) {
            delete S;
            return ABFS_ERR_INVALID_ARG;
        }
        if (i == 0) {
            S->device = dev;
            S->sms = sms;
        } else if (dev != S->device) {
            delete S;
            return ABFS_ERR_INVALID_ARG;
        }
        S->layouts.push_back(layout_for(n, nnz, c.params));
        largest = std::max(largest, S->layouts.back().total);
    }
    if (largest + 256 > c.memory_budget) {
        delete S;
        return ABFS_ERR_OOM;  // the budget cannot hold even the largest graph's query
    }
    const uint32_t ns = c.max_slots;
    cudaError_t e = cudaSuccess;
    auto ck = [&](cudaError_t r) {
        if (e == cudaSuccess) e = r;
    };
    ck(cudaMalloc((void**)&S->d_slots, sizeof(Inst) * ns));
    ck(cudaMalloc((void**)&S->d_ctl, sizeof(InstCtl) * ns));
    ck(cudaMalloc((void**)&S->d_state, 4 * ns));
    ck(cudaMalloc((void**)&S->d_stop, 256));
    ck(cudaMalloc((void**)&S->d_done, 256));
    ck(cudaMalloc((void**)&S->d_beat, 256));
    ck(cudaMalloc((void**)&S->d_arena, c.memory_budget));
    ck(cudaHostAlloc((void**)&S->h_notify, 8 * ns, cudaHostAllocMapped));
    ck(cudaHostAlloc((void**)&S->h_stage, sizeof(Inst) * ns, cudaHostAllocDefault));
    ck(cudaHostAlloc((void**)&S->h_words, 64, cudaHostAllocDefault));
    if (e == cudaSuccess) ck(cudaHostGetDevicePointer((void**)&S->d_notify, S->h_notify, 0));
    ck(cudaStreamCreateWithFlags(&S->kstream, cudaStreamNonBlocking));
    ck(cudaStreamCreateWithFlags(&S->cstream, cudaStreamNonBlocking));
    if (e == cudaSuccess) {
        std::memset(S->h_notify, 0, 8 * ns);
        S->h_words[0] = kSlotSubmitted;
        S->h_words[1] = 1u;
        ck(cudaMemset(S->d_slots, 0, sizeof(Inst) * ns));
        ck(cudaMemset(S->d_ctl, 0, sizeof(InstCtl) * ns));
        ck(cudaMemset(S->d_state, 0, 4 * ns));
        ck(cudaMemset(S->d_stop, 0, 256));
        ck(cudaMemset(S->d_done, 0, 256));
        ck(cudaMemset(S->d_beat, 0, 256));
        ck(cudaDeviceSynchronize());
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        release_server(S);
        return e == cudaErrorMemoryAllocation ? ABFS_ERR_OOM : ABFS_ERR_CUDA;
    }
    S->slots.resize(ns);
    S->arena.init(c.memory_budget);
    S->t_start = Clock::now();
    S->th = std::thread(serve_loop, S);
    *out = S;
    return ABFS_OK;
}

extern "C" int abfs_serve_submit(abfs_server_t S, uint32_t graph_idx, uint32_t source, int32_t* level,
                                 int32_t* parent, uint64_t* ticket) {
    if (!S || !ticket || !level || !parent || graph_idx >= S->graphs.size())
        return ABFS_ERR_INVALID_ARG;
    uint32_t n;
    abfs_graph_info(S->graphs[graph_idx], &n, nullptr, nullptr);
    if (source >= n) return ABFS_ERR_INVALID_ARG;
    if (S->stopping.load()) return ABFS_ERR_BUSY;
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->fatal) return S->fatal;
    if (S->pending.size() >= S->cfg.queue_capacity) return ABFS_ERR_BUSY;
    Request r;
    r.ticket = S->next_ticket++;
    r.g = graph_idx;
    r.src = source;
    r.level = level;
    r.parent = parent;
    r.t0 = Clock::now();
    S->pending.push_back(r);
    S->submitted += 1;
    *ticket = r.ticket;
    return ABFS_OK;
}

extern "C" int abfs_serve_poll(abfs_server_t S, uint64_t ticket, int* done, int32_t* status) {
    if (!S || !done) return ABFS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->done_status.find(ticket);
    if (it != S->done_status.end()) {
        *done = 1;
        if (status) *status = it->second;
        return ABFS_OK;
    }
    if (ticket == 0 || ticket >= S->next_ticket) return ABFS_ERR_NOT_FOUND;
    *done = 0;
    return S->fatal ? S->fatal : ABFS_OK;
}

extern "C" int abfs_serve_wait(abfs_server_t S, uint64_t ticket, uint32_t timeout_ms,
                               int32_t* status) {
    if (!S) return ABFS_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    if (ticket == 0 || ticket >= S->next_ticket) return ABFS_ERR_NOT_FOUND;
    const bool ok = S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] {
        return S->done_status.count(ticket) > 0 || S->fatal != 0;
    });
    if (S->fatal) return S->fatal;
    if (!ok) return ABFS_ERR_TIMEOUT;
    if (status) *status = S->done_status[ticket];
    return ABFS_OK;
}

extern "C" int abfs_serve_stop(abfs_server_t S, abfs_serve_report* report) {
    if (!S) return ABFS_ERR_INVALID_ARG;
    S->stopping.store(true);
    if (S->th.joinable()) S->th.join();
    const double wall =
        std::chrono::duration<double>(Clock::now() - S->t_start).count();
    if (report) {
        std::memset(report, 0, sizeof(*report));
        report->submitted = S->submitted;
        report->completed = S->completed;
        report->failed = S->failed;
        report->launches = S->launches;
        report->wall_s = wall;
        report->qps = wall > 0 ? S->completed / wall : 0.0;
        std::vector<double> v = S->lat_ms;
        if (!v.empty()) {
            std::sort(v.begin(), v.end());
            auto pct = [&](double p) {
                const size_t i = (size_t)std::min<double>(v.size() - 1, p * (v.size() - 1) + 0.5);
                return v[i];
            };
            report->p50_ms = pct(0.50);
            report->p99_ms = pct(0.99);
            report->max_ms = v.back();
            double sum = 0;
            for (double x : v) sum += x;
            report->mean_ms = sum / v.size();
        }
    }
    const int rc = S->fatal;
    release_server(S);
    return rc;
}
