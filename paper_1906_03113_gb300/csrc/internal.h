// Internal declarations shared by the device engine (engine.cu) and the host
// runtime (abfs.cpp).  Not part of the public C-ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace abfs {

// Threads per CTA of the persistent engine.
constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
// Largest frontier tile (vertices) a CTA expands at once.
constexpr int kTileMax = 2048;
// CTA staging buffer for newly reached vertices before one global append.
constexpr int kOutBuf = 4096;
// Marker of an unset parent / unclaimed vertex (reads as -1 through int32).
constexpr uint32_t kUnset = 0xFFFFFFFFu;

enum Mode : uint32_t { kModeSub = 0, kModePlain = 1 };

enum PhaseKind : uint32_t {
    kPhLevel = 0,      // submatrix method: mask rows, then multiply (one phase per level)
    kPhPlainMult = 1,  // comparator: multiply every entry of the frontier columns
    kPhPlainMask = 2,  // comparator: apply the visited mask to the touched rows
    kPhShrink = 3,     // physical shrink of the unvisited columns
};

enum InstStatus : uint32_t { kRunning = 0, kDone = 1, kFailed = 2 };

// Device-resident control block of one search.  Zeroed at initialisation.
struct InstCtl {
    unsigned long long grab;     // [epoch:32][units taken:32] of the published phase
    unsigned long long desc[2];  // per epoch parity: [epoch:32][units:32]
    uint32_t pending[2];         // per epoch parity: units not yet completed
    uint32_t kind[2];            // per epoch parity: PhaseKind
    uint32_t plevel[2];          // per epoch parity: BFS level of the phase
    uint32_t nheavy[2];          // per epoch parity: heavy-chunk units (come first)
    uint32_t nitems[2];          // per epoch parity: light vertices (or touched rows / shrink items)
    uint32_t epoch;              // last published epoch (written by the advancer only)
    uint32_t fcnt[2];            // per level parity: light frontier length
    uint32_t hcnt[2];            // per level parity: heavy chunks
    uint32_t hvert[2];           // per level parity: heavy vertices
    uint32_t tcnt;               // comparator: rows touched by the current multiply
    uint32_t status;             // InstStatus
    uint32_t err;                // abfs_status when status == kFailed
    uint32_t levels;             // non-empty frontiers
    uint32_t reached;            // vertices reached
    uint32_t wide_levels;        // phases published to the whole grid
    uint32_t shrinks;            // shrink events
    uint32_t mat_cur;            // matrix used for levels >= mat_switch (0 = input)
    uint32_t mat_prev;           // matrix used for levels < mat_switch
    uint32_t mat_switch;         // first level that reads mat_cur
    uint32_t shrink_out;         // shrink: entries written so far
    uint32_t pad_;
    unsigned long long entries_read;
    unsigned long long entries_unmasked;
    unsigned long long claims;
    unsigned long long nnz_reached;
    unsigned long long shrink_read;
    unsigned long long shrink_kept;
};

// Read-only descriptor of one search (graph, outputs, workspace).
struct Inst {
    const uint32_t* colptr;  // input CSC
    const uint32_t* rowidx;
    uint32_t n;
    uint32_t src;
    uint32_t nwords;         // ceil(n/32)
    uint32_t hcap;           // capacity of each heavy-chunk queue
    int32_t* level;          // output
    uint32_t* parent;        // output (0xFFFFFFFF reads as -1)
    uint32_t* bm[2];         // visited bitmaps, ping-pong by level parity
    uint32_t* fq[2];         // light frontier queues, by level parity
    uint2* hq[2];            // heavy chunk queues (vertex, chunk index), by level parity
    unsigned long long* y;   // comparator: stamped (min, index) accumulator
    uint32_t* touched;       // comparator: rows touched by the multiply
    uint32_t* sbeg[2];       // shrunk copies: column begin per vertex
    uint32_t* slen[2];       // shrunk copies: column length per vertex
    uint32_t* srows[2];      // shrunk copies: row arrays
    unsigned long long scap; // capacity of each shrunk row array
    InstCtl* ctl;
};

struct EngineParams {
    uint32_t mode;
    uint32_t tile;
    uint32_t heavy;
    uint32_t chunk;
    uint32_t narrow_max;
    float shrink_theta;
    uint32_t shrink_max;
    uint32_t shrink_tile;          // vertices per shrink unit
    unsigned long long timeout_ns;
};

struct EngineArgs {
    const Inst* insts;
    uint32_t ninst;
    uint32_t* done_count;          // instances finished (any status)
    unsigned long long* heartbeat; // progress counter for the bounded waits
    EngineParams p;
};

// Launch helpers implemented in engine.cu.
cudaError_t launch_set_query(Inst* inst, uint32_t src, int32_t* level, uint32_t* parent,
                             cudaStream_t s);
cudaError_t launch_init(const EngineArgs& a, uint32_t max_n, cudaStream_t s);
cudaError_t launch_engine(const EngineArgs& a, int grid, cudaStream_t s);
cudaError_t engine_occupancy(uint32_t mode, int* blocks_per_sm);

}  // namespace abfs
