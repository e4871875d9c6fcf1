// Internal declarations shared by the device engine (engine.cu) and the host
// runtime (abfs.cpp).  Not part of the public C-ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/abfs.h"

namespace abfs {

// Threads per CTA of the persistent engine, and the CTAs per SM its register
// budget is compiled for (512 x 2: 64 registers per thread).  The build may
// override both (and kIlp) with -D for measurements of other shapes.
#ifndef ABFS_THREADS
#define ABFS_THREADS 512
#endif
#ifndef ABFS_MIN_CTAS
#define ABFS_MIN_CTAS 2
#endif
#ifndef ABFS_ILP
#define ABFS_ILP 4
#endif
constexpr int kThreads = ABFS_THREADS;
constexpr int kMinCtas = ABFS_MIN_CTAS;
constexpr int kWarps = kThreads / 32;
static_assert(kThreads % 32 == 0 && kWarps <= 32, "CTA size");
// Largest group of frontier vertices a CTA stages in shared memory at once.
constexpr int kTileMax = 1024;
// Entries each thread keeps in flight in the expand loop (memory-level parallelism).
constexpr int kIlp = ABFS_ILP;
// Entries in flight per thread in levels that claim by reductions (nothing is
// staged there, so the registers go to more loads in flight).
#ifndef ABFS_ILP_SCAN
#define ABFS_ILP_SCAN 4
#endif
constexpr int kIlpScan = ABFS_ILP_SCAN;
// Prefer the smallest shared-memory carveout that holds the resident CTAs (1)
// or leave the split to the driver (0).
#ifndef ABFS_CARVEOUT
#define ABFS_CARVEOUT 1
#endif
// Per-warp staging buffer for newly reached vertices.  A warp writes its
// buffer out as one frontier block once a further expand step (32 * kIlp
// appends) might not fit; at the end of a unit the leftovers of all warps
// leave as one block.
constexpr int kWarpBuf = 64 * kIlp < 256 ? 256 : 64 * kIlp;
constexpr int kWarpFlushAt = kWarpBuf - 32 * kIlp;
// Largest work unit (entry slots) and the per-unit start bitmap it needs.
#ifndef ABFS_UNIT_MAX
#define ABFS_UNIT_MAX 65536
#endif
constexpr uint32_t kUnitMax = ABFS_UNIT_MAX;
static_assert((kUnitMax & (kUnitMax - 1)) == 0 && kUnitMax >= 1024, "unit size");
// The expand loop reads row indices four at a time (one 16-byte load per
// lane): slots come in chunks of four, and the start bitmap has a bit per chunk.
constexpr uint32_t kChunk = 4;
constexpr int kStartWords = kUnitMax / kChunk / 32 + 2;
// Marker of an unset parent / unclaimed vertex (reads as -1 through int32).
constexpr uint32_t kUnset = 0xFFFFFFFFu;
// Weight of a frontier vertex in its level's work space: the chunks that hold
// its column.  Entry x of a column whose first row index sits at position h of
// its aligned 16-byte group occupies slot start + h + x, and every vertex
// starts on a chunk boundary, so every chunk of four slots maps onto one
// aligned 16-byte group of the column's row indices.  A vertex owns at least
// one chunk (a vertex without entries still owns a start), so units balance
// vertices as well as entries.
__host__ __device__ constexpr uint32_t vslots(uint32_t h, uint32_t len) {
    return (h & (kChunk - 1)) + len == 0 ? kChunk
                                         : ((h & (kChunk - 1)) + len + kChunk - 1) / kChunk * kChunk;
}
// Upper bound of vslots(h, len) - len.
constexpr uint32_t kVertexSlotsMax = 2 * (kChunk - 1);
// Packed frontier counter: [entries : 40 bits][blocks : 24 bits].
constexpr uint32_t kBlockBits = 24;
constexpr uint32_t kBlockMask = (1u << kBlockBits) - 1u;

enum Mode : uint32_t { kModeSub = 0, kModePlain = 1 };

enum PhaseKind : uint32_t {
    kPhLevel = 0,      // submatrix method: mask rows, then multiply (one phase per level)
    kPhPlainMult = 1,  // comparator: multiply every entry of the frontier columns
    kPhPlainMask = 2,  // comparator: apply the visited mask to the touched rows
    kPhShrink = 3,     // physical shrink of the unvisited columns
    kPhInit = 4,       // serving: clear the outputs and bitmaps of a newly started search
    kPhLevelScan = 5,  // submatrix method, large level: mask, multiply and claim by reductions
    kPhExtract = 6,    // the vertices a kPhLevelScan level reached, read off the bitmaps
    kPhBuPrep = 7,     // hybrid: the frontier bitmap of a bottom-up level that follows a top-down one
    kPhBottomUp = 8,   // hybrid: unvisited vertices scan their sorted columns for a frontier entry
    kPhStart = 9,      // one empty unit: its CTA advances into level 0 (a resident run if small)
    kPhMsLevel = 10,   // multi-source search: expand the union frontier into the next-bit masks
    kPhMsUpdate = 11,  // multi-source search: new bits -> levels, parents, next union frontier
};

// Largest number of sources one multi-source search carries (one bit each).
constexpr uint32_t kMsMax = 64;

enum InstStatus : uint32_t { kIdle = 0, kRunning = 1, kDone = 2, kFailed = 3 };

// Serving slot states (device array, one word per slot).
enum SlotState : uint32_t { kSlotFree = 0, kSlotSubmitted = 1, kSlotRunning = 2 };

// A block of the frontier: nv consecutive vertices at fq[vb..], whose column
// entries occupy [eb, eb + sum of their weights) of the level's entry space.
// Blocks are numbered in the order of their entry ranges.
struct Block {
    uint32_t vb;
    uint32_t nv;
    unsigned long long eb;
};

// Device-resident control block of one search.  Zeroed at initialisation.
struct InstCtl {
    unsigned long long grab;     // [epoch:32][units taken:32] of the published phase
    unsigned long long desc[2];  // per epoch parity: [epoch:32][units:32]
    unsigned long long bctr[2];  // per level parity: [entries:40][blocks:24] of the frontier
    unsigned long long fent[2];  // per level parity: column entries of the frontier (hybrid only)
    uint32_t pending[2];         // per epoch parity: units not yet completed
    uint32_t kind[2];            // per epoch parity: PhaseKind
    uint32_t plevel[2];          // per epoch parity: BFS level of the phase
    uint32_t nitems[2];          // per epoch parity: touched rows (mask) / copy index (shrink)
    uint32_t fcnt[2];            // per level parity: frontier vertices
    uint32_t epoch;              // last published epoch (written by the advancer only)
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
    uint32_t trace_n;            // trace entries written
    uint32_t bu_on;              // hybrid: 1 while levels run bottom-up
    uint32_t init_ticket;        // blocks of init_single_kernel that are done (wraps to 0)
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
    unsigned long long nnz;  // row indices at rowidx (reads stay inside them)
    uint32_t n;
    uint32_t src;
    uint32_t nwords;         // ceil(n/32)
    uint32_t bcap;           // blocks per frontier
    unsigned long long ucap; // unit starts per frontier
    int32_t* level;          // output
    uint32_t* parent;        // output (0xFFFFFFFF reads as -1)
    unsigned long long* sigma;  // optional output: shortest-path counts mod 2^64 (nullptr = off)
    uint32_t* bm[2];         // visited bitmaps, ping-pong by level parity
    uint32_t* fbm[2];        // hybrid: frontier bitmaps of bottom-up levels, by level parity
    const uint32_t* inb;     // rows that occur in some column (nullptr: not known); the
                             // others can never be reached and start out masked
    uint32_t bu_ok;          // hybrid: bottom-up levels allowed (undirected, sorted columns, no counts)
    uint32_t* fq[2];         // frontier vertices, by level parity
    uint32_t* fbeg[2];       // their column begins (kUnset: no entries)
    uint32_t* fpre[2];       // their entry offsets within their block
    uint32_t* flen[2];       // their column lengths
    // relabelled graph (vertices numbered by column-length class): the input
    // label of each vertex, looked up where a frontier vertex is staged
    // (nullptr: the labels are the input's).  Parents are always input labels.
    const uint32_t* lab;
    Block* blk[2];           // frontier blocks
    uint2* ustart[2];        // unit u starts in (block, vertex index in block)
    unsigned long long* y;   // comparator: stamped (min, index) accumulator
    uint32_t* touched;       // comparator: rows touched by the multiply
    uint32_t* sbeg[2];       // shrunk copies: column begin per vertex
    uint32_t* slen[2];       // shrunk copies: column length per vertex
    uint32_t* srows[2];      // shrunk copies: row arrays
    unsigned long long scap; // capacity of each shrunk row array
    InstCtl* ctl;
    uint4* trace;            // optional per-phase trace (nullptr = off)
    uint32_t trace_cap;
    uint32_t slot;           // serving: slot index
    unsigned long long ticket;       // serving: request ticket
    unsigned long long* notify;      // serving: host-mapped word that receives ticket<<8 | status
    // multi-source search (ms > 0): ms sources, one bit of a 64-bit mask each;
    // level/parent/src above are unused, each source has its own outputs
    uint32_t ms;
    uint32_t ms_sorted;               // columns ascend: a parent scan may stop at the first hit
    unsigned long long* ms_vis;       // vertices reached, per source bit (levels <= k)
    unsigned long long* ms_fr[2];     // frontier bits, by level parity
    unsigned long long* ms_nx;        // bits newly reached at the current level
    const uint32_t* ms_src;           // the sources (ms of them)
    int32_t* const* ms_level;         // per source: level output (n int32)
    int32_t* const* ms_parent;        // per source: parent output (n int32)
};

struct EngineParams {
    uint32_t mode;
    uint32_t tile;                 // vertices per staged group / touched rows per mask unit
    uint32_t unit;                 // granule of work units in entry slots (a power of two)
    uint32_t unit_shift;           // log2(unit)
    uint32_t narrow_max;
    uint32_t narrow_edges;
    uint32_t narrow_loop;          // 1: narrow levels run back to back on one CTA (resident runs)
    uint32_t scan_min;             // wide levels with >= scan_min entry slots claim by reductions (0: never)
    uint32_t bu_alpha;             // hybrid: top-down -> bottom-up when frontier edges * alpha > unexplored edges (0: off)
    uint32_t bu_beta;              // hybrid: bottom-up -> top-down when frontier vertices * beta < n
    float shrink_theta;
    uint32_t shrink_max;
    uint32_t shrink_tile;          // vertices per shrink unit
    uint32_t init_tile;            // serving: vertices per initialisation unit
    unsigned long long timeout_ns;
    uint32_t cluster;              // CTAs per thread-block cluster of the launch (1: no cluster runs)
    uint32_t cluster_min;          // a level of >= cluster_min entry slots starts a cluster run
    uint32_t cluster_max;          // cluster runs continue while a level has <= cluster_max vertices ...
    uint32_t cluster_edges;        // ... and <= cluster_edges entry slots
};

struct EngineArgs {
    const Inst* insts;
    uint32_t ninst;
    uint32_t* done_count;          // instances finished (any status)
    unsigned long long* heartbeat; // progress counter for the bounded waits
    unsigned long long* prof;      // optional per-category CTA cycle totals (kProfSlots), or null
    uint32_t serve;                // 1: long-lived serving launch over a slot table
    uint32_t* slot_state;          // serving: SlotState per slot
    const uint32_t* stop_flag;     // serving: host sets 1 to end the launch
    unsigned long long idle_exit_ns;  // serving: the launch ends after this long without progress
    EngineParams p;
    // test control (abfs_test_hold_first_phase): units the first phase of every
    // search waits for beyond its own, so it never completes and the bounded
    // idle wait runs out; 0 in normal operation
    uint32_t hold_units = 0;
};

// Cycle accounting of the engine's CTAs (profiling runs only).
enum ProfSlot : int {
    kProfIdle = 0,     // no unit available
    kProfTake = 1,     // scanning searches and taking a unit
    kProfGather = 2,   // staging frontier vertices of a unit
    kProfExpand = 3,   // warp 0's own expand time
    kProfWait = 4,     // waiting for the other warps' expand
    kProfFlush = 5,    // writing the unit's leftovers as a block
    kProfAdvance = 6,  // advancing a search to its next phase
    kProfUnits = 7,    // units run (a count)
    // resident narrow runs
    kProfNLoad = 8,     // staging a chunk of the frontier list (columns, scan, starts)
    kProfNExpand = 9,   // expanding it
    kProfNAppend = 10,  // appending the warps' leftovers (and the comparator's mask)
    kProfNDecide = 11,  // counters and the decision to go on
    kProfNBlocks = 12,  // rewriting the last list as blocks
    kProfNLevels = 13,  // levels run (a count)
    // per warp inside the expand loop (sums over warps)
    kProfXSetup = 14,    // locating the warp's first vertex and issuing the first row loads
    kProfXLoop = 15,     // the whole loop over the warp's slots
    kProfXProcess = 16,  // of which: mask, multiply and claim (waits for the loads)
    kProfXFlush = 17,    // of which: writing staged vertices out
    kProfXCalls = 18,    // expand calls per warp (a count)
    kProfSlots = 19
};

// Per-search workspace layout: byte offsets of each buffer from the base.
struct Layout {
    uint64_t nnz;
    size_t bm[2], fbm[2], fq[2], fbeg[2], fpre[2], flen[2], blk[2], ustart[2], y, touched, sbeg[2], slen[2],
        srows[2], ctl, inst, inst_r;
    size_t ms_vis, ms_fr[2], ms_nx, ms_src, ms_lev, ms_par;  // multi-source searches only
    size_t lev_i, par_i;  // searches on a relabelled graph: internal outputs
    size_t total;
    uint32_t nwords, bcap, ncopies;
    unsigned long long ucap, scap;
};

// Host helpers implemented in abfs.cpp.
abfs_params default_params();
bool shrink_enabled(const abfs_params& p);
int check_params(const abfs_params& p);
EngineParams engine_params(const abfs_params& p);
Layout layout_for(uint32_t n, uint64_t nnz, const abfs_params& p, uint32_t ms = 0,
                  bool relabel = false);
Inst make_inst_raw(const uint32_t* colptr, const uint32_t* rowidx, uint32_t n, char* base,
                   const Layout& L, uint32_t src, int32_t* level, int32_t* parent);
int grid_for(int sms, const abfs_params& p);
int graph_arrays(abfs_graph_t g, const uint32_t** colptr, const uint32_t** rowidx, uint32_t* n,
                 uint64_t* nnz, int* device, int* sms);

// Test control set by abfs_test_hold_first_phase (abfs.cpp).
uint32_t test_hold_units();

// Launch helpers implemented in engine.cu.
cudaError_t launch_put_inst(const Inst& inst, Inst* dst, cudaStream_t s);
cudaError_t launch_sorted_check(const uint32_t* colptr, const uint32_t* rowidx, uint32_t n,
                                uint32_t* unsorted, cudaStream_t s);
cudaError_t launch_row_bitmap(const uint32_t* rowidx, uint64_t nnz, uint32_t* bits, uint32_t nwords,
                              cudaStream_t s);
cudaError_t launch_set_query(Inst* inst, uint32_t src, int32_t* level, uint32_t* parent,
                             unsigned long long* sigma, uint32_t bu_ok,
                             uint4* trace, uint32_t trace_cap, cudaStream_t s);
cudaError_t launch_init(const EngineArgs& a, uint32_t max_n, cudaStream_t s);
// One search on a workspace's instance 0: the descriptor's per-call fields,
// the cleared outputs and bitmaps, and level 0, in one launch.
cudaError_t launch_init_single(const EngineArgs& a, uint32_t src, uint32_t src_label, int32_t* level,
                               uint32_t* parent, unsigned long long* sigma, uint32_t bu_ok,
                               uint4* trace, uint32_t trace_cap, uint32_t n, cudaStream_t s);
// A search on a relabelled graph: the caller's outputs in input labels,
// level[o] = lev_i[pos[o]], parent[o] = par_i[pos[o]] (-1 without a look-up for
// internal vertices >= n_keep other than the source s_i).
cudaError_t launch_relabel_out(const uint32_t* pos, const int32_t* lev_i, const uint32_t* par_i,
                               int32_t* level, int32_t* parent, uint32_t n, uint32_t n_keep,
                               uint32_t s_i, cudaStream_t s);
cudaError_t launch_engine(const EngineArgs& a, int grid, cudaStream_t s);
cudaError_t engine_occupancy(uint32_t mode, int* blocks_per_sm);
// Clusters of `cluster` CTAs of the engine that can be resident at once.
cudaError_t engine_max_clusters(uint32_t mode, uint32_t cluster, int* clusters);
size_t engine_smem_bytes();

}  // namespace abfs
