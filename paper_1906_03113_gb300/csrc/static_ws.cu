// abfs_run_static: one search whose scratch memory is a fixed device array
// compiled into this library, for callers that must not allocate.
//
// The scratch (visited bitmaps, frontier queues and blocks, unit starts, the
// control block and the search descriptor) lives in g_static_ws below, a
// file-scope __device__ array of kStaticWorkspaceBytes.  Every GPU that loads
// this library holds that array until the process exits.  In host code the
// name g_static_ws is only a host-side stand-in for the symbol, not a device
// address: its device address is obtained with cudaGetSymbolAddress, once per
// device, with that device current, and then passed to the kernels.
//
// The kernels are the same persistent engine that abfs_run uses; only the
// origin of the scratch differs.  Nothing here calls cudaMalloc, cudaFree or
// any allocating library routine.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/abfs.h"
#include "internal.h"

namespace abfs {
namespace {

// 72 MiB: enough for graphs up to about 1.1 million vertices (the layout
// needs about 65 bytes per vertex plus two unit-start tables of 8 bytes per
// 1024 entry slots, i.e. 16 bytes per 1024 of nnz + 6n).
constexpr size_t kStaticWorkspaceBytes = 72ull << 20;
// The first 256 bytes hold the launch's completion counter and heartbeat.
constexpr size_t kStaticHeader = 256;

static __device__ __align__(256) unsigned char g_static_ws[kStaticWorkspaceBytes];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_addr[kMaxDevices];  // device address of g_static_ws, per device

// Device address of g_static_ws on the current device (looked up once).
int static_base(int dev, void** out) {
    if (dev < 0 || dev >= kMaxDevices) return ABFS_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_ws);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return ABFS_ERR_CUDA;
        }
        g_static_addr[dev] = p;
    }
    *out = g_static_addr[dev];
    return ABFS_OK;
}

}  // namespace
}  // namespace abfs

using namespace abfs;

extern "C" int abfs_run_static(const uint32_t* colptr, const uint32_t* rowidx, uint32_t n,
                               uint64_t nnz, uint32_t source, int32_t* level, int32_t* parent,
                               abfs_stream_t stream) {
    if (!colptr || (nnz && !rowidx) || !level || !parent || n == 0 || source >= n)
        return ABFS_ERR_INVALID_ARG;
    if (n >= (1u << 31) || nnz + n >= (1ull << 32)) return ABFS_ERR_UNSUPPORTED;
    const abfs_params p = default_params();
    const Layout L = layout_for(n, nnz, p);
    if (kStaticHeader + L.total > kStaticWorkspaceBytes) return ABFS_ERR_UNSUPPORTED;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ABFS_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return ABFS_ERR_CUDA;
    void* ws = nullptr;
    int rc = static_base(dev, &ws);
    if (rc) return rc;
    char* base = static_cast<char*>(ws) + kStaticHeader;
    cudaStream_t s = (cudaStream_t)stream;
    Inst* d_inst = reinterpret_cast<Inst*>(base + L.inst);
    const Inst I = make_inst_raw(colptr, rowidx, n, base, L, source, level, parent);
    EngineArgs a;
    a.insts = d_inst;
    a.ninst = 1;
    a.done_count = static_cast<uint32_t*>(ws);
    a.heartbeat = reinterpret_cast<unsigned long long*>(static_cast<char*>(ws) + 8);
    a.prof = nullptr;
    a.serve = 0;
    a.slot_state = nullptr;
    a.stop_flag = nullptr;
    a.idle_exit_ns = 0;
    a.p = engine_params(p);
    // the initialisation kernels clear every word a search expects at zero
    // (bitmaps, control block, counters); the rest is written before it is read
    if (launch_put_inst(I, d_inst, s) != cudaSuccess) return ABFS_ERR_CUDA;
    if (launch_init(a, n, s) != cudaSuccess) return ABFS_ERR_CUDA;
    if (launch_engine(a, grid_for(sms, p), s) != cudaSuccess) return ABFS_ERR_CUDA;
    // the search's own status, read back into a host variable
    InstCtl ctl;
    if (cudaMemcpyAsync(&ctl, base + L.ctl, sizeof(ctl), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return ABFS_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return ABFS_ERR_CUDA;
    if (ctl.status == kDone) return ABFS_OK;
    return ctl.err ? (int)ctl.err : ABFS_ERR_DEVICE;
}
