"""Thin ctypes binding over libabfs.so (the C-ABI in include/abfs.h).

Argument marshalling only: every step of a search runs in the library's CUDA
kernels.  PyTorch supplies device memory (output tensors) and streams.  The
binding loads the in-tree libabfs.so and raises if it is missing; there is no
fallback path.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libabfs.so")
HEADER_PATH = os.path.join(os.path.dirname(_HERE), "include", "abfs.h")

OK = 0
ERR_INVALID_ARG = 1
ERR_NOT_SYMMETRIC = 2
ERR_OOM = 3
ERR_CUDA = 4
ERR_TIMEOUT = 5
ERR_BUSY = 6
ERR_DEVICE = 7
ERR_UNSUPPORTED = 8
ERR_NOT_FOUND = 9

VALIDATE = 1
INPUT_ON_DEVICE = 2
MODE_SUBMATRIX = 0
MODE_PLAIN = 1


class Params(ctypes.Structure):
    _fields_ = [
        ("mode", ctypes.c_uint32),
        ("tile", ctypes.c_uint32),
        ("unit_entries", ctypes.c_uint32),
        ("narrow_max", ctypes.c_uint32),
        ("narrow_edges", ctypes.c_uint32),
        ("ctas_per_sm", ctypes.c_uint32),
        ("shrink_theta", ctypes.c_float),
        ("shrink_max", ctypes.c_uint32),
        ("timeout_ms", ctypes.c_uint32),
        ("narrow_resident", ctypes.c_uint32),
        ("claim_scan", ctypes.c_uint32),
        ("bottom_up_alpha", ctypes.c_uint32),
        ("bottom_up_beta", ctypes.c_uint32),
        ("cluster_ctas", ctypes.c_uint32),
        ("cluster_min", ctypes.c_uint32),
        ("cluster_max", ctypes.c_uint32),
        ("cluster_edges", ctypes.c_uint32),
        ("multi_source", ctypes.c_uint32),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class Stats(ctypes.Structure):
    _fields_ = [
        ("levels", ctypes.c_uint32),
        ("reached", ctypes.c_uint32),
        ("nnz_reached", ctypes.c_uint64),
        ("entries_read", ctypes.c_uint64),
        ("entries_unmasked", ctypes.c_uint64),
        ("claims", ctypes.c_uint64),
        ("shrinks", ctypes.c_uint32),
        ("wide_levels", ctypes.c_uint32),
        ("shrink_entries_read", ctypes.c_uint64),
        ("shrink_entries_kept", ctypes.c_uint64),
        ("status", ctypes.c_uint32),
        ("reserved", ctypes.c_uint32),
    ]

    def as_dict(self) -> dict:
        return {k: int(getattr(self, k)) for k, _ in self._fields_ if k != "reserved"}


class ServeCfg(ctypes.Structure):
    _fields_ = [
        ("max_slots", ctypes.c_uint32),
        ("queue_capacity", ctypes.c_uint32),
        ("memory_budget", ctypes.c_uint64),
        ("idle_exit_ms", ctypes.c_uint32),
        ("params", Params),
    ]


class ServeReport(ctypes.Structure):
    _fields_ = [
        ("submitted", ctypes.c_uint64),
        ("completed", ctypes.c_uint64),
        ("failed", ctypes.c_uint64),
        ("launches", ctypes.c_uint64),
        ("p50_ms", ctypes.c_double),
        ("p99_ms", ctypes.c_double),
        ("mean_ms", ctypes.c_double),
        ("max_ms", ctypes.c_double),
        ("wall_s", ctypes.c_double),
        ("qps", ctypes.c_double),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class AbfsError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib.abfs_strerror(status).decode() if _lib else str(status)
        extra = ""
        if status == ERR_CUDA and _lib:
            extra = " (" + _lib.abfs_last_cuda_error().decode() + ")"
        super().__init__(f"{where}: {msg}{extra} [status {status}]")


class Calibration(ctypes.Structure):
    _fields_ = [("words", ctypes.c_uint32), ("reserved", ctypes.c_uint32), ("ops", ctypes.c_uint64),
                ("red_gops", ctypes.c_double), ("load_gops", ctypes.c_double)]


_lib = None


def declared_symbols() -> list[str]:
    """Every function name include/abfs.h declares."""
    text = open(HEADER_PATH).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(abfs_[a-z_0-9]+)\s*\(", text)))


def load():
    """Loads libabfs.so (built by __graft_entry__.build()); raises if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    u32, u64, i32, vp = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32, ctypes.c_void_p
    c_int = ctypes.c_int
    sig = {
        "abfs_strerror": ([c_int], ctypes.c_char_p),
        "abfs_last_cuda_error": ([], ctypes.c_char_p),
        "abfs_version": ([], c_int),
        "abfs_default_params": ([P(Params)], c_int),
        "abfs_graph_create": ([vp, vp, u32, u64, c_int, u32, vp, P(vp)], c_int),
        "abfs_graph_destroy": ([vp], c_int),
        "abfs_graph_info": ([vp, P(u32), P(u64), P(c_int)], c_int),
        "abfs_graph_footprint": ([vp, P(Params), P(ctypes.c_size_t)], c_int),
        "abfs_run": ([vp, u32, vp, vp, vp, P(Params), P(Stats)], c_int),
        "abfs_run_counts": ([vp, u32, vp, vp, vp, vp, P(Params), P(Stats)], c_int),
        "abfs_calibrate": ([u32, P(Calibration), vp], c_int),
        "abfs_run_host": ([vp, u32, vp, vp, vp, P(Params), P(Stats)], c_int),
        "abfs_graph_relabel": ([vp], c_int),
        "abfs_relabel_order": ([vp, u32, vp, vp], c_int),
        "abfs_run_host_many": ([vp, P(u32), u32, vp, vp, vp, P(Params), P(i32)], c_int),
        "abfs_run_trace": ([vp, u32, vp, vp, vp, P(Params), vp, u32, P(u32)], c_int),
        "abfs_run_batch": ([P(vp), P(u32), u32, P(vp), P(vp), vp, P(Params), P(i32)], c_int),
        "abfs_batch_create": ([P(vp), P(u32), u32, P(vp), P(vp), P(Params), vp, P(vp)], c_int),
        "abfs_batch_create_counts": ([P(vp), P(u32), u32, P(vp), P(vp), P(vp), P(Params), vp, P(vp)],
                                     c_int),
        "abfs_batch_launch": ([vp, vp], c_int),
        "abfs_batch_status": ([vp, vp, P(i32)], c_int),
        "abfs_batch_destroy": ([vp], c_int),
        "abfs_tune": ([vp, P(u32), u32, u32, ctypes.c_char_p, vp, P(Params),
                       P(ctypes.c_float)], c_int),
        "abfs_batch_tune": ([P(vp), P(u32), u32, u32, ctypes.c_char_p, vp, P(Params),
                             P(ctypes.c_float)], c_int),
        "abfs_set_allocator": ([vp, vp, vp], c_int),
        "abfs_test_hold_first_phase": ([u32], c_int),
        "abfs_check_params": ([P(Params)], c_int),
        "abfs_run_static": ([vp, vp, u32, u64, u32, vp, vp, vp], c_int),
        "abfs_serve_default_cfg": ([P(ServeCfg)], c_int),
        "abfs_serve_start": ([P(vp), u32, P(ServeCfg), P(vp)], c_int),
        "abfs_serve_submit": ([vp, u32, u32, vp, vp, P(u64)], c_int),
        "abfs_serve_poll": ([vp, u64, P(c_int), P(i32)], c_int),
        "abfs_serve_wait": ([vp, u64, u32, P(i32)], c_int),
        "abfs_serve_stop": ([vp, P(ServeReport)], c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _check(rc: int, where: str) -> None:
    if rc != OK:
        raise AbfsError(rc, where)


def _stream_ptr(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream or None
    if isinstance(stream, int):
        return stream or None
    return stream.cuda_stream or None


def default_params(**overrides) -> Params:
    p = Params()
    _check(load().abfs_default_params(ctypes.byref(p)), "abfs_default_params")
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def strerror(status: int) -> str:
    return load().abfs_strerror(status).decode()


# ---------------------------------------------------------------------------
# graphs
# ---------------------------------------------------------------------------

class Graph:
    """A device-resident graph (abfs_graph_t).  Column j of the CSC lists the
    out-neighbours of j."""

    def __init__(self, handle: int, n: int, nnz: int, directed: bool):
        self.handle = ctypes.c_void_p(handle)
        self.n, self.nnz, self.directed = n, nnz, directed

    def destroy(self) -> None:
        if self.handle and self.handle.value:
            _check(load().abfs_graph_destroy(self.handle), "abfs_graph_destroy")
            self.handle = ctypes.c_void_p(0)

    def __del__(self):
        try:
            if _lib is not None and self.handle and self.handle.value:
                _lib.abfs_graph_destroy(self.handle)
        except Exception:
            pass

    def footprint(self, params: Params | None = None) -> int:
        out = ctypes.c_size_t()
        _check(load().abfs_graph_footprint(self.handle, ctypes.byref(params) if params else None,
                                           ctypes.byref(out)), "abfs_graph_footprint")
        return int(out.value)


def graph_create(colptr, rowidx, directed: bool = False, validate: bool = False,
                 stream=None) -> Graph:
    """From host numpy arrays (uint32) or CUDA tensors (int32/uint32 bits)."""
    lib = load()
    flags = VALIDATE if validate else 0
    if isinstance(colptr, np.ndarray):
        colptr = np.ascontiguousarray(colptr, dtype=np.uint32)
        rowidx = np.ascontiguousarray(rowidx, dtype=np.uint32)
        n = colptr.shape[0] - 1
        nnz = rowidx.shape[0]
        cp, rp = colptr.ctypes.data, (rowidx.ctypes.data if nnz else None)
        keep = (colptr, rowidx)
    else:  # torch tensors on the device
        flags |= INPUT_ON_DEVICE
        n = colptr.numel() - 1
        nnz = rowidx.numel()
        cp, rp = colptr.data_ptr(), (rowidx.data_ptr() if nnz else None)
        keep = (colptr, rowidx)
    h = ctypes.c_void_p()
    rc = lib.abfs_graph_create(cp, rp, n, nnz, 1 if directed else 0, flags, _stream_ptr(stream),
                               ctypes.byref(h))
    del keep
    _check(rc, "abfs_graph_create")
    return Graph(h.value, n, nnz, directed)


def graph_destroy(g: Graph) -> None:
    g.destroy()


# ---------------------------------------------------------------------------
# searches
# ---------------------------------------------------------------------------

def _outputs(n: int, level, parent, device):
    import torch
    if level is None:
        level = torch.empty(n, dtype=torch.int32, device=device)
    if parent is None:
        parent = torch.empty(n, dtype=torch.int32, device=device)
    assert level.dtype == torch.int32 and parent.dtype == torch.int32
    assert level.is_cuda and parent.is_cuda and level.numel() >= n and parent.numel() >= n
    return level, parent


def run(g: Graph, source: int, level=None, parent=None, stream=None, params: Params | None = None,
        stats: bool = False):
    """abfs_run: returns (level, parent) CUDA int32 tensors (and a stats dict)."""
    import torch
    level, parent = _outputs(g.n, level, parent, torch.device("cuda", torch.cuda.current_device()))
    st = Stats() if stats else None
    rc = load().abfs_run(g.handle, int(source), level.data_ptr(), parent.data_ptr(),
                         _stream_ptr(stream), ctypes.byref(params) if params else None,
                         ctypes.byref(st) if st else None)
    _check(rc, "abfs_run")
    return (level, parent, st.as_dict()) if stats else (level, parent)


def run_counts(g: Graph, source: int, level=None, parent=None, sigma=None, stream=None,
               params: Params | None = None, stats: bool = False):
    """abfs_run_counts: (level, parent, sigma) CUDA tensors -- int32, int32 and
    int64 holding the uint64 shortest-path counts mod 2^64 -- (and a stats dict)."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    level, parent = _outputs(g.n, level, parent, dev)
    if sigma is None:
        sigma = torch.empty(g.n, dtype=torch.int64, device=dev)
    if sigma.numel() < g.n or sigma.element_size() != 8 or not sigma.is_cuda:
        raise ValueError("sigma must be a CUDA tensor of n 64-bit integers")
    st = Stats() if stats else None
    rc = load().abfs_run_counts(g.handle, int(source), level.data_ptr(), parent.data_ptr(),
                                sigma.data_ptr(), _stream_ptr(stream),
                                ctypes.byref(params) if params else None,
                                ctypes.byref(st) if st else None)
    _check(rc, "abfs_run_counts")
    return (level, parent, sigma, st.as_dict()) if stats else (level, parent, sigma)


def calibrate(words_log2: int = 22, stream=None) -> dict:
    """abfs_calibrate: random L2 load and red.min rates (10^9/s) over 2^words_log2 words."""
    c = Calibration()
    _check(load().abfs_calibrate(int(words_log2), ctypes.byref(c), _stream_ptr(stream)),
           "abfs_calibrate")
    return {"words": c.words, "ops": c.ops, "red_gops": c.red_gops, "load_gops": c.load_gops}


TRACE_KINDS = {0: "level", 1: "plain_mult", 2: "plain_mask", 3: "shrink", 4: "init",
               5: "level_scan", 6: "extract", 7: "bu_prep", 8: "bottom_up", 10: "ms_level",
               11: "ms_update", 0xFE: "start",
               0xFF: "end"}


def run_trace(g: Graph, source: int, params: Params | None = None, cap: int = 4096, stream=None):
    """abfs_run_trace: (level, parent, list of per-phase dicts with t_us from start)."""
    import torch
    level, parent = _outputs(g.n, None, None, torch.device("cuda", torch.cuda.current_device()))
    buf = np.zeros(cap * 8, dtype=np.uint32)
    cnt = ctypes.c_uint32()
    rc = load().abfs_run_trace(g.handle, int(source), level.data_ptr(), parent.data_ptr(),
                               _stream_ptr(stream), ctypes.byref(params) if params else None,
                               buf.ctypes.data, cap, ctypes.byref(cnt))
    _check(rc, "abfs_run_trace")
    rows = buf[: cnt.value * 8].reshape(-1, 8).astype(np.uint64)
    out = []
    t0 = None
    prof_at = [i for i, r in enumerate(rows) if (int(r[2]) >> 24) == 0xFD]
    if prof_at:
        flat = rows[prof_at[0]:].reshape(-1)[4:]
        names = ["idle", "take", "gather", "expand", "wait", "flush", "advance", "units",
                 "narrow_load", "narrow_expand", "narrow_append", "narrow_decide", "narrow_blocks",
                 "narrow_levels", "x_setup", "x_loop", "x_process", "x_flush", "x_calls"]
        vals = [int(flat[2 * q] | (flat[2 * q + 1] << 32)) for q in range(len(names))]
        out_prof = dict(zip(names, vals))
        rows = rows[:prof_at[0]]
    else:
        out_prof = {}
    for r in rows:
        t = int(r[0] | (r[1] << 32))
        t0 = t if t0 is None else t0
        out.append({"t_us": (t - t0) / 1e3, "kind": TRACE_KINDS.get(int(r[2]) >> 24, int(r[2]) >> 24),
                    "level": int(r[2]) & 0xFFFFFF, "alone": int(r[3]), "items": int(r[4]),
                    "vertices": int(r[5]), "entries": int(r[6])})
    if out_prof:
        out.append({"kind": "profile", **out_prof})
    return level, parent, out


def run_host(g: Graph, source: int, level_host: np.ndarray | None = None,
             parent_host: np.ndarray | None = None, stream=None, params: Params | None = None,
             stats: bool = False):
    """abfs_run_host: results in host arrays (pinned tensors give full copy speed)."""
    if level_host is None:
        level_host = np.empty(g.n, dtype=np.int32)
    if parent_host is None:
        parent_host = np.empty(g.n, dtype=np.int32)
    lp = level_host.ctypes.data if isinstance(level_host, np.ndarray) else level_host.data_ptr()
    pp = parent_host.ctypes.data if isinstance(parent_host, np.ndarray) else parent_host.data_ptr()
    st = Stats() if stats else None
    rc = load().abfs_run_host(g.handle, int(source), lp, pp, _stream_ptr(stream),
                              ctypes.byref(params) if params else None,
                              ctypes.byref(st) if st else None)
    _check(rc, "abfs_run_host")
    return (level_host, parent_host, st.as_dict()) if stats else (level_host, parent_host)


def graph_relabel(g: Graph) -> None:
    """abfs_graph_relabel: single searches on g run on a copy numbered by
    column-length class; outputs stay in g's labels."""
    _check(load().abfs_graph_relabel(g.handle), "abfs_graph_relabel")


def relabel_order(colptr):
    """abfs_relabel_order (host only): (lab, pos) of the numbering
    abfs_graph_relabel uses -- lab[i] is the input label of internal vertex i,
    pos its inverse."""
    cp = np.ascontiguousarray(colptr, dtype=np.uint32)
    n = cp.size - 1
    lab = np.empty(max(n, 0), dtype=np.uint32)
    pos = np.empty(max(n, 0), dtype=np.uint32)
    _check(load().abfs_relabel_order(cp.ctypes.data, max(n, 0), lab.ctypes.data, pos.ctypes.data),
           "abfs_relabel_order")
    return lab, pos


def run_host_many(g: Graph, sources, level_host=None, parent_host=None, stream=None,
                  params: Params | None = None):
    """abfs_run_host_many: search i's results in row i of host arrays of shape
    (len(sources), n) (pinned tensors let the copies overlap the searches).
    Returns (level_host, parent_host, per-search statuses)."""
    srcs = np.ascontiguousarray(np.asarray(sources, dtype=np.uint32))
    count = int(srcs.shape[0])
    if level_host is None:
        level_host = np.empty((count, g.n), dtype=np.int32)
    if parent_host is None:
        parent_host = np.empty((count, g.n), dtype=np.int32)
    lp = level_host.ctypes.data if isinstance(level_host, np.ndarray) else level_host.data_ptr()
    pp = parent_host.ctypes.data if isinstance(parent_host, np.ndarray) else parent_host.data_ptr()
    st = (ctypes.c_int32 * max(count, 1))()
    rc = load().abfs_run_host_many(g.handle, srcs.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                   count, lp, pp, _stream_ptr(stream),
                                   ctypes.byref(params) if params else None, st)
    statuses = [int(st[i]) for i in range(count)]
    # a search's own failure comes back in `statuses`; anything else raises
    if rc and rc != next((x for x in statuses if x), 0):
        _check(rc, "abfs_run_host_many")
    return level_host, parent_host, statuses


def _ptr_array(ptrs):
    arr = (ctypes.c_void_p * len(ptrs))()
    for i, p in enumerate(ptrs):
        arr[i] = p
    return arr


def run_batch(graphs: list[Graph], sources, levels=None, parents=None, stream=None,
              params: Params | None = None):
    """abfs_run_batch: one persistent launch for all searches.  Returns
    (levels, parents, statuses)."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    count = len(graphs)
    levels = levels or [torch.empty(g.n, dtype=torch.int32, device=dev) for g in graphs]
    parents = parents or [torch.empty(g.n, dtype=torch.int32, device=dev) for g in graphs]
    src = (ctypes.c_uint32 * count)(*[int(s) for s in sources])
    st = (ctypes.c_int32 * count)()
    rc = load().abfs_run_batch(_ptr_array([g.handle.value for g in graphs]), src, count,
                               _ptr_array([t.data_ptr() for t in levels]),
                               _ptr_array([t.data_ptr() for t in parents]), _stream_ptr(stream),
                               ctypes.byref(params) if params else None, st)
    statuses = list(st)
    if rc not in (OK, ERR_TIMEOUT, ERR_DEVICE):
        _check(rc, "abfs_run_batch")
    return levels, parents, statuses


class BatchPlan:
    """abfs_batch_create / launch / status / destroy: workspaces allocated once,
    initialisation + persistent launch captured in a CUDA graph."""

    def __init__(self, graphs: list[Graph], sources, levels=None, parents=None,
                 params: Params | None = None, stream=None, counts: bool = False):
        """counts=True: abfs_batch_create_counts, with int64 tensors (uint64 path
        counts mod 2^64) in self.sigmas."""
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        self.graphs = list(graphs)
        self.count = len(graphs)
        self.levels = levels or [torch.empty(g.n, dtype=torch.int32, device=dev) for g in graphs]
        self.parents = parents or [torch.empty(g.n, dtype=torch.int32, device=dev) for g in graphs]
        self.sigmas = [torch.empty(g.n, dtype=torch.int64, device=dev) for g in graphs] if counts else None
        src = (ctypes.c_uint32 * self.count)(*[int(s) for s in sources])
        h = ctypes.c_void_p()
        gp = _ptr_array([g.handle.value for g in graphs])
        lp = _ptr_array([t.data_ptr() for t in self.levels])
        pp = _ptr_array([t.data_ptr() for t in self.parents])
        pr = ctypes.byref(params) if params else None
        if counts:
            rc = load().abfs_batch_create_counts(gp, src, self.count, lp, pp,
                                                 _ptr_array([t.data_ptr() for t in self.sigmas]),
                                                 pr, _stream_ptr(stream), ctypes.byref(h))
            _check(rc, "abfs_batch_create_counts")
        else:
            rc = load().abfs_batch_create(gp, src, self.count, lp, pp, pr, _stream_ptr(stream),
                                          ctypes.byref(h))
            _check(rc, "abfs_batch_create")
        self.handle = h

    def launch(self, stream=None) -> None:
        _check(load().abfs_batch_launch(self.handle, _stream_ptr(stream)), "abfs_batch_launch")

    def status(self, stream=None) -> list[int]:
        st = (ctypes.c_int32 * self.count)()
        load().abfs_batch_status(self.handle, _stream_ptr(stream), st)
        return list(st)

    def destroy(self) -> None:
        if self.handle and self.handle.value:
            _check(load().abfs_batch_destroy(self.handle), "abfs_batch_destroy")
            self.handle = ctypes.c_void_p(0)

    def __del__(self):
        try:
            if _lib is not None and self.handle and self.handle.value:
                _lib.abfs_batch_destroy(self.handle)
        except Exception:
            pass


def run_static(colptr, rowidx, source: int, level, parent, stream=None) -> int:
    """abfs_run_static: one search with the library's fixed device scratch array
    (no allocation).  colptr/rowidx/level/parent are CUDA tensors; returns the
    status code."""
    n = colptr.numel() - 1
    return load().abfs_run_static(colptr.data_ptr(), rowidx.data_ptr() if rowidx.numel() else None,
                                  n, rowidx.numel(), int(source), level.data_ptr(),
                                  parent.data_ptr(), _stream_ptr(stream))


def serve_default_cfg(**overrides) -> ServeCfg:
    c = ServeCfg()
    _check(load().abfs_serve_default_cfg(ctypes.byref(c)), "abfs_serve_default_cfg")
    for k, v in overrides.items():
        setattr(c, k, v)
    return c


class Server:
    """abfs_serve_*: continuous batching of BFS queries on resident graphs."""

    def __init__(self, graphs: list[Graph], cfg: ServeCfg | None = None):
        self.graphs = list(graphs)
        h = ctypes.c_void_p()
        rc = load().abfs_serve_start(_ptr_array([g.handle.value for g in self.graphs]),
                                     len(self.graphs), ctypes.byref(cfg) if cfg else None,
                                     ctypes.byref(h))
        _check(rc, "abfs_serve_start")
        self.handle = h

    def submit(self, graph_idx: int, source: int, level, parent) -> int | None:
        """Queues a query into the caller's device tensors; None when the queue is full."""
        t = ctypes.c_uint64()
        rc = load().abfs_serve_submit(self.handle, int(graph_idx), int(source), level.data_ptr(),
                                      parent.data_ptr(), ctypes.byref(t))
        if rc == ERR_BUSY:
            return None
        _check(rc, "abfs_serve_submit")
        return int(t.value)

    def poll(self, ticket: int):
        done = ctypes.c_int()
        st = ctypes.c_int32()
        _check(load().abfs_serve_poll(self.handle, ticket, ctypes.byref(done), ctypes.byref(st)),
               "abfs_serve_poll")
        return bool(done.value), int(st.value)

    def wait(self, ticket: int, timeout_ms: int = 60000) -> int:
        st = ctypes.c_int32()
        _check(load().abfs_serve_wait(self.handle, ticket, timeout_ms, ctypes.byref(st)),
               "abfs_serve_wait")
        return int(st.value)

    def stop(self) -> dict:
        rep = ServeReport()
        h, self.handle = self.handle, ctypes.c_void_p(0)
        _check(load().abfs_serve_stop(h, ctypes.byref(rep)), "abfs_serve_stop")
        return rep.as_dict()

    def __del__(self):
        try:
            if _lib is not None and self.handle and self.handle.value:
                _lib.abfs_serve_stop(self.handle, None)
        except Exception:
            pass


def tune(g: Graph, sources, mode: int = MODE_SUBMATRIX, cache_path: str | None = None,
         stream=None):
    """abfs_tune: returns (best Params, mean ms per search)."""
    count = len(sources)
    src = (ctypes.c_uint32 * count)(*[int(s) for s in sources])
    best = Params()
    ms = ctypes.c_float()
    rc = load().abfs_tune(g.handle, src, count, mode,
                          cache_path.encode() if cache_path else None, _stream_ptr(stream),
                          ctypes.byref(best), ctypes.byref(ms))
    _check(rc, "abfs_tune")
    return best, float(ms.value)


def batch_tune(graphs: list[Graph], sources, mode: int = MODE_SUBMATRIX,
               cache_path: str | None = None, stream=None):
    """abfs_batch_tune: (best Params for the whole batch, mean ms per launch)."""
    count = len(graphs)
    src = (ctypes.c_uint32 * count)(*[int(s) for s in sources])
    best = Params()
    ms = ctypes.c_float()
    rc = load().abfs_batch_tune(_ptr_array([g.handle.value for g in graphs]), src, count, mode,
                                cache_path.encode() if cache_path else None, _stream_ptr(stream),
                                ctypes.byref(best), ctypes.byref(ms))
    _check(rc, "abfs_batch_tune")
    return best, float(ms.value)
