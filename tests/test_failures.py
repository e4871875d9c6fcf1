"""Failure paths of the library, made to happen without faulting or hanging a
GPU.

  * A bounded device wait that runs out: the host control
    abfs_test_hold_first_phase makes each search's first phase wait for work
    units that never come; the engine's idle wait (bounded by timeout_ms without
    progress) expires, the search reports ABFS_ERR_TIMEOUT, the launch returns,
    and the context stays usable (the next search is bit-exact with the oracle).
  * An allocator hook that fails at its N-th call: every call that allocates
    returns ABFS_ERR_OOM and frees what it had allocated (no leak).
  * Serving with a memory budget that holds no query: start-up refuses it.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth

import paper_1906_03113_gb300 as abfs
from paper_1906_03113_gb300 import binding

ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class FailingHook:
    """Allocator hook that fails at its fail_at-th call (0: never) and counts
    the blocks it handed out and got back.  host=True hands out host memory
    (for host-only error paths on a machine without a GPU)."""

    def __init__(self, fail_at: int, host: bool, shift: int = 0):
        self.fail_at, self.host, self.shift = fail_at, host, shift
        self.calls = 0
        self.live = {}
        if host:
            self.libc = ctypes.CDLL(None)
            self.libc.malloc.restype = ctypes.c_void_p
            self.libc.malloc.argtypes = [ctypes.c_size_t]
            self.libc.free.argtypes = [ctypes.c_void_p]
        self._a = ALLOC(self._alloc)
        self._f = FREE(self._free)

    def _alloc(self, nbytes, ctx):
        self.calls += 1
        if self.fail_at and self.calls >= self.fail_at:
            return None
        if self.host:
            p = self.libc.malloc(nbytes + 16) + self.shift
        else:
            import torch
            t = torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")
            p = t.data_ptr()
            self.live[p] = t
            return p
        self.live[p] = nbytes
        return p

    def _free(self, p, ctx):
        obj = self.live.pop(p)
        if self.host:
            self.libc.free(p - self.shift)
        del obj

    def install(self, lib):
        assert lib.abfs_set_allocator(ctypes.cast(self._a, ctypes.c_void_p),
                                      ctypes.cast(self._f, ctypes.c_void_p), None) == 0

    @staticmethod
    def remove(lib):
        assert lib.abfs_set_allocator(None, None, None) == 0


@pytest.fixture(scope="module")
def lib():
    abfs.build()
    return abfs.load()


def test_hold_control_needs_no_device(lib):
    assert lib.abfs_test_hold_first_phase(3) == 0
    assert lib.abfs_test_hold_first_phase(0) == 0


def test_allocator_failure_on_the_host_path(lib):
    """graph_create allocates the column pointers and the row indices before
    any copy: a hook failing at the first or second call gives ABFS_ERR_OOM and
    the block already handed out is returned."""
    cp = (ctypes.c_uint32 * 3)(0, 1, 2)
    rows = (ctypes.c_uint32 * 2)(1, 0)
    for n_fail in (1, 2):
        hook = FailingHook(n_fail, host=True)
        hook.install(lib)
        try:
            out = ctypes.c_void_p()
            rc = lib.abfs_graph_create(cp, rows, 2, 2, 0, 0, None, ctypes.byref(out))
        finally:
            FailingHook.remove(lib)
        assert rc == binding.ERR_OOM and not out.value
        assert hook.calls == n_fail and not hook.live


def test_allocator_blocks_off_16_byte_alignment_are_refused(lib):
    """A hook block that is not 16-byte aligned goes back to the hook and the
    call fails with ABFS_ERR_INVALID_ARG before anything reads it."""
    cp = (ctypes.c_uint32 * 3)(0, 1, 2)
    rows = (ctypes.c_uint32 * 2)(1, 0)
    for shift in (4, 8):
        hook = FailingHook(0, host=True, shift=shift)
        hook.install(lib)
        try:
            out = ctypes.c_void_p()
            rc = lib.abfs_graph_create(cp, rows, 2, 2, 0, 0, None, ctypes.byref(out))
        finally:
            FailingHook.remove(lib)
        assert rc == binding.ERR_INVALID_ARG and not out.value
        assert hook.calls == 1 and not hook.live


# ---------------------------------------------------------------------------
# on a GPU
# ---------------------------------------------------------------------------

def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    return torch


@pytest.mark.gpu
def test_bounded_wait_runs_out_with_timeout_status(lib):
    torch = _gpu()
    g = synth.rmat(12, 8.0, seed=5)
    G = abfs.graph_create(g.colptr, g.rowidx, directed=False)
    s = int(np.argmax(g.degrees()))
    p = abfs.default_params(timeout_ms=5)
    assert lib.abfs_test_hold_first_phase(1) == 0
    try:
        with pytest.raises(abfs.AbfsError) as ei:
            abfs.run(G, s, params=p, stats=True)
        assert ei.value.status == binding.ERR_TIMEOUT
        with pytest.raises(abfs.AbfsError) as ei:
            abfs.run_host(G, s, params=p)
        assert ei.value.status == binding.ERR_TIMEOUT
        # a batch of three: every search times out, the launch returns
        _, _, st = abfs.run_batch([G] * 3, [s, 0, 1], params=p)
        assert st == [binding.ERR_TIMEOUT] * 3
        # many searches into host memory: each search's own status comes back
        _, _, st = abfs.run_host_many(G, [s, 0, 1], params=p)
        assert st == [binding.ERR_TIMEOUT] * 3
    finally:
        assert lib.abfs_test_hold_first_phase(0) == 0
    torch.cuda.synchronize()
    # the context is still usable and the next search is exact
    level, parent = abfs.run(G, s)
    lo, po = oracle.bfs(g, s)
    assert np.array_equal(level.cpu().numpy(), lo) and np.array_equal(parent.cpu().numpy(), po)
    G.destroy()


@pytest.mark.gpu
def test_allocator_failing_at_each_call(lib):
    """graph_create and the first abfs_run (which allocates the search
    workspace) under a hook that fails at call N, for every N that any of them
    reaches: the failing call returns ABFS_ERR_OOM, nothing leaks, and with the
    hook removed the same graph searches exactly."""
    torch = _gpu()
    g = synth.er(3000, 4.0, seed=21)
    lo, po = oracle.bfs(g, 0)
    level = torch.empty(g.n, dtype=torch.int32, device="cuda")
    parent = torch.empty(g.n, dtype=torch.int32, device="cuda")
    # how many allocations a full create + run makes
    probe = FailingHook(0, host=False)
    probe.install(lib)
    try:
        G = abfs.graph_create(g.colptr, g.rowidx, directed=False)
        abfs.run(G, 0, level, parent, stats=True)
        G.destroy()
    finally:
        FailingHook.remove(lib)
    total = probe.calls
    assert total >= 5 and not probe.live
    for n_fail in range(1, total + 1):
        hook = FailingHook(n_fail, host=False)
        hook.install(lib)
        G = None
        try:
            try:
                G = abfs.graph_create(g.colptr, g.rowidx, directed=False)
                rc = None
            except abfs.AbfsError as exc:
                rc = exc.status
            if G is not None:
                with pytest.raises(abfs.AbfsError) as ei:
                    abfs.run(G, 0, level, parent, stats=True)
                rc = ei.value.status
                G.destroy()
        finally:
            FailingHook.remove(lib)
        assert rc == binding.ERR_OOM, n_fail
        assert not hook.live, (n_fail, list(hook.live))
    G = abfs.graph_create(g.colptr, g.rowidx, directed=False)
    abfs.run(G, 0, level, parent)
    assert np.array_equal(level.cpu().numpy(), lo) and np.array_equal(parent.cpu().numpy(), po)
    G.destroy()


@pytest.mark.gpu
def test_serving_budget_that_holds_no_query_is_refused(lib):
    _gpu()
    g = synth.er(3000, 4.0, seed=21)
    G = abfs.graph_create(g.colptr, g.rowidx, directed=False)
    for budget in (0, G.footprint() // 2):
        with pytest.raises(abfs.AbfsError) as ei:
            abfs.Server([G], abfs.serve_default_cfg(memory_budget=budget))
        assert ei.value.status == binding.ERR_OOM
    G.destroy()
