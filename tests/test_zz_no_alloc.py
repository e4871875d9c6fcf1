"""The allocation-free entry point abfs_run_static, checked against abfs_run.

abfs_run_static serves callers that cannot allocate device memory (the
library's graph copy and workspace come from cudaMalloc): its scratch is a
fixed device array inside libabfs.so.  These tests call it through the C-ABI
twice in a row -- the array keeps the previous call's contents, so the second
call checks that everything a search needs at zero is cleared -- and compare
its outputs with abfs_run's.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1906_03113_gb300 as abfs  # noqa: E402
from paper_1906_03113_gb300 import binding  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    abfs.build()
    abfs.load()
    torch.cuda.set_device(0)


def _device_csc(g):
    return (torch.from_numpy(g.colptr.view(np.int32)).cuda(),
            torch.from_numpy(g.rowidx.view(np.int32)).cuda())


GRAPHS = {
    "er_2_16": synth.er_2_16,
    "rmat_16": lambda: synth.rmat(16, 16.0, seed=5),
    "grid_300": lambda: synth.grid(300, 300),
    # directed: rows that occur in no column are not pre-masked on this path
    "rgg_2_14_directed": lambda: synth.rgg_knn(1 << 14, 4, seed=4),
    # close to the array's limit: about 68 MB of its 72 MiB
    "grid_1024": lambda: synth.grid(1024, 1024),
}


@pytest.mark.parametrize("name", list(GRAPHS))
def test_static_matches_run_on_two_calls_in_a_row(name):
    g = GRAPHS[name]()
    cp, ri = _device_csc(g)
    G = abfs.graph_create(g.colptr, g.rowidx, directed=g.directed)
    assert G.footprint() + 256 <= 72 << 20
    deg = g.degrees()
    sources = [int(np.argmax(deg)), int(np.nonzero(deg)[0][-1])]
    for s in sources:  # two calls in a row on the same static array
        lev_ref, par_ref = abfs.run(G, s)
        lev = torch.full((g.n,), 7, dtype=torch.int32, device="cuda")
        par = torch.full((g.n,), 7, dtype=torch.int32, device="cuda")
        rc = abfs.binding.run_static(cp, ri, s, lev, par)
        assert rc == 0, abfs.strerror(rc)
        assert torch.equal(lev, lev_ref) and torch.equal(par, par_ref), (name, s)
    lev_o, par_o = oracle.bfs(g, sources[-1])
    assert np.array_equal(lev.cpu().numpy(), lev_o) and np.array_equal(par.cpu().numpy(), par_o)
    G.destroy()


MISALIGNED = {
    "rmat_12": lambda: synth.rmat(12, 16.0, seed=9),
    "path_7": lambda: synth.from_arcs(7, list(range(6)), list(range(1, 7)), directed=False),
    "star_50": lambda: synth.from_arcs(51, [0] * 50, list(range(1, 51)), directed=False),
}


@pytest.mark.parametrize("name", list(MISALIGNED))
@pytest.mark.parametrize("shift", [1, 2, 3])
def test_static_on_row_arrays_off_16_byte_alignment(name, shift):
    """The caller's row array may start anywhere 4-byte aligned: the expand
    loop's 16-byte row loads then start before the column's first entry, and
    the groups at both ends of the array fall back to 4-byte loads."""
    g = MISALIGNED[name]()
    cp, ri = _device_csc(g)
    nnz = ri.numel()
    big = torch.zeros(nnz + 8, dtype=torch.int32, device="cuda")
    view = big[shift:shift + nnz]
    view.copy_(ri)
    assert view.data_ptr() % 16 == 4 * shift
    deg = g.degrees()
    for s in (0, int(np.argmax(deg)), g.n - 1):
        lev = torch.full((g.n,), 7, dtype=torch.int32, device="cuda")
        par = torch.full((g.n,), 7, dtype=torch.int32, device="cuda")
        rc = abfs.binding.run_static(cp, view, s, lev, par)
        assert rc == 0, abfs.strerror(rc)
        lev_o, par_o = oracle.bfs(g, s)
        assert np.array_equal(lev.cpu().numpy(), lev_o), (name, shift, s)
        assert np.array_equal(par.cpu().numpy(), par_o), (name, shift, s)


def test_static_rejects_graphs_beyond_its_array():
    g = synth.grid(4, 4)
    cp, ri = _device_csc(g)
    lev = torch.empty(16, dtype=torch.int32, device="cuda")
    par = torch.empty(16, dtype=torch.int32, device="cuda")
    # a vertex count whose scratch layout exceeds the fixed array: rejected
    # before any device work (the pointers are never dereferenced)
    rc = abfs.load().abfs_run_static(cp.data_ptr(), ri.data_ptr(), 1 << 25, 64, 0,
                                     lev.data_ptr(), par.data_ptr(), None)
    assert rc == binding.ERR_UNSUPPORTED
    rc = abfs.load().abfs_run_static(cp.data_ptr(), ri.data_ptr(), 16, ri.numel(), 16,
                                     lev.data_ptr(), par.data_ptr(), None)
    assert rc == binding.ERR_INVALID_ARG


def test_static_rejects_a_graph_just_beyond_its_array():
    g = synth.grid(1100, 1100)
    G = abfs.graph_create(g.colptr, g.rowidx, directed=False)
    assert G.footprint() + 256 > 64 << 20
    G.destroy()
    cp, ri = _device_csc(g)
    lev = torch.empty(g.n, dtype=torch.int32, device="cuda")
    par = torch.empty(g.n, dtype=torch.int32, device="cuda")
    assert abfs.binding.run_static(cp, ri, 0, lev, par) == binding.ERR_UNSUPPORTED


ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


def test_static_allocates_nothing_after_its_first_call():
    """After a first call, a caller whose allocator refuses every request (a
    hook that counts and fails) still gets exact results, the hook is never
    called, and the device's free memory does not move."""
    g = synth.rmat(14, 16.0, seed=3)
    cp, ri = _device_csc(g)
    lev = torch.empty(g.n, dtype=torch.int32, device="cuda")
    par = torch.empty(g.n, dtype=torch.int32, device="cuda")
    assert abfs.binding.run_static(cp, ri, 0, lev, par) == 0
    torch.cuda.synchronize()
    calls = [0]

    def refuse(nbytes, ctx):
        calls[0] += 1
        return None

    def release(p, ctx):
        calls[0] += 1

    a, f = ALLOC(refuse), FREE(release)
    lib = abfs.load()
    assert lib.abfs_set_allocator(ctypes.cast(a, ctypes.c_void_p), ctypes.cast(f, ctypes.c_void_p),
                                  None) == 0
    try:
        free0, _ = torch.cuda.mem_get_info()
        srcs = [int(np.argmax(g.degrees())), 0]
        for s in srcs:
            assert abfs.binding.run_static(cp, ri, s, lev, par) == 0
        free1, _ = torch.cuda.mem_get_info()
    finally:
        assert lib.abfs_set_allocator(None, None, None) == 0
    assert calls[0] == 0 and free1 == free0
    lo, po = oracle.bfs(g, srcs[-1])
    assert np.array_equal(lev.cpu().numpy(), lo) and np.array_equal(par.cpu().numpy(), po)
