"""The allocation-free entry point abfs_run_static, checked against abfs_run.

abfs_run_static serves callers that cannot allocate device memory (the
library's graph copy and workspace come from cudaMalloc): its scratch is a
fixed device array inside libabfs.so.  These tests call it through the C-ABI
twice in a row -- the array keeps the previous call's contents, so the second
call checks that everything a search needs at zero is cleared -- and compare
its outputs with abfs_run's.  This file is collected last on purpose.
"""
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


@pytest.mark.parametrize("name", ["er_2_16", "rmat_16", "grid_300"])
def test_static_matches_run_on_two_calls_in_a_row(name):
    g = {"er_2_16": synth.er_2_16, "rmat_16": lambda: synth.rmat(16, 16.0, seed=5),
         "grid_300": lambda: synth.grid(300, 300)}[name]()
    cp, ri = _device_csc(g)
    G = abfs.graph_create(g.colptr, g.rowidx, directed=g.directed)
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
