"""Multi-source searches: batch queries on one undirected graph with ascending
columns run as one search of up to 64 sources, one bit per source in a 64-bit
mask per vertex (x_{k+1} = A X_k, Theorem 1 applied column by column).  Every
source's levels and least-index parents must equal the oracle's, bit for bit.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1906_03113_gb300 as abfs  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    abfs.build()
    abfs.load()
    torch.cuda.set_device(0)


def _check(g, src, level, parent, ctx):
    lo, po = oracle.bfs(g, src)
    lev = level.cpu().numpy()
    par = parent.cpu().numpy()
    bad = np.nonzero(lev != lo)[0]
    assert bad.size == 0, f"{ctx}: level mismatch at {bad[:8]} ({lev[bad[:8]]} vs {lo[bad[:8]]})"
    bad = np.nonzero(par != po)[0]
    assert bad.size == 0, f"{ctx}: parent mismatch at {bad[:8]} ({par[bad[:8]]} vs {po[bad[:8]]})"


MS = abfs.default_params(multi_source=2)


def test_every_undirected_graph_on_5_vertices_all_sources_in_one_search():
    pairs = [(i, j) for i in range(5) for j in range(i + 1, 5)]
    graphs, srcs, hosts = [], [], []
    dev = []
    for mask in range(1 << len(pairs)):
        arcs = [pairs[b] for b in range(len(pairs)) if mask >> b & 1]
        g = synth.from_arcs(5, [a for a, _ in arcs], [b for _, b in arcs], directed=False)
        G = abfs.graph_create(g.colptr, g.rowidx, directed=False)
        dev.append(G)
        for s in range(5):
            graphs.append(G)
            srcs.append(s)
            hosts.append(g)
    levels, parents, st = abfs.run_batch(graphs, srcs, params=MS)
    torch.cuda.synchronize()
    assert all(x == 0 for x in st)
    for g, s, L, P in zip(hosts, srcs, levels, parents):
        _check(g, s, L, P, "tiny multi-source")
    for G in dev:
        G.destroy()


CASES = {
    "rmat_14_100_sources": (lambda: synth.rmat(14, 16.0, seed=3), 100),
    "er_2000_repeated": (lambda: synth.er(2000, 3.0, seed=2), 40),
    "grid_100x37": (lambda: synth.grid(100, 37), 9),
    "two_components": (lambda: synth.from_arcs(100, list(range(49)) + list(range(50, 99)),
                                               list(range(1, 50)) + list(range(51, 100)),
                                               directed=False), 12),
    "star": (lambda: synth.from_arcs(3001, [0] * 3000, list(range(1, 3001)), directed=False), 64),
    "path_3000": (lambda: synth.from_arcs(3000, list(range(2999)), list(range(1, 3000)),
                                          directed=False), 33),
}


@pytest.mark.parametrize("name", list(CASES))
def test_multi_source_equals_oracle(name):
    make, count = CASES[name]
    g = make()
    G = abfs.graph_create(g.colptr, g.rowidx, directed=False)
    rng = np.random.default_rng(5)
    srcs = [int(x) for x in rng.integers(g.n, size=count)]
    if name == "er_2000_repeated":
        srcs = srcs[:20] + srcs[:20]          # every source twice in one search
    if name == "star":
        srcs[0] = 0                           # the centre and many leaves
    for p in (MS, abfs.default_params(multi_source=2, tile=64, unit_entries=256, narrow_max=0,
                                      narrow_edges=0)):
        levels, parents, st = abfs.run_batch([G] * len(srcs), srcs, params=p)
        torch.cuda.synchronize()
        assert all(x == 0 for x in st), st
        for s, L, P in zip(srcs, levels, parents):
            _check(g, s, L, P, f"{name} src {s}")
    G.destroy()


def test_mixed_batch_groups_only_where_allowed():
    """Undirected sorted graphs group; a directed graph and an undirected graph
    with shuffled columns run as single searches; all in one launch, replayed
    from a CUDA graph twice."""
    u = synth.rmat(12, 8.0, seed=11)
    d = synth.rgg_knn(1 << 12, 4, seed=12)
    rng = np.random.default_rng(3)
    rows = u.rowidx.copy()
    for v in range(u.n):
        a, b = int(u.colptr[v]), int(u.colptr[v + 1])
        rows[a:b] = rng.permutation(rows[a:b])
    U = abfs.graph_create(u.colptr, u.rowidx, directed=False)
    D = abfs.graph_create(d.colptr, d.rowidx, directed=True)
    S = abfs.graph_create(u.colptr, rows, directed=False)
    graphs, srcs, hosts = [], [], []
    for G, h in ((U, u), (D, d), (S, u)):
        for s in rng.integers(h.n, size=10):
            graphs.append(G)
            srcs.append(int(s))
            hosts.append(h)
    plan = abfs.BatchPlan(graphs, srcs, params=MS)
    for rep in range(2):
        for L in plan.levels:
            L.fill_(9)
        plan.launch()
        assert plan.status() == [0] * len(graphs)
        for h, s, L, P in zip(hosts, srcs, plan.levels, plan.parents):
            _check(h, s, L, P, f"mixed rep {rep}")
    plan.destroy()
    for G in (U, D, S):
        G.destroy()
