"""The CPU baselines (Algorithm 2 sequential, Algorithm 3 with OpenMP) against
the oracle: levels equal oracle.bfs element by element; every parent is a
valid predecessor (an entry v of column parent[v] with level[parent[v]] =
level[v] - 1), since both methods resolve concurrent or repeated writes in
their own order (Section 10 allows any).  Planted mistakes in a copy of the
outputs are caught by the same checks."""
import numpy as np
import pytest

import cpu_baselines
import oracle
import synth


def _valid(g, src, lev, par):
    lo, _ = oracle.bfs(g, src)
    assert np.array_equal(lev, lo)
    reached = np.nonzero(lo >= 0)[0]
    assert par[src] == src
    assert np.all(par[lo < 0] == -1)
    deg = g.degrees()
    for v in reached:
        if v == src:
            continue
        p = int(par[v])
        assert 0 <= p < g.n and lo[p] == lo[v] - 1, (v, p)
        col = g.rowidx[g.colptr[p]:g.colptr[p] + deg[p]]
        assert v in col, (v, p)


GRAPHS = [
    ("fig1", lambda: synth.from_arcs(5, [0, 1, 2, 2], [3, 4, 3, 4], directed=False)),
    ("er_3000", lambda: synth.er(3000, 4.0, seed=2)),
    ("rmat_12", lambda: synth.rmat(12, 16.0, seed=3)),
    ("grid_30x17", lambda: synth.grid(30, 17)),
    ("rgg_4096", lambda: synth.rgg_knn(4096, 4, seed=4)),
    ("two_components", lambda: synth.from_arcs(40, list(range(19)) + list(range(20, 39)),
                                               list(range(1, 20)) + list(range(21, 40)),
                                               directed=False)),
    ("no_edges", lambda: synth.from_arcs(9, [], [], directed=False)),
    ("one_vertex", lambda: synth.from_arcs(1, [], [], directed=False)),
]


@pytest.mark.parametrize("name,make", GRAPHS, ids=[x[0] for x in GRAPHS])
def test_alg2_and_alg3_match_oracle(name, make):
    g = make()
    deg = g.degrees()
    srcs = sorted({0, g.n - 1, int(np.argmax(deg))})
    for s in srcs:
        lev, par, t = cpu_baselines.alg2(g, s)
        assert t >= 0
        _valid(g, s, lev, par)
        for threads in (1, 3, 8):
            lev, par, t, used = cpu_baselines.alg3(g, s, threads)
            assert t >= 0 and used >= 1
            _valid(g, s, lev, par)


def test_alg2_parent_is_first_discoverer_on_figure1():
    # Figure 1 from vertex 1 (0-based): the list order decides the parents
    g = synth.from_arcs(5, [0, 1, 2, 2], [3, 4, 3, 4], directed=False)
    lev, par, _ = cpu_baselines.alg2(g, 1)
    assert lev.tolist() == [4, 0, 2, 3, 1]
    assert par.tolist() == [3, 1, 4, 2, 1]


def test_checks_catch_planted_mistakes():
    g = synth.rmat(10, 8.0, seed=7)
    s = int(np.argmax(g.degrees()))
    lev, par, _ = cpu_baselines.alg2(g, s)
    bad = lev.copy()
    v = int(np.nonzero(lev == 2)[0][0])
    bad[v] = 3
    with pytest.raises(AssertionError):
        _valid(g, s, bad, par)
    badp = par.copy()
    badp[v] = s  # a vertex two levels down cannot hang from the source
    with pytest.raises(AssertionError):
        _valid(g, s, lev, badp)


def test_timing_harness_reports_cores():
    g = synth.er(3000, 4.0, seed=2)
    rows = cpu_baselines.time_baselines(g, [0, 1], budget_s=2.0, reps=3)
    kinds = [r["kind"] for r in rows]
    assert kinds == ["alg2_sequential", "alg3_openmp"]
    for r in rows:
        assert r["value"] > 0 and r["cores"] >= 1 and r["host_cores"] >= 1
