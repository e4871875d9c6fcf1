"""Section 11's operation counts (Table 2's columns) measured on the device
against the oracle's op_counts, which runs each method's loop on the CPU.

  * Algorithm 2 multiplies one nonzero per reached row other than the source
    (Theorem 2): 2 (n_c - 1) operations, from the device's reached count.
  * Masked SpMSpV multiplies every nonzero of every reached column: 2 nnz_c,
    from the comparator's multiplied-entry counter.
  * Theorem 1's exact mask multiplies the entries j -> i with
    level(i) = level(j) + 1 (E_adj), counted by the submatrix engine as the
    entries that pass the mask; E_adj <= m (Lemma 3).
  * The all-nonzero variant of Algorithm 2 (Section 9) multiplies each edge of
    an undirected reached component once, 2 m_c = nnz_c operations
    (Section 11): the oracle's count must equal the device's nnz_c.
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


def _e_adj(g, lev):
    cols = np.repeat(np.arange(g.n), g.degrees())
    lj = lev[cols]
    li = lev[g.rowidx.astype(np.int64)]
    return int(((lj >= 0) & (li == lj + 1)).sum())


GRAPHS = {
    "er_2000": lambda: synth.er(2000, 3.0, seed=2),
    "rmat_14": lambda: synth.rmat(14, 16.0, seed=3),
    "grid_100x37": lambda: synth.grid(100, 37),
    "rgg_2_15": lambda: synth.rgg_knn(1 << 15, 4, seed=4),
    "two_components": lambda: synth.from_arcs(100, list(range(49)) + list(range(50, 99)),
                                              list(range(1, 50)) + list(range(51, 100)),
                                              directed=False),
}


@pytest.mark.parametrize("name", list(GRAPHS))
def test_device_counts_equal_oracle_op_counts(name):
    g = GRAPHS[name]()
    G = abfs.graph_create(g.colptr, g.rowidx, directed=g.directed)
    deg = g.degrees()
    srcs = sorted({0, int(np.argmax(deg)), int(np.nonzero(deg > 0)[0][0])})
    m = g.nnz if g.directed else g.nnz // 2
    for s in srcs:
        oc = oracle.op_counts(g, s)
        lev_o, _ = oracle.bfs(g, s)
        _, _, sub = abfs.run(G, s, params=abfs.default_params(), stats=True)
        _, _, pl = abfs.run(G, s, params=abfs.default_params(mode=abfs.MODE_PLAIN), stats=True)
        assert sub["status"] == 0 and pl["status"] == 0
        assert sub["reached"] == oc["n_c"] and sub["nnz_reached"] == oc["nnz_c"]
        assert sub["levels"] == oc["levels"] == pl["levels"]
        assert 2 * (sub["reached"] - 1) == oc["alg2"], (name, s)
        assert 2 * pl["entries_read"] == oc["spmmspv"], (name, s)
        assert 2 * g.nnz * sub["levels"] == oc["spmv"], (name, s)
        e_adj = _e_adj(g, lev_o)
        assert sub["entries_unmasked"] == e_adj <= m, (name, s)
        if not g.directed:
            assert oc["alg2_all_nonzero"] == sub["nnz_reached"], (name, s)
            # Theorem 1's multiplies never exceed the all-nonzero variant's
            assert 2 * e_adj <= oc["alg2_all_nonzero"]
    G.destroy()
