"""Pins of the CPU oracle against what the paper and mathematics fix.

Nothing here compares the oracle with itself: every check is against a value
the paper prints (Figure 1, the Section 6 example, Tables 1-2), a closed form,
brute force (Floyd-Warshall over every small graph) or an identity the paper
proves (Theorem 1, Claim 1, Theorem 2, Lemma 3, Proposition 1).  The last
block plants plausible mistakes in copies of the oracle's logic and checks that
the pins catch each of them.
"""
import itertools

import numpy as np
import pytest

import oracle
import synth
from conftest import golden_path


# ---------------------------------------------------------------------------
# fixture readers
# ---------------------------------------------------------------------------

def _read_kv(name):
    out = {}
    rows = []
    in_rows = False
    for line in open(golden_path(name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line == "rows":
            in_rows = True
            continue
        parts = line.split()
        if in_rows and all(p in "01" for p in parts):
            rows.append([int(p) for p in parts])
            continue
        in_rows = False
        out[parts[0]] = parts[1:]
    return out, rows


def _fig1():
    kv, _ = _read_kv("fig1_path.txt")
    n = int(kv["n"][0])
    edges = [tuple(int(x) - 1 for x in e.split("-")) for e in kv["edges"]]
    src = int(kv["source"][0]) - 1
    frontiers = [[int(x) - 1 for x in grp.split(",")] for grp in " ".join(kv["frontiers"]).split("|")]
    V = [[int(x) - 1 for x in grp.strip().split(",")] for grp in " ".join(kv["V"]).split("|")]
    levels = {int(a) - 1: int(b) for a, b in (p.split(":") for p in kv["levels"])}
    parents = {int(a) - 1: int(b) - 1 for a, b in (p.split(":") for p in kv["parents"])}
    g = synth.from_arcs(n, [a for a, b in edges], [b for a, b in edges], directed=False)
    return g, src, frontiers, V, levels, parents


# ---------------------------------------------------------------------------
# values the paper prints
# ---------------------------------------------------------------------------

def test_fig1_levels_parents_frontiers():
    g, src, frontiers, V, levels, parents = _fig1()
    for fn in (oracle.bfs, oracle.bfs_levelsync, oracle.bfs_dense_mask):
        lev, par = fn(g, src)
        assert [int(x) for x in lev] == [levels[v] for v in range(g.n)], fn.__name__
        assert [int(x) for x in par] == [parents[v] for v in range(g.n)], fn.__name__
    _, _, fs = oracle.bfs(g, src, with_frontiers=True)
    assert fs.tolist() == [len(f) for f in frontiers]


def test_fig1_mask_sets():
    g, src, frontiers, V, _, _ = _fig1()
    _, _, steps = oracle.bfs_dense_mask(g, src, record=True)
    assert [s for s, _ in steps] == [sorted(f) for f in frontiers]
    assert [v for _, v in steps] == [sorted(x) for x in V]


def test_sec6_outer_product_example():
    kv, rows = _read_kv("sec6_outer_product.txt")
    A = np.array(rows, dtype=bool)
    assert (A == A.T).all()
    x = [int(v) - 1 for v in kv["x"]]
    assert np.nonzero(A[:, 1])[0].tolist() == [int(v) - 1 for v in kv["col2"]]
    assert np.nonzero(A[:, 2])[0].tolist() == [int(v) - 1 for v in kv["col3"]]
    assert oracle.spmv_step(A, x).tolist() == [int(v) - 1 for v in kv["product"]]
    allowed = sorted(set(range(5)) - set(x))
    assert oracle.spmv_step(A, x, row_mask=allowed).tolist() == [int(v) - 1 for v in kv["masked_product"]]


def _table2():
    rows = []
    for line in open(golden_path("table2_ops.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, n, m, D, a2, spmm, spmv, kind = line.split()
        rows.append((name, int(n), int(m), int(D), int(a2), int(spmm), int(spmv), kind))
    return rows


@pytest.mark.parametrize("row", _table2(), ids=lambda r: r[0])
def test_table2_closed_forms(row):
    name, n, m, D, a2, spmm, spmv, kind = row
    if kind == "full":
        cf = oracle.closed_form_counts(n_c=n, nnz_c=2 * m, nnz=2 * m, levels=D + 1)
        assert cf["alg2"] == a2
        assert cf["spmmspv"] == spmm
        assert cf["spmv"] == spmv
    else:
        cf = oracle.closed_form_counts(n_c=1, nnz_c=0, nnz=2 * m, levels=D + 1)
        assert cf["spmv"] == spmv
        # the road-network source reaches part of the graph: fewer ops than a full search
        assert a2 < 2 * (n - 1) and spmm < 4 * m


# ---------------------------------------------------------------------------
# brute force over every small graph
# ---------------------------------------------------------------------------

def _all_graphs(n, directed):
    pairs = ([(i, j) for i in range(n) for j in range(n) if i != j] if directed
             else [(i, j) for i in range(n) for j in range(i + 1, n)])
    for mask in range(1 << len(pairs)):
        arcs = [pairs[b] for b in range(len(pairs)) if mask >> b & 1]
        yield arcs


def _graph(n, arcs, directed):
    return synth.from_arcs(n, [a for a, _ in arcs], [b for _, b in arcs], directed=directed)


@pytest.mark.parametrize("n,directed", [(1, False), (2, False), (3, False), (4, False), (5, False),
                                        (2, True), (3, True), (4, True)])
def test_exhaustive_vs_floyd_warshall(n, directed):
    for arcs in _all_graphs(n, directed):
        g = _graph(n, arcs, directed)
        M = oracle.dense_matrix(g)
        D = oracle.floyd_warshall(M)
        for s in range(n):
            lev, par = oracle.bfs(g, s)
            assert lev.tolist() == D[s].tolist(), (arcs, s)
            assert par.tolist() == oracle.parents_from_distances(M, D[s], s).tolist(), (arcs, s)
            lev2, par2 = oracle.bfs_dense_mask(M, s)
            assert lev2.tolist() == D[s].tolist() and par2.tolist() == par.tolist(), (arcs, s)


def test_exhaustive_undirected_6_sampled():
    """A seeded third of the 32768 undirected graphs on 6 vertices, every source."""
    n = 6
    rng = np.random.default_rng(6)
    masks = rng.choice(1 << 15, size=(1 << 15) // 3, replace=False)
    pairs = [(i, j) for i in range(n) for j in range(i + 1, n)]
    for mask in masks:
        arcs = [pairs[b] for b in range(15) if int(mask) >> b & 1]
        g = _graph(n, arcs, False)
        M = oracle.dense_matrix(g)
        D = oracle.floyd_warshall(M)
        for s in range(n):
            lev, par = oracle.bfs(g, s)
            assert lev.tolist() == D[s].tolist()
            assert par.tolist() == oracle.parents_from_distances(M, D[s], s).tolist()


# ---------------------------------------------------------------------------
# closed forms
# ---------------------------------------------------------------------------

def _path(n):
    return synth.from_arcs(n, list(range(n - 1)), list(range(1, n)), directed=False)


@pytest.mark.parametrize("n,s", [(1, 0), (2, 1), (7, 0), (7, 3), (50, 49), (1000, 417)])
def test_path(n, s):
    lev, par = oracle.bfs(_path(n), s)
    idx = np.arange(n)
    assert (lev == np.abs(idx - s)).all()
    exp = np.where(idx > s, idx - 1, idx + 1)
    exp[s] = s
    assert (par == exp).all()


@pytest.mark.parametrize("leaves,c", [(1, 0), (5, 0), (5, 3), (40, 17)])
def test_star(leaves, c):
    n = leaves + 1
    others = [v for v in range(n) if v != c]
    g = synth.from_arcs(n, [c] * leaves, others, directed=False)
    lev, par = oracle.bfs(g, c)
    assert lev[c] == 0 and par[c] == c
    assert all(lev[v] == 1 and par[v] == c for v in others)
    leaf = others[-1]
    lev, par = oracle.bfs(g, leaf)
    assert lev[c] == 1 and par[c] == leaf and lev[leaf] == 0 and par[leaf] == leaf
    assert all(lev[v] == 2 and par[v] == c for v in others if v != leaf)


@pytest.mark.parametrize("n,s", [(2, 0), (6, 4), (33, 10)])
def test_complete(n, s):
    src = [i for i in range(n) for j in range(i + 1, n)]
    dst = [j for i in range(n) for j in range(i + 1, n)]
    g = synth.from_arcs(n, src, dst, directed=False)
    lev, par = oracle.bfs(g, s)
    assert (np.delete(lev, s) == 1).all() and (np.delete(par, s) == s).all()
    assert lev[s] == 0 and par[s] == s


@pytest.mark.parametrize("W,H", [(1, 1), (1, 9), (9, 1), (2, 2), (17, 5), (64, 64)])
def test_grid_manhattan(W, H):
    g = synth.grid(W, H)
    lev, par = oracle.bfs(g, 0)
    v = np.arange(W * H)
    r, c = v // W, v % W
    assert (lev == r + c).all()
    exp = np.where(r > 0, v - W, v - 1)
    exp[0] = 0
    assert (par == exp).all()


def test_disjoint_components_stay_unreached():
    a = _path(10)
    # two paths: 0..9 and 10..19, plus isolated vertices 20..24
    src = list(range(9)) + list(range(10, 19))
    dst = list(range(1, 10)) + list(range(11, 20))
    g = synth.from_arcs(25, src, dst, directed=False)
    lev, par = oracle.bfs(g, 3)
    assert (lev[10:] == -1).all() and (par[10:] == -1).all()
    assert lev[:10].tolist() == oracle.bfs(a, 3)[0].tolist()


@pytest.mark.parametrize("n,s", [(1 + 1, 0), (5, 2), (100, 37)])
def test_directed_cycle(n, s):
    g = synth.from_arcs(n, list(range(n)), [(i + 1) % n for i in range(n)], directed=True)
    lev, par = oracle.bfs(g, s)
    idx = np.arange(n)
    assert (lev == (idx - s) % n).all()
    exp = (idx - 1) % n
    exp[s] = s
    assert (par == exp).all()


def test_rmat_isolated_vertices_unreached():
    g = synth.rmat(12, 8.0, seed=3)
    deg = g.degrees()
    s = int(synth.sources_with_degree(g, 1, seed=3)[0])
    lev, par = oracle.bfs(g, s)
    iso = np.nonzero(deg == 0)[0]
    assert iso.size > 0
    assert (lev[iso] == -1).all() and (par[iso] == -1).all()


# ---------------------------------------------------------------------------
# invariants from the paper's theorems, on seeded random graphs
# ---------------------------------------------------------------------------

def _graphs_small():
    return [synth.er(2000, 3.0, seed=2), synth.rmat(11, 6.0, seed=4), synth.grid(31, 17),
            synth.rgg_knn(3000, 4, seed=5), synth.rgg_knn(500, 2, seed=6)]


@pytest.mark.parametrize("gi", range(5))
def test_invariants(gi):
    g = _graphs_small()[gi]
    deg = g.degrees()
    s = int(np.argmax(deg > 0))
    lev, par, fs = oracle.bfs(g, s, with_frontiers=True)
    reached = lev >= 0
    n_c = int(reached.sum())
    # Claim 1 / Theorem 2: every reached vertex is in exactly one frontier.
    assert int(fs.sum()) == n_c
    assert fs.shape[0] == int(lev.max()) + 1            # steps = eccentricity + 1
    cols = np.repeat(np.arange(g.n), deg)
    rows = g.rowidx.astype(np.int64)
    lj, li = lev[cols], lev[rows]
    on = lj >= 0
    if not g.directed:
        assert (np.abs(lj[on] - li[on]) <= 1).all()
    assert (li[on] >= 0).all() and (li[on] <= lj[on] + 1).all()
    # parents: a valid predecessor on the previous level, and the least one
    nz = reached & (np.arange(g.n) != s)
    assert (lev[par[nz]] == lev[nz] - 1).all()
    assert (oracle.parent_by_scan(g, lev) == par).all()
    l2, p2 = oracle.bfs_levelsync(g, s)
    assert (l2 == lev).all() and (p2 == par).all()


@pytest.mark.parametrize("gi", range(5))
def test_op_counts_meet_closed_forms(gi):
    """Theorem 2 (Algorithm 2 uses n_c - 1 nonzeros), masked SpMSpV's 2 nnz_c,
    SpMV's nnz per step, and Lemma 3 (each undirected edge once, at most m)."""
    g = _graphs_small()[gi]
    s = int(np.argmax(g.degrees() > 0))
    c = oracle.op_counts(g, s)
    lev, _ = oracle.bfs(g, s)
    n_c = int((lev >= 0).sum())
    nnz_c = int(g.degrees()[lev >= 0].sum())
    assert c["n_c"] == n_c and c["nnz_c"] == nnz_c and c["levels"] == int(lev.max()) + 1
    cf = oracle.closed_form_counts(n_c, nnz_c, g.nnz, c["levels"])
    assert c["alg2"] == cf["alg2"]
    assert c["spmmspv"] == cf["spmmspv"]
    assert c["spmv"] == cf["spmv"]
    assert c["alg2_all_nonzero"] <= 2 * nnz_c
    if not g.directed:
        assert c["alg2_all_nonzero"] == cf["alg2_all_nonzero_undirected"]


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_proposition1_linear_transformation(seed):
    """Proposition 1: A_k x_k = A_k y_k with the conventional y_k = A^{k-1} x_1,
    and S_{k+1} A_k x_k is the next frontier of the masked recurrence."""
    g = synth.er(60, 3.0, seed=seed)
    s = int(np.argmax(g.degrees() > 0))
    _, _, steps = oracle.bfs_dense_mask(g, s, record=True)
    sym = oracle.bfs_symmetric_form(g, s)
    assert len(sym) == len(steps)
    for k, (ax, ay, masked) in enumerate(sym):
        assert ax == ay
        nxt = steps[k + 1][0] if k + 1 < len(steps) else []
        assert masked == nxt


def test_permutation_equivariance_of_levels():
    g = synth.er(3000, 4.0, seed=9)
    pi = np.random.default_rng(9).permutation(g.n).astype(np.uint32)
    cols = np.repeat(np.arange(g.n), g.degrees())
    h = synth.from_arcs(g.n, pi[cols], pi[g.rowidx], directed=True)
    lev, _ = oracle.bfs(g, 5)
    lev_h, par_h = oracle.bfs(h, int(pi[5]))
    assert (lev_h[pi] == lev).all()
    assert (oracle.parent_by_scan(h, lev_h) == par_h).all()


def test_duplicates_and_self_loops_do_not_change_results():
    g = synth.er(500, 4.0, seed=11)
    cols = np.repeat(np.arange(g.n), g.degrees())
    src = np.concatenate([cols, cols[:200], np.arange(50)])
    dst = np.concatenate([g.rowidx, g.rowidx[:200], np.arange(50)])
    h = synth.from_arcs(g.n, src, dst, directed=True)
    assert (h.colptr == g.colptr).all() and (h.rowidx == g.rowidx).all()


# ---------------------------------------------------------------------------
# planted mistakes: each must be caught by one of the pins above
# ---------------------------------------------------------------------------

def _bfs_variant(g, s, mode):
    """Copies of the queue BFS with one planted mistake each."""
    n = g.n
    lev = np.full(n, -1, np.int64)
    par = np.full(n, -1, np.int64)
    lev[s], par[s] = 0, s
    cur = [s]
    k = 0
    while cur:
        if mode != "unsorted":
            cur = sorted(cur, reverse=(mode == "max_parent"))
        nxt = []
        for j in cur:
            for e in range(int(g.colptr[j]), int(g.colptr[j + 1])):
                i = int(g.rowidx[e])
                if lev[i] == -1:
                    lev[i] = k + (1 if mode != "off_by_one" else 2)
                    par[i] = j
                    nxt.append(i)
        if mode == "unsorted":
            nxt = nxt[::-1]
        cur = nxt
        k += 1
    return lev, par


@pytest.mark.parametrize("mode", ["max_parent", "unsorted", "off_by_one"])
def test_pins_catch_planted_mistakes(mode):
    caught = False
    for arcs in _all_graphs(4, False):
        g = _graph(4, arcs, False)
        M = oracle.dense_matrix(g)
        D = oracle.floyd_warshall(M)
        for s in range(4):
            lev, par = _bfs_variant(g, s, mode)
            if lev.tolist() != D[s].tolist() or par.tolist() != oracle.parents_from_distances(M, D[s], s).tolist():
                caught = True
    assert caught, mode
