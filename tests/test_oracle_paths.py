"""Pins of the oracle's shortest-path counts (the all-nonzero variant of
Algorithm 2 over the arithmetic semiring).

Every check is against something other than the oracle: closed forms (grid
binomials, hypercube factorials, cycles, bipartite graphs), brute force (walk
counts A^d over every small graph: a walk of length dist(s, v) that ends at v is
a shortest path), an identity of undirected graphs (the s-v count equals the v-s
count), and wrap-around mod 2^64 checked against exact integers.  The last block
plants plausible mistakes in copies of the counting and checks that the pins
catch each of them.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
import synth

MOD = 1 << 64


def _walk_counts(M, s):
    """sigma by brute force: (M^d)[v, s] for d = dist(s, v), exact integers."""
    n = M.shape[0]
    D = oracle.floyd_warshall(M > 0)
    Mo = M.astype(object)
    P = np.identity(n, dtype=object)
    out = [0] * n
    for d in range(n):
        for v in range(n):
            if D[s, v] == d:
                out[v] = int(P[v, s])
        P = Mo.dot(P)
    return out


def _graph(n, arcs, directed):
    return synth.from_arcs(n, [a for a, _ in arcs], [b for _, b in arcs], directed=directed)


def _all_graphs(n, directed):
    pairs = ([(i, j) for i in range(n) for j in range(n) if i != j] if directed
             else [(i, j) for i in range(n) for j in range(i + 1, n)])
    for mask in range(1 << len(pairs)):
        yield [pairs[b] for b in range(len(pairs)) if mask >> b & 1]


def _hand_matrix(g):
    """Integer A^T built here from the CSC, independent of the oracle's helper."""
    M = np.zeros((g.n, g.n), dtype=np.int64)
    for j in range(g.n):
        for e in range(int(g.colptr[j]), int(g.colptr[j + 1])):
            M[int(g.rowidx[e]), j] += 1
    return M


# ---------------------------------------------------------------------------
# brute force
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n,directed", [(1, False), (2, False), (3, False), (4, False), (5, False),
                                        (2, True), (3, True), (4, True)])
def test_exhaustive_vs_walk_counts(n, directed):
    for arcs in _all_graphs(n, directed):
        g = _graph(n, arcs, directed)
        M = _hand_matrix(g)
        for s in range(n):
            want = _walk_counts(M, s)
            assert oracle.path_counts_dense(g, s) == want, (arcs, s)
            assert oracle.path_counts(g, s).tolist() == want, (arcs, s)


def test_duplicate_entries_count_as_integer_entries():
    """A column storing a row twice is the integer entry 2 of the stored matrix."""
    # 0 -> 1 twice, 0 -> 2, 1 -> 3, 2 -> 3 three times, 3 -> 3 (self-loop)
    colptr = np.array([0, 3, 4, 7, 8], dtype=np.uint32)
    rowidx = np.array([1, 1, 2, 3, 3, 3, 3, 3], dtype=np.uint32)
    g = synth.Graph(colptr, rowidx, True)
    M = _hand_matrix(g)
    want = _walk_counts(M, 0)
    assert want == [1, 2, 1, 2 * 1 + 1 * 3]
    assert oracle.path_counts(g, 0).tolist() == want
    assert oracle.path_counts_dense(g, 0) == want


# ---------------------------------------------------------------------------
# closed forms
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("W,H", [(1, 1), (1, 9), (5, 7), (12, 12), (40, 40), (64, 3)])
def test_grid_binomials(W, H):
    """Monotone lattice paths: sigma(r, c) = C(r + c, r), reduced mod 2^64
    (C(78, 39) on the 40 x 40 grid is about 2.6e22)."""
    g = synth.grid(W, H)
    sig = oracle.path_counts(g, 0)
    want = [math.comb(v // W + v % W, v // W) for v in range(W * H)]
    assert sig.tolist() == [w % MOD for w in want]
    if W * H <= 144:
        assert oracle.path_counts_dense(g, 0) == want


@pytest.mark.parametrize("d", [1, 3, 5, 8, 10])
def test_hypercube_factorials(d):
    """From vertex 0 of Q_d, the shortest paths to v flip v's set bits in any
    order: sigma(v) = popcount(v)!."""
    n = 1 << d
    arcs = [(v, v ^ (1 << b)) for v in range(n) for b in range(d) if v < v ^ (1 << b)]
    g = _graph(n, arcs, False)
    sig = oracle.path_counts(g, 0)
    assert sig.tolist() == [math.factorial(bin(v).count("1")) for v in range(n)]
    if d <= 5:
        assert oracle.path_counts_dense(g, 0) == sig.tolist()


@pytest.mark.parametrize("n", [3, 4, 9, 10, 101, 1000])
def test_cycles(n):
    """Undirected C_n from 0: the antipode of an even cycle has two shortest
    paths, every other vertex one."""
    g = _graph(n, [(i, (i + 1) % n) for i in range(n)], False)
    sig = oracle.path_counts(g, 0).tolist()
    want = [1] * n
    if n % 2 == 0:
        want[n // 2] = 2
    assert sig == want


@pytest.mark.parametrize("a,b", [(1, 1), (2, 3), (5, 4), (30, 17)])
def test_complete_bipartite(a, b):
    """K_{a,b} from a vertex of the first side: the other side has one path
    each, the first side's other vertices b each."""
    arcs = [(i, a + j) for i in range(a) for j in range(b)]
    g = _graph(a + b, arcs, False)
    sig = oracle.path_counts(g, 0).tolist()
    assert sig == [1] + [b] * (a - 1) + [1] * b


@pytest.mark.parametrize("n,s", [(1, 0), (7, 3), (1000, 417)])
def test_path_graph_and_complete_graph(n, s):
    p = synth.from_arcs(n, list(range(n - 1)), list(range(1, n)), directed=False)
    assert (oracle.path_counts(p, s) == 1).all()
    m = min(n, 40)
    src = [i for i in range(m) for j in range(i + 1, m)]
    dst = [j for i in range(m) for j in range(i + 1, m)]
    k = synth.from_arcs(m, src, dst, directed=False)
    assert (oracle.path_counts(k, min(s, m - 1)) == 1).all()


def test_unreached_vertices_count_zero():
    src = list(range(9)) + list(range(10, 19))
    dst = list(range(1, 10)) + list(range(11, 20))
    g = synth.from_arcs(25, src, dst, directed=False)
    sig = oracle.path_counts(g, 3)
    assert (sig[:10] == 1).all() and (sig[10:] == 0).all()


# ---------------------------------------------------------------------------
# identity on seeded random graphs
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("seed", [1, 2, 3])
def test_undirected_symmetry(seed):
    """Reversing a shortest s-v path gives a shortest v-s path, so on an
    undirected graph sigma_s(v) = sigma_v(s)."""
    g = synth.er(300, 5.0, seed=seed)
    rng = np.random.default_rng(seed)
    verts = rng.choice(g.n, size=12, replace=False)
    table = {int(s): oracle.path_counts(g, int(s)) for s in verts}
    for s, t in itertools.permutations(verts.tolist(), 2):
        assert table[s][t] == table[t][s]


def test_rmat_counts_exceed_one_and_match_dense():
    g = synth.rmat(7, 6.0, seed=9)
    s = int(synth.sources_with_degree(g, 1, seed=9)[0])
    sig = oracle.path_counts(g, s)
    assert sig.max() > 1
    assert sig.tolist() == oracle.path_counts_dense(g, s)


# ---------------------------------------------------------------------------
# planted mistakes: each must be caught by the pins above
# ---------------------------------------------------------------------------

def _counts_variant(g, s, mode):
    lev, _ = oracle.bfs(g, s)
    n = g.n
    sig = [0] * n
    sig[s] = 1
    for k in range(int(lev.max()) + 1):
        for j in range(n):
            if lev[j] != k:
                continue
            for e in range(int(g.colptr[j]), int(g.colptr[j + 1])):
                i = int(g.rowidx[e])
                same_level = mode == "same_level_edges" and lev[i] == k and i > j
                if lev[i] == k + 1 or same_level:
                    if mode == "first_only":
                        sig[i] = sig[i] or sig[j]
                    elif mode == "add_one":
                        sig[i] += 1
                    else:
                        sig[i] += sig[j]
    return sig


@pytest.mark.parametrize("mode", ["same_level_edges", "first_only", "add_one"])
def test_pins_catch_planted_mistakes(mode):
    caught = False
    for arcs in _all_graphs(5, False):
        g = _graph(5, arcs, False)
        M = _hand_matrix(g)
        for s in range(5):
            if _counts_variant(g, s, mode) != _walk_counts(M, s):
                caught = True
                break
        if caught:
            break
    assert caught, mode
