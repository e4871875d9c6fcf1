"""CPU oracle for the algebraic BFS of "Optimal algebraic Breadth-First Search
for sparse graphs" (Burkhardt) -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  It shares no code with the CUDA path (it reads
the same seeded inputs from ``synth``, which holds no BFS arithmetic).

Contents:
  * ``bfs``              -- Moore's queue BFS with sorted frontiers (C), the
                            plain definition of levels and min-index parents.
  * ``parent_by_scan``   -- parents recomputed from levels over every stored
                            entry (C), a traversal-order-free cross-check.
  * ``bfs_levelsync``    -- the same definition, level-synchronous, in numpy.
  * ``bfs_dense_mask``   -- the paper's recurrence x_{k+1} = A[V_{k+1},V_k] x_k
                            (Theorem 1) with dense selection matrices
                            (Appendix A, Definitions 2-3) over the
                            (min, second-index) semiring, small n only.
  * ``spmv_step``        -- one dense (masked) matrix-vector product, Section 6.
  * ``floyd_warshall``   -- all-pairs hop distances, tiny n only.
  * ``op_counts``        -- Table 2 operation counts measured by running each
                            method's loop (C).
  * ``closed_form_counts`` -- the closed forms those counts must meet.
  * ``path_counts``      -- the all-nonzero variant of Algorithm 2 over the
                            arithmetic semiring (Section 8, Proposition 1's
                            caveat): x_k(v) = number of shortest paths from
                            the source to v, mod 2^64, in numpy.
  * ``path_counts_dense`` -- the same recurrence with dense selection matrices
                            and exact integers, small n only.

Every function is pinned by ``tests/test_oracle_pins.py`` against values the
paper prints, closed forms, brute force and identities (Proposition 1).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bfs_oracle.c")
_LIB = os.path.join(_HERE, "_oracle.so")


def build(force: bool = False) -> str:
    """Compiles bfs_oracle.c into _oracle.so (plain C, -O2, no GPU)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    cmd = ["gcc", "-O2", "-shared", "-fPIC", "-std=c11", _SRC, "-o", tmp]
    try:
        subprocess.run(cmd, check=True, capture_output=True, text=True)
    except subprocess.CalledProcessError as exc:  # pragma: no cover
        os.unlink(tmp)
        raise RuntimeError(f"building oracle/bfs_oracle.c failed:\n{exc.stderr}") from exc
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        u32 = ctypes.c_uint32
        lib.oracle_bfs_queue.argtypes = [u32, P(u32), P(u32), u32, P(ctypes.c_int32),
                                         P(ctypes.c_int32), P(u32)]
        lib.oracle_bfs_queue.restype = ctypes.c_int64
        lib.oracle_parent_by_scan.argtypes = [u32, P(u32), P(u32), P(ctypes.c_int32),
                                              P(ctypes.c_int32)]
        lib.oracle_parent_by_scan.restype = None
        lib.oracle_op_counts.argtypes = [u32, P(u32), P(u32), u32, P(ctypes.c_uint64)]
        lib.oracle_op_counts.restype = ctypes.c_int
        _lib = lib
    return _lib


def _arrays(g_or_colptr, rowidx=None):
    if rowidx is None:
        colptr, rowidx = g_or_colptr.colptr, g_or_colptr.rowidx
    else:
        colptr = g_or_colptr
    colptr = np.ascontiguousarray(colptr, dtype=np.uint32)
    rowidx = np.ascontiguousarray(rowidx, dtype=np.uint32)
    if rowidx.shape[0] == 0:
        rowidx = np.zeros(1, dtype=np.uint32)  # valid pointer for an empty graph
    return colptr, rowidx


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def bfs(g_or_colptr, src: int, rowidx=None, with_frontiers: bool = False):
    """Queue BFS with sorted frontiers.  Returns (level int32[n], parent int32[n])
    and, with ``with_frontiers``, the frontier sizes per level."""
    colptr, rowidx = _arrays(g_or_colptr, rowidx)
    n = colptr.shape[0] - 1
    level = np.empty(n, dtype=np.int32)
    parent = np.empty(n, dtype=np.int32)
    fs = np.zeros(n + 1, dtype=np.uint32)
    k = _load().oracle_bfs_queue(n, _p(colptr, ctypes.c_uint32), _p(rowidx, ctypes.c_uint32),
                                 int(src), _p(level, ctypes.c_int32), _p(parent, ctypes.c_int32),
                                 _p(fs, ctypes.c_uint32))
    if k < 0:
        raise ValueError("oracle_bfs_queue: bad argument")
    if with_frontiers:
        return level, parent, fs[:k].astype(np.int64)
    return level, parent


def parent_by_scan(g_or_colptr, level, rowidx=None) -> np.ndarray:
    colptr, rowidx = _arrays(g_or_colptr, rowidx)
    n = colptr.shape[0] - 1
    level = np.ascontiguousarray(level, dtype=np.int32)
    parent = np.empty(n, dtype=np.int32)
    _load().oracle_parent_by_scan(n, _p(colptr, ctypes.c_uint32), _p(rowidx, ctypes.c_uint32),
                                  _p(level, ctypes.c_int32), _p(parent, ctypes.c_int32))
    return parent


OP_KEYS = ("alg2", "alg2_all_nonzero", "spmmspv", "spmv", "n_c", "nnz_c", "levels")


def op_counts(g_or_colptr, src: int, rowidx=None) -> dict:
    """Operation counts of Section 11, Table 2, measured by running the loops."""
    colptr, rowidx = _arrays(g_or_colptr, rowidx)
    n = colptr.shape[0] - 1
    out = np.zeros(7, dtype=np.uint64)
    rc = _load().oracle_op_counts(n, _p(colptr, ctypes.c_uint32), _p(rowidx, ctypes.c_uint32),
                                  int(src), _p(out, ctypes.c_uint64))
    if rc != 0:
        raise ValueError("oracle_op_counts failed")
    return {k: int(v) for k, v in zip(OP_KEYS, out)}


def closed_form_counts(n_c: int, nnz_c: int, nnz: int, levels: int) -> dict:
    """Closed forms of Section 11: Algorithm 2 uses n_c - 1 nonzeros (Theorem 2),
    two operations each; masked SpMSpV multiplies every nonzero of every reached
    column (2 nnz_c, i.e. 4 m_c undirected); SpMV multiplies all nnz stored
    nonzeros at each of the ``levels`` steps; the all-nonzero variant of
    Algorithm 2 multiplies each undirected edge once (2 m_c = nnz_c, Lemma 3)."""
    return {
        "alg2": 2 * (n_c - 1),
        "spmmspv": 2 * nnz_c,
        "spmv": 2 * nnz * levels,
        "alg2_all_nonzero_undirected": nnz_c,
    }


def bfs_levelsync(g_or_colptr, src: int, rowidx=None):
    """The result definition evaluated one level at a time with numpy: the
    candidates of level k+1 are the pairs (i, j) with j on level k, i in column
    j and i not yet reached; parent[i] is the least such j."""
    colptr, rowidx = _arrays(g_or_colptr, rowidx)
    colptr = colptr.astype(np.int64)
    n = colptr.shape[0] - 1
    level = np.full(n, -1, dtype=np.int32)
    parent = np.full(n, -1, dtype=np.int32)
    level[src] = 0
    parent[src] = src
    frontier = np.array([src], dtype=np.int64)
    k = 0
    while frontier.size:
        beg, end = colptr[frontier], colptr[frontier + 1]
        deg = end - beg
        total = int(deg.sum())
        if total == 0:
            break
        owner = np.repeat(frontier, deg)
        start = np.repeat(beg - np.concatenate(([0], np.cumsum(deg)[:-1])), deg)
        pos = start + np.arange(total, dtype=np.int64)
        rows = rowidx[pos].astype(np.int64)
        fresh = level[rows] == -1
        rows, owner = rows[fresh], owner[fresh]
        if rows.size == 0:
            break
        order = np.lexsort((owner, rows))
        rows, owner = rows[order], owner[order]
        first = np.ones(rows.size, dtype=bool)
        first[1:] = rows[1:] != rows[:-1]
        new, par = rows[first], owner[first]
        level[new] = k + 1
        parent[new] = par
        frontier = new
        k += 1
    return level, parent


def dense_matrix(g) -> np.ndarray:
    """A^T as a dense Boolean matrix M with M[i, j] = 1 iff i is in column j
    (so M x projects columns exactly as x_{k+1} = A^T x_k in Section 7)."""
    n = g.n
    M = np.zeros((n, n), dtype=bool)
    cols = np.repeat(np.arange(n), np.diff(g.colptr.astype(np.int64)))
    M[g.rowidx.astype(np.int64), cols] = True
    return M


INF = np.iinfo(np.int64).max


def minsecond_product(M: np.ndarray, x: np.ndarray) -> np.ndarray:
    """y = M (min, second) x: y(i) = min{ j : M(i,j) = 1 and x(j) is nonzero },
    the semiring in which the 'product' of A(i,j) and x(j) carries the index j
    and 'addition' keeps the least index.  Zero is INF."""
    n = M.shape[0]
    idx = np.where(x != INF, np.arange(n, dtype=np.int64), INF)
    cand = np.where(M, idx[None, :], INF)
    return cand.min(axis=1) if n else np.zeros(0, dtype=np.int64)


def spmv_step(M: np.ndarray, x_support, row_mask=None) -> np.ndarray:
    """Support of one Boolean product y = M x (Section 6), with the rows outside
    ``row_mask`` (a set of allowed row indices) removed when it is given."""
    n = M.shape[0]
    x = np.zeros(n, dtype=bool)
    x[list(x_support)] = True
    y = (M & x[None, :]).any(axis=1)
    if row_mask is not None:
        keep = np.zeros(n, dtype=bool)
        keep[list(row_mask)] = True
        y &= keep
    return np.nonzero(y)[0]


def bfs_dense_mask(g_or_M, src: int, record: bool = False):
    """Theorem 1 with the selection matrices of Appendix A:
        V_1 = all, x_1 = e_src, V_{k+1} = V_k minus supp(x_k),
        x_{k+1} = S_{k+1} M S_k x_k        (M = A^T, S_k = diag(V_k)),
    over the (min, second-index) semiring, so x_{k+1}(i) is the least frontier
    index adjacent to row i.  Levels are the step at which a vertex enters a
    support; parents are the values of x.  Dense O(n^2) per step: small n only.
    With ``record``, also returns the list of (supp(x_k), V_k) per step."""
    M = g_or_M if isinstance(g_or_M, np.ndarray) else dense_matrix(g_or_M)
    n = M.shape[0]
    level = np.full(n, -1, dtype=np.int32)
    parent = np.full(n, -1, dtype=np.int32)
    V = np.ones(n, dtype=bool)                        # V_1
    x = np.full(n, INF, dtype=np.int64)
    x[src] = src                                      # x_1
    level[src], parent[src] = 0, src
    steps = []
    k = 0
    while (x != INF).any():
        supp = x != INF
        V_next = V & ~supp                            # V_{k+1} = V_k \ supp(x_k)
        if record:
            steps.append((np.nonzero(supp)[0].tolist(), np.nonzero(V)[0].tolist()))
        xs = np.where(V, x, INF)                      # S_k x_k
        y = minsecond_product(M, xs)                  # M S_k x_k
        x_next = np.where(V_next, y, INF)             # S_{k+1} M S_k x_k
        k += 1
        new = x_next != INF
        level[new] = k
        parent[new] = x_next[new]
        x, V = x_next, V_next
    if record:
        return level, parent, steps
    return level, parent


def bfs_symmetric_form(g_or_M, src: int):
    """Proposition 1 in the Boolean semiring.  With A_k = S_k A S_k and the
    conventional recurrence y_{k+1} = A y_k (y_1 = x_1 = e_src), returns, for
    each step k, the triple of supports
        (A_k x_k,  A_k y_k,  S_{k+1} A_k x_k)
    where x_k is kept masked by V_k.  Proposition 1 says the first two are
    equal; the third must be the next frontier of the masked recurrence."""
    M = g_or_M if isinstance(g_or_M, np.ndarray) else dense_matrix(g_or_M)
    n = M.shape[0]
    Mi = M.astype(np.int64)
    V = np.ones(n, dtype=bool)                          # V_1
    x = np.zeros(n, dtype=bool)
    x[src] = True                                       # x_1
    y = x.copy()                                        # y_1
    steps = []
    for _ in range(n + 1):
        if not x.any():
            break
        S = V.astype(np.int64)
        Ak = S[:, None] * Mi * S[None, :]               # A_k = S_k A S_k
        ax = (Ak @ x.astype(np.int64)) > 0
        ay = (Ak @ y.astype(np.int64)) > 0
        V_next = V & ~x                                 # V_{k+1} = V_k \ supp(x_k)
        steps.append((np.nonzero(ax)[0].tolist(), np.nonzero(ay)[0].tolist(),
                      np.nonzero(ax & V_next)[0].tolist()))
        V = V_next
        x = ax & V                                      # x_{k+1} masked by V_{k+1}
        y = (Mi @ y.astype(np.int64)) > 0               # y_{k+1} = A y_k
    return steps


def path_counts(g_or_colptr, src: int, rowidx=None) -> np.ndarray:
    """Shortest-path counts sigma (uint64, mod 2^64) from ``src``.

    Section 8 turns Algorithm 2 into its all-nonzero variant: every entry of
    column j whose row is still unvisited contributes to the product, instead of
    the first one only.  With the arithmetic semiring and x_1 = e_src (Proposition
    1 asks for one semiring throughout), x_{k+1}(i) sums x_k(j) over the stored
    entries i of the frontier columns j, for rows i of level k+1; by induction on
    k it counts the shortest paths from the source.  A column that stores row i
    twice counts twice (the stored matrix, read as integer entries).  Evaluated
    level by level: the entries from level k to level k+1 are applied after
    every entry of level k-1 to level k.  sigma[v] = 0 for unreached v."""
    colptr, rowidx = _arrays(g_or_colptr, rowidx)
    n = colptr.shape[0] - 1
    nnz = int(colptr[-1])
    level, _ = bfs(colptr, src, rowidx)
    cols = np.repeat(np.arange(n, dtype=np.int64), np.diff(colptr.astype(np.int64)))
    rows = rowidx[:nnz].astype(np.int64)
    lj = level[cols].astype(np.int64)
    keep = (lj >= 0) & (level[rows].astype(np.int64) == lj + 1)
    cols, rows, lj = cols[keep], rows[keep], lj[keep]
    order = np.argsort(lj, kind="stable")
    cols, rows, lj = cols[order], rows[order], lj[order]
    depth = int(level.max()) + 1
    bounds = np.searchsorted(lj, np.arange(depth + 1))
    sigma = np.zeros(n, dtype=np.uint64)
    sigma[src] = 1
    for k in range(depth):
        a, b = int(bounds[k]), int(bounds[k + 1])
        if a < b:
            np.add.at(sigma, rows[a:b], sigma[cols[a:b]])   # wraps mod 2^64
    return sigma


def count_matrix(g) -> np.ndarray:
    """A^T with integer entries: M[i, j] = copies of row i stored in column j."""
    M = np.zeros((g.n, g.n), dtype=np.int64)
    cols = np.repeat(np.arange(g.n), np.diff(g.colptr.astype(np.int64)))
    np.add.at(M, (g.rowidx.astype(np.int64), cols), 1)
    return M


def path_counts_dense(g_or_M, src: int) -> list:
    """Theorem 1's masked recurrence x_{k+1} = S_{k+1} M S_k x_k over the
    arithmetic semiring (ordinary + and *, exact Python integers), x_1 = e_src,
    M = ``count_matrix``.  Returns sigma as a list of ints: the value x_k(v) at
    the step k where v enters a support (1 for the source, 0 if unreached).
    Dense O(n^2) per step: small n only."""
    M = g_or_M if isinstance(g_or_M, np.ndarray) else count_matrix(g_or_M)
    n = M.shape[0]
    Mo = M.astype(object)
    V = np.ones(n, dtype=bool)                          # V_1
    x = np.zeros(n, dtype=object)
    x[src] = 1                                          # x_1
    sigma = [0] * n
    sigma[src] = 1
    while any(v != 0 for v in x):
        supp = np.array([v != 0 for v in x], dtype=bool)
        V_next = V & ~supp                              # V_{k+1} = V_k \ supp(x_k)
        xs = np.where(V, x, 0)                          # S_k x_k
        y = Mo.dot(xs)                                  # M S_k x_k
        x = np.where(V_next, y, 0)                      # S_{k+1} M S_k x_k
        for v in range(n):
            if x[v] != 0:
                sigma[v] = int(x[v])
        V = V_next
    return sigma


def floyd_warshall(M: np.ndarray) -> np.ndarray:
    """All-pairs hop distances D[s, v] along arcs (M[i, j] = arc j -> i);
    -1 where unreachable.  Tiny n only."""
    n = M.shape[0]
    big = n + 1
    D = np.full((n, n), big, dtype=np.int64)
    src_idx, dst_idx = np.nonzero(M.T)                  # arc j -> i  is  M[i, j]
    D[src_idx, dst_idx] = 1
    np.fill_diagonal(D, 0)
    for k in range(n):
        D = np.minimum(D, D[:, k:k + 1] + D[k:k + 1, :])
    D[D >= big] = -1
    return D


def parents_from_distances(M: np.ndarray, dist: np.ndarray, src: int) -> np.ndarray:
    """parent[v] = least j with an arc j -> v and dist[j] = dist[v] - 1."""
    n = M.shape[0]
    parent = np.full(n, -1, dtype=np.int32)
    for v in range(n):
        if v == src:
            parent[v] = src
        elif dist[v] > 0:
            for j in range(n):
                if M[v, j] and dist[j] == dist[v] - 1:
                    parent[v] = j
                    break
    return parent


__all__ = [
    "build", "bfs", "parent_by_scan", "op_counts", "closed_form_counts", "bfs_levelsync",
    "dense_matrix", "minsecond_product", "spmv_step", "bfs_dense_mask", "bfs_symmetric_form",
    "floyd_warshall", "parents_from_distances", "OP_KEYS",
]
