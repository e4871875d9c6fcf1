"""Seeded synthetic graph generators shared by the oracle and the CUDA path.

This package holds none of the BFS arithmetic.  It draws random numbers
(SplitMix64 used as a counter-based generator, see ``gen.c``) and assembles
CSC arrays: ``colptr`` uint32[n+1] and ``rowidx`` uint32[nnz], where column j
lists the out-neighbours of vertex j (the CSC of A^T used by the paper's
Section 7 for directed graphs; for undirected graphs A = A^T).

The workloads mirror the shapes of the graphs in the paper's Section 11
(Table 1): low-diameter social graphs (Erdos-Renyi, R-MAT) and
large-diameter road networks (2-D grid, k-nearest-neighbour geometric graph).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import sys
import tempfile
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "_gen.so")


class _CSC(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_uint32),
        ("nnz", ctypes.c_uint64),
        ("colptr", ctypes.POINTER(ctypes.c_uint32)),
        ("rowidx", ctypes.POINTER(ctypes.c_uint32)),
    ]


def build(force: bool = False) -> str:
    """Compiles gen.c into _gen.so next to it (host C, no GPU needed)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(cmd, check=True, capture_output=True, text=True)
    except subprocess.CalledProcessError as exc:  # pragma: no cover - build failure is fatal
        os.unlink(tmp)
        raise RuntimeError(f"building synth/gen.c failed:\n{exc.stderr}") from exc
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        u32, u64, dbl, i32 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double, ctypes.c_int
        lib.synth_rmat.argtypes = [u32, dbl, dbl, dbl, dbl, u64, i32, u32, P(_CSC)]
        lib.synth_er.argtypes = [u32, dbl, u64, P(_CSC)]
        lib.synth_grid.argtypes = [u32, u32, P(_CSC)]
        lib.synth_rgg_knn.argtypes = [u32, u32, u64, P(_CSC)]
        lib.synth_from_arcs.argtypes = [u32, u64, P(u32), P(u32), i32, P(_CSC)]
        lib.synth_free.argtypes = [P(_CSC)]
        lib.synth_free.restype = None
        lib.synth_uniform.argtypes = [u64, u64, u64, P(dbl)]
        lib.synth_uniform.restype = None
        for f in ("synth_rmat", "synth_er", "synth_grid", "synth_rgg_knn", "synth_from_arcs"):
            getattr(lib, f).restype = i32
        _lib = lib
    return _lib


@dataclass
class Graph:
    """A CSC graph: column j = out-neighbours of j, rows ascending."""

    colptr: np.ndarray  # uint32[n+1]
    rowidx: np.ndarray  # uint32[nnz]
    directed: bool
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.colptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.rowidx.shape[0])

    def degrees(self) -> np.ndarray:
        return np.diff(self.colptr.astype(np.int64))


def _take(res: _CSC, directed: bool, name: str, meta: dict) -> Graph:
    lib = _load()
    n, nnz = int(res.n), int(res.nnz)
    colptr = np.ctypeslib.as_array(res.colptr, shape=(n + 1,)).copy()
    rowidx = (np.ctypeslib.as_array(res.rowidx, shape=(nnz,)).copy() if nnz
              else np.zeros(0, dtype=np.uint32))
    lib.synth_free(ctypes.byref(res))
    return Graph(colptr.astype(np.uint32, copy=False), rowidx.astype(np.uint32, copy=False),
                 directed, name, meta)


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise ValueError(f"{what}: generator returned error {rc}")


def rmat(scale: int, edgefactor: float = 16.0, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 1, permute: bool = True, n_keep: int = 0) -> Graph:
    """Undirected R-MAT, duplicates and self-loops removed, optional label permutation."""
    res = _CSC()
    _check(_load().synth_rmat(scale, edgefactor, a, b, c, seed, int(permute), n_keep,
                              ctypes.byref(res)), "rmat")
    return _take(res, False, f"rmat{scale}",
                 dict(kind="rmat", scale=scale, edgefactor=edgefactor, a=a, b=b, c=c, seed=seed))


def er(n: int, avg_degree: float = 8.0, seed: int = 1, p: float | None = None) -> Graph:
    """Undirected G(n, p) with p = avg_degree/(n-1) unless p is given."""
    if p is None:
        p = avg_degree / (n - 1) if n > 1 else 0.0
    res = _CSC()
    _check(_load().synth_er(n, p, seed, ctypes.byref(res)), "er")
    return _take(res, False, f"er{n}", dict(kind="er", n=n, p=p, seed=seed))


def grid(W: int, H: int | None = None) -> Graph:
    """Undirected W x H 4-neighbour grid, row-major labels v = r*W + c."""
    H = W if H is None else H
    res = _CSC()
    _check(_load().synth_grid(W, H, ctypes.byref(res)), "grid")
    return _take(res, False, f"grid{W}x{H}", dict(kind="grid", W=W, H=H))


def rgg_knn(n: int, k: int = 4, seed: int = 1) -> Graph:
    """Directed k-NN geometric graph on n uniform points of the unit square."""
    res = _CSC()
    _check(_load().synth_rgg_knn(n, k, seed, ctypes.byref(res)), "rgg_knn")
    return _take(res, True, f"rgg{n}k{k}", dict(kind="rgg", n=n, k=k, seed=seed))


def from_arcs(n: int, src, dst, directed: bool, name: str = "arcs") -> Graph:
    """CSC from explicit arcs src[e] -> dst[e] (undirected: both directions)."""
    src = np.ascontiguousarray(np.asarray(src, dtype=np.uint32))
    dst = np.ascontiguousarray(np.asarray(dst, dtype=np.uint32))
    assert src.shape == dst.shape
    P = ctypes.POINTER(ctypes.c_uint32)
    res = _CSC()
    _check(_load().synth_from_arcs(n, src.shape[0], src.ctypes.data_as(P), dst.ctypes.data_as(P),
                                   0 if directed else 1, ctypes.byref(res)), "from_arcs")
    return _take(res, directed, name, dict(kind="arcs"))


def uniform(seed: int, stream: int, count: int) -> np.ndarray:
    """count seeded uniforms in [0,1) from one counter-based stream."""
    out = np.empty(count, dtype=np.float64)
    _load().synth_uniform(seed, stream, count, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def sources_with_degree(g: Graph, count: int, seed: int = 1) -> np.ndarray:
    """count distinct sources drawn uniformly from the vertices of out-degree >= 1."""
    cand = np.nonzero(g.degrees() >= 1)[0].astype(np.int64)
    if count > cand.shape[0]:
        raise ValueError("not enough vertices with degree >= 1")
    keys = uniform(seed, 0x535243, cand.shape[0])  # stream "SRC"
    order = np.argsort(keys, kind="stable")
    return cand[order[:count]].astype(np.uint32)


# ---------------------------------------------------------------------------
# The five workloads (synthetic stand-ins for the paper's SNAP graphs).
# ---------------------------------------------------------------------------

def er_2_16(seed: int = 1) -> Graph:
    """Undirected G(n,p), n = 2^16, p = 8/(n-1); source 0."""
    return er(1 << 16, 8.0, seed)


def rmat_22(seed: int = 1) -> Graph:
    """Undirected R-MAT scale 22, edge factor 16, a/b/c/d = .57/.19/.19/.05, permuted."""
    return rmat(22, 16.0, 0.57, 0.19, 0.19, seed, True)


def grid_4096() -> Graph:
    """Undirected 4096 x 4096 4-neighbour grid; source 0."""
    return grid(4096, 4096)


def rgg_2_22(seed: int = 1) -> Graph:
    """Directed 4-NN geometric graph, n = 2^22; source 0."""
    return rgg_knn(1 << 22, 4, seed)


@dataclass
class BatchSpec:
    kind: str
    n: int
    avg_degree: float
    seed: int


def batch_specs(count: int = 512, seed: int = 1, lo_log2: float = 10.0, hi_log2: float = 18.0,
                dmin: float = 4.0, dmax: float = 32.0) -> list[BatchSpec]:
    """Graph g: n = round(2^U[lo,hi]), avg degree U[dmin,dmax], ER for even g, R-MAT for odd g."""
    un = uniform(seed, 0x42544E, count)   # "BTN"
    ud = uniform(seed, 0x425444, count)   # "BTD"
    out = []
    for g in range(count):
        n = int(round(2.0 ** (lo_log2 + (hi_log2 - lo_log2) * un[g])))
        d = dmin + (dmax - dmin) * ud[g]
        out.append(BatchSpec("er" if g % 2 == 0 else "rmat", n, float(d), seed + g))
    return out


def make_batch_graph(spec: BatchSpec) -> Graph:
    if spec.kind == "er":
        return er(spec.n, spec.avg_degree, spec.seed)
    scale = max(1, int(math.ceil(math.log2(spec.n))))
    return rmat(scale, spec.avg_degree / 2.0, 0.57, 0.19, 0.19, spec.seed, True, spec.n)


def serve_graph_specs() -> list[tuple[str, dict]]:
    """32 resident graphs: 16 R-MAT (scales 16..22 cycling), 15 ER (2^16..2^20 cycling, d=8),
    one 2048 x 2048 grid."""
    specs: list[tuple[str, dict]] = []
    for i in range(16):
        specs.append(("rmat", dict(scale=16 + (i % 7), seed=1 + i)))
    for i in range(15):
        specs.append(("er", dict(n=1 << (16 + (i % 5)), avg_degree=8.0, seed=101 + i)))
    specs.append(("grid", dict(W=2048, H=2048)))
    return specs


def make_serve_graph(kind: str, kw: dict) -> Graph:
    if kind == "rmat":
        return rmat(kw["scale"], 16.0, 0.57, 0.19, 0.19, kw["seed"], True)
    if kind == "er":
        return er(kw["n"], kw["avg_degree"], kw["seed"])
    return grid(kw["W"], kw["H"])


__all__ = [
    "Graph", "build", "rmat", "er", "grid", "rgg_knn", "from_arcs", "uniform",
    "sources_with_degree", "er_2_16", "rmat_22", "grid_4096", "rgg_2_22", "batch_specs",
    "make_batch_graph", "BatchSpec", "serve_graph_specs", "make_serve_graph",
]
