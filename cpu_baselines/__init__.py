"""The paper's CPU methods as timed baselines: sequential Algorithm 2
(Section 9) and OpenMP Algorithm 3 (Section 10), in plain C
(``algebraic_bfs.c``), for the host cores of the machine that holds the GPU.

They share no code with the CUDA path or with the oracle.  Levels are the BFS
distances; parents are valid predecessors chosen by discovery order
(Algorithm 2) or thread timing (Algorithm 3), as the paper allows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "algebraic_bfs.c")
_LIB = os.path.join(_HERE, "_cpubfs.so")


def build(force: bool = False) -> str:
    """Compiles algebraic_bfs.c with OpenMP (without it if the compiler lacks
    it: Algorithm 3 then runs on one thread)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    base = ["gcc", "-O3", "-shared", "-fPIC", "-std=c11", _SRC, "-o", tmp]
    try:
        try:
            subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True,
                           text=True)
        except subprocess.CalledProcessError:
            subprocess.run(base, check=True, capture_output=True, text=True)
    except subprocess.CalledProcessError as exc:  # pragma: no cover
        os.unlink(tmp)
        raise RuntimeError(f"building cpu_baselines/algebraic_bfs.c failed:\n{exc.stderr}") from exc
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        u32, i32, i64 = ctypes.c_uint32, ctypes.c_int32, ctypes.c_int64
        lib.alg2_bfs.argtypes = [u32, P(u32), P(u32), u32, P(i32), P(i32), P(ctypes.c_uint8), P(u32)]
        lib.alg2_bfs.restype = i64
        lib.alg3_bfs.argtypes = [u32, P(u32), P(u32), u32, P(i32), P(i32), P(ctypes.c_uint8), P(u32),
                                 ctypes.c_int, P(ctypes.c_int)]
        lib.alg3_bfs.restype = i64
        lib.alg3_has_openmp.argtypes = []
        lib.alg3_has_openmp.restype = ctypes.c_int
        _lib = lib
    return _lib


def has_openmp() -> bool:
    return bool(_load().alg3_has_openmp())


def host_cores() -> int:
    """Cores this process may run on (the affinity mask), as nproc reports."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


class _Arrays:
    def __init__(self, g):
        self.colptr = np.ascontiguousarray(g.colptr, dtype=np.uint32)
        rows = np.ascontiguousarray(g.rowidx, dtype=np.uint32)
        self.rowidx = rows if rows.size else np.zeros(1, dtype=np.uint32)
        self.n = self.colptr.shape[0] - 1
        self.level = np.empty(self.n, dtype=np.int32)
        self.parent = np.empty(self.n, dtype=np.int32)
        self.T = np.empty(self.n, dtype=np.uint8)
        self.L = np.empty(self.n, dtype=np.uint32)

    def ptrs(self):
        P = ctypes.POINTER
        return (self.n, self.colptr.ctypes.data_as(P(ctypes.c_uint32)),
                self.rowidx.ctypes.data_as(P(ctypes.c_uint32)))

    def outs(self):
        P = ctypes.POINTER
        return (self.level.ctypes.data_as(P(ctypes.c_int32)),
                self.parent.ctypes.data_as(P(ctypes.c_int32)),
                self.T.ctypes.data_as(P(ctypes.c_uint8)), self.L.ctypes.data_as(P(ctypes.c_uint32)))


def alg2(g, src: int, arrays: _Arrays | None = None):
    """Sequential Algorithm 2: (level, parent, seconds)."""
    a = arrays or _Arrays(g)
    n, cp, ri = a.ptrs()
    ns = _load().alg2_bfs(n, cp, ri, int(src), *a.outs())
    if ns < 0:
        raise ValueError("alg2_bfs: bad argument")
    return a.level.copy(), a.parent.copy(), ns * 1e-9


def alg3(g, src: int, threads: int = 0, arrays: _Arrays | None = None):
    """OpenMP Algorithm 3: (level, parent, seconds, threads used)."""
    a = arrays or _Arrays(g)
    n, cp, ri = a.ptrs()
    used = ctypes.c_int(0)
    ns = _load().alg3_bfs(n, cp, ri, int(src), *a.outs(), int(threads), ctypes.byref(used))
    if ns < 0:
        raise ValueError("alg3_bfs: bad argument or allocation failure")
    return a.level.copy(), a.parent.copy(), ns * 1e-9, used.value


def time_baselines(g, sources, budget_s: float = 10.0, reps: int = 5) -> list[dict]:
    """Times both methods on the workload's sources: per source the median of
    `reps` runs (fewer when the budget of each method runs out), GTEPS with
    m_c = nnz_c / 2 on undirected graphs.  Returns one dict per method."""
    a = _Arrays(g)
    deg = np.diff(g.colptr.astype(np.int64))
    out = []
    cores = host_cores()
    for name, fn, threads in (("alg2_sequential", "alg2", 1), ("alg3_openmp", "alg3", cores)):
        edges = 0.0
        secs = 0.0
        used_src = 0
        team = 1
        spent = 0.0
        for s in sources:
            times = []
            for _ in range(reps):
                if fn == "alg2":
                    lev, _, t = alg2(g, int(s), a)
                else:
                    lev, _, t, team = alg3(g, int(s), threads, a)
                times.append(t)
                spent += t
                if spent > budget_s:
                    break
            times.sort()
            secs += times[len(times) // 2]
            nnz_c = float(deg[lev >= 0].sum())
            edges += nnz_c if g.directed else nnz_c / 2.0
            used_src += 1
            if spent > budget_s:
                break
        out.append({"kind": name, "value": edges / secs / 1e9, "unit": "GTEPS",
                    "cores": 1 if fn == "alg2" else team, "host_cores": cores,
                    "openmp": fn == "alg3" and has_openmp(),
                    "sample": f"{used_src} of {len(sources)} sources, median of up to {reps} runs "
                              f"each ({spent:.1f} s)"})
    return out
