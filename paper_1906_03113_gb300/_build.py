"""Builds libabfs.so in-tree: CUDA engine (nvcc, sm_103a) + host runtime (g++).

Two translation units compile in parallel, then one shared-library link.
Artefacts: paper_1906_03113_gb300/_build/*.o and paper_1906_03113_gb300/libabfs.so.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libabfs.so")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _cuda_home() -> str:
    home = os.environ.get("CUDA_HOME") or os.environ.get("CUDA_PATH")
    if home and os.path.isdir(home):
        return home
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    return "/usr/local/cuda"


def _sources():
    srcs = []
    for name in sorted(os.listdir(CSRC)):
        if name.endswith((".cu", ".cpp", ".h", ".cuh")):
            srcs.append(os.path.join(CSRC, name))
    srcs.append(os.path.join(INCLUDE, "abfs.h"))
    return srcs


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in _sources())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    if not os.path.exists(nvcc):
        nvcc = shutil.which("nvcc") or nvcc
    os.makedirs(BUILD, exist_ok=True)
    inc = ["-I", INCLUDE, "-I", CSRC, "-I", os.path.join(cuda, "include")]
    jobs = []
    cu_files = [f for f in sorted(os.listdir(CSRC)) if f.endswith(".cu")]
    cpp_files = [f for f in sorted(os.listdir(CSRC)) if f.endswith(".cpp")]
    objs = []
    for f in cu_files:
        obj = os.path.join(BUILD, f + ".o")
        cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
               "-Xptxas", "-v", *inc, "-c", os.path.join(CSRC, f), "-o", obj]
        jobs.append((cmd, obj))
        objs.append(obj)
    for f in cpp_files:
        obj = os.path.join(BUILD, f + ".o")
        cmd = ["g++", "-std=c++17", "-O2", "-fPIC", "-Wall", "-pthread", *inc, "-c",
               os.path.join(CSRC, f), "-o", obj]
        jobs.append((cmd, obj))
        objs.append(obj)
    procs = [(subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True), cmd)
             for cmd, _ in jobs]
    logs = []
    failed = False
    for p, cmd in procs:
        out, _ = p.communicate()
        logs.append(" ".join(cmd) + "\n" + out)
        if p.returncode != 0:
            failed = True
    with open(os.path.join(BUILD, "build.log"), "w") as fh:
        fh.write("\n".join(logs))
    if failed:
        raise RuntimeError("libabfs build failed:\n" + "\n".join(logs))
    tmp = LIB + ".tmp"
    link = [nvcc, *ARCH, "-shared", "-cudart", "shared", "-Xcompiler", "-pthread", "-o", tmp, *objs,
            "-Xlinker", "-rpath", "-Xlinker", os.path.join(cuda, "lib64")]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("libabfs link failed:\n" + r.stdout + r.stderr)
    os.replace(tmp, LIB)
    if verbose:
        print("\n".join(logs))
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
