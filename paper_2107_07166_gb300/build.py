"""Builds the gbfmm CUDA library in place: ``libgbfmm.so`` next to this file.

Generates the order-specialised expansion headers, compiles every translation unit
for sm_103a in parallel with nvcc, and links one shared library.  Used by
``__graft_entry__.build()`` and by the Python binding when the library is missing.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libgbfmm.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-Xcompiler", "-fvisibility=hidden"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources():
    gen = os.path.join(CSRC, "gen")
    own = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu")]
    generated = [os.path.join(gen, f) for f in os.listdir(gen) if f.endswith(".cu")] if os.path.isdir(gen) else []
    # heaviest translation units (highest order) first, so the parallel build ends sooner
    def cost(f):
        b = os.path.basename(f)
        return -int(b[len("expansion_p")]) if b.startswith("expansion_p") else 0
    return sorted(own + generated, key=lambda f: (cost(f), f))


def _stale(obj, deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, jobs: int | None = None, extra_flags=None) -> str:
    subprocess.check_call([sys.executable, os.path.join(CSRC, "gen_expansion.py"), os.path.join(CSRC, "gen")])
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers.append(os.path.join(INCLUDE, "gbfmm.h"))
    flags = NVCC_FLAGS + list(extra_flags or [])
    cmds = []
    objs = []
    for s in sources():
        src = os.path.basename(s)
        o = os.path.join(BUILD, src[:-3] + ".o")
        objs.append(o)
        deps = [s] + headers
        if src.startswith("expansion_p"):
            deps.append(os.path.join(CSRC, "gen", "exp_p" + src[len("expansion_p")] + ".cuh"))
        if _stale(o, deps):
            cmds.append([nvcc(), *ARCH, *flags, "-I", INCLUDE, "-c", s, "-o", o])
    jobs = jobs or max(2, os.cpu_count() or 2)

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if verbose or r.returncode:
            sys.stderr.write(r.stdout + r.stderr)
        if r.returncode:
            raise RuntimeError("nvcc failed: " + " ".join(cmd))
        return cmd

    with cf.ThreadPoolExecutor(jobs) as ex:
        list(ex.map(run, cmds))
    if cmds or not os.path.exists(LIB):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call([nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
