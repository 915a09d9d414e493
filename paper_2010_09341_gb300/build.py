"""Build the sm_103a CUDA library ``libvegas.so`` in-tree.

Each ``.cu`` file under ``csrc/`` is compiled by nvcc in parallel for
``-gencode arch=compute_103a,code=sm_103a`` and the objects are linked into
``paper_2010_09341_gb300/libvegas.so``.  No fast-math flags: the FP64 path
must agree with the FP64 oracle to 1e-12.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libvegas.so")
INCLUDE = os.path.join(os.path.dirname(PKG), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I", INCLUDE]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libvegas.so")


# Kernel headers compiled again at run time, with a user integrand (NVRTC):
# embedded in the library as string literals by gen_jit_sources().
JIT_HEADERS = ["vegas_device.cuh", "vegas_sample.cuh", "vegas_strat.cuh", "vegas_trace.cuh"]
JIT_GEN = os.path.join(CSRC, "_jit_sources.h")


def gen_jit_sources() -> None:
    """Write csrc/_jit_sources.h: each header of JIT_HEADERS as a raw string
    literal, in a table of (name, text) for the run-time compiler."""
    deps = [os.path.join(CSRC, h) for h in JIT_HEADERS]
    if not _stale(JIT_GEN, deps + [os.path.abspath(__file__)]):
        return
    delim = "vegasjitsrc"
    out = ["// Generated by build.py from the kernel headers: do not edit.",
           "#pragma once", "namespace vegas {", "struct JitHeader { const char *name; const char *text; };",
           "static const JitHeader kJitHeaders[] = {"]
    for h in JIT_HEADERS:
        txt = open(os.path.join(CSRC, h)).read()
        assert ")" + delim not in txt
        out.append('    {"%s", R"%s(%s)%s"},' % (h, delim, txt, delim))
    out += ["};", "static const int kJitHeaderCount = %d;" % len(JIT_HEADERS), "}  // namespace vegas", ""]
    tmp = JIT_GEN + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        f.write("\n".join(out))
    os.replace(tmp, JIT_GEN)


def _sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hs += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return hs


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(dp) > t for dp in deps)


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    """Compile every csrc/*.cu and link libvegas.so; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    gen_jit_sources()
    cc = nvcc()
    srcs = _sources()
    hdrs = _headers()
    objs = []
    jobs = []
    for s in srcs:
        o = os.path.join(BUILD, os.path.basename(s)[:-3] + ".o")
        objs.append(o)
        if force or _stale(o, [s] + hdrs):
            cmd = [cc, *ARCH, *NVCC_FLAGS, *extra_flags, "-c", s, "-o", o]
            jobs.append(cmd)

    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n%s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, flush=True)
        return r

    if jobs:
        with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
            list(ex.map(run, jobs))
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + ".tmp%d" % os.getpid()
        run([cc, *ARCH, "-shared", "-o", tmp, *objs, "-ldl"])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
    print(LIB)
