"""Build the native library libsd.so (C ABI of include/sd.h) in-tree.

Every translation unit is compiled by nvcc for sm_103a only, in parallel,
then linked into paper_2206_11664_gb300/_build/libsd.so.  Run as
``python -m paper_2206_11664_gb300.build`` or through ``__graft_entry__.build()``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libsd.so")
SOURCES = ["planner.cpp", "schedule.cpp", "api.cpp", "jit.cpp", "kernels.cu", "noalloc.cu"]
JIT_HEADERS = [("kJitDevTypes", "dev_types.h"), ("kJitFixedPoint", "fixed_point.cuh"),
               ("kJitTileDevice", "tile_device.cuh")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _embed_headers() -> None:
    """Write _build/jit_headers.inc: the device headers the run-time compiler
    needs, as C++ raw string literals."""
    out = []
    for var, name in JIT_HEADERS:
        text = open(os.path.join(CSRC, name)).read()
        assert ")SDJITSRC" not in text
        out.append(f'static const char *{var} = R"SDJITSRC({text})SDJITSRC";\n')
    path = os.path.join(OUT, "jit_headers.inc")
    body = "".join(out)
    if not os.path.exists(path) or open(path).read() != body:
        with open(path, "w") as f:
            f.write(body)


def _compile(src: str, obj: str, verbose_ptxas: bool) -> None:
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
           "-Xcompiler", "-O2", "-I", os.path.join(HERE, "..", "include"), "-I", OUT,
           "-c", src, "-o", obj]
    if verbose_ptxas and src.endswith(".cu"):
        cmd[1:1] = ["-Xptxas", "-v"]
    subprocess.check_call(cmd)


def _stale(objs) -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(HERE, "..", "include", "sd.h"))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    objs = [os.path.join(OUT, os.path.splitext(s)[0] + ".o") for s in SOURCES]
    if not force and not _stale(objs):
        return LIB
    _embed_headers()
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        futs = [ex.submit(_compile, os.path.join(CSRC, s), o, verbose_ptxas)
                for s, o in zip(SOURCES, objs)]
        for f in futs:
            f.result()
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call([nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-ldl"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv))
