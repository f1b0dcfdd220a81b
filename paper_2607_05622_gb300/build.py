"""Build the CUDA library in-tree: paper_2607_05622_gb300/_build/libltjk.so.

nvcc compiles each translation unit for sm_103a only (no PTX for other
targets, no fast-math: FP64 results must round to nearest), in parallel, and
links them into one shared library exporting the C ABI of include/ltjk.h.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libltjk.so")
SOURCES = ["context.cu", "host.cpp", "program.cpp"]
# host generator of the class-specialised integral code (run before nvcc)
GEN_SOURCES = ["gen_main.cpp", "program.cpp", "codegen.cpp"]
GEN_INC = os.path.join(OUT, "gen_classes.inc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found")
    return cand


def _deps():
    files = [os.path.join(SRC, f) for f in os.listdir(SRC)]
    files.append(os.path.join(ROOT, "include", "ltjk.h"))
    return max(os.path.getmtime(f) for f in files)


def cxx() -> str:
    for c in ("g++", "c++", "clang++"):
        p = shutil.which(c)
        if p:
            return p
    raise RuntimeError("no host C++ compiler found")


def generate() -> str:
    """Compile and run the class-code generator: writes _build/gen_classes.inc."""
    os.makedirs(OUT, exist_ok=True)
    exe = os.path.join(OUT, "gen_main")
    cmd = [cxx(), "-O1", "-std=c++17", "-I", SRC, "-I", os.path.join(ROOT, "include"),
           *[os.path.join(SRC, f) for f in GEN_SOURCES], "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"generator build failed:\n{r.stdout}\n{r.stderr}")
    tmp = GEN_INC + f".tmp{os.getpid()}"
    r = subprocess.run([exe, tmp], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"generator failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, GEN_INC)
    return GEN_INC


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps():
        return LIB
    generate()
    common = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "-I", os.path.join(ROOT, "include"), "-I", OUT]
    objs = []

    def compile_one(src):
        obj = os.path.join(OUT, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc(), *ARCH, *common, "-c", os.path.join(SRC, src), "-o", obj]
        if src.endswith(".cu"):
            cmd[1:1] = ["-Xptxas", "-v"] if verbose else []
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
