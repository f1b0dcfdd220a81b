"""The class-specialised source generator (paper_2607_05622_gb300/csrc/codegen.cpp)
on the CPU: the straight-line code it emits for every value class, (ss|ss) to
(dd|dd), and for the derivative classes up to (pp|pp), compiled as host C++,
gives the blocks of the interpreted programs (tests/program_eval.cpp) and of
the oracle's McMurchie-Davidson integrals; and the light classes' emitted
code compiles for sm_103a without register spills (ptxas report)."""
import ctypes
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

from paper_2607_05622_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
OUT = os.path.join(ROOT, "tests", "_build")
CSRC = os.path.join(ROOT, "paper_2607_05622_gb300", "csrc")
INC = os.path.join(ROOT, "include")


def _gxx():
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    return cxx


@pytest.fixture(scope="module")
def emitter():
    cxx = _gxx()
    os.makedirs(OUT, exist_ok=True)
    exe = os.path.join(OUT, "codegen_emit")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, "-I", INC,
                    os.path.join(ROOT, "tests", "codegen_emit.cpp"), os.path.join(CSRC, "program.cpp"),
                    os.path.join(CSRC, "codegen.cpp"), "-o", exe], check=True)
    return exe


def _gen_lib(emitter, deriv, lmax):
    hdr = os.path.join(OUT, f"gen_d{deriv}_l{lmax}.h")
    subprocess.run([emitter, hdr, str(deriv), str(lmax)], check=True)
    so = os.path.join(OUT, f"libprogram_eval_gen_d{deriv}_l{lmax}.so")
    subprocess.run([_gxx(), "-O0", "-std=c++17", "-shared", "-fPIC", f"-DLTJK_GEN_DERIV={deriv}",
                    f'-DLTJK_GEN_HEADER="{hdr}"', "-I", CSRC, "-I", INC,
                    os.path.join(ROOT, "tests", "program_eval.cpp"), os.path.join(CSRC, "program.cpp"),
                    "-o", so], check=True)
    lib = ctypes.CDLL(so)
    assert lib.pe_init() == 0
    return lib


def _args(mol, cn, shells):
    ls = [int(mol.shell_l[s]) for s in shells]
    ctr = np.concatenate([mol.coords[mol.shell_atom[s]] for s in shells]).astype(np.float64)
    off = np.concatenate([[0], np.cumsum(mol.shell_nprim)])
    np_ = np.array([mol.shell_nprim[s] for s in shells], dtype=np.int32)
    ex = np.concatenate([mol.exps[off[s]:off[s + 1]] for s in shells])
    co = np.concatenate([cn[off[s]:off[s + 1]] for s in shells])
    return ls, ctr, np_, ex, co


def _call(fn, ls, ctr, np_, ex, co, nout, deriv=None):
    P = ctypes.POINTER(ctypes.c_double)
    out = np.zeros(nout)
    extra = [] if deriv is None else [deriv]
    rc = fn(*ls, *extra, ctr.ctypes.data_as(P), np_.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
            ex.ctypes.data_as(P), co.ctypes.data_as(P), out.ctypes.data_as(P))
    assert rc == 0
    return out


def _molecule():
    rng = np.random.default_rng(11)
    coords = [np.zeros(3)]
    while len(coords) < 4:  # four heavy atoms placed in 3D, 1.3-2.6 bohr apart
        p = coords[-1] + rng.normal(size=3)
        if 1.3 <= min(np.linalg.norm(p - q) for q in coords) <= 2.6:
            coords.append(p)
    return W.build_molecule([tuple(c) for c in coords], ["heavy"] * 4,
                            W.draw_kind_bases(np.random.default_rng(7)))


def _pick(mol):
    off = np.concatenate([[0], np.cumsum(mol.shell_nprim)])
    first = {}  # the most diffuse shell of each l on each atom
    for s, (a, l) in enumerate(zip(mol.shell_atom, mol.shell_l)):
        key, lo = (int(a), int(l)), mol.exps[off[s]:off[s + 1]].min()
        if key not in first or lo < first[key][1]:
            first[key] = (s, lo)
    return first


def test_emitted_value_classes_match_programs_and_oracle(emitter, oracle):
    lib = _gen_lib(emitter, 0, 2)
    mol = _molecule()
    cn = oracle.norm_coefs(mol)
    first = _pick(mol)
    pairs = [(la, lb) for la in range(3) for lb in range(la + 1)]
    for (la, lb) in pairs:
        for (lc, ld) in pairs:
            shells = [first[(atom, l)][0] for atom, l in enumerate((la, lb, lc, ld))]
            ls, ctr, np_, ex, co = _args(mol, cn, shells)
            n = int(np.prod([(l + 1) * (l + 2) // 2 for l in ls]))
            got = _call(lib.pe_quartet_gen, ls, ctr, np_, ex, co, n)
            interp = _call(lib.pe_quartet_d, ls, ctr, np_, ex, co, n, deriv=0)
            ref = oracle.shell_quartet(mol, *shells).ravel()
            scale = np.abs(ref).max()
            assert np.abs(got - interp).max() <= 1e-13 * scale, (la, lb, lc, ld)
            assert np.abs(got - ref).max() <= 1e-11 * scale, (la, lb, lc, ld)


def test_emitted_derivative_classes_match_programs(emitter, oracle):
    lib = _gen_lib(emitter, 1, 1)
    mol = _molecule()
    cn = oracle.norm_coefs(mol)
    first = _pick(mol)
    pairs = [(la, lb) for la in range(2) for lb in range(la + 1)]
    for (la, lb) in pairs:
        for (lc, ld) in pairs:
            shells = [first[(atom, l)][0] for atom, l in enumerate((la, lb, lc, ld))]
            ls, ctr, np_, ex, co = _args(mol, cn, shells)
            n = 9 * int(np.prod([(l + 1) * (l + 2) // 2 for l in ls]))
            got = _call(lib.pe_quartet_gen, ls, ctr, np_, ex, co, n)
            interp = _call(lib.pe_quartet_d, ls, ctr, np_, ex, co, n, deriv=1)
            assert np.abs(got - interp).max() <= 1e-13 * np.abs(interp).max(), (la, lb, lc, ld)


def test_light_classes_compile_for_sm103a_without_spills(emitter):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("no nvcc")
    hdr = os.path.join(OUT, "gen_d0_l1.h")
    subprocess.run([emitter, hdr, "0", "1"], check=True)
    src = os.path.join(OUT, "gen_light_kernels.cu")
    body = ['#define LTJK_HD __host__ __device__', f'#include "{hdr}"']
    names = re.findall(r"inline void (c\d{4}d0)_vrr", open(hdr).read())
    for nm in names:  # one kernel per class: a primitive loop and the horizontal steps
        body.append(f"""
__global__ void k_{nm}(const double *base, const double *cf, const double *h, const double *X,
                       double *out, int nprim) {{
  double acc[128] = {{0}};
  for (int i = 0; i < nprim; ++i) {nm}_vrr<double>(base + 16 * i, cf + 32 * i, h + 32 * i, acc);
  {nm}_hrr<double>(acc, X, out + 128 * (blockIdx.x * blockDim.x + threadIdx.x));
}}""")
    open(src, "w").write("\n".join(body) + "\n")
    r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                        "-Xptxas", "-v", "-c", src, "-o", os.path.join(OUT, "gen_light_kernels.o")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    spills = re.findall(r"(\d+) bytes spill stores", r.stderr)
    assert len(spills) >= len(names)
    assert all(int(s) == 0 for s in spills), r.stderr[-3000:]
