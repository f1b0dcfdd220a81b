"""Binary32 quartets and the mixed-precision tolerance, on the CPU.

The library's recurrence programs interpreted in binary32 in the integral
kernel's operation order (tests/program_eval.cpp, pe_quartet_f32) against the
oracle's McMurchie-Davidson blocks on the 40-AO chain that the mixed-mode GPU
test uses: for every kept quartet sampled, of every class, the error is at
most EPS32 times its Schwarz product Q_ab Q_cd.  From that, tests/mixed_bound.py
bounds the mixed build's J and K error per element; the bound on the GPU
test's densities is the gate that test applies (about 1e-8 of max|J|, where
the measured error is about 4e-12)."""
import ctypes
import itertools
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2607_05622_gb300 import workloads as W
from mixed_bound import EPS32, EPS_DIG, EPS_TF32, mixed_jk_bound

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
OUT = os.path.join(ROOT, "tests", "_build")


@pytest.fixture(scope="module")
def pe():
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    os.makedirs(OUT, exist_ok=True)
    so = os.path.join(OUT, "libprogram_eval_f32.so")
    src = [os.path.join(ROOT, "tests", "program_eval.cpp"),
           os.path.join(ROOT, "paper_2607_05622_gb300", "csrc", "program.cpp")]
    subprocess.run([cxx, "-O2", "-std=c++17", "-shared", "-fPIC",
                    "-I", os.path.join(ROOT, "paper_2607_05622_gb300", "csrc"),
                    "-I", os.path.join(ROOT, "include"), *src, "-o", so], check=True)
    lib = ctypes.CDLL(so)
    assert lib.pe_init() == 0
    return lib


def _quartet(fn, mol, cn, shells):
    ls = [int(mol.shell_l[s]) for s in shells]
    ctr = np.concatenate([mol.coords[mol.shell_atom[s]] for s in shells]).astype(np.float64)
    off = np.concatenate([[0], np.cumsum(mol.shell_nprim)])
    np_ = np.array([mol.shell_nprim[s] for s in shells], dtype=np.int32)
    ex = np.concatenate([mol.exps[off[s]:off[s + 1]] for s in shells])
    co = np.concatenate([cn[off[s]:off[s + 1]] for s in shells])
    n = [(l + 1) * (l + 2) // 2 for l in ls]
    out = np.zeros(int(np.prod(n)))
    P = ctypes.POINTER(ctypes.c_double)
    rc = fn(*ls, 0, ctr.ctypes.data_as(P), np_.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
            ex.ctypes.data_as(P), co.ctypes.data_as(P), out.ctypes.data_as(P))
    assert rc == 0
    return out.reshape(n)


def _mixed_chain():
    return W.small_chain(2, 2, seed=4, tau=1e-12).mol


def test_binary32_quartets_within_eps_of_schwarz(pe, oracle):
    """Every quartet of the 40-AO chain that mixed mode evaluates in binary32
    (1e-12 <= Q_ab Q_cd <= 1e-6, about 3000 of them, 21 classes): error at
    most EPS32 Q_ab Q_cd.  Above the threshold the same arithmetic is far
    worse relative to Q_ab Q_cd (4e-2 on (dd|dd) with tight d shells 1.4 bohr
    apart, cancellation in the horizontal steps), which is why those quartets
    are promoted."""
    mol = _mixed_chain()
    cn = oracle.norm_coefs(mol)
    Q = oracle.schwarz(mol)
    l = np.asarray(mol.shell_l)
    ns = len(l)
    worst, seen, count = 0.0, set(), 0
    for s in itertools.product(range(ns), repeat=4):
        if l[s[0]] < l[s[1]] or l[s[2]] < l[s[3]]:
            continue
        qq = Q[s[0], s[1]] * Q[s[2], s[3]]
        if not 1e-12 <= qq <= 1e-6:
            continue
        ref = oracle.shell_quartet(mol, *s)
        got = _quartet(pe.pe_quartet_f32, mol, cn, s)
        worst = max(worst, np.abs(got - ref).max() / qq)
        seen.add(tuple(int(l[x]) for x in s))
        count += 1
    assert count > 2000 and len(seen) >= 20, (count, len(seen))
    assert worst <= EPS32, worst
    # genuinely binary32 (the double interpreter is 1e-11 against the oracle)
    assert worst > 1e-6


def test_binary32_f_quartets_within_eps_of_schwarz(pe, oracle):
    """The same on the f-shell chain (heavy 4s3p2d1f, H 3s2p1d): 1500 quartets
    with an f shell sampled from those mixed mode evaluates in binary32, every
    f class among them, error at most EPS32 Q_ab Q_cd."""
    mol = W.small_chain_tz(2, 2, seed=4, tau=1e-12).mol
    cn = oracle.norm_coefs(mol)
    Q = oracle.schwarz(mol)
    l = np.asarray(mol.shell_l)
    ns = len(l)
    cand = []
    for s in itertools.product(range(ns), repeat=4):
        if l[s[0]] < l[s[1]] or l[s[2]] < l[s[3]] or max(l[s[0]], l[s[2]]) < 3:
            continue
        if 1e-12 <= Q[s[0], s[1]] * Q[s[2], s[3]] <= 1e-6:
            cand.append(s)
    rng = np.random.default_rng(3)
    sel = rng.choice(len(cand), size=min(1500, len(cand)), replace=False)
    worst, seen = 0.0, set()
    for i in sel:
        s = cand[i]
        qq = Q[s[0], s[1]] * Q[s[2], s[3]]
        ref = oracle.shell_quartet(mol, *s)
        got = _quartet(pe.pe_quartet_f32, mol, cn, s)
        worst = max(worst, np.abs(got - ref).max() / qq)
        seen.add(tuple(int(l[x]) for x in s))
    print(f"f quartets in binary32: worst error / (Q_ab Q_cd) = {worst:.2e}, {len(seen)} classes")
    assert len(seen) >= 30, len(seen)
    assert worst <= EPS32, worst
    assert worst > 1e-6


def test_mixed_gate_from_the_bound(oracle):
    """The bound on the mixed GPU test's densities: small against max|J|, |K|,
    and zero when nothing is binary32 (promotion threshold below screening)."""
    mol = _mixed_chain()
    Q = oracle.schwarz(mol)
    D = np.random.default_rng(9).standard_normal((8, mol.nao, mol.nao))
    Jr, Kr = oracle.jk(mol, D, 1e-12)
    bj, bk = mixed_jk_bound(Q, mol, D, EPS32 + EPS_DIG, 1e-12, 1e-6)
    rj, rk = bj / np.abs(Jr).max(), bk / np.abs(Kr).max()
    assert 1e-11 < rj < 1e-7 and 1e-11 < rk < 1e-7, (rj, rk)
    assert mixed_jk_bound(Q, mol, D, EPS32, 1e-12, 1e-13) == (0.0, 0.0)


def test_bound_holds_for_planted_binary32_errors(oracle):
    """The bound is an upper bound: on the full ERI tensor of a small molecule,
    perturb every binary32 quartet's elements by eps Q_ab Q_cd with random
    signs (the same value on all eight permutational images) and the J and K
    changes stay within it."""
    mol = W.build_molecule(*W.water_like(), W.draw_kind_bases(np.random.default_rng(2)))
    Q = oracle.schwarz(mol)
    I = oracle.eri_tensor(mol)
    l = np.asarray(mol.shell_l)
    so = np.concatenate([[0], np.cumsum((l + 1) * (l + 2) // 2)])
    sh = np.repeat(np.arange(len(l)), np.diff(so))
    q2 = Q[sh][:, sh]                                  # Q of the shells of (mu, nu)
    QQ = q2[:, :, None, None] * q2[None, None, :, :]
    tmix = float(np.quantile(QQ[QQ >= 1e-12], 0.3))   # a third of the quartets binary32
    rng = np.random.default_rng(0)
    R = rng.choice([-1.0, 1.0], size=I.shape)
    # symmetrise the signs over the eight images of each element
    R = R + R.transpose(1, 0, 2, 3) + R.transpose(0, 1, 3, 2) + R.transpose(1, 0, 3, 2)
    R = R + R.transpose(2, 3, 0, 1)
    R = np.sign(R + 1e-3)
    eps = 1e-3
    dI = np.where((QQ >= 1e-12) & (QQ <= tmix), eps * QQ * R, 0.0)
    D = rng.standard_normal((2, mol.nao, mol.nao))
    J0, K0 = oracle.jk_from_tensor(I, D)
    J1, K1 = oracle.jk_from_tensor(I + dI, D)
    bj, bk = mixed_jk_bound(Q, mol, D, eps, 1e-12, tmix)
    assert np.abs(J1 - J0).max() <= bj * (1 + 1e-9)
    assert np.abs(K1 - K0).max() <= bk * (1 + 1e-9)
    # and it is not vacuous: the planted change reaches a fair part of it
    assert np.abs(J1 - J0).max() >= 1e-3 * bj


def _tf32_truncate(x):
    """binary64 -> binary32 (round to nearest) -> TF32 by dropping the 13 low
    significand bits (round toward zero), returned as binary64."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32)).view(np.uint32)
    return (f & np.uint32(0xFFFFE000)).view(np.float32).astype(np.float64)


def test_tf32_digestion_within_its_bound(oracle):
    """The accuracy of a TF32 tensor-core digestion of the binary32 quartets,
    emulated on the 40-AO chain of the mixed GPU test: the oracle's ERI
    tensor, the binary32 quartets' integrals and the densities they meet
    truncated to TF32, the sums exact.  The J and K change stays within the
    a priori bound with EPS_TF32 (and reaches a fair part of it), and adding
    EPS_TF32 to the mixed mode's per-quartet budget widens the mixed gate by
    about a fifth: a TF32 digestion fits the mixed mode's error class."""
    mol = _mixed_chain()
    Q = oracle.schwarz(mol)
    I = oracle.eri_tensor(mol)
    l = np.asarray(mol.shell_l)
    so = np.concatenate([[0], np.cumsum((l + 1) * (l + 2) // 2)])
    sh = np.repeat(np.arange(len(l)), np.diff(so))
    q2 = Q[sh][:, sh]
    QQ = q2[:, :, None, None] * q2[None, None, :, :]
    tau, tmix = 1e-12, 1e-6
    keep = QQ >= tau
    b32 = keep & (QQ <= tmix)
    assert 0.01 < b32.sum() / keep.sum() < 0.5
    D = np.random.default_rng(9).standard_normal((8, mol.nao, mol.nao))
    J0, K0 = oracle.jk_from_tensor(np.where(keep, I, 0.0), D)
    Ja, Ka = oracle.jk_from_tensor(np.where(keep & ~b32, I, 0.0), D)
    Jb, Kb = oracle.jk_from_tensor(np.where(b32, _tf32_truncate(I), 0.0), _tf32_truncate(D))
    dJ, dK = np.abs(Ja + Jb - J0).max(), np.abs(Ka + Kb - K0).max()
    bj, bk = mixed_jk_bound(Q, mol, D, EPS_TF32, tau, tmix)
    assert dJ <= bj and dK <= bk, (dJ, bj, dK, bk)
    assert dJ >= 1e-3 * bj and dK >= 1e-3 * bk, (dJ, bj, dK, bk)
    # measured: 3.8e-11 / 3.5e-11 of max|J| / max|K|
    assert dJ < 1e-10 * np.abs(J0).max() and dK < 1e-10 * np.abs(K0).max()
    gj, gk = mixed_jk_bound(Q, mol, D, EPS32 + EPS_DIG, tau, tmix)
    tj, tk = mixed_jk_bound(Q, mol, D, EPS32 + EPS_DIG + EPS_TF32, tau, tmix)
    assert tj <= 1.25 * gj and tk <= 1.25 * gk
