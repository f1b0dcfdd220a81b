"""Pins for the oracle's integrals: brute-force quadrature, closed forms, limits,
normalisation, permutational symmetry and the Cauchy-Schwarz inequality."""
import math
import os
import sys

import numpy as np
import pytest
from numpy.polynomial.hermite import hermgauss

sys.path.insert(0, os.path.dirname(__file__))
from quad_eri import eri_quadrature  # noqa: E402

from paper_2607_05622_gb300 import workloads as W  # noqa: E402


def comps(l):
    return [(lx, ly, l - lx - ly) for lx in range(l, -1, -1) for ly in range(l - lx, -1, -1)]


CLASSES = [(0, 0, 0, 0), (1, 0, 0, 0), (0, 0, 1, 0), (1, 1, 0, 0), (1, 0, 1, 0), (1, 1, 1, 1),
           (2, 0, 0, 0), (2, 1, 1, 0), (2, 2, 0, 0), (2, 0, 2, 0), (2, 2, 2, 2), (2, 1, 2, 1),
           (3, 0, 0, 0), (3, 2, 2, 2), (2, 2, 3, 2), (2, 3, 2, 2)]


@pytest.mark.parametrize("ls", CLASSES)
def test_primitive_block_against_quadrature(oracle, ls):
    """Every tested component of a primitive block equals the brute-force
    quadrature of 1/r12 (independent of the Hermite scheme)."""
    rng = np.random.default_rng(hash(ls) % 2**32)
    es = np.exp(rng.uniform(math.log(0.1), math.log(60.0), 4))
    cs = [rng.uniform(-1.2, 1.2, 3) for _ in range(4)]
    blk = oracle.eri_prim(ls, es, cs)
    scale = np.abs(blk).max()
    idx = [comps(l) for l in ls]
    picks = rng.integers(0, 1 << 30, size=(6, 4))
    for p in picks:
        sel = [int(p[t] % len(idx[t])) for t in range(4)]
        v = eri_quadrature([idx[t][sel[t]] for t in range(4)], es, cs)
        assert abs(v - blk[tuple(sel)]) <= 1e-10 * scale, (ls, sel, v, blk[tuple(sel)])


def test_ss_closed_form(oracle):
    """(ss|ss) = 2 pi^{5/2}/(pq sqrt(p+q)) exp(-ab/p AB^2) exp(-cd/q CD^2) F0(pq/(p+q) PQ^2)."""
    rng = np.random.default_rng(11)
    for _ in range(20):
        a, b, c, d = np.exp(rng.uniform(math.log(0.1), math.log(5e3), 4))
        A, B, C, D = (rng.uniform(-2, 2, 3) for _ in range(4))
        p, q = a + b, c + d
        P, Q = (a * A + b * B) / p, (c * C + d * D) / q
        T = p * q / (p + q) * np.sum((P - Q) ** 2)
        F0 = 1.0 if T == 0 else 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))
        ref = (2 * math.pi ** 2.5 / (p * q * math.sqrt(p + q)) * math.exp(-a * b / p * np.sum((A - B) ** 2))
               * math.exp(-c * d / q * np.sum((C - D) ** 2)) * F0)
        v = oracle.eri_prim((0, 0, 0, 0), (a, b, c, d), (A, B, C, D))[0, 0, 0, 0]
        # exp() of an argument with rounding error |x| eps: relative error ~ |x| eps
        assert abs(v - ref) <= 1e-12 * abs(ref) + 1e-300


def test_same_centre_ss_golden(oracle):
    """Normalised s primitives of one exponent on one centre: (ss|ss) = 2 sqrt(alpha/pi)."""
    path = os.path.join(os.path.dirname(__file__), "golden", "ss_same_centre.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    for alpha, ref in ((float(r[0]), float(r[1])) for r in rows):
        n = (2 * alpha / math.pi) ** 0.75
        z = np.zeros(3)
        v = oracle.eri_prim((0, 0, 0, 0), (alpha,) * 4, (z, z, z, z))[0, 0, 0, 0] * n ** 4
        assert abs(v - ref) <= 1e-14 * ref


def _two_atom(seed, R, kinds=("heavy", "heavy")):
    rng = np.random.default_rng(seed)
    bases = W.draw_kind_bases(rng)
    return W.build_molecule([(0, 0, 0), (0, 0, R)], list(kinds), bases)


def test_far_field_coulomb_limit(oracle):
    """(aa|bb) -> 1/R for unit-normalised s functions far apart."""
    R = 60.0
    m = _two_atom(3, R)
    ns_a = sum(1 for s in range(m.nshells) if m.shell_atom[s] == 0)
    for sa in range(ns_a):
        if m.shell_l[sa] != 0:
            continue
        sb = ns_a + sa
        v = oracle.shell_quartet(m, sa, sa, sb, sb)[0, 0, 0, 0]
        assert abs(v - 1.0 / R) <= 1e-12 / R


def test_contracted_normalisation(oracle):
    """The contracted x^l function of every shell has unit self-overlap (1D Gauss-Hermite)."""
    c, k = W.chain(2, 2)
    m = W.build_molecule(c, k, W.draw_kind_bases(np.random.default_rng(7)))
    nc = oracle.norm_coefs(m)
    y, wy = hermgauss(40)
    p0 = 0
    for s in range(m.nshells):
        l, npr = int(m.shell_l[s]), int(m.shell_nprim[s])
        e, cc = m.exps[p0:p0 + npr], nc[p0:p0 + npr]
        S = 0.0
        for i in range(npr):
            for j in range(npr):
                g = e[i] + e[j]
                ix = np.sum(wy * y ** (2 * l)) / g ** (l + 0.5)
                i0 = np.sum(wy) / g ** 0.5
                S += cc[i] * cc[j] * ix * i0 * i0
        assert abs(S - 1.0) < 1e-13
        p0 += npr


@pytest.fixture(scope="module")
def c1_tensor(oracle):
    w = W.config1()
    return w, oracle.eri_tensor(w.mol)


def test_eightfold_symmetry_positivity_schwarz(oracle, c1_tensor):
    w, I = c1_tensor
    s = np.abs(I).max()
    for perm in [(1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1), (3, 2, 1, 0), (2, 3, 1, 0)]:
        assert np.abs(I - I.transpose(perm)).max() <= 1e-13 * s
    N = I.shape[0]
    diag = np.einsum("mnmn->mn", I)
    assert diag.min() >= -1e-14 * s
    bound = np.sqrt(np.abs(diag)).reshape(N * N)
    assert np.all(np.abs(I.reshape(N * N, N * N)) <= np.outer(bound, bound) * (1 + 1e-12) + 1e-14)
    Q = oracle.schwarz(w.mol)
    off = oracle.shell_offsets(w.mol)
    for a in range(w.mol.nshells):
        for b in range(w.mol.nshells):
            blk = diag[off[a]:off[a + 1], off[b]:off[b + 1]]
            assert abs(Q[a, b] - math.sqrt(np.abs(blk).max())) <= 1e-14 * max(Q.max(), 1)


def test_translation_and_axis_permutation(oracle):
    """A rigid translation leaves every integral unchanged; swapping the x and y
    axes of all centres permutes Cartesian components accordingly."""
    m = W.config1().mol
    rng = np.random.default_rng(2)
    quartets = [(0, 3, 5, 1), (5, 5, 4, 2), (3, 4, 5, 5), (9, 11, 5, 6)]
    for q in quartets:
        ref = oracle.shell_quartet(m, *q)
        mt = m.with_coords(m.coords + rng.uniform(-3, 3, 3))
        tol = 1e-12 * np.abs(ref).max() + 1e-14  # parity-forbidden blocks are 0 up to rounding
        assert np.abs(oracle.shell_quartet(mt, *q) - ref).max() <= tol
        ms = m.with_coords(m.coords[:, [1, 0, 2]])
        sw = oracle.shell_quartet(ms, *q)
        ls = [int(m.shell_l[s]) for s in q]
        cl = [comps(l) for l in ls]
        for i, ci in enumerate(cl[0]):
            for j, cj in enumerate(cl[1]):
                for k, ck in enumerate(cl[2]):
                    for l, cm in enumerate(cl[3]):
                        swp = [cl[t].index((c[1], c[0], c[2])) for t, c in enumerate((ci, cj, ck, cm))]
                        assert abs(sw[tuple(swp)] - ref[i, j, k, l]) <= tol
