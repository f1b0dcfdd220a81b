"""The library's recurrence programs evaluated on the CPU (tests/program_eval.cpp
interprets them with its own Boys function and primitive set-up) against the
oracle's McMurchie-Davidson contracted blocks, one shell quartet of every value
class from (ss|ss) to (dd|dd), bra and ket classes in both orders, and of every
class with an f shell up to (ff|ff) (whose output tiles are assembled into the
block), at 1e-11 relative to the block's largest element (f classes: 1e-12 with
the programs run in long double, 1e-8 in binary64, whose rounding the f
blocks' horizontal recurrence amplifies); and the derivative programs' nine
tiles, every class, against central differences of the oracle's blocks: the generator's
vertical and horizontal steps, its compacted slots, channel weights and
component order are right before any kernel runs them.  The derivative
programs of f classes, which the library does not use yet, are checked the
same way against central differences, (ff|ff) with its sub-tiles."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2607_05622_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
OUT = os.path.join(ROOT, "tests", "_build")


@pytest.fixture(scope="module")
def pe():
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    os.makedirs(OUT, exist_ok=True)
    so = os.path.join(OUT, "libprogram_eval.so")
    src = [os.path.join(ROOT, "tests", "program_eval.cpp"),
           os.path.join(ROOT, "paper_2607_05622_gb300", "csrc", "program.cpp")]
    subprocess.run([cxx, "-O2", "-std=c++17", "-shared", "-fPIC",
                    "-I", os.path.join(ROOT, "paper_2607_05622_gb300", "csrc"),
                    "-I", os.path.join(ROOT, "include"), *src, "-o", so], check=True)
    lib = ctypes.CDLL(so)
    assert lib.pe_init() == 0
    return lib


def _quartet(pe, oracle, mol, cn, shells, long_double=False):
    ls = [int(mol.shell_l[s]) for s in shells]
    ctr = np.concatenate([mol.coords[mol.shell_atom[s]] for s in shells]).astype(np.float64)
    off = np.concatenate([[0], np.cumsum(mol.shell_nprim)])
    np_ = np.array([mol.shell_nprim[s] for s in shells], dtype=np.int32)
    ex = np.concatenate([mol.exps[off[s]:off[s + 1]] for s in shells])
    co = np.concatenate([cn[off[s]:off[s + 1]] for s in shells])
    n = [(l + 1) * (l + 2) // 2 for l in ls]
    out = np.zeros(int(np.prod(n)))
    P = ctypes.POINTER(ctypes.c_double)
    args = (ctr.ctypes.data_as(P), np_.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
            ex.ctypes.data_as(P), co.ctypes.data_as(P), out.ctypes.data_as(P))
    rc = pe.pe_quartet_ld(*ls, 0, *args) if long_double else pe.pe_quartet(*ls, *args)
    assert rc == 0
    return out.reshape(n)


def test_every_value_class_against_the_oracle(pe, oracle):
    c, k = W.chain(2, 2)  # heavy 3s2p1d + H 2s1p, several centres
    mol = W.build_molecule(c, k, W.draw_kind_bases(np.random.default_rng(7)))
    cn = oracle.norm_coefs(mol)
    by_l = {}
    for s, l in enumerate(mol.shell_l):
        by_l.setdefault(int(l), []).append(s)
    rng = np.random.default_rng(1)
    pairs = [(la, lb) for la in range(3) for lb in range(la + 1)]
    checked = 0
    for (la, lb) in pairs:
        for (lc, ld) in pairs:
            shells = [int(rng.choice(by_l[l])) for l in (la, lb, lc, ld)]
            got = _quartet(pe, oracle, mol, cn, shells)
            ref = oracle.shell_quartet(mol, *shells)
            scale = np.abs(ref).max()
            assert np.abs(got - ref).max() <= 1e-11 * scale, ((la, lb, lc, ld), np.abs(got - ref).max() / scale)
            checked += 1
    assert checked == 36


def test_every_f_value_class_against_the_oracle(pe, oracle):
    w = W.small_chain_tz(2, 2, seed=7)  # heavy 4s3p2d1f + H 3s2p1d, several centres
    mol = w.mol
    cn = oracle.norm_coefs(mol)
    by_l = {}
    for s, l in enumerate(mol.shell_l):
        by_l.setdefault(int(l), []).append(s)
    rng = np.random.default_rng(2)
    pairs = [(la, lb) for la in range(4) for lb in range(la + 1)]
    checked = 0
    for (la, lb) in pairs:
        for (lc, ld) in pairs:
            if max(la, lc) < 3:
                continue
            while True:  # at least two centres (one-centre blocks of odd total l vanish)
                shells = [int(rng.choice(by_l[l])) for l in (la, lb, lc, ld)]
                if len({int(mol.shell_atom[s]) for s in shells}) > 1:
                    break
            ref = oracle.shell_quartet(mol, *shells)
            scale = np.abs(ref).max()
            # the programs in long double pin their steps: 1e-12 of the block
            got = _quartet(pe, oracle, mol, cn, shells, long_double=True)
            err = np.abs(got - ref).max() / scale
            assert err <= 1e-12, ((la, lb, lc, ld), err)
            # in binary64 the horizontal transfer of these blocks amplifies
            # rounding (up to ~5e-10 of the block measured on f quartets with
            # d partners of exponent ~1e3): bounded, not a wrong step
            got = _quartet(pe, oracle, mol, cn, shells)
            err = np.abs(got - ref).max() / scale
            assert err <= 1e-8, ((la, lb, lc, ld), err)
            checked += 1
    assert checked == 100 - 36


def test_derivative_tiles_against_finite_differences(pe, oracle):
    """Derivative programs (four weighted channels, nine (centre, direction)
    tiles): each tile equals the central difference of the oracle's value block
    when only that shell's centre moves (four shells on four atoms)."""
    c, k = W.chain(2, 2)
    base = W.build_molecule(c, k, W.draw_kind_bases(np.random.default_rng(7)))
    # one shell per atom: a d shell, a p shell, a p shell and an s shell
    atoms = {}
    for s, (a, l) in enumerate(zip(base.shell_atom, base.shell_l)):
        atoms.setdefault(int(a), {})[int(l)] = s
    pick = []
    for l, a in ((2, 0), (1, 2), (1, 1), (0, 3)):
        pick.append(atoms[a][l])
    cn = oracle.norm_coefs(base)
    got = _quartet_d(pe, base, cn, pick)
    h = 1e-4
    scale = None
    for centre in range(3):
        for x in range(3):
            blocks = []
            for sgn in (1.0, -1.0):
                cc = base.coords.copy()
                cc[base.shell_atom[pick[centre]], x] += sgn * h
                blocks.append(oracle.shell_quartet(base.with_coords(cc), *pick))
            fd = (blocks[0] - blocks[1]) / (2 * h)
            scale = np.abs(fd).max() if scale is None else max(scale, np.abs(fd).max())
            tile = got[3 * centre + x]
            assert np.abs(tile - fd).max() <= 1e-6 * np.abs(fd).max() + 1e-9, (centre, x)


def _quartet_d(pe, mol, cn, shells):
    ls = [int(mol.shell_l[s]) for s in shells]
    ctr = np.concatenate([mol.coords[mol.shell_atom[s]] for s in shells]).astype(np.float64)
    off = np.concatenate([[0], np.cumsum(mol.shell_nprim)])
    np_ = np.array([mol.shell_nprim[s] for s in shells], dtype=np.int32)
    ex = np.concatenate([mol.exps[off[s]:off[s + 1]] for s in shells])
    co = np.concatenate([cn[off[s]:off[s + 1]] for s in shells])
    n = [(l + 1) * (l + 2) // 2 for l in ls]
    out = np.zeros(9 * int(np.prod(n)))
    P = ctypes.POINTER(ctypes.c_double)
    rc = pe.pe_quartet_d(*ls, 1, ctr.ctypes.data_as(P), np_.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                         ex.ctypes.data_as(P), co.ctypes.data_as(P), out.ctypes.data_as(P))
    assert rc == 0
    return out.reshape([9] + n)


def test_every_derivative_class_against_finite_differences(pe, oracle):
    """All 36 derivative classes, (ss|ss) to (dd|dd) with bra and ket classes in
    both orders: each of the nine (centre, direction) tiles equals the central
    difference of the oracle's value block when only that shell's atom moves.
    The four shells sit on four atoms placed off any plane, so no direction's
    derivative vanishes by symmetry."""
    rng = np.random.default_rng(11)
    coords = [np.zeros(3)]
    while len(coords) < 4:  # four heavy atoms 1.3 to 2.6 bohr apart, in 3D
        p = coords[-1] + rng.normal(size=3)
        d = min(np.linalg.norm(p - q) for q in coords)
        if 1.3 <= d <= 2.6:
            coords.append(p)
    mol = W.build_molecule([tuple(c) for c in coords], ["heavy"] * 4,
                           W.draw_kind_bases(np.random.default_rng(7)))
    off = np.concatenate([[0], np.cumsum(mol.shell_nprim)])
    first = {}  # the most diffuse shell of each l on each atom: blocks of order 0.1, not 1e-9
    for s, (a, l) in enumerate(zip(mol.shell_atom, mol.shell_l)):
        key, lo = (int(a), int(l)), mol.exps[off[s]:off[s + 1]].min()
        if key not in first or lo < first[key][1]:
            first[key] = (s, lo)
    cn = oracle.norm_coefs(mol)
    pairs = [(la, lb) for la in range(3) for lb in range(la + 1)]
    h = 1e-4
    checked = 0
    for (la, lb) in pairs:
        for (lc, ld) in pairs:
            pick = [first[(atom, l)][0] for atom, l in enumerate((la, lb, lc, ld))]
            got = _quartet_d(pe, mol, cn, pick)
            for centre in range(3):
                for x in range(3):
                    blocks = []
                    for sgn in (1.0, -1.0):
                        cc = mol.coords.copy()
                        cc[centre, x] += sgn * h
                        blocks.append(oracle.shell_quartet(mol.with_coords(cc), *pick))
                    fd = (blocks[0] - blocks[1]) / (2 * h)
                    err = np.abs(got[3 * centre + x] - fd).max()
                    assert np.abs(fd).max() > 1e-5, ((la, lb, lc, ld), centre, x)
                    assert err <= 1e-6 * np.abs(fd).max(), ((la, lb, lc, ld), centre, x, err)
            checked += 1
    assert checked == 36


def test_f_derivative_programs_against_finite_differences(pe, oracle):
    """The generator's derivative programs of f classes (not used by the
    library, whose gradient stops at d; built here class by class and
    validated by the generator's checks): the nine (centre, direction) tiles
    equal central differences of the oracle's value blocks, including
    (ff|ff), whose (centre, direction) tiles split over ranges of a's
    components to fit the 16-bit slots."""
    rng = np.random.default_rng(12)
    coords = [np.zeros(3)]
    while len(coords) < 4:  # four atoms 1.3 to 2.6 bohr apart, in 3D
        p = coords[-1] + rng.normal(size=3)
        d = min(np.linalg.norm(p - q) for q in coords)
        if 1.3 <= d <= 2.6:
            coords.append(p)
    mol = W.build_molecule([tuple(c) for c in coords], ["heavy_tz"] * 4,
                           W.draw_tz_bases(np.random.default_rng(8)))
    off = np.concatenate([[0], np.cumsum(mol.shell_nprim)])
    first = {}
    for s, (a, l) in enumerate(zip(mol.shell_atom, mol.shell_l)):
        key, lo = (int(a), int(l)), mol.exps[off[s]:off[s + 1]].min()
        if key not in first or lo < first[key][1]:
            first[key] = (s, lo)
    cn = oracle.norm_coefs(mol)
    P = ctypes.POINTER(ctypes.c_double)
    h = 1e-4
    tiles = {}
    for cls in [(3, 0, 0, 0), (3, 1, 1, 0), (2, 1, 3, 0), (3, 2, 2, 0), (3, 3, 0, 0), (3, 3, 3, 3)]:
        pick = [first[(atom, l)][0] for atom, l in enumerate(cls)]
        ls = list(cls)
        ctr = np.concatenate([mol.coords[mol.shell_atom[s]] for s in pick]).astype(np.float64)
        np_ = np.array([mol.shell_nprim[s] for s in pick], dtype=np.int32)
        ex = np.concatenate([mol.exps[off[s]:off[s + 1]] for s in pick])
        co = np.concatenate([cn[off[s]:off[s + 1]] for s in pick])
        n = [(l + 1) * (l + 2) // 2 for l in ls]
        out = np.zeros(9 * int(np.prod(n)))
        nt = ctypes.c_int(0)
        rc = pe.pe_quartet_fderiv(*ls, ctr.ctypes.data_as(P), np_.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                  ex.ctypes.data_as(P), co.ctypes.data_as(P), out.ctypes.data_as(P),
                                  ctypes.byref(nt))
        assert rc == 0, cls
        tiles[cls] = nt.value
        got = out.reshape([9] + n)
        for centre in range(3):
            for x in range(3):
                blocks = []
                for sgn in (1.0, -1.0):
                    cc = mol.coords.copy()
                    cc[centre, x] += sgn * h
                    blocks.append(oracle.shell_quartet(mol.with_coords(cc), *pick))
                fd = (blocks[0] - blocks[1]) / (2 * h)
                err = np.abs(got[3 * centre + x] - fd).max()
                assert np.abs(fd).max() > 1e-5, (cls, centre, x)
                assert err <= 1e-6 * np.abs(fd).max(), (cls, centre, x, err / np.abs(fd).max())
    assert tiles[(3, 0, 0, 0)] == 9 and tiles[(3, 3, 3, 3)] > 9, tiles


def _cart(l):
    return [(lx, ly, l - lx - ly) for lx in range(l, -1, -1) for ly in range(l - lx, -1, -1)]


def _exact_derivative_tiles(oracle, mol, cn, shells):
    """d/dA_x, d/dB_x, d/dC_x of a contracted block from the oracle's
    primitive integrals over raw Gaussians, by the rule d/dA g_a = 2 alpha
    g_{a+1} - a_x g_{a-1} (the centre of each shell moves with it)."""
    ls = [int(mol.shell_l[s]) for s in shells]
    n = [(l + 1) * (l + 2) // 2 for l in ls]
    off = np.concatenate([[0], np.cumsum(mol.shell_nprim)])
    X = [mol.coords[mol.shell_atom[s]] for s in shells]
    out = np.zeros([9] + n)
    for centre in range(3):
        l = ls[centre]
        up_l, dn_l = _cart(l + 1), (_cart(l - 1) if l > 0 else [])
        for x in range(3):
            raise_i = np.array([up_l.index(tuple(c[t] + (t == x) for t in range(3))) for c in _cart(l)])
            pw = np.array([c[x] for c in _cart(l)], dtype=float)
            lower_i = np.array([dn_l.index(tuple(c[t] - (t == x) for t in range(3))) if c[x] else 0
                                for c in _cart(l)])
            for i in range(off[shells[0]], off[shells[0] + 1]):
                for j in range(off[shells[1]], off[shells[1] + 1]):
                    for k in range(off[shells[2]], off[shells[2] + 1]):
                        for m in range(off[shells[3]], off[shells[3] + 1]):
                            e = [mol.exps[i], mol.exps[j], mol.exps[k], mol.exps[m]]
                            w = cn[i] * cn[j] * cn[k] * cn[m]
                            Lu = list(ls); Lu[centre] += 1
                            blk = 2 * e[centre] * np.take(oracle.eri_prim(Lu, e, X), raise_i, axis=centre)
                            if l > 0:
                                Ld = list(ls); Ld[centre] -= 1
                                dn = np.take(oracle.eri_prim(Ld, e, X), lower_i, axis=centre)
                                shape = [1, 1, 1, 1]; shape[centre] = len(pw)
                                blk = blk - pw.reshape(shape) * dn
                            out[3 * centre + x] += w * blk
    return out


def test_f_derivative_programs_against_exact_derivatives(pe, oracle):
    """The f-class derivative programs against derivative blocks assembled
    from the oracle's primitive integrals with the Gaussian derivative rule:
    run in long double they agree to 1e-11 of the block's largest element (a
    far tighter pin than the finite differences); in binary64 the deep f
    recurrences lose digits to cancellation, as the value classes do, and
    the gate there is 1e-8."""
    rng = np.random.default_rng(13)
    coords = [np.zeros(3)]
    while len(coords) < 4:
        p = coords[-1] + rng.normal(size=3)
        d = min(np.linalg.norm(p - q) for q in coords)
        if 1.3 <= d <= 2.6:
            coords.append(p)
    mol = W.build_molecule([tuple(c) for c in coords], ["heavy_tz"] * 4,
                           W.draw_tz_bases(np.random.default_rng(9)))
    off = np.concatenate([[0], np.cumsum(mol.shell_nprim)])
    first = {}
    for s, (a, l) in enumerate(zip(mol.shell_atom, mol.shell_l)):
        key, lo = (int(a), int(l)), mol.exps[off[s]:off[s + 1]].min()
        if key not in first or lo < first[key][1]:
            first[key] = (s, lo)
    cn = oracle.norm_coefs(mol)
    P = ctypes.POINTER(ctypes.c_double)
    for cls in [(3, 0, 1, 0), (3, 2, 2, 1), (2, 1, 3, 1)]:
        pick = [first[(atom, l)][0] for atom, l in enumerate(cls)]
        ctr = np.concatenate([mol.coords[mol.shell_atom[s]] for s in pick]).astype(np.float64)
        np_ = np.array([mol.shell_nprim[s] for s in pick], dtype=np.int32)
        ex = np.concatenate([mol.exps[off[s]:off[s + 1]] for s in pick])
        co = np.concatenate([cn[off[s]:off[s + 1]] for s in pick])
        n = [(l + 1) * (l + 2) // 2 for l in cls]
        ref = _exact_derivative_tiles(oracle, mol, cn, pick)
        for fn, tol in ((pe.pe_quartet_fderiv_ld, 1e-11), (pe.pe_quartet_fderiv, 1e-8)):
            out = np.zeros(9 * int(np.prod(n)))
            nt = ctypes.c_int(0)
            assert fn(*cls, ctr.ctypes.data_as(P), np_.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                      ex.ctypes.data_as(P), co.ctypes.data_as(P), out.ctypes.data_as(P), ctypes.byref(nt)) == 0
            err = np.abs(out.reshape([9] + n) - ref).max() / np.abs(ref).max()
            assert err <= tol, (cls, fn.__name__, err)


def test_f_shell_gradient_assembled_from_the_programs(pe, oracle):
    """The gradient of E = sum_r [cJ J(P_r,Q_r) + cK K(P_r,Q_r)] (Eq. jkderiv)
    on the 65-AO f-shell water, assembled from the library's derivative
    programs (the f classes built class by class as above): over canonical
    shell quartets, each weighted by the number of distinct quartets its
    eight-fold permutation orbit holds, its nine (centre, direction) tiles
    contracted with Gamma averaged over the orbit, the fourth centre's
    derivative by translational invariance.  Against the oracle's gradient
    (tests/golden/grad_water_tz.txt, McMurchie-Davidson derivative integrals):
    with the programs run in long double it agrees to 1e-11 of max|g|
    (measured 2e-13), which pins the f derivative programs and the assembly
    rule; in binary64 the deep recurrences of the f classes leave 1.0e-9,
    within 1e-8 but above 1e-10: a gradient with f shells needs a tolerance
    derived from binary64's rounding, not the s/p/d gradient's 1e-10."""
    wl = W.grad_water_tz()
    mol = wl.mol
    g_ref = np.loadtxt(os.path.join(ROOT, "tests", "golden", "grad_water_tz.txt"))
    G = (wl.cJ * np.einsum("rmn,rls->mnls", wl.P, wl.Q)
         + wl.cK * np.einsum("rml,rns->mnls", wl.P, wl.Q))     # E = sum I_mnls G_mnls
    G = G + G.transpose(1, 0, 2, 3)
    G = G + G.transpose(0, 1, 3, 2)
    G = (G + G.transpose(2, 3, 0, 1)) / 8                         # orbit average
    ls = np.asarray(mol.shell_l)
    so = np.concatenate([[0], np.cumsum((ls + 1) * (ls + 2) // 2)])
    off = np.concatenate([[0], np.cumsum(mol.shell_nprim)])
    cn = oracle.norm_coefs(mol)
    Pd, Pi = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)

    def tiles(sh, long_double):
        L = [int(ls[s]) for s in sh]
        n = [(l + 1) * (l + 2) // 2 for l in L]
        ctr = np.concatenate([mol.coords[mol.shell_atom[s]] for s in sh]).astype(np.float64)
        np_ = np.array([mol.shell_nprim[s] for s in sh], dtype=np.int32)
        ex = np.concatenate([mol.exps[off[s]:off[s + 1]] for s in sh])
        co = np.concatenate([cn[off[s]:off[s + 1]] for s in sh])
        out = np.zeros(9 * int(np.prod(n)))
        args = (ctr.ctypes.data_as(Pd), np_.ctypes.data_as(Pi), ex.ctypes.data_as(Pd),
                co.ctypes.data_as(Pd), out.ctypes.data_as(Pd))
        if max(L) == 3:
            nt = ctypes.c_int(0)
            fn = pe.pe_quartet_fderiv_ld if long_double else pe.pe_quartet_fderiv
            assert fn(*L, *args, ctypes.byref(nt)) == 0
        else:
            fn = pe.pe_quartet_ld if long_double else pe.pe_quartet_d
            assert fn(*L, 1, *args) == 0
        return out.reshape([9] + n)

    pairs = [(a, b) for a in range(len(ls)) for b in range(a + 1)]
    err = {}
    for long_double in (True, False):
        g = np.zeros((mol.natoms, 3))
        for i, (a, b) in enumerate(pairs):
            for c, d in pairs[:i + 1]:
                orbit = (1 + (a != b)) * (1 + (c != d)) * (1 + ((a, b) != (c, d)))
                sh = [a, b, c, d]
                if ls[sh[0]] < ls[sh[1]]:          # programs take l_a >= l_b, l_c >= l_d
                    sh[0], sh[1] = sh[1], sh[0]
                if ls[sh[2]] < ls[sh[3]]:
                    sh[2], sh[3] = sh[3], sh[2]
                blk = G[tuple(slice(so[s], so[s + 1]) for s in sh)]
                v = orbit * np.einsum("tabcd,abcd->t", tiles(sh, long_double), blk).reshape(3, 3)
                for k in range(3):
                    g[mol.shell_atom[sh[k]]] += v[k]
                g[mol.shell_atom[sh[3]]] -= v.sum(axis=0)
        err[long_double] = np.abs(g - g_ref).max() / np.abs(g_ref).max()
    assert err[True] <= 1e-11, err
    assert 1e-10 < err[False] <= 1e-8, err
