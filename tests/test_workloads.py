"""The seeded input recipe (host only): the workloads have the shapes the
design states, draw the same inputs on every call, and the f-shell recipe
changes none of the s/p/d workloads' draws."""
import numpy as np

from paper_2607_05622_gb300 import workloads as W


def test_configs_have_their_stated_shapes():
    w1, w2, w3 = W.config1(), W.config2(), W.config3()
    assert (w1.mol.nao, w1.nocc, w1.ndens) == (25, 5, 8)
    assert (w2.mol.nao, w2.nocc, w2.ndens) == (200, 35, 48)
    assert (w3.mol.nao, w3.nocc, w3.ndens) == (445, 86, 128)
    g = W.config4()
    assert g.P.shape == (16, 200, 200) and np.allclose(g.P, g.P.transpose(0, 2, 1))
    wf = W.config_fshell()
    assert (wf.mol.nao, wf.ndens) == (200, 48)
    assert W.water_tz().mol.nao == 65
    gw = W.grad_water_tz()
    assert gw.mol.nao == 65 and gw.P.shape == (2, 65, 65) and not np.allclose(gw.P, gw.P.transpose(0, 2, 1))
    assert max(gw.mol.shell_l) == 3 and (gw.cJ, gw.cK) == (1.0, -0.5)


def test_draws_are_deterministic():
    a, b = W.config2(), W.config2()
    for x, y in ((a.C, b.C), (a.X, b.X), (a.mol.exps, b.mol.exps), (a.mol.coefs, b.mol.coefs)):
        assert np.array_equal(x, y)
    f1, f2 = W.config_fshell(), W.config_fshell()
    assert np.array_equal(f1.mol.exps, f2.mol.exps) and np.array_equal(f1.X, f2.X)


def test_f_shell_recipe():
    """Heavy atoms 4s3p2d1f, H 3s2p1d; f exponents in [0.2, 5], the other
    shells in [0.1, 5e3], three primitives each, coefficients in (0, 1]."""
    mol = W.config_fshell().mol
    l = np.asarray(mol.shell_l)
    per_atom = {}
    for s, a in enumerate(mol.shell_atom):
        per_atom.setdefault(int(a), []).append(int(l[s]))
    for a, kind in enumerate(mol.kinds):
        assert tuple(per_atom[a]) == W.TZ_KIND_SHELLS[kind]
    off = np.concatenate([[0], np.cumsum(mol.shell_nprim)])
    assert (np.asarray(mol.shell_nprim) == 3).all()
    for s in range(mol.nshells):
        e = mol.exps[off[s]:off[s + 1]]
        lo, hi = W.EXP_RANGE_F if l[s] == 3 else W.EXP_RANGE
        assert (e >= lo).all() and (e <= hi).all() and (np.diff(e) <= 0).all()
        c = mol.coefs[off[s]:off[s + 1]]
        assert (c > 0).all() and (c <= 1).all()


def test_kind_shells_draw_unchanged_by_the_f_recipe():
    """draw_kind_bases with the default kinds consumes the generator exactly
    as before the f-shell kinds existed: same exponents for the same seed as
    an explicit draw in the recipe's order."""
    rng = np.random.default_rng(123)
    bases = W.draw_kind_bases(rng)
    ref = np.random.default_rng(123)
    lo, hi = np.log(W.EXP_RANGE[0]), np.log(W.EXP_RANGE[1])
    for kind in ("heavy", "central", "H"):
        for (l, e, c), lk in zip(bases[kind], W.KIND_SHELLS[kind]):
            assert l == lk
            e_ref = np.sort(np.exp(ref.uniform(lo, hi, W.NPRIM)))[::-1]
            c_ref = 1.0 - ref.random(W.NPRIM)
            assert np.array_equal(e, e_ref) and np.array_equal(c, c_ref)
