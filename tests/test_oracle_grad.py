"""Pins for the oracle's gradient of E = sum_r [cJ J(P_r,Q_r) + cK K(P_r,Q_r)]
(Eq. jkderiv): central finite differences of the energy, translational
invariance (the sum over atoms vanishes), and pair symmetries."""
import numpy as np
import pytest

from paper_2607_05622_gb300 import workloads as W


def small_mol(seed=31):
    c, k = W.chain(2, 1)
    return W.build_molecule(c, k, W.draw_kind_bases(np.random.default_rng(seed)))


def energy(oracle, mol, P, Q, cJ, cK):
    """E via the oracle's J/K of Q_r: sum_r <P_r, cJ J[Q_r] + cK K[Q_r]>, which equals
    cJ J(P,Q) + cK K(P,Q) by the 8-fold symmetry of the integrals."""
    J, K = oracle.jk(mol, Q)
    return float(np.sum(P * (cJ * J + cK * K)))


@pytest.mark.parametrize("cJ,cK,sym,natom", [(1.0, 0.0, True, 2), (1.0, -0.5, False, 3),
                                             (0.0, 1.0, False, 2)])
def test_gradient_against_central_differences(oracle, cJ, cK, sym, natom):
    mol = small_mol() if natom == 3 else W.build_molecule(
        *W.chain(1, 1), W.draw_kind_bases(np.random.default_rng(32)))
    rng = np.random.default_rng(7)
    N, R = mol.nao, 2
    P = rng.standard_normal((R, N, N))
    Q = rng.standard_normal((R, N, N))
    if sym:
        P, Q = 0.5 * (P + P.transpose(0, 2, 1)), 0.5 * (Q + Q.transpose(0, 2, 1))
    g = oracle.grad(mol, P, Q, cJ, cK)
    h = 1e-4
    fd = np.zeros_like(g)
    for a in range(mol.natoms):
        for x in range(3):
            cp = mol.coords.copy(); cp[a, x] += h
            cm = mol.coords.copy(); cm[a, x] -= h
            fd[a, x] = (energy(oracle, mol.with_coords(cp), P, Q, cJ, cK)
                        - energy(oracle, mol.with_coords(cm), P, Q, cJ, cK)) / (2 * h)
    gmax = np.abs(g).max()
    assert np.abs(g - fd).max() <= 1e-7 * gmax + 1e-9, np.abs(g - fd).max() / gmax
    assert np.abs(g.sum(axis=0)).max() <= 1e-10 * gmax           # translational invariance


def test_energy_forms_agree(oracle):
    """E from J/K builds equals the literal four-index form over the tensor."""
    mol = small_mol()
    rng = np.random.default_rng(8)
    N = mol.nao
    P, Q = rng.standard_normal((2, N, N)), rng.standard_normal((2, N, N))
    I = oracle.eri_tensor(mol)
    e1 = oracle.energy_from_tensor(I, P, Q, 1.0, -0.5)
    e2 = energy(oracle, mol, P, Q, 1.0, -0.5)
    assert abs(e1 - e2) <= 1e-12 * abs(e1)


def test_pair_symmetries_and_filter(oracle):
    c, k = W.chain(1, 1)
    mol = W.build_molecule(c, k, W.draw_kind_bases(np.random.default_rng(33)))
    rng = np.random.default_rng(9)
    N = mol.nao
    A = rng.standard_normal((1, N, N)); B = rng.standard_normal((1, N, N))
    Ps, Qs = 0.5 * (A + A.transpose(0, 2, 1)), 0.5 * (B + B.transpose(0, 2, 1))
    g1 = oracle.grad(mol, Ps, Qs, 1.0, 0.0)
    g2 = oracle.grad(mol, Qs, Ps, 1.0, 0.0)
    s = np.abs(g1).max()
    assert np.abs(g1 - g2).max() <= 1e-10 * s                    # J^x(P,Q) = J^x(Q,P)
    anti = A - A.transpose(0, 2, 1)
    g3 = oracle.grad(mol, Ps + anti, Qs, 1.0, 0.0)
    assert np.abs(g3 - g1).max() <= 1e-10 * s                    # antisymmetric part drops from J^x
    g4 = oracle.grad(mol, A, B, 0.0, 1.0)
    g5 = oracle.grad(mol, A.transpose(0, 2, 1).copy(), B.transpose(0, 2, 1).copy(), 0.0, 1.0)
    assert np.abs(g4 - g5).max() <= 1e-10 * np.abs(g4).max()     # K^x(A,B) = K^x(A^T,B^T)
    for atom in range(mol.natoms):
        gf = oracle.grad(mol, A, B, 1.0, -0.5, atom_filter=atom)
        gall = oracle.grad(mol, A, B, 1.0, -0.5)
        assert np.abs(gf[atom] - gall[atom]).max() <= 1e-10 * np.abs(gall).max()
