"""Pins for the oracle's J/K build (Eq. jkbuild) on non-symmetric densities."""
import numpy as np
import pytest

from paper_2607_05622_gb300 import workloads as W


@pytest.fixture(scope="module")
def c1(oracle):
    w = W.config1()
    I = oracle.eri_tensor(w.mol)
    rng = np.random.default_rng(21)
    D = rng.standard_normal((3, w.mol.nao, w.mol.nao))
    return w, I, D


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def test_quartet_loop_equals_literal_sums(oracle, c1):
    """The canonical-integral loop with explicit permutation images equals the
    literal four-index sums over the independently built full tensor."""
    w, I, D = c1
    J, K = oracle.jk(w.mol, D)
    Jr, Kr = oracle.jk_from_tensor(I, D)
    assert rel(J, Jr) < 1e-14 and rel(K, Kr) < 1e-14


def test_jk_identities(oracle, c1):
    w, I, D = c1
    DT = D.transpose(0, 2, 1).copy()
    J, K = oracle.jk_from_tensor(I, D)
    JT, KT = oracle.jk_from_tensor(I, DT)
    Js, _ = oracle.jk_from_tensor(I, 0.5 * (D + DT))
    assert rel(JT, J) < 1e-14 and rel(Js, J) < 1e-14          # J[D] = J[D^T] = J[sym D]
    assert rel(J.transpose(0, 2, 1), J) < 1e-14                # J symmetric
    assert rel(KT, K.transpose(0, 2, 1)) < 1e-14               # K[D^T] = K[D]^T
    assert rel(K.transpose(0, 2, 1), K) > 1e-3                 # K not symmetric for general D
    A = D - DT
    JA, KA = oracle.jk_from_tensor(I, A)
    assert np.abs(JA).max() < 1e-13 * np.abs(J).max()          # antisymmetric D: J = 0
    assert np.abs(KA).max() > 1e-2 * np.abs(K).max()           # ... but K != 0
    D2 = np.random.default_rng(3).standard_normal(D.shape)
    J2, K2 = oracle.jk_from_tensor(I, D2)
    J3, K3 = oracle.jk_from_tensor(I, 2.0 * D - 0.5 * D2)
    assert rel(J3, 2 * J - 0.5 * J2) < 1e-13 and rel(K3, 2 * K - 0.5 * K2) < 1e-13
    # self-adjointness <D', J[D]> = <D, J[D']> and the same for K
    for q in range(D.shape[0]):
        a, b = np.sum(D2[q] * J[q]), np.sum(D[q] * J2[q])
        assert abs(a - b) <= 1e-12 * max(abs(a), 1)
        a, b = np.sum(D2[q] * K[q]), np.sum(D[q] * K2[q])
        assert abs(a - b) <= 1e-12 * max(abs(a), 1)


def test_translation_invariance(oracle, c1):
    w, I, D = c1
    mol_t = w.mol.with_coords(w.mol.coords + np.array([0.7, -1.3, 2.1]))
    J, K = oracle.jk(w.mol, D)
    Jt, Kt = oracle.jk(mol_t, D)
    assert rel(Jt, J) < 1e-12 and rel(Kt, K) < 1e-12


def test_blocks_and_screening(oracle, c1):
    """Sampled blocks from the definition equal the full build; the Schwarz rule
    changes the result by less than tau times the density and quartet count."""
    w, I, D = c1
    Jr, Kr = oracle.jk_from_tensor(I, D)
    off = oracle.shell_offsets(w.mol)
    for (a, b) in [(5, 0), (2, 9), (11, 11), (4, 3)]:
        jb = oracle.j_block(w.mol, D, a, b)
        kb = oracle.k_block(w.mol, D, a, b)
        assert rel(jb, Jr[:, off[a]:off[a + 1], off[b]:off[b + 1]]) < 1e-13
        assert rel(kb, Kr[:, off[a]:off[a + 1], off[b]:off[b + 1]]) < 1e-13
    tau = 1e-7
    Js, Ks = oracle.jk(w.mol, D, tau)
    ns = w.mol.nshells
    bound = tau * np.abs(D).max() * 8 * ns ** 4 * 15 ** 2
    assert np.abs(Js - Jr).max() <= bound and np.abs(Ks - Kr).max() <= bound
    assert np.abs(Js - Jr).max() > 0  # screening actually removed something
