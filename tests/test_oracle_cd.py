"""Pins of the oracle's Cholesky-factorised J/K (Eqs. cdfact, cdj, cdknonsym):
the complete factorisation reproduces the ERI matrix and the exact J/K of the
McMurchie-Davidson integral loop (Eq. jkbuild); an incomplete one obeys the
positive-semidefinite residual bound |V - B^T B| <= delta elementwise, hence
|J_cd - J| <= delta sum|D|; the factors are symmetric and the factored exchange
equals the literal sum over D = U V^T."""
import numpy as np
import pytest

from paper_2607_05622_gb300 import workloads as W


@pytest.fixture(scope="module")
def tiny(oracle):
    c, k = W.chain(1, 1)
    mol = W.build_molecule(c, k, W.draw_kind_bases(np.random.default_rng(21)))
    return mol, oracle.eri_tensor(mol)


def test_complete_factor_reproduces_eri_and_exact_jk(oracle, tiny):
    mol, I = tiny
    N = I.shape[0]
    B, res = oracle.cd_factor(I, 1e-13)
    assert res <= 1e-13
    V = I.reshape(N * N, N * N)
    BtB = np.einsum("qa,qb->ab", B.reshape(len(B), -1), B.reshape(len(B), -1))
    assert np.abs(BtB - V).max() <= 1e-11 * np.abs(V).max()
    # every vector is a symmetric matrix (the tensor's (mu nu| and (nu mu| agree
    # to rounding), and there are at most N(N+1)/2 of them
    assert np.abs(B - B.transpose(0, 2, 1)).max() <= 1e-11 * np.abs(B).max()
    assert len(B) <= N * (N + 1) // 2
    rng = np.random.default_rng(3)
    U = rng.standard_normal((2, N, 3))
    Vf = rng.standard_normal((2, N, 3))
    D = np.einsum("qkm,qrm->qkr", U, Vf)
    Jc, Kc = oracle.cd_jk(B, U, Vf)
    J, K = oracle.jk(mol, D)
    assert np.abs(Jc - J).max() <= 1e-10 * np.abs(J).max()
    assert np.abs(Kc - K).max() <= 1e-10 * np.abs(K).max()


def test_incomplete_factor_error_bounds(oracle, tiny):
    mol, I = tiny
    N = I.shape[0]
    delta = 1e-4
    B, res = oracle.cd_factor(I, delta)
    assert res <= delta
    V = I.reshape(N * N, N * N)
    R = V - np.einsum("qa,qb->ab", B.reshape(len(B), -1), B.reshape(len(B), -1))
    # the residual is positive semidefinite: |R_ij| <= sqrt(R_ii R_jj) <= max diag
    assert np.abs(R).max() <= res * (1 + 1e-9) + 1e-14
    assert np.linalg.eigvalsh(0.5 * (R + R.T)).min() >= -1e-10
    rng = np.random.default_rng(4)
    U = rng.standard_normal((1, N, N))
    Vf = np.eye(N)[None]
    D = np.einsum("qkm,qrm->qkr", U, Vf)
    Jc, Kc = oracle.cd_jk(B, U, Vf)
    J, K = oracle.jk(mol, D)
    bound = res * np.abs(D).sum()
    assert np.abs(Jc - J).max() <= bound
    assert np.abs(Kc - K).max() <= bound
    # a looser threshold keeps fewer vectors
    B2, _ = oracle.cd_factor(I, 1e-2)
    assert len(B2) < len(B)


def test_factored_exchange_is_the_literal_sum(oracle, tiny):
    _, I = tiny
    N = I.shape[0]
    B, _ = oracle.cd_factor(I, 1e-6)
    rng = np.random.default_rng(5)
    U = rng.standard_normal((1, N, 2))
    Vf = rng.standard_normal((1, N, 2))
    _, Kc = oracle.cd_jk(B, U, Vf)
    D = U[0] @ Vf[0].T
    Klit = np.zeros((N, N))
    for Q in range(len(B)):
        Klit += B[Q] @ D @ B[Q].T
    assert np.abs(Kc[0] - Klit).max() <= 1e-12 * np.abs(Klit).max()
