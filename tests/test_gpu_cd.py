"""Cholesky-factorised J/K on the GPU (Eqs. cdfact, cdj, cdknonsym) against the
oracle: the factor reproduces the oracle's ERI matrix within its own residual
bound, the contraction kernels equal the oracle's contraction of the same
factor element by element, and the J/K read off a tight factor equal the exact
J/K of the McMurchie-Davidson loop; on the 200-AO chain the factored J/K of the
48 Laplace pseudo-densities agree with the direct build within the bound."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2607_05622_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_05622_gb300 import ltjk
    ltjk.lib()
    return ltjk


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


@pytest.fixture(scope="module")
def small(oracle):
    c, k = W.chain(1, 1)
    mol = W.build_molecule(c, k, W.draw_kind_bases(np.random.default_rng(21)))
    return mol, oracle.eri_tensor(mol)


@pytest.mark.parametrize("delta", [1e-4, 1e-10])
def test_factor_reproduces_eri_within_residual(L, oracle, small, delta):
    mol, I = small
    N = mol.nao
    ctx = L.Context(mol, schwarz_tau=0.0)
    B, naux, res = ctx.cd_factor(delta, N * (N + 1) // 2)
    torch.cuda.synchronize()
    assert 0 < naux <= N * (N + 1) // 2 and res <= delta
    Bh = B.cpu().numpy().reshape(naux, -1)
    R = I.reshape(N * N, N * N) - Bh.T @ Bh
    # positive semidefinite residual: every element within the largest residual diagonal
    assert np.abs(R).max() <= res + 1e-12 * np.abs(I).max()
    # the oracle's own factorisation keeps a similar number of vectors
    Bo, reso = oracle.cd_factor(I, delta)
    assert abs(len(Bo) - naux) <= max(2, naux // 20)


@pytest.mark.parametrize("precision,tol", [("FP64_NATIVE", 1e-12), ("FP64", 1e-11)])
def test_contraction_matches_oracle_on_the_same_factor(L, oracle, small, precision, tol):
    """IEEE FP64 kernels and the double-float GEMMs, per-density and shared left
    factors, against the oracle's contraction of the same factor."""
    mol, I = small
    N = mol.nao
    ctx = L.Context(mol, schwarz_tau=0.0, precision=getattr(L, precision))
    B, naux, _ = ctx.cd_factor(1e-8, N * (N + 1) // 2)
    Bh = B.cpu().numpy()
    rng = np.random.default_rng(7)
    for rank in (1, 5, N):
        for shared in (False, True):
            U = rng.standard_normal((1 if shared else 3, N, rank))
            V = rng.standard_normal((3, N, rank))
            J, K = ctx.cd_jk(B, dev(U), dev(V))
            torch.cuda.synchronize()
            Jo, Ko = oracle.cd_jk(Bh, np.broadcast_to(U, V.shape).copy(), V)
            assert np.abs(J.cpu().numpy() - Jo).max() <= tol * np.abs(Jo).max(), (rank, shared)
            assert np.abs(K.cpu().numpy() - Ko).max() <= tol * np.abs(Ko).max(), (rank, shared)


def test_tight_factor_gives_exact_jk(L, oracle, small):
    mol, _ = small
    N = mol.nao
    ctx = L.Context(mol, schwarz_tau=0.0)
    B, naux, res = ctx.cd_factor(1e-12, N * (N + 1) // 2)
    rng = np.random.default_rng(8)
    D = rng.standard_normal((2, N, N))  # general non-symmetric D = D I^T
    U = D
    V = np.broadcast_to(np.eye(N), (2, N, N)).copy()
    J, K = ctx.cd_jk(B, dev(U), dev(V))
    torch.cuda.synchronize()
    Jr, Kr = oracle.jk(mol, D)
    assert np.abs(J.cpu().numpy() - Jr).max() <= 1e-9 * np.abs(Jr).max()
    assert np.abs(K.cpu().numpy() - Kr).max() <= 1e-9 * np.abs(Kr).max()
    # the error bound of an incomplete factor: |J_cd - J| <= res * sum|D|
    B4, _, res4 = ctx.cd_factor(1e-4, N * (N + 1) // 2)
    J4, K4 = ctx.cd_jk(B4, dev(U), dev(V))
    torch.cuda.synchronize()
    for q in range(2):
        bound = res4 * np.abs(D[q]).sum()
        assert np.abs(J4[q].cpu().numpy() - Jr[q]).max() <= bound
        assert np.abs(K4[q].cpu().numpy() - Kr[q]).max() <= bound


def test_chain200_factored_pseudo_densities_match_direct(L):
    """Full size: the 48 pseudo-densities of the 200-AO chain as rank-35 factors
    U = C_occ, V_q = C_vir Y_q^T, against the direct FP64-class build."""
    w = W.config2()
    mol = w.mol
    N, no = mol.nao, w.nocc
    ctx = L.Context(mol, schwarz_tau=w.schwarz_tau)
    xmin = 2.0 * (w.eps_vir.min() - w.eps_occ.max())
    xmax = 2.0 * (w.eps_vir.max() - w.eps_occ.min())
    t, _, _ = L.laplace_quadrature(xmin, xmax, w.nlap)
    D = ctx.pseudo_densities(dev(w.C_occ), dev(w.C_vir), dev(w.eps_occ), dev(w.eps_vir), dev(w.X), t)
    Jd, Kd = ctx.jk_build(D)
    B, naux, res = ctx.cd_factor(1e-9, 20 * N)
    U, V = ctx.pseudo_density_factors(dev(w.C_occ), dev(w.C_vir), dev(w.eps_occ), dev(w.eps_vir),
                                      dev(w.X), t)
    # the factors reproduce the pseudo-densities
    assert float((torch.bmm(U, V.transpose(1, 2)) - D).abs().max()) <= 1e-12 * float(D.abs().max())
    J, K = ctx.cd_jk(B, U[:1].contiguous(), V)  # one left factor, C_occ, for every density
    torch.cuda.synchronize()
    assert res <= 1e-9 and naux < 20 * N
    Dh = D.cpu().numpy()
    for q in range(0, D.shape[0], 7):
        bound = res * np.abs(Dh[q]).sum() + 1e-10 * float(Jd[q].abs().max())
        assert float((J[q] - Jd[q]).abs().max()) <= bound
        assert float((K[q] - Kd[q]).abs().max()) <= bound
