"""Spherical AO matrices on the GPU: the transformation equals T A T^T of the
oracle's matrix element by element, and J/K of a spherical density reached
through the Cartesian build (density to Cartesian, ltjk_jk_build, results to
spherical) equal the J/K of the oracle's spherical ERI tensor, the Cartesian
tensor transformed on all four indices."""
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


def test_transform_matches_oracle(L, oracle):
    w = W.config1()
    ctx = L.Context(w.mol, schwarz_tau=0.0)
    T = oracle.sph_transform(w.mol)
    assert ctx.nsph == T.shape[0]
    rng = np.random.default_rng(31)
    A = rng.standard_normal((3, w.mol.nao, w.mol.nao))
    B = ctx.to_spherical(dev(A)).cpu().numpy()
    ref = np.einsum("ai,qij,bj->qab", T, A, T)
    assert np.abs(B - ref).max() <= 1e-13 * np.abs(ref).max()
    S = rng.standard_normal((2, T.shape[0], T.shape[0]))
    C = ctx.from_spherical(dev(S)).cpu().numpy()
    refc = np.einsum("ai,qab,bj->qij", T, S, T)
    assert np.abs(C - refc).max() <= 1e-13 * np.abs(refc).max()


def test_spherical_jk_through_the_cartesian_build(L, oracle):
    w = W.config1()
    mol = w.mol
    ctx = L.Context(mol, schwarz_tau=0.0)
    T = oracle.sph_transform(mol)
    Ns = T.shape[0]
    rng = np.random.default_rng(32)
    Ds = rng.standard_normal((2, Ns, Ns))  # non-symmetric
    Dc = ctx.from_spherical(dev(Ds))
    J, K = ctx.jk_build(Dc)
    Js = ctx.to_spherical(J).cpu().numpy()
    Ks = ctx.to_spherical(K).cpu().numpy()
    Is = np.einsum("ai,bj,ijkl,ck,dl->abcd", T, T, oracle.eri_tensor(mol), T, T, optimize=True)
    Jr = np.einsum("abcd,qcd->qab", Is, Ds)
    Kr = np.einsum("acbd,qcd->qab", Is, Ds)
    assert np.abs(Js - Jr).max() <= 1e-10 * np.abs(Jr).max()
    assert np.abs(Ks - Kr).max() <= 1e-10 * np.abs(Kr).max()
