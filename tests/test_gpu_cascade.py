"""Laplace-Fock back-transform (Eq. laplacefock) and one level of the density
cascade (Eq. aodensk with R = the occupied-virtual Laplace-Fock block) on the
GPU against the oracle chain on the 25-AO molecule."""
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


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def test_two_level_cascade(L, oracle):
    w = W.config1()
    xmin, xmax = oracle.laplace_range(w.eps_occ, w.eps_vir)
    t, _, _ = oracle.laplace_quadrature(xmin, xmax, 4)
    ctx = L.Context(w.mol, schwarz_tau=0.0)
    Co, Cv, C = dev(w.C_occ), dev(w.C_vir), dev(w.C)
    eo, ev = dev(w.eps_occ), dev(w.eps_vir)
    # level 1
    D1 = ctx.pseudo_densities(Co, Cv, eo, ev, dev(w.X), t)
    J1, K1 = ctx.jk_build(D1)
    F = ctx.laplace_fock(J1, K1, C, C)                 # full MO block
    R = ctx.laplace_fock(J1, K1, Co, Cv)               # occupied-virtual block
    # level 2: new grid points, amplitudes R
    t2 = t[::-1].copy()
    D2 = ctx.pseudo_densities(Co, Cv, eo, ev, R, t2)
    J2, K2 = ctx.jk_build(D2)
    torch.cuda.synchronize()
    I = oracle.eri_tensor(w.mol)
    D1r = oracle.pseudo_densities(w.C_occ, w.C_vir, w.eps_occ, w.eps_vir, w.X, t)
    J1r, K1r = oracle.jk_from_tensor(I, D1r)
    Fr = oracle.laplace_fock(J1r, K1r, w.C, w.C)
    Rr = oracle.laplace_fock(J1r, K1r, w.C_occ, w.C_vir)
    D2r = oracle.pseudo_densities(w.C_occ, w.C_vir, w.eps_occ, w.eps_vir, Rr, t2)
    J2r, K2r = oracle.jk_from_tensor(I, D2r)
    assert rel(F.cpu().numpy(), Fr) < 1e-10
    assert rel(R.cpu().numpy(), Rr) < 1e-10
    assert np.allclose(Fr[:, : w.nocc, w.nocc:], Rr, rtol=1e-12, atol=1e-12 * np.abs(Rr).max())
    assert rel(D2.cpu().numpy(), D2r) < 1e-10
    assert rel(J2.cpu().numpy(), J2r) < 1e-10 and rel(K2.cpu().numpy(), K2r) < 1e-10
