"""The autograd.Function: dE/dcoords from the ERI-derivative kernel and
dE/dP, dE/dQ from J/K builds (the adjoint of a J/K build is a J/K build),
against the oracle and finite differences."""
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


def test_jk_energy_backward(L, oracle):
    c, k = W.chain(2, 1)
    mol = W.build_molecule(c, k, W.draw_kind_bases(np.random.default_rng(31)))
    rng = np.random.default_rng(3)
    N = mol.nao
    Ph, Qh = rng.standard_normal((2, N, N)), rng.standard_normal((2, N, N))
    cJ, cK = 1.0, -0.5
    coords = torch.tensor(mol.coords, dtype=torch.float64, requires_grad=True)
    P = torch.tensor(Ph, device="cuda:0", requires_grad=True)
    Q = torch.tensor(Qh, device="cuda:0", requires_grad=True)
    E = L.JKEnergy.apply(coords, P, Q, mol, cJ, cK, {"schwarz_tau": 0.0})
    E.backward()
    I = oracle.eri_tensor(mol)
    Eref = oracle.energy_from_tensor(I, Ph, Qh, cJ, cK)
    assert abs(E.item() - Eref) <= 1e-10 * abs(Eref)
    gref = oracle.grad(mol, Ph, Qh, cJ, cK)
    gc = coords.grad.cpu().numpy()
    assert np.abs(gc - gref).max() <= 1e-10 * np.abs(gref).max()
    JQ, KQ = oracle.jk_from_tensor(I, Qh)
    JP, KP = oracle.jk_from_tensor(I, Ph)
    gP, gQ = P.grad.cpu().numpy(), Q.grad.cpu().numpy()
    rP, rQ = cJ * JQ + cK * KQ, cJ * JP + cK * KP
    assert np.abs(gP - rP).max() <= 1e-10 * np.abs(rP).max()
    assert np.abs(gQ - rQ).max() <= 1e-10 * np.abs(rQ).max()
    # directional finite difference in P (E is bilinear: exact up to rounding)
    dP = rng.standard_normal(Ph.shape)
    h = 1e-3
    Ep = oracle.energy_from_tensor(I, Ph + h * dP, Qh, cJ, cK)
    Em = oracle.energy_from_tensor(I, Ph - h * dP, Qh, cJ, cK)
    assert abs((Ep - Em) / (2 * h) - np.sum(gP * dP)) <= 1e-9 * abs(Ep)
