"""Edge cases of the J/K build on the GPU: a molecule of one s shell (a single
(ss|ss) quartet), every quartet screened away (J = K = 0 exactly), the largest
accepted density count (4096) and the first rejected one, J-only and K-only
builds, zero densities, and the two ends of the mixed-precision threshold
(mixed_tau = 0: every quartet FP64-class, so the FP64 result; mixed_tau huge:
every quartet FP32, with the cancellation error that the promotion avoids).""" 
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
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def test_single_s_shell(L, oracle):
    bases = {"H": [(0, np.array([3.0, 0.7, 0.15]), np.array([0.2, 0.5, 0.4]))]}
    mol = W.build_molecule(np.zeros((1, 3)), ["H"], bases)
    assert mol.nao == 1
    ctx = L.Context(mol, schwarz_tau=0.0)
    D = np.array([[[0.7]], [[-1.3]]])
    J, K = ctx.jk_build(dev(D))
    Jr, Kr = oracle.jk(mol, D)
    assert rel(J.cpu().numpy(), Jr) < 1e-12 and rel(K.cpu().numpy(), Kr) < 1e-12
    # one function: J = K = (aa|aa) D
    assert np.allclose(Jr, Kr, rtol=1e-14, atol=0)


def test_everything_screened(L):
    w = W.config1()
    ctx = L.Context(w.mol, schwarz_tau=1e30)
    assert ctx.stats()["quartets_kept"] == 0
    D = np.random.default_rng(1).standard_normal((3, w.mol.nao, w.mol.nao))
    J, K = ctx.jk_build(dev(D))
    assert float(J.abs().max()) == 0.0 and float(K.abs().max()) == 0.0


def test_max_density_count_and_rejection(L, oracle):
    w = W.config1()
    N = w.mol.nao
    ctx = L.Context(w.mol, schwarz_tau=0.0)
    rng = np.random.default_rng(2)
    D = rng.standard_normal((4096, N, N))
    J, K = ctx.jk_build(dev(D))
    pick = [0, 1, 2047, 4095]
    Jr, Kr = oracle.jk(w.mol, D[pick])
    Jh, Kh = J.cpu().numpy()[pick], K.cpu().numpy()[pick]
    for i in range(len(pick)):
        assert rel(Jh[i], Jr[i]) <= 1e-10 and rel(Kh[i], Kr[i]) <= 1e-10
    with pytest.raises(L.LtjkError) as e:
        ctx.jk_build(dev(rng.standard_normal((4097, N, N))))
    assert e.value.code == L.EINVAL


def test_j_only_k_only_and_zero(L, oracle):
    w = W.config1()
    N = w.mol.nao
    ctx = L.Context(w.mol, schwarz_tau=0.0)
    D = np.random.default_rng(3).standard_normal((5, N, N))
    Jr, Kr = oracle.jk(w.mol, D)
    J, K = ctx.jk_build(dev(D), want_k=False)
    assert K is None and rel(J.cpu().numpy(), Jr) <= 1e-10
    J, K = ctx.jk_build(dev(D), want_j=False)
    assert J is None and rel(K.cpu().numpy(), Kr) <= 1e-10
    J0, K0 = ctx.jk_build(dev(np.zeros((2, N, N))))
    assert float(J0.abs().max()) == 0.0 and float(K0.abs().max()) == 0.0


def test_mixed_threshold_extremes(L):
    w = W.small_chain(2, 2, seed=4, tau=1e-12)
    m = w.mol
    D = dev(np.random.default_rng(4).standard_normal((6, m.nao, m.nao)))
    J64, K64 = L.Context(m, schwarz_tau=1e-12, precision=L.FP64).jk_build(D)
    c0 = L.Context(m, schwarz_tau=1e-12, mixed_tau=0.0, precision=L.MIXED)
    assert c0.stats()["quartets_fp64"] == c0.stats()["quartets_kept"]
    J0, K0 = c0.jk_build(D)
    assert rel(J0.cpu().numpy(), J64.cpu().numpy()) < 1e-12
    assert rel(K0.cpu().numpy(), K64.cpu().numpy()) < 1e-12
    c1 = L.Context(m, schwarz_tau=1e-12, mixed_tau=1e30, precision=L.MIXED)
    assert c1.stats()["quartets_fp64"] == 0
    J1, K1 = c1.jk_build(D)
    e1 = max(rel(J1.cpu().numpy(), J64.cpu().numpy()), rel(K1.cpu().numpy(), K64.cpu().numpy()))
    # genuinely FP32: measured 2.4e-5 relative to max on this chain -- FP32
    # recurrences lose digits to cancellation on tight exponents (up to 5e3),
    # which is why quartets with a large Schwarz product stay FP64-class in
    # mixed mode (there the error is ~4e-12)
    assert 1e-12 < e1 < 1e-3
