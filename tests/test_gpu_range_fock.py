"""Densities of any binary64 magnitude, and the library's J/K combination and
energy functional (ltjk_jk_fock, ltjk_jk_energy), against the oracle.

The FP64-class and mixed modes keep densities in double-float and binary32
words; each density is scaled by an exact power of two before those copies
are made and J, K are scaled back, so densities far outside binary32's range
(2^-140, 2^+140) give the same relative accuracy as unit-size ones.  The
oracle side is exact under the same scaling (J and K are linear in D and a
power of two scales binary64 exactly), so the reference is the oracle's J/K of
the unscaled density times the scale."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2607_05622_gb300 import workloads as W  # noqa: E402
from mixed_bound import EPS32, EPS_DIG, mixed_jk_bound  # noqa: E402

TOL64 = 1e-10


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_05622_gb300 import ltjk
    ltjk.lib()
    return ltjk


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def relerr(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.fixture(scope="module")
def chain(oracle):
    wl = W.small_chain(2, 2, seed=4, tau=1e-12)
    m = wl.mol
    D = np.random.default_rng(21).standard_normal((4, m.nao, m.nao))
    Jr, Kr = oracle.jk(m, D, 1e-12)
    return m, D, Jr, Kr


@pytest.mark.parametrize("exp2", [-140, 140, -1000])
@pytest.mark.parametrize("prec", ["fp64", "mixed", "native"])
def test_density_range(L, oracle, chain, prec, exp2):
    m, D, Jr, Kr = chain
    P = {"fp64": L.FP64, "mixed": L.MIXED, "native": L.FP64_NATIVE}[prec]
    ctx = L.Context(m, schwarz_tau=1e-12, mixed_tau=1e-6, precision=P)
    s = 2.0 ** exp2
    Ds = D * s
    assert np.all(Ds / s == D)  # the scaling is exact in binary64
    J, K = ctx.jk_build(dev(Ds))
    torch.cuda.synchronize()
    J, K = J.cpu().numpy() / s, K.cpu().numpy() / s
    ej, ek = relerr(J, Jr), relerr(K, Kr)
    if prec == "mixed":
        bj, bk = mixed_jk_bound(oracle.schwarz(m), m, D, EPS32 + EPS_DIG, 1e-12, 1e-6)
        gj, gk = bj / np.abs(Jr).max() + TOL64, bk / np.abs(Kr).max() + TOL64
    else:
        gj = gk = TOL64
    print(f"{prec} D x 2^{exp2}: J {ej:.2e} K {ek:.2e}")
    assert ej <= gj and ek <= gk


@pytest.mark.parametrize("cJ,cK", [(2.0, -1.0), (1.0, 0.0), (0.0, -0.5), (0.0, 0.0)])
def test_jk_fock(L, chain, cJ, cK):
    m, D, Jr, Kr = chain
    ctx = L.Context(m, schwarz_tau=1e-12)
    F = ctx.jk_fock(dev(D), cJ, cK)
    torch.cuda.synchronize()
    Fr = cJ * Jr + cK * Kr
    if cJ == 0.0 and cK == 0.0:
        assert np.all(F.cpu().numpy() == 0.0)
    else:
        assert relerr(F.cpu().numpy(), Fr) <= TOL64


def test_jk_energy(L, oracle, chain):
    m, D, Jr, Kr = chain
    ctx = L.Context(m, schwarz_tau=1e-12)
    Pm = np.random.default_rng(5).standard_normal(D.shape)
    cJ, cK = 1.0, -0.5
    E, F = ctx.jk_energy(dev(Pm), dev(D), cJ, cK)
    torch.cuda.synchronize()
    Fr = cJ * Jr + cK * Kr
    Er = float(np.sum(Pm * Fr))
    scale = float(np.sum(np.abs(Pm * Fr)))
    assert abs(E.item() - Er) <= TOL64 * scale
    assert relerr(F.cpu().numpy(), Fr) <= TOL64
    # a second call (into the caller's F) agrees to the rounding of the build
    E2, _ = ctx.jk_energy(dev(Pm), dev(D), cJ, cK, F=F)
    assert abs(E2.item() - E.item()) <= 1e-12 * scale
