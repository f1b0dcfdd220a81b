"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

FP64 gate: max|GPU - oracle| / max|oracle| <= 1e-10 per output matrix and for
the gradient vector (normwise, since single elements can vanish)."""
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


@pytest.mark.parametrize("prec,tol", [("native", 1e-12), ("dfloat", 1e-11), ("fp32", 1e-4)])
def test_shell_quartet_blocks(L, oracle, prec, tol):
    """Sampled unique canonical shell quartets of the 25-AO molecule in IEEE FP64,
    double-float and FP32 recurrences (error relative to the largest integral)."""
    w = W.config1()
    ctx = L.Context(w.mol, schwarz_tau=0.0)
    P = {"native": L.FP64_NATIVE, "dfloat": L.FP64, "fp32": L.MIXED}[prec]
    m = w.mol
    ns = m.nshells
    pairs = [(a, b) for a in range(ns) for b in range(ns)
             if m.shell_l[a] > m.shell_l[b] or (m.shell_l[a] == m.shell_l[b] and a >= b)]
    quartets = [(a, b, c, d) for (a, b) in pairs for (c, d) in pairs]
    rng = np.random.default_rng(0)
    sel = rng.choice(len(quartets), size=min(600, len(quartets)), replace=False)
    qs = [quartets[i] for i in sel]
    blocks = ctx.shell_quartets(qs, precision=P)
    worst = 0.0
    scale = 0.0
    for q, blk in zip(qs, blocks):
        ref = oracle.shell_quartet(m, *q)
        scale = max(scale, np.abs(ref).max())
        worst = max(worst, np.abs(blk - ref).max())
    print(f"{prec}: worst block error / max integral = {worst / scale:.2e}")
    assert worst <= tol * scale, worst / scale


def test_schwarz(L, oracle):
    w = W.config1()
    ctx = L.Context(w.mol, schwarz_tau=0.0)
    Q = ctx.schwarz()
    Qr = oracle.schwarz(w.mol)
    assert relerr(Q, Qr) < 1e-12


def test_pseudo_densities(L, oracle):
    w = W.config2()
    ctx = L.Context(w.mol, schwarz_tau=1e-12)
    t = np.array([0.0, 0.05, 0.3, 1.1, 2.5])
    D = ctx.pseudo_densities(dev(w.C_occ), dev(w.C_vir), dev(w.eps_occ), dev(w.eps_vir), dev(w.X), t)
    torch.cuda.synchronize()
    Dr = oracle.pseudo_densities(w.C_occ, w.C_vir, w.eps_occ, w.eps_vir, w.X, t)
    for q in range(Dr.shape[0]):
        assert relerr(D[q].cpu().numpy(), Dr[q]) < 1e-13


@pytest.mark.parametrize("nd,native", [(1, False), (8, False), (37, False), (8, True)])
def test_jk_water_unscreened(L, oracle, nd, native):
    w = W.config1()
    ctx = L.Context(w.mol, schwarz_tau=0.0, precision=L.FP64_NATIVE if native else L.FP64)
    D = np.random.default_rng(nd).standard_normal((nd, w.mol.nao, w.mol.nao))
    J, K = ctx.jk_build(dev(D))
    torch.cuda.synchronize()
    Jr, Kr = oracle.jk(w.mol, D)
    J, K = J.cpu().numpy(), K.cpu().numpy()
    for q in range(nd):
        assert relerr(J[q], Jr[q]) <= TOL64
        assert relerr(K[q], Kr[q]) <= TOL64


def test_jk_identities_on_gpu(L):
    w = W.config1()
    ctx = L.Context(w.mol, schwarz_tau=0.0)
    D = np.random.default_rng(5).standard_normal((4, w.mol.nao, w.mol.nao))
    J, K = ctx.jk_build(dev(D))
    JT, KT = ctx.jk_build(dev(D.transpose(0, 2, 1)))
    A = D - D.transpose(0, 2, 1)
    JA, KA = ctx.jk_build(dev(A))
    torch.cuda.synchronize()
    J, K, JT, KT, JA, KA = (x.cpu().numpy() for x in (J, K, JT, KT, JA, KA))
    assert relerr(KT, K.transpose(0, 2, 1)) < 1e-13
    assert relerr(JT, J) < 1e-13
    assert np.abs(JA).max() < 1e-13 * np.abs(J).max()
    assert np.abs(KA).max() > 1e-2 * np.abs(K).max()


def test_jk_chain_screened(L, oracle):
    """40-AO chain, Schwarz 1e-12, 37 densities (several tiles and a ragged tail)."""
    wl = W.small_chain(2, 2, seed=4, tau=1e-12)
    m = wl.mol
    ctx = L.Context(m, schwarz_tau=1e-12)
    st = ctx.stats()
    assert st["quartets_kept"] <= st["quartets_total"]
    D = np.random.default_rng(9).standard_normal((37, m.nao, m.nao))
    J, K = ctx.jk_build(dev(D))
    torch.cuda.synchronize()
    Jr, Kr = oracle.jk(m, D, 1e-12)
    J, K = J.cpu().numpy(), K.cpu().numpy()
    for q in range(37):
        assert relerr(J[q], Jr[q]) <= TOL64
        assert relerr(K[q], Kr[q]) <= TOL64


@pytest.mark.parametrize("cJ,cK", [(1.0, 0.0), (1.0, -0.5), (0.0, 1.0)])
def test_gradient(L, oracle, cJ, cK):
    c, k = W.chain(2, 1)
    m = W.build_molecule(c, k, W.draw_kind_bases(np.random.default_rng(31)))
    rng = np.random.default_rng(7)
    P = rng.standard_normal((3, m.nao, m.nao))
    Q = rng.standard_normal((3, m.nao, m.nao))
    ctx = L.Context(m, schwarz_tau=0.0)
    g = ctx.jk_grad(dev(P), dev(Q), cJ, cK)
    torch.cuda.synchronize()
    g = g.cpu().numpy()
    gr = oracle.grad(m, P, Q, cJ, cK)
    assert relerr(g, gr) <= TOL64
    assert np.abs(g.sum(axis=0)).max() <= 1e-10 * np.abs(g).max()


def test_mixed_precision_error(L, oracle):
    """Mixed mode: FP32 quartets below the Schwarz product 1e-6, FP64 above.
    Gate: the a priori bound of tests/mixed_bound.py with the binary32 error
    per quartet pinned on the CPU (tests/test_mixed_bound.py), about 1e-8 of
    max|J|, plus the FP64 gate for the promoted quartets."""
    wl = W.small_chain(2, 2, seed=4, tau=1e-12)
    m = wl.mol
    ctx = L.Context(m, schwarz_tau=1e-12, mixed_tau=1e-6, precision=L.MIXED)
    st = ctx.stats()
    assert 0 < st["quartets_fp64"] < st["quartets_kept"]
    D = np.random.default_rng(9).standard_normal((8, m.nao, m.nao))
    J, K = ctx.jk_build(dev(D))
    torch.cuda.synchronize()
    Jr, Kr = oracle.jk(m, D, 1e-12)
    ej = relerr(J.cpu().numpy(), Jr)
    ek = relerr(K.cpu().numpy(), Kr)
    bj, bk = mixed_jk_bound(oracle.schwarz(m), m, D, EPS32 + EPS_DIG, 1e-12, 1e-6)
    gj, gk = bj / np.abs(Jr).max() + TOL64, bk / np.abs(Kr).max() + TOL64
    print(f"mixed: J rel {ej:.2e} (bound {gj:.2e}) K rel {ek:.2e} (bound {gk:.2e})")
    assert gj < 1e-7 and gk < 1e-7
    assert ej <= gj and ek <= gk
