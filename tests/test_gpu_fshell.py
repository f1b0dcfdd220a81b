"""f shells on the GPU (through the C ABI) against the CPU oracle.

The f-shell workloads (heavy atoms 4s3p2d1f, H 3s2p1d) run every class up to
(ff|ff), the heavier ones in output tiles over the first index.  Gates as for
s/p/d: shell-quartet blocks relative to the largest integral, J and K at 1e-10
per output matrix in the FP64 modes, the mixed mode within its a priori bound,
the f spherical transform against the oracle's, and the gradient's refusal of
f shells (its derivative programs stop at d)."""
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
def test_f_shell_quartet_blocks(L, oracle, prec, tol):
    """600 sampled canonical quartets of the 65-AO f-shell water, and every
    (ff|ff) quartet of it, assembled from their output tiles."""
    w = W.water_tz()
    m = w.mol
    ctx = L.Context(m, schwarz_tau=0.0)
    P = {"native": L.FP64_NATIVE, "dfloat": L.FP64, "fp32": L.MIXED}[prec]
    l = np.asarray(m.shell_l)
    ns = m.nshells
    pairs = [(a, b) for a in range(ns) for b in range(ns)
             if l[a] > l[b] or (l[a] == l[b] and a >= b)]
    quartets = [(a, b, c, d) for (a, b) in pairs for (c, d) in pairs]
    rng = np.random.default_rng(0)
    sel = rng.choice(len(quartets), size=600, replace=False)
    qs = [quartets[i] for i in sel]
    fs = [s for s in range(ns) if l[s] == 3]
    qs += [(a, b, c, d) for a in fs for b in fs for c in fs for d in fs]
    blocks = ctx.shell_quartets(qs, precision=P)
    worst = scale = 0.0
    classes = set()
    for q, blk in zip(qs, blocks):
        ref = oracle.shell_quartet(m, *q)
        assert blk.shape == ref.shape
        scale = max(scale, np.abs(ref).max())
        worst = max(worst, np.abs(blk - ref).max())
        classes.add(tuple(int(l[s]) for s in q))
    print(f"{prec}: worst block error / max integral = {worst / scale:.2e}, {len(classes)} classes")
    assert (3, 3, 3, 3) in classes and sum(3 in c for c in classes) >= 30
    assert worst <= tol * scale, worst / scale


@pytest.mark.parametrize("nd,prec", [(1, "dfloat"), (8, "dfloat"), (37, "dfloat"), (8, "native")])
def test_f_shell_jk_unscreened(L, oracle, nd, prec):
    w = W.water_tz()
    P = {"native": L.FP64_NATIVE, "dfloat": L.FP64}[prec]
    ctx = L.Context(w.mol, schwarz_tau=0.0, precision=P)
    D = np.random.default_rng(nd).standard_normal((nd, w.mol.nao, w.mol.nao))  # non-symmetric
    J, K = ctx.jk_build(dev(D))
    torch.cuda.synchronize()
    Jr, Kr = oracle.jk(w.mol, D)
    J, K = J.cpu().numpy(), K.cpu().numpy()
    ej = max(relerr(J[q], Jr[q]) for q in range(nd))
    ek = max(relerr(K[q], Kr[q]) for q in range(nd))
    print(f"f-shell water {prec} nd={nd}: J {ej:.2e} K {ek:.2e}")
    assert ej <= TOL64 and ek <= TOL64


def test_f_shell_jk_chain_screened(L, oracle):
    """100-AO f-shell chain (2 heavy + 2 H), Schwarz 1e-12, 37 densities."""
    wl = W.small_chain_tz(2, 2, seed=4, tau=1e-12)
    m = wl.mol
    ctx = L.Context(m, schwarz_tau=1e-12)
    D = np.random.default_rng(9).standard_normal((37, m.nao, m.nao))
    J, K = ctx.jk_build(dev(D))
    torch.cuda.synchronize()
    Jr, Kr = oracle.jk(m, D, 1e-12)
    J, K = J.cpu().numpy(), K.cpu().numpy()
    for q in range(37):
        assert relerr(J[q], Jr[q]) <= TOL64
        assert relerr(K[q], Kr[q]) <= TOL64


def test_f_shell_mixed_precision_error(L, oracle):
    """Mixed mode on the f-shell chain: within the a priori bound (EPS32 pinned
    for f quartets in tests/test_mixed_bound.py)."""
    wl = W.small_chain_tz(2, 2, seed=4, tau=1e-12)
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
    print(f"f-shell mixed: J rel {ej:.2e} (bound {gj:.2e}) K rel {ek:.2e} (bound {gk:.2e})")
    assert ej <= gj and ek <= gk


def test_f_spherical_transform_and_jk(L, oracle):
    """The f block of the spherical transform equals the oracle's sph_block(3)
    element by element, and J/K of a spherical density through the Cartesian
    build equal those of the oracle's spherical ERI tensor."""
    w = W.water_tz()
    m = w.mol
    ctx = L.Context(m, schwarz_tau=0.0)
    T = oracle.sph_transform(m)
    assert ctx.nsph == T.shape[0] == 4 + 9 + 10 + 7 + 2 * (3 + 6 + 5)
    rng = np.random.default_rng(41)
    A = rng.standard_normal((2, m.nao, m.nao))
    B = ctx.to_spherical(dev(A)).cpu().numpy()
    ref = np.einsum("ai,qij,bj->qab", T, A, T)
    assert relerr(B, ref) <= 1e-13
    Ns = T.shape[0]
    Ds = rng.standard_normal((2, Ns, Ns))
    J, K = ctx.jk_build(ctx.from_spherical(dev(Ds)))
    Js = ctx.to_spherical(J).cpu().numpy()
    Ks = ctx.to_spherical(K).cpu().numpy()
    Is = np.einsum("ai,bj,ijkl,ck,dl->abcd", T, T, oracle.eri_tensor(m), T, T, optimize=True)
    Jr = np.einsum("abcd,qcd->qab", Is, Ds)
    Kr = np.einsum("acbd,qcd->qab", Is, Ds)
    assert relerr(Js, Jr) <= TOL64 and relerr(Ks, Kr) <= TOL64


def test_gradient_refuses_f_shells(L):
    w = W.water_tz()
    ctx = L.Context(w.mol, schwarz_tau=0.0)
    N = w.mol.nao
    P = dev(np.eye(N)[None])
    with pytest.raises(L.LtjkError) as e:
        ctx.jk_grad(P, P, 1.0, 0.0)
    assert e.value.code == L.EUNSUPPORTED
    # the context stays usable
    J, K = ctx.jk_build(P)
    torch.cuda.synchronize()
    assert np.isfinite(J.cpu().numpy()).all()


def test_service_refuses_f_shell_gradient(L):
    w = W.water_tz()
    ctx = L.Context(w.mol, schwarz_tau=0.0)
    N = w.mol.nao
    P = dev(np.eye(N)[None])
    svc = L.Service(1 << 30)
    try:
        with pytest.raises(L.LtjkError) as e:
            svc.submit_grad(ctx, P, P, 1.0, 0.0)
        assert e.value.code == L.EUNSUPPORTED
    finally:
        svc.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_service_and_noalloc_with_f_shells(L, precision):
    """J/K of an f-shell context through the service (f classes in binary64
    beside double-float s/p/d classes in one step, alongside an s/p/d
    context's request) and through the allocation-free entry point equal the
    direct build."""
    prec = L.FP64 if precision == "fp64" else L.MIXED
    wf = W.water_tz()
    ws = W.small_chain(2, 2, seed=4)
    cf = L.Context(wf.mol, schwarz_tau=1e-12, mixed_tau=1e-6, precision=prec)
    cs = L.Context(ws.mol, schwarz_tau=1e-12, mixed_tau=1e-6, precision=prec)
    rng = np.random.default_rng(21)
    Df = dev(rng.standard_normal((6, wf.mol.nao, wf.mol.nao)))
    Ds = dev(rng.standard_normal((4, ws.mol.nao, ws.mol.nao)))
    Jf0, Kf0 = cf.jk_build(Df)
    Js0, Ks0 = cs.jk_build(Ds)
    torch.cuda.synchronize()
    svc = L.Service(1 << 30)
    try:
        t1, Jf, Kf = svc.submit_jk(cf, Df)
        t2, Js, Ks = svc.submit_jk(cs, Ds)
        svc.wait(t1, 120)
        svc.wait(t2, 120)
        for a, b in ((Jf, Jf0), (Kf, Kf0), (Js, Js0), (Ks, Ks0)):
            assert relerr(a.cpu().numpy(), b.cpu().numpy()) <= 1e-12
    finally:
        svc.close()
    J = torch.full_like(Df, np.nan)
    K = torch.full_like(Df, np.nan)
    cf.jk_build_noalloc(Df, J, K)
    torch.cuda.synchronize()
    assert relerr(J.cpu().numpy(), Jf0.cpu().numpy()) <= 1e-12
    assert relerr(K.cpu().numpy(), Kf0.cpu().numpy()) <= 1e-12


@pytest.mark.parametrize("prec", ["dfloat", "mixed"])
def test_f_only_molecules_max_primitives(L, oracle, prec):
    """Degenerate f cases: one f shell of 8 primitives (the largest count; a
    single (ff|ff) quartet, 4096 primitive quartets, on one centre) and two
    atoms carrying one f shell each (only (ff|ff) quartets, three of them
    unique), J and K of non-symmetric densities against the oracle."""
    P = {"dfloat": L.FP64, "mixed": L.MIXED}[prec]
    rng = np.random.default_rng(51)
    e8 = np.sort(np.exp(rng.uniform(np.log(0.2), np.log(5.0), 8)))[::-1].copy()
    c8 = 1.0 - rng.random(8)
    e3 = np.array([2.1, 0.9, 0.35])
    c3 = np.array([0.3, 0.6, 0.4])
    one = W.build_molecule(np.zeros((1, 3)), ["X"], {"X": [(3, e8, c8)]})
    two = W.build_molecule(np.array([[0.0, 0.0, 0.0], [0.3, -1.1, 2.4]]), ["X", "X"],
                           {"X": [(3, e3, c3)]})
    for mol in (one, two):
        assert mol.nao == 10 * mol.natoms
        ctx = L.Context(mol, schwarz_tau=0.0, mixed_tau=1e-6, precision=P)
        D = rng.standard_normal((3, mol.nao, mol.nao))
        J, K = ctx.jk_build(dev(D))
        torch.cuda.synchronize()
        Jr, Kr = oracle.jk(mol, D)
        J, K = J.cpu().numpy(), K.cpu().numpy()
        print(f"f only, {mol.natoms} atom(s), {prec}: J {relerr(J, Jr):.2e} K {relerr(K, Kr):.2e}")
        assert relerr(J, Jr) <= TOL64 and relerr(K, Kr) <= TOL64
