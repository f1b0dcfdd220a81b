"""Full-size parity in the launch configuration bench.py times: J/K of the
200-AO chain (48 pseudo-densities, Schwarz 1e-12), of the 200-AO f-shell
chain (48 densities, FP64 class and mixed) and of the 445-AO macrocycle
(128 densities, mixed precision) against oracle blocks computed one by one
from the definition; the 200-AO gradient against central finite differences
of the GPU FP64 energy and translational invariance."""
import os

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


def densities(L, ctx, w):
    xmin = 2.0 * (w.eps_vir.min() - w.eps_occ.max())
    xmax = 2.0 * (w.eps_vir.max() - w.eps_occ.min())
    t, _, _ = L.laplace_quadrature(xmin, xmax, w.nlap)
    return ctx.pseudo_densities(dev(w.C_occ), dev(w.C_vir), dev(w.eps_occ), dev(w.eps_vir),
                                dev(w.X), t)


def sampled_blocks(oracle, w, D, J, K, pairs, tau):
    off = oracle.shell_offsets(w.mol)
    Dh = D.cpu().numpy()
    errs = []
    for (a, b) in pairs:
        jb = oracle.j_block(w.mol, Dh, a, b, tau)
        kb = oracle.k_block(w.mol, Dh, a, b, tau)
        Jg = J[:, off[a]:off[a + 1], off[b]:off[b + 1]].cpu().numpy()
        Kg = K[:, off[a]:off[a + 1], off[b]:off[b + 1]].cpu().numpy()
        errs.append((np.abs(Jg - jb).max(), np.abs(Kg - kb).max()))
    return errs


def test_chain200_fp64_and_mixed_sampled(L, oracle):
    w = W.config2()
    ns = w.mol.nshells
    rng = np.random.default_rng(2)
    pairs = [(int(rng.integers(ns)), int(rng.integers(ns))) for _ in range(4)] + [(ns - 1, 0)]
    c64 = L.Context(w.mol, schwarz_tau=w.schwarz_tau)
    D = densities(L, c64, w)
    J, K = c64.jk_build(D)
    cmx = L.Context(w.mol, schwarz_tau=w.schwarz_tau, mixed_tau=1e-6, precision=L.MIXED)
    Jm, Km = cmx.jk_build(D)
    torch.cuda.synchronize()
    sj, sk = float(J.abs().max()), float(K.abs().max())
    for ej, ek in sampled_blocks(oracle, w, D, J, K, pairs, w.schwarz_tau):
        assert ej <= 1e-10 * sj and ek <= 1e-10 * sk, (ej / sj, ek / sk)
    for ej, ek in sampled_blocks(oracle, w, D, Jm, Km, pairs, w.schwarz_tau):
        assert ej <= 1e-8 * sj and ek <= 1e-8 * sk, (ej / sj, ek / sk)
    # every density, every element: K[D^T] = K[D]^T holds for the full build too
    JT, KT = c64.jk_build(D.transpose(1, 2).contiguous())
    assert float((KT - K.transpose(1, 2)).abs().max()) <= 1e-12 * sk
    assert float((JT - J).abs().max()) <= 1e-12 * sj


def test_fshell_chain200_sampled(L, oracle):
    w = W.config_fshell()
    l = np.asarray(w.mol.shell_l)
    fs = [s for s in range(len(l)) if l[s] == 3]
    ds = [s for s in range(len(l)) if l[s] == 2]
    pairs = [(fs[0], fs[0]), (fs[1], fs[-1]), (fs[2], ds[-1]), (ds[0], 0), (len(l) - 1, fs[1])]
    c64 = L.Context(w.mol, schwarz_tau=w.schwarz_tau)
    D = densities(L, c64, w)
    J, K = c64.jk_build(D)
    cmx = L.Context(w.mol, schwarz_tau=w.schwarz_tau, mixed_tau=1e-6, precision=L.MIXED)
    Jm, Km = cmx.jk_build(D)
    torch.cuda.synchronize()
    sj, sk = float(J.abs().max()), float(K.abs().max())
    off = oracle.shell_offsets(w.mol)
    Dh = D.cpu().numpy()
    e64, emx = [], []
    for (a, b) in pairs:  # each oracle block once, against both builds
        jb = oracle.j_block(w.mol, Dh, a, b, w.schwarz_tau)
        kb = oracle.k_block(w.mol, Dh, a, b, w.schwarz_tau)
        for (Jx, Kx, out) in ((J, K, e64), (Jm, Km, emx)):
            Jg = Jx[:, off[a]:off[a + 1], off[b]:off[b + 1]].cpu().numpy()
            Kg = Kx[:, off[a]:off[a + 1], off[b]:off[b + 1]].cpu().numpy()
            out.append((np.abs(Jg - jb).max(), np.abs(Kg - kb).max()))
    print("f-shell chain 200 AO: FP64 class %.2e, mixed %.2e of max |J|,|K|"
          % (max(max(a / sj, b / sk) for a, b in e64), max(max(a / sj, b / sk) for a, b in emx)))
    for ej, ek in e64:
        assert ej <= 1e-10 * sj and ek <= 1e-10 * sk, (ej / sj, ek / sk)
    for ej, ek in emx:
        assert ej <= 1e-8 * sj and ek <= 1e-8 * sk, (ej / sj, ek / sk)


def test_macrocycle445_mixed_sampled(L, oracle):
    w = W.config3()
    ns = w.mol.nshells
    pairs = [(0, 0), (8, 3), (ns - 1, ns // 2)]
    cmx = L.Context(w.mol, schwarz_tau=w.schwarz_tau, mixed_tau=1e-6, precision=L.MIXED)
    D = densities(L, cmx, w)
    Jm, Km = cmx.jk_build(D)
    torch.cuda.synchronize()
    sj, sk = float(Jm.abs().max()), float(Km.abs().max())
    errs = sampled_blocks(oracle, w, D, Jm, Km, pairs, w.schwarz_tau)
    worst = max(max(ej / sj, ek / sk) for ej, ek in errs)
    print(f"macrocycle 445 AO mixed: max error relative to max |J|,|K| = {worst:.2e}")
    assert worst <= 1e-8


def gpu_energy(L, mol, P, Q, cJ, cK, tau):
    c = L.Context(mol, schwarz_tau=tau)
    J, K = c.jk_build(Q)
    return float(torch.sum(P * (cJ * J + cK * K)))


def test_chain200_gradient_fd(L):
    wl = W.config4()
    mol = wl.mol
    P, Q = dev(wl.P), dev(wl.Q)
    tau = 0.0  # unscreened: a screened energy jumps where a quartet crosses tau
    c = L.Context(mol, schwarz_tau=tau)
    g = c.jk_grad(P, Q, wl.cJ, wl.cK).cpu().numpy()
    gmax = np.abs(g).max()
    assert np.abs(g.sum(axis=0)).max() <= 1e-10 * gmax
    h = 1e-4
    for atom, x in [(0, 0), (4, 1), (9, 0), (12, 1), (19, 0), (19, 2)]:
        cp = mol.coords.copy(); cp[atom, x] += h
        cm = mol.coords.copy(); cm[atom, x] -= h
        fd = (gpu_energy(L, mol.with_coords(cp), P, Q, wl.cJ, wl.cK, tau)
              - gpu_energy(L, mol.with_coords(cm), P, Q, wl.cJ, wl.cK, tau)) / (2 * h)
        assert abs(g[atom, x] - fd) <= 1e-7 * gmax + 1e-9, (atom, x, g[atom, x], fd)


def test_chain200_gradient_row_vs_oracle(L):
    """The full-size gradient (200-AO chain, 16 terms, unscreened) against the
    oracle's explicit four-centre derivative integrals for one atom's row,
    stored by tests/golden/make_grad_chain200.py (the oracle needs minutes for
    it): FP64 gate relative to the largest gradient component."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "grad_chain200_atom19.txt")
    rows = [l for l in open(path) if not l.startswith("#")]
    ref = np.array([float(v) for v in rows[0].split()])
    wl = W.config4()
    P, Q = dev(wl.P), dev(wl.Q)
    for prec in (L.FP64, L.FP64_NATIVE):
        c = L.Context(wl.mol, schwarz_tau=0.0, precision=prec)
        g = c.jk_grad(P, Q, wl.cJ, wl.cK).cpu().numpy()
        gmax = np.abs(g).max()
        err = np.abs(g[19] - ref).max() / gmax
        print(f"precision {prec}: atom 19 row vs oracle {err:.2e} of max|g| = {gmax:.3g}")
        assert err <= 1e-10, (prec, g[19], ref)
