"""Python side of the CPU oracle.  TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
(``cpu_baseline`` and ``--impl reference``) may import this module.  It shares
no code with the CUDA library and never imports it.

Contents (each function cites the passage it follows):
  * ctypes wrappers around ``oracle.c`` (McMurchie-Davidson ERIs, J/K, gradient);
  * J/K and the energy functional written as literal sums over a full AO
    tensor (Eq. jkbuild, Eq. jkderiv);
  * the least-squares Laplace quadrature (Eq. laplace), step by step, the
    minimax grid by the Remez exchange and the omega-shifted weights
    (Eq. eomshift);
  * Laplace pseudo-densities (Eqs. scaledcoeff, aodens/aodensk with R = X);
  * the brute-force energy-denominator sums that the quadrature must reproduce
    (Eq. factorize);
  * the Laplace-Fock back-transform to the MO basis (Eq. laplacefock);
  * the Cholesky-factorised two-electron operator and J/K read off it
    (Eqs. cdfact, cdj, cdknonsym), step by step;
  * the Cartesian -> real-spherical transformation of AO matrices.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (OpenMP) into oracle/_build/liboracle.so."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Basis(ctypes.Structure):
    _fields_ = [("natoms", ctypes.c_int), ("coords", ctypes.c_void_p),
                ("nshells", ctypes.c_int), ("sh_atom", ctypes.c_void_p),
                ("sh_l", ctypes.c_void_p), ("sh_nprim", ctypes.c_void_p),
                ("exps", ctypes.c_void_p), ("coefs", ctypes.c_void_p)]


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        I = ctypes.c_int
        D = ctypes.c_double
        _lib.orc_boys.argtypes = [I, D, P]
        _lib.orc_eri_prim.argtypes = [I, I, I, I, D, D, D, D, P, P, P, P, P]
        _lib.orc_norm_coefs.argtypes = [I, P, P, P, P, P]
        _lib.orc_shell_quartet.argtypes = [P, I, I, I, I, P]
        _lib.orc_eri_tensor.argtypes = [P, P]
        _lib.orc_schwarz.argtypes = [P, P]
        _lib.orc_jk.argtypes = [P, I, P, D, P, P]
        _lib.orc_j_block.argtypes = [P, I, P, D, I, I, P]
        _lib.orc_k_block.argtypes = [P, I, P, D, I, I, P]
        _lib.orc_grad.argtypes = [P, I, P, P, D, D, I, P]
        _lib.orc_num_threads.restype = I
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class _BasisRef:
    """Keeps the numpy arrays alive while the C struct points at them."""

    def __init__(self, mol):
        self.arrs = [np.ascontiguousarray(mol.coords, dtype=np.float64),
                     np.ascontiguousarray(mol.shell_atom, dtype=np.int32),
                     np.ascontiguousarray(mol.shell_l, dtype=np.int32),
                     np.ascontiguousarray(mol.shell_nprim, dtype=np.int32),
                     np.ascontiguousarray(mol.exps, dtype=np.float64),
                     np.ascontiguousarray(mol.coefs, dtype=np.float64)]
        c, a, l, n, e, k = self.arrs
        self.s = _Basis(c.shape[0], c.ctypes.data, l.shape[0], a.ctypes.data, l.ctypes.data,
                        n.ctypes.data, e.ctypes.data, k.ctypes.data)

    @property
    def p(self):
        return ctypes.byref(self.s)


def ncart(l):
    return (l + 1) * (l + 2) // 2


def nao(mol) -> int:
    return int(sum(ncart(int(l)) for l in mol.shell_l))


def shell_offsets(mol):
    off = np.zeros(mol.nshells + 1, dtype=np.int64)
    for s, l in enumerate(mol.shell_l):
        off[s + 1] = off[s] + ncart(int(l))
    return off


def num_threads() -> int:
    return int(lib().orc_num_threads())


# ------------------------------------------------------------------ wrappers
def boys(mmax: int, T: float) -> np.ndarray:
    out = np.zeros(mmax + 1)
    lib().orc_boys(mmax, float(T), _ptr(out))
    return out


def eri_prim(ls, es, centers) -> np.ndarray:
    """Primitive block over unnormalised Cartesian Gaussians, shape [na, nb, nc, nd]."""
    la, lb, lc, ld = ls
    out = np.zeros(ncart(la) * ncart(lb) * ncart(lc) * ncart(ld))
    cs = [np.ascontiguousarray(c, dtype=np.float64) for c in centers]
    lib().orc_eri_prim(la, lb, lc, ld, *[float(e) for e in es], *[_ptr(c) for c in cs], _ptr(out))
    return out.reshape(ncart(la), ncart(lb), ncart(lc), ncart(ld))


def norm_coefs(mol) -> np.ndarray:
    out = np.zeros_like(mol.exps)
    lib().orc_norm_coefs(mol.nshells, _ptr(np.ascontiguousarray(mol.shell_l, dtype=np.int32)),
                         _ptr(np.ascontiguousarray(mol.shell_nprim, dtype=np.int32)),
                         _ptr(mol.exps), _ptr(mol.coefs), _ptr(out))
    return out


def shell_quartet(mol, a, b, c, d) -> np.ndarray:
    ls = [int(mol.shell_l[s]) for s in (a, b, c, d)]
    out = np.zeros(int(np.prod([ncart(l) for l in ls])))
    br = _BasisRef(mol)
    lib().orc_shell_quartet(br.p, a, b, c, d, _ptr(out))
    return out.reshape([ncart(l) for l in ls])


def eri_tensor(mol) -> np.ndarray:
    """Full (mu nu|ka rho) tensor, every ordered shell quartet evaluated directly."""
    N = nao(mol)
    out = np.zeros(N ** 4)
    br = _BasisRef(mol)
    lib().orc_eri_tensor(br.p, _ptr(out))
    return out.reshape(N, N, N, N)


def schwarz(mol) -> np.ndarray:
    """Q[a, b] = max sqrt|(mu nu|mu nu)| over mu in shell a, nu in shell b."""
    ns = mol.nshells
    out = np.zeros(ns * ns)
    br = _BasisRef(mol)
    lib().orc_schwarz(br.p, _ptr(out))
    return out.reshape(ns, ns)


def jk(mol, D: np.ndarray, tau: float = 0.0):
    """J[D], K[D] for D [nd, N, N] by the canonical-integral loop with explicit
    permutation images (Eq. jkbuild); Schwarz rule: skip iff Q_ab Q_cd < tau."""
    D = np.ascontiguousarray(D, dtype=np.float64)
    nd, N, _ = D.shape
    J = np.zeros_like(D)
    K = np.zeros_like(D)
    br = _BasisRef(mol)
    lib().orc_jk(br.p, nd, _ptr(D), float(tau), _ptr(J), _ptr(K))
    return J, K


def j_block(mol, D, sa, sb, tau=0.0):
    """J[q][mu][nu] for mu in shell sa, nu in shell sb, from the definition."""
    D = np.ascontiguousarray(D, dtype=np.float64)
    nd = D.shape[0]
    na, nb = ncart(int(mol.shell_l[sa])), ncart(int(mol.shell_l[sb]))
    out = np.zeros(nd * na * nb)
    br = _BasisRef(mol)
    lib().orc_j_block(br.p, nd, _ptr(D), float(tau), sa, sb, _ptr(out))
    return out.reshape(nd, na, nb)


def k_block(mol, D, sa, sc, tau=0.0):
    """K[q][mu][nu] for mu in shell sa, nu in shell sc, from the definition."""
    D = np.ascontiguousarray(D, dtype=np.float64)
    nd = D.shape[0]
    na, nc = ncart(int(mol.shell_l[sa])), ncart(int(mol.shell_l[sc]))
    out = np.zeros(nd * na * nc)
    br = _BasisRef(mol)
    lib().orc_k_block(br.p, nd, _ptr(D), float(tau), sa, sc, _ptr(out))
    return out.reshape(nd, na, nc)


def grad(mol, P, Q, cJ, cK, atom_filter: int = -1) -> np.ndarray:
    """d/dR sum_r [cJ J(P_r,Q_r) + cK K(P_r,Q_r)] (Eq. jkderiv), shape [natoms, 3]."""
    P = np.ascontiguousarray(P, dtype=np.float64)
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    out = np.zeros(mol.natoms * 3)
    br = _BasisRef(mol)
    lib().orc_grad(br.p, P.shape[0], _ptr(P), _ptr(Q), float(cJ), float(cK), int(atom_filter),
                   _ptr(out))
    return out.reshape(mol.natoms, 3)


# -------------------------------------------------- literal sums over a tensor
def jk_from_tensor(I: np.ndarray, D: np.ndarray):
    """Eq. jkbuild written out: J_mn = sum_kr (mn|kr) D_kr, K_mn = sum_kr (mk|nr) D_kr."""
    J = np.einsum("mnkr,qkr->qmn", I, D, optimize=True)
    K = np.einsum("mknr,qkr->qmn", I, D, optimize=True)
    return J, K


def energy_from_tensor(I, P, Q, cJ, cK) -> float:
    """E = sum_r [cJ J(P_r,Q_r) + cK K(P_r,Q_r)], with
    J(A,B) = sum (mn|kr) A_mn B_kr and K(A,B) = sum (mk|nr) A_mn B_kr (Eq. jkderiv)."""
    eJ = np.einsum("mnkr,qmn,qkr->", I, P, Q, optimize=True)
    eK = np.einsum("mknr,qmn,qkr->", I, P, Q, optimize=True)
    return float(cJ * eJ + cK * eK)


# ----------------------------------------------------------- Laplace (Eq. laplace)
def laplace_range(eps_occ, eps_vir):
    """Fit range [2*gap, 2*span] of the doubles denominator D = e_a + e_b - e_i - e_j."""
    return 2.0 * (np.min(eps_vir) - np.max(eps_occ)), 2.0 * (np.max(eps_vir) - np.min(eps_occ))


def laplace_quadrature(xmin: float, xmax: float, n: int, nsample: int = 2000,
                       ncheck: int = 100000, return_all: bool = False):
    """Least-squares exponential sum sum_q w_q exp(-t_q x) ~ 1/x on [xmin, xmax] (Eq. laplace).

    The paper asks for a short exponential-sum grid over the denominator range;
    this oracle fits it in the least-squares sense:
      (1) the problem is scale invariant, so fit on [1, R], R = xmax/xmin, and
          map back with t -> t/xmin, w -> w/xmin;
      (2) nsample log-spaced sample points x_s in [1, R];
      (3) continuation in the number of points: a one-point fit, then for
          k = 2..n one node is appended beyond the largest exponent (geometric
          extrapolation) and all 2k parameters (log t, log w) are refined by
          Levenberg-Marquardt (MINPACK, via scipy) on the relative residual
          r_s = 1 - x_s sum_q w_q exp(-t_q x_s);
      (4) the maximum relative error |x sum w exp(-t x) - 1| on ncheck
          log-spaced points of [xmin, xmax].
    Returns (t, w, max_rel_err), t ascending; with return_all, a dict k -> that triple."""
    from scipy.optimize import least_squares

    R = xmax / xmin
    xs = np.geomspace(1.0, R, nsample)

    def res(th, k):
        with np.errstate(over="ignore", invalid="ignore"):
            t, w = np.exp(th[:k]), np.exp(th[k:])
            r = 1.0 - xs * (np.exp(-np.outer(xs, t)) @ w)
        return np.where(np.isfinite(r), r, 1e150)

    def jac(th, k):
        with np.errstate(over="ignore", invalid="ignore"):
            t, w = np.exp(th[:k]), np.exp(th[k:])
            E = np.exp(-np.outer(xs, t))
            Jm = np.concatenate([(xs ** 2)[:, None] * (w * t)[None, :] * E,
                                 -xs[:, None] * w[None, :] * E], axis=1)
        return np.where(np.isfinite(Jm), Jm, 0.0)

    th = np.array([np.log(1.0 / np.sqrt(R)), 0.0])
    out = {}
    for k in range(1, n + 1):
        if k > 1:
            t, w = np.exp(th[:k - 1]), np.exp(th[k - 1:])
            ratio = t[-1] / t[-2] if k > 2 else 3.0
            t = np.append(t, t[-1] * ratio)
            w = np.append(w, 0.5 * w[-1])
            th = np.concatenate([np.log(t), np.log(w)])
        th = least_squares(res, th, jac=jac, args=(k,), method="lm", xtol=1e-15, ftol=1e-15,
                           gtol=1e-15, max_nfev=4000 * k).x
        order = np.argsort(th[:k])
        th = np.concatenate([th[:k][order], th[k:][order]])
        if return_all or k == n:
            t, w = np.exp(th[:k]) / xmin, np.exp(th[k:]) / xmin
            out[k] = (t, w, laplace_error(t, w, xmin, xmax, ncheck))
    return out if return_all else out[n]


def laplace_error(t, w, xmin, xmax, ncheck=100000) -> float:
    """max over a log-spaced grid of |x sum_q w_q exp(-t_q x) - 1|."""
    xc = np.geomspace(xmin, xmax, ncheck)
    return float(np.max(np.abs(xc * (np.exp(-np.outer(xc, t)) @ w) - 1.0)))


# ---------------------------------------- pseudo-densities (Eqs. scaledcoeff, aodensk)
def pseudo_densities(C_occ, C_vir, eps_occ, eps_vir, X, t) -> np.ndarray:
    """D[q*npair + p] = U_q X_p V_q^T with U_q = C_o diag(e^{t_q eps_o}) and
    V_q = C_v diag(e^{-t_q eps_v}) (Eq. scaledcoeff; Eq. aodensk with the residual
    replaced by the amplitudes X_p).  No quadrature weight is folded in."""
    nlap, npair = len(t), X.shape[0]
    N = C_occ.shape[0]
    D = np.zeros((nlap * npair, N, N))
    for q in range(nlap):
        U = C_occ * np.exp(t[q] * eps_occ)[None, :]
        V = C_vir * np.exp(-t[q] * eps_vir)[None, :]
        for p in range(npair):
            D[q * npair + p] = U @ X[p] @ V.T
    return D


def denominator_sums(I, C_occ, C_vir, eps_occ, eps_vir, X):
    """Brute-force sums the quadrature must reproduce (Eq. factorize):
    SJ = sum_{ia,jb} X_ia X_jb (ia|jb) / (d_ia + d_jb),
    SK = sum_{ia,jb} X_ia X_jb (ij|ab) / (d_ia + d_jb), d_ia = e_a - e_i,
    and the matching sums of absolute values (for the error bound)."""
    ovov = np.einsum("mi,na,kj,rb,mnkr->iajb", C_occ, C_vir, C_occ, C_vir, I, optimize=True)
    oovv = np.einsum("mi,nj,ka,rb,mnkr->ijab", C_occ, C_occ, C_vir, C_vir, I, optimize=True)
    d = eps_vir[None, :] - eps_occ[:, None]
    den = d[:, :, None, None] + d[None, None, :, :]
    XX = np.einsum("ia,jb->iajb", X, X)
    tJ = XX * ovov / den
    tK = XX * oovv.transpose(0, 2, 1, 3) / den
    return float(tJ.sum()), float(tK.sum()), float(np.abs(tJ).sum()), float(np.abs(tK).sum())


# --------------------------------------------- minimax quadrature (Eq. laplace)
def _rel_err_fn(t, w, x):
    return 1.0 - x * (np.exp(-np.outer(x, t)) @ w)


def _alternation_points(t, w, R, n, ngrid=40000):
    """The 2n+1 extrema of e(x) = 1 - x sum w e^{-t x} on [1, R] with alternating
    signs: split a fine log grid at the sign changes of e and take the point of
    largest |e| in every piece."""
    x = np.geomspace(1.0, R, ngrid)
    e = _rel_err_fn(t, w, x)
    sgn = np.sign(e)
    cuts = np.nonzero(sgn[1:] != sgn[:-1])[0] + 1
    pieces = np.split(np.arange(ngrid), cuts)
    pts = np.array([x[p[np.argmax(np.abs(e[p]))]] for p in pieces])
    return pts, e


def laplace_minimax(xmin: float, xmax: float, n: int, iters: int = 60, tol: float = 1e-6):
    """Best uniform (minimax) relative approximation sum_q w_q exp(-t_q x) ~ 1/x
    on [xmin, xmax], the grid the paper asks for (Eq. laplace), by the Remez
    exchange: starting from the least-squares fit, repeatedly (1) take the 2n+1
    alternating extrema x_i of the relative error e(x) = 1 - x sum w e^{-t x} and
    (2) solve e(x_i) = (-1)^i E for (log t, log w, E) by Newton's method, until
    the levelled error E equals the maximum error.  Returns (t, w, max_rel_err)."""
    from scipy.optimize import least_squares

    R = xmax / xmin
    t, w, _ = laplace_quadrature(xmin, xmax, n)
    t, w = t * xmin, w * xmin  # normalised problem on [1, R]
    E = 0.0
    for _ in range(iters):
        pts, e = _alternation_points(t, w, R, n)
        if len(pts) != 2 * n + 1:
            break
        signs = np.sign(_rel_err_fn(t, w, pts))
        E0 = float(np.mean(np.abs(_rel_err_fn(t, w, pts))))

        def eqs(th):
            tt, ww, EE = np.exp(th[:n]), np.exp(th[n:2 * n]), th[2 * n]
            return _rel_err_fn(tt, ww, pts) - signs * EE

        th0 = np.concatenate([np.log(t), np.log(w), [E0]])
        sol = least_squares(eqs, th0, method="lm", xtol=1e-15, ftol=1e-15, gtol=1e-15)
        t, w, E = np.exp(sol.x[:n]), np.exp(sol.x[n:2 * n]), abs(sol.x[2 * n])
        emax = float(np.max(np.abs(_rel_err_fn(t, w, np.geomspace(1.0, R, 40000)))))
        if emax <= E * (1 + tol):
            break
    order = np.argsort(t)
    t, w = t[order] / xmin, w[order] / xmin
    return t, w, laplace_error(t, w, xmin, xmax)


def laplace_shift(t, w, omega):
    """EOM-shifted weights w_q e^{omega t_q} (Eq. eomshift): sum_q w~_q e^{-t_q D}
    approximates 1/(D - omega) wherever D - omega lies in the fitted range."""
    return np.asarray(w) * np.exp(omega * np.asarray(t))


def laplace_fock(J, K, C_left, C_right, cJ=2.0, cK=-1.0):
    """Eq. laplacefock: F[q] = C_left^T (cJ J[q] + cK K[q]) C_right."""
    return np.einsum("mp,qmn,nr->qpr", C_left, cJ * J + cK * K, C_right, optimize=True)


# ------------------------------------------------------------ Cholesky J/K
def cd_factor(I: np.ndarray, delta: float, max_vectors: int | None = None):
    """Pivoted incomplete Cholesky factor of the ERI matrix (Eq. cdfact):
    V[(mu nu), (ka rho)] = (mu nu|ka rho) ~ sum_Q B[Q, mu nu] B[Q, ka rho].
    The plain algorithm: residual diagonal d = diag(V); while the largest d over
    the unique pairs mu >= nu exceeds delta, take that pair p, form the new
    vector (V[:, p] - sum_Q B[Q, :] B[Q, p]) / sqrt(d[p]) and subtract its
    square from d.  Returns (B [naux, N, N], final max residual diagonal)."""
    N = I.shape[0]
    V = I.reshape(N * N, N * N)
    d = np.diag(V).copy()
    uniq = np.array([m * N + n for m in range(N) for n in range(m + 1)])
    vecs = []
    cap = max_vectors if max_vectors is not None else N * (N + 1) // 2
    while len(vecs) < cap:
        p = uniq[np.argmax(d[uniq])]
        if d[p] <= delta:
            break
        col = V[:, p].copy()
        for v in vecs:
            col -= v * v[p]
        v = col / np.sqrt(d[p])
        vecs.append(v)
        d -= v * v
    B = np.array(vecs).reshape(len(vecs), N, N) if vecs else np.zeros((0, N, N))
    return B, float(d[uniq].max())


def cd_jk(B: np.ndarray, U: np.ndarray, V: np.ndarray):
    """J and K of the densities D[q] = U[q] V[q]^T read off the factor B:
    J = sum_Q B_Q gamma_Q with gamma_Q = sum B_Q,ka rho D_ka rho (Eq. cdj), and
    K = sum_{Q,m} (B_Q U)_{mu m} (B_Q V)_{nu m} (Eq. cdknonsym)."""
    D = np.einsum("qkm,qrm->qkr", U, V)
    gamma = np.einsum("Qkr,qkr->qQ", B, D)
    J = np.einsum("qQ,Qmn->qmn", gamma, B)
    BU = np.einsum("Qmk,qkr->qQmr", B, U)
    BV = np.einsum("Qmk,qkr->qQmr", B, V)
    K = np.einsum("qQmr,qQnr->qmn", BU, BV)
    return J, K


# ------------------------------------------------ spherical (real solid) AOs
def sph_block(l: int) -> np.ndarray:
    """Rows: normalised real solid harmonics of one shell in terms of its
    Cartesian components (descending l_x, then l_y; every component carries the
    normalisation of x^l).  s: 1; p: x, y, z kept in Cartesian order; d, in the
    order m = -2..2: sqrt3 xy, sqrt3 yz, (2 zz - xx - yy)/2, sqrt3 xz,
    sqrt3/2 (xx - yy); f, m = -3..3, from the degree-3 solid harmonics below
    (the library has no f shells yet: this is the oracle for that row)."""
    if l == 0:
        return np.ones((1, 1))
    if l == 1:
        return np.eye(3)
    if l == 2:
        r3 = np.sqrt(3.0)
        #               xx        xy  xz  yy        yz  zz
        return np.array([[0.0, r3, 0.0, 0.0, 0.0, 0.0],
                         [0.0, 0.0, 0.0, 0.0, r3, 0.0],
                         [-0.5, 0.0, 0.0, -0.5, 0.0, 1.0],
                         [0.0, 0.0, r3, 0.0, 0.0, 0.0],
                         [r3 / 2, 0.0, 0.0, -r3 / 2, 0.0, 0.0]])
    if l == 3:
        return _sph_from_polynomials(3, _F_HARMONICS)
    raise ValueError("spherical transform defined for l <= 3")


# Real solid harmonics of degree 3, m = -3..3, as integer polynomials
# {(lx, ly, lz): coefficient}: y(3x^2 - y^2), xyz, y(4z^2 - x^2 - y^2),
# z(2z^2 - 3x^2 - 3y^2), x(4z^2 - x^2 - y^2), z(x^2 - y^2), x(x^2 - 3y^2).
_F_HARMONICS = [
    {(2, 1, 0): 3, (0, 3, 0): -1},
    {(1, 1, 1): 1},
    {(0, 1, 2): 4, (2, 1, 0): -1, (0, 3, 0): -1},
    {(0, 0, 3): 2, (2, 0, 1): -3, (0, 2, 1): -3},
    {(1, 0, 2): 4, (3, 0, 0): -1, (1, 2, 0): -1},
    {(2, 0, 1): 1, (0, 2, 1): -1},
    {(3, 0, 0): 1, (1, 2, 0): -3},
]


def _sph_from_polynomials(l: int, polys) -> np.ndarray:
    """Rows of T for polynomials given on the monomials: every Cartesian
    component carries the normalisation of x^l, so their one-centre overlap is
    (lx+lx'-1)!! (ly+ly'-1)!! (lz+lz'-1)!! / (2l-1)!! (zero for an odd sum);
    each row is scaled to unit norm under that overlap."""
    comps = [(lx, ly, l - lx - ly) for lx in range(l, -1, -1) for ly in range(l - lx, -1, -1)]

    def dfact(n):  # (n)!! with (-1)!! = 1
        return 1.0 if n <= 0 else n * dfact(n - 2)

    def ov(a, b):
        e = [a[k] + b[k] for k in range(3)]
        if any(v % 2 for v in e):
            return 0.0
        return dfact(e[0] - 1) * dfact(e[1] - 1) * dfact(e[2] - 1) / dfact(2 * l - 1)

    G = np.array([[ov(a, b) for b in comps] for a in comps])
    T = np.array([[float(p.get(c, 0)) for c in comps] for p in polys])
    return T / np.sqrt(np.einsum("ij,jk,ik->i", T, G, T))[:, None]


def sph_transform(mol) -> np.ndarray:
    """T [N_sph, N_cart], block diagonal over the shells in input order."""
    blocks = [sph_block(l) for l in mol.shell_l]
    ns = sum(b.shape[0] for b in blocks)
    nc = sum(b.shape[1] for b in blocks)
    T = np.zeros((ns, nc))
    r = c = 0
    for b in blocks:
        T[r:r + b.shape[0], c:c + b.shape[1]] = b
        r += b.shape[0]
        c += b.shape[1]
    return T
