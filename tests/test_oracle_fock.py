"""Pins of the oracle's Laplace-Fock back-transform (Eq. laplacefock):
explicit quadruple loops on a tiny case, the sub-block property, and the
pairing identity sum_ia X_ia F_ia = tr(D^T (cJ J + cK K)) for D = C_o X C_v^T."""
import numpy as np


def test_fock_loops(oracle):
    rng = np.random.default_rng(11)
    nq, n, a, b = 2, 4, 3, 2
    J, K = rng.standard_normal((nq, n, n)), rng.standard_normal((nq, n, n))
    Cl, Cr = rng.standard_normal((n, a)), rng.standard_normal((n, b))
    F = oracle.laplace_fock(J, K, Cl, Cr, cJ=1.5, cK=-0.25)
    for q in range(nq):
        for p in range(a):
            for r in range(b):
                s = 0.0
                for m in range(n):
                    for v in range(n):
                        s += Cl[m, p] * (1.5 * J[q, m, v] - 0.25 * K[q, m, v]) * Cr[v, r]
                assert abs(F[q, p, r] - s) < 1e-13 * (1 + abs(s))


def test_fock_subblock_and_pairing(oracle):
    rng = np.random.default_rng(12)
    nq, n, no = 3, 7, 3
    C = rng.standard_normal((n, n))
    J, K = rng.standard_normal((nq, n, n)), rng.standard_normal((nq, n, n))
    Ff = oracle.laplace_fock(J, K, C, C)
    Fov = oracle.laplace_fock(J, K, C[:, :no], C[:, no:])
    assert np.allclose(Ff[:, :no, no:], Fov, rtol=0, atol=1e-12 * np.abs(Ff).max())
    X = rng.standard_normal((no, n - no))
    D = C[:, :no] @ X @ C[:, no:].T
    for q in range(nq):
        lhs = float(np.sum(X * Fov[q]))
        rhs = float(np.trace(D.T @ (2.0 * J[q] - K[q])))
        assert abs(lhs - rhs) < 1e-11 * (1 + abs(rhs))
