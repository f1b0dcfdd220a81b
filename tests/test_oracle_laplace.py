"""Pins for the Laplace quadrature (Eq. laplace) and the pseudo-densities
(Eqs. scaledcoeff, aodensk): accuracy against 1/x and the brute-force
energy-denominator sums of Eq. factorize."""
import numpy as np
import pytest

from paper_2607_05622_gb300 import workloads as W


@pytest.fixture(scope="module")
def c1_fits(oracle):
    w = W.config1()
    xmin, xmax = oracle.laplace_range(w.eps_occ, w.eps_vir)
    return xmin, xmax, oracle.laplace_quadrature(xmin, xmax, 16, return_all=True)


def test_error_decreases_with_n(oracle, c1_fits):
    """max_x |x sum w e^{-tx} - 1| falls geometrically with n until the
    least-squares fit reaches its floor (~1e-10 here)."""
    xmin, xmax, fits = c1_fits
    errs = []
    for n in (4, 8, 12, 16):
        t, w_, err = fits[n]
        assert np.all(t > 0) and np.all(w_ > 0)
        xs = np.linspace(xmin, xmax, 7777)
        assert np.max(np.abs(xs * (np.exp(-np.outer(xs, t)) @ w_) - 1)) <= err * (1 + 1e-9)
        errs.append(err)
    for a, b in zip(errs, errs[1:]):
        assert b < 0.1 * a or b < 1e-9, errs
    assert errs[0] < 1e-3 and errs[1] < 1e-7 and errs[3] < 1e-9, errs


@pytest.fixture(scope="module")
def c1_setup(oracle):
    w = W.config1()
    I = oracle.eri_tensor(w.mol)
    xmin, xmax = oracle.laplace_range(w.eps_occ, w.eps_vir)
    return w, I, xmin, xmax


@pytest.mark.parametrize("n", [8, 12])
def test_denominator_sums(oracle, c1_setup, c1_fits, n):
    """sum_q w_q <D_q, J[D_q]> = sum X X (ia|jb)/(d_ia + d_jb) and the K analogue
    with (ij|ab), to within the quadrature's maximum relative error."""
    w, I, xmin, xmax = c1_setup
    t, wq, err = c1_fits[2][n]
    D = oracle.pseudo_densities(w.C_occ, w.C_vir, w.eps_occ, w.eps_vir, w.X, t)
    J, K = oracle.jk_from_tensor(I, D)
    eJ = sum(wq[q] * np.sum(D[q] * J[q]) for q in range(n))
    eK = sum(wq[q] * np.sum(D[q] * K[q]) for q in range(n))
    sJ, sK, aJ, aK = oracle.denominator_sums(I, w.C_occ, w.C_vir, w.eps_occ, w.eps_vir, w.X[0])
    assert abs(eJ - sJ) <= err * aJ * 1.0001 + 1e-12 * aJ
    assert abs(eK - sK) <= err * aK * 1.0001 + 1e-12 * aK
    # and the agreement is real, not vacuous
    assert err * aJ < 1e-4 * abs(sJ) and err * aK < 1e-4 * abs(sK)


def test_zero_point_density(oracle):
    """t = 0 gives D = C_o X C_v^T."""
    w = W.config1()
    D = oracle.pseudo_densities(w.C_occ, w.C_vir, w.eps_occ, w.eps_vir, w.X, np.array([0.0]))
    assert np.allclose(D[0], w.C_occ @ w.X[0] @ w.C_vir.T, rtol=1e-14, atol=1e-12)
