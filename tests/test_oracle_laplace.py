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


@pytest.mark.parametrize("rng_,n", [((1.2672, 8.502), 4), ((0.2, 20.0), 4), ((0.2, 20.0), 8)])
def test_minimax_equioscillates(oracle, rng_, n):
    """The Remez result is the minimax grid: its relative error alternates in
    sign at 2n+1 points with equal magnitude (Chebyshev alternation), and its
    maximum error is below the least-squares grid's."""
    xmin, xmax = rng_
    tl, wl, el = oracle.laplace_quadrature(xmin, xmax, n)
    tm, wm, em = oracle.laplace_minimax(xmin, xmax, n)
    pts, _ = oracle._alternation_points(tm * xmin, wm * xmin, xmax / xmin, n)
    ee = oracle._rel_err_fn(tm * xmin, wm * xmin, pts)
    assert len(pts) == 2 * n + 1
    assert np.all(np.sign(ee[1:]) != np.sign(ee[:-1]))
    assert np.abs(ee).max() / np.abs(ee).min() < 1.001
    assert em < el
    assert abs(np.abs(ee).max() - em) <= 1e-3 * em


def test_eom_shift_identity(oracle):
    """sum w e^{omega t} e^{-t D} = sum w e^{-t (D - omega)} (Eq. eomshift): the shifted grid
    has the unshifted grid's error for D - omega in the fitted range."""
    xmin, xmax = 1.2672, 8.502
    t, w, err = oracle.laplace_minimax(xmin, xmax, 6)
    omega = 0.9
    ws = oracle.laplace_shift(t, w, omega)
    D = np.geomspace(xmin + omega, xmax + omega, 5001)
    approx = np.exp(-np.outer(D, t)) @ ws
    assert np.max(np.abs((D - omega) * approx - 1.0)) <= err * (1 + 1e-9)
