"""Pins of the oracle's Cartesian -> real-spherical transformation: with the
one-centre overlap of the x^l-normalised Cartesian components computed by
Gauss-Hermite quadrature (not by the double-factorial formula), every shell's
spherical functions are orthonormal, the d set is orthogonal to the s-type
contaminant xx + yy + zz and the f set to the p-type contaminants x r^2,
y r^2, z r^2, and every d and f function is a harmonic polynomial (zero
Laplacian); the spherical ERI tensor built from it keeps the 8-fold
permutational symmetry."""
import numpy as np
import pytest

from paper_2607_05622_gb300 import workloads as W


def cart_components(l):
    return [(lx, ly, l - lx - ly) for lx in range(l, -1, -1) for ly in range(l - lx, -1, -1)]


def overlap_quadrature(l, alpha=0.8, npts=40):
    """<m_i|m_j> / <x^l|x^l> for one primitive, 1-D Gauss-Hermite in each direction."""
    x, w = np.polynomial.hermite.hermgauss(npts)
    x = x / np.sqrt(2 * alpha)  # weight exp(-2 alpha r^2) per direction
    comps = cart_components(l)

    def mom(k):
        return float(np.sum(w * x ** k))

    S = np.array([[mom(a[0] + b[0]) * mom(a[1] + b[1]) * mom(a[2] + b[2]) for b in comps] for a in comps])
    return S / S[0, 0]


@pytest.mark.parametrize("l", [0, 1, 2, 3])
def test_spherical_functions_orthonormal(oracle, l):
    T = oracle.sph_block(l)
    S = overlap_quadrature(l)
    assert np.abs(T @ S @ T.T - np.eye(2 * l + 1)).max() < 1e-13


def test_d_set_free_of_s_contaminant(oracle):
    T = oracle.sph_block(2)
    S = overlap_quadrature(2)
    r2 = np.array([1.0, 0, 0, 1.0, 0, 1.0])  # xx + yy + zz
    assert np.abs(T @ S @ r2).max() < 1e-13


def test_spherical_eri_symmetry(oracle):
    c, k = W.water_like()
    mol = W.build_molecule(c, k, W.draw_kind_bases(np.random.default_rng(1)))
    T = oracle.sph_transform(mol)
    assert T.shape == (sum(2 * l + 1 for l in mol.shell_l), mol.nao)
    I = oracle.eri_tensor(mol)
    Is = np.einsum("ai,bj,ijkl,ck,dl->abcd", T, T, I, T, T, optimize=True)
    m = np.abs(Is).max()
    for perm in [(1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1)]:
        assert np.abs(Is - Is.transpose(perm)).max() <= 1e-11 * m


def test_f_set_free_of_p_contaminants(oracle):
    T = oracle.sph_block(3)
    S = overlap_quadrature(3)
    comps = cart_components(3)
    for k in range(3):  # x r^2, y r^2, z r^2
        v = np.zeros(len(comps))
        for j in range(3):
            e = [0, 0, 0]
            e[k] += 1
            e[j] += 2
            v[comps.index(tuple(e))] += 1.0
        assert np.abs(T @ S @ v).max() < 1e-13, k


@pytest.mark.parametrize("l", [2, 3])
def test_spherical_functions_are_harmonic(oracle, l):
    """Every component shares the normalisation of x^l, so a row of T is
    proportional to the polynomial's monomial coefficients; its Laplacian,
    taken term by term, vanishes."""
    T = oracle.sph_block(l)
    comps = cart_components(l)
    for row in T:
        lap = {}
        for c, coef in zip(comps, row):
            for k in range(3):
                if c[k] >= 2:
                    e = list(c)
                    e[k] -= 2
                    lap[tuple(e)] = lap.get(tuple(e), 0.0) + coef * c[k] * (c[k] - 1)
        assert max(abs(v) for v in lap.values()) < 1e-12 * np.abs(row).max()
    assert np.linalg.matrix_rank(T) == 2 * l + 1
