"""Brute-force numerical quadrature of single Cartesian Gaussian ERIs.

Independent of the oracle's McMurchie-Davidson scheme: it uses
1/r12 = (2/sqrt(pi)) int_0^inf exp(-t^2 r12^2) dt, which makes the six-
dimensional integral a product over x, y, z of two-dimensional Gaussian
integrals for each t.  Each 2D integral (a polynomial times a Gaussian) is
done exactly by a tensor Gauss-Hermite rule after a Cholesky change of
variables; the t integral is a trapezoid rule in u = ln t, which converges
exponentially for this analytic, exponentially decaying integrand.
"""
import math

import numpy as np
from numpy.polynomial.hermite import hermgauss


def eri_quadrature(comps, exps, centers, nh=12, du=0.02, umin=-36.0, umax=21.0):
    """(ab|cd) over unnormalised primitives (x-A_x)^lx ... exp(-a|r-A|^2)."""
    y, wy = hermgauss(nh)
    Y1, Y2 = np.meshgrid(y, y, indexing="ij")
    W = np.outer(wy, wy)
    u = np.arange(umin, umax + 0.5 * du, du)
    t = np.exp(u)
    t2 = (t * t)[:, None, None]
    a, b, c, d = exps
    p, q = a + b, c + d
    prod = np.ones_like(t)
    for ax in range(3):
        A, B, C, D = (float(cen[ax]) for cen in centers)
        ia, ib, ic, id_ = (cm[ax] for cm in comps)
        P = (a * A + b * B) / p
        Q = (c * C + d * D) / q
        kab = math.exp(-a * b / p * (A - B) ** 2)
        kcd = math.exp(-c * d / q * (C - D) ** 2)
        det = p * q + t2 * (p + q)
        mu1 = ((q + t2) * p * P + t2 * q * Q) / det
        mu2 = (t2 * p * P + (p + t2) * q * Q) / det
        L11 = np.sqrt(p + t2)
        L21 = -t2 / L11
        L22 = np.sqrt(det) / L11
        x2 = mu2 + Y2[None] / L22
        x1 = mu1 + (Y1[None] - L21 * Y2[None] / L22) / L11
        poly = (x1 - A) ** ia * (x1 - B) ** ib * (x2 - C) ** ic * (x2 - D) ** id_
        kappa = p * q * t2[:, 0, 0] / det[:, 0, 0]
        val = (poly * W[None]).sum(axis=(1, 2)) / np.sqrt(det[:, 0, 0])
        prod = prod * kab * kcd * np.exp(-kappa * (P - Q) ** 2) * val
    integrand = prod * t
    return 2.0 / math.sqrt(math.pi) * float(np.trapezoid(integrand, dx=du))
