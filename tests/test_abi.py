"""Host-side checks of the C-ABI library (no GPU needed): it builds for
sm_103a, loads, exports every entry point declared in include/ltjk.h, and its
host-only Laplace quadrature meets the stated accuracy."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2607_05622_gb300 import build, ltjk
    build.build()
    ltjk.lib()
    return ltjk


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ltjk.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ltjk_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(L):
    names = declared_functions()
    assert len(names) >= 12
    lib = ctypes.CDLL(L.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding knows every one of them
    assert not [n for n in names if n not in L.SIGNATURES], set(names) - set(L.SIGNATURES)


def test_version_and_counter(L):
    assert L.lib().ltjk_version() >= 100
    assert L.launch_count() >= 0


def test_invalid_arguments_report_errors(L):
    with pytest.raises(L.LtjkError) as e:
        L.laplace_quadrature(-1.0, 2.0, 4)
    assert e.value.code == L.EINVAL and "xmin" in str(e.value)
    with pytest.raises(L.LtjkError):
        L.laplace_quadrature(1.0, 2.0, 0)
    rc = L.lib().ltjk_context_create(None, None, None)
    assert rc == L.EINVAL
    assert L.lib().ltjk_last_error()


def test_library_laplace_quadrature(L, oracle):
    from paper_2607_05622_gb300 import workloads as W
    w = W.config1()
    xmin, xmax = oracle.laplace_range(w.eps_occ, w.eps_vir)
    prev = None
    for n in (4, 8, 12):
        t, wq, err = L.laplace_quadrature(xmin, xmax, n)
        assert np.all(np.diff(t) > 0) and np.all(t > 0) and np.all(wq > 0)
        assert abs(err - oracle.laplace_error(t, wq, xmin, xmax)) <= 1e-12 + 1e-9 * err
        if prev is not None:
            assert err < prev
        prev = err
    _, _, e8 = L.laplace_quadrature(xmin, xmax, 8)
    # the variable-projection fit reaches the oracle's least-squares optimum
    # (MINPACK on all 2n parameters) within a small factor
    _, _, eo8 = oracle.laplace_quadrature(xmin, xmax, 8)
    assert e8 < 1e-7 and e8 <= 10.0 * eo8, (e8, eo8)
    # a cached call returns the same nodes
    t1, w1, _ = L.laplace_quadrature(xmin, xmax, 8)
    t2, w2, _ = L.laplace_quadrature(xmin, xmax, 8)
    assert np.array_equal(t1, t2) and np.array_equal(w1, w2)


def test_library_minimax_and_shift(L, oracle):
    """Where the library's Remez exchange converges, it finds the oracle's minimax
    grid (the best approximation is unique); the shift matches Eq. eomshift."""
    for (xmin, xmax), n in [((1.2672, 8.502), 4), ((0.2, 20.0), 4), ((0.2, 20.0), 8)]:
        t, w, err, conv = L.laplace_minimax(xmin, xmax, n)
        assert conv, (xmin, xmax, n)
        to, wo, eo = oracle.laplace_minimax(xmin, xmax, n)
        assert abs(err - eo) <= 1e-3 * eo
        assert np.allclose(t, to, rtol=1e-4) and np.allclose(w, wo, rtol=1e-4)
    t, w, err, conv = L.laplace_minimax(1.2672, 8.502, 12)
    _, _, els = L.laplace_quadrature(1.2672, 8.502, 12)
    assert err <= els * (1 + 1e-12)  # never worse than the least-squares grid
    ws = L.laplace_shift(t, w, 0.75)
    assert np.allclose(ws, oracle.laplace_shift(t, w, 0.75), rtol=1e-14, atol=0)
    with pytest.raises(L.LtjkError):
        L.laplace_shift(t, w, float("nan"))


def test_library_quadrature_on_the_chain_range(L, oracle):
    """On the 200-AO chain's denominator range the variable-projection fit keeps
    improving with n up to the double-precision floor (least squares 4.8e-8 at
    n = 8, ~2e-10 at n = 16), returns n distinct positive nodes and positive
    weights, and its reported error is the oracle's measure of the same grid."""
    from paper_2607_05622_gb300 import workloads as W
    w = W.config2()
    xmin, xmax = oracle.laplace_range(w.eps_occ, w.eps_vir)
    errs = {}
    for n in (4, 8, 16):
        t, wq, err = L.laplace_quadrature(xmin, xmax, n)
        assert t.shape == (n,) and np.all(np.diff(t) > 0) and np.all(wq > 0)
        assert abs(err - oracle.laplace_error(t, wq, xmin, xmax)) <= 1e-12 + 1e-9 * err
        errs[n] = err
    assert errs[8] < 1e-7 and errs[16] < 1e-9 and errs[16] < errs[8] < errs[4]


def test_library_minimax_equioscillates_on_the_chain_range(L, oracle):
    """n = 8 on the 200-AO chain's range: Lawson reweighting plus the exchange
    converge, the relative error alternates in sign at 2n+1 points with equal
    magnitude (the characterisation of the best uniform approximation), and it
    is below the least-squares grid's maximum error."""
    from paper_2607_05622_gb300 import workloads as W
    w = W.config2()
    xmin, xmax = oracle.laplace_range(w.eps_occ, w.eps_vir)
    t, wq, err, conv = L.laplace_minimax(xmin, xmax, 8)
    assert conv
    _, _, els = L.laplace_quadrature(xmin, xmax, 8)
    assert err < els
    x = np.geomspace(xmin, xmax, 200001)
    e = 1.0 - x * (np.exp(-np.outer(x, t)) @ wq)
    sg = np.sign(e)
    runs = np.split(np.abs(e), np.nonzero(sg[1:] != sg[:-1])[0] + 1)
    peaks = np.array([r.max() for r in runs])
    assert len(peaks) == 17
    assert peaks.max() <= peaks.min() * (1 + 1e-3)
