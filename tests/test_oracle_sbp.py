"""Pins of the oracle's SBP 4-2 first derivative (Sec. 2.1, App. C.1) against exact
mathematics: the summation-by-parts identity in rational arithmetic, polynomial accuracy,
and the periodic spectrum the paper quotes in Sec. 4.4."""
import ctypes
from fractions import Fraction

import numpy as np
import pytest

import oracle
from conftest import golden

NORM = [Fraction(17, 48), Fraction(59, 48), Fraction(43, 48), Fraction(49, 48)]


def _classes(n, left=True, right=True, per=False):
    c = np.zeros(n, np.int8)
    if not per:
        for r in range(4):
            c[r] = 1 + r
            c[n - 1 - r] = 5 + r
    return c


def _dmatrix(n, cls):
    L = oracle.lib()
    D = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        out = np.zeros(n)
        L.orc_apply_d1(n, ctypes.c_void_p(cls.ctypes.data), ctypes.c_void_p(e.ctypes.data),
                       ctypes.c_void_p(out.ctypes.data))
        D[:, k] = out
    return D


@pytest.mark.parametrize("n", [8, 9, 12, 17])
def test_sbp_identity_exact(n):
    D = _dmatrix(n, _classes(n))
    Dq = [[Fraction(v).limit_denominator(200) for v in row] for row in D]
    # the rational reading reproduces the floating coefficients to the last bit or so
    assert max(abs(float(Dq[i][j]) - D[i][j]) for i in range(n) for j in range(n)) < 1e-15
    h = NORM + [Fraction(1)] * (n - 8) + NORM[::-1]
    for i in range(n):
        for j in range(n):
            s = h[i] * Dq[i][j] + Dq[j][i] * h[j]
            b = Fraction(-1) if (i == j == 0) else Fraction(1) if (i == j == n - 1) else Fraction(0)
            assert s == b, (i, j, s)


def test_accuracy_orders():
    n = 16
    D = _dmatrix(n, _classes(n))
    x = np.arange(n, dtype=np.float64) - 3.3
    for k in range(3):  # exact for x^0..x^2 on every row
        assert np.allclose(D @ x ** k, k * x ** (k - 1) if k else 0 * x, atol=1e-10)
    inner = slice(4, n - 4)
    for k in range(3, 5):  # exact for x^3, x^4 on interior rows only
        err = D @ x ** k - k * x ** (k - 1)
        assert np.allclose(err[inner], 0.0, atol=1e-9)
        assert np.abs(err[:4]).max() > 1e-6


def test_periodic_spectrum_matches_paper():
    n = 256
    D = _dmatrix(n, _classes(n, per=True))
    lam = np.abs(np.linalg.eigvals(D)).max()
    paper = float(golden("periodic_spectrum.txt")[0][0])
    assert abs(lam - paper) < 5e-5
    # the periodic operator is exactly antisymmetric
    assert np.abs(D + D.T).max() < 1e-15


def test_hole_segment_closures():
    """A segment next to a hole uses the same closure rows as a mesh end (reading of Sec. 2.2)."""
    n = 30
    act = np.ones((1, n), np.int8)
    act[0, 10:14] = 0
    ci = np.zeros((1, n), np.int8)
    cj = np.zeros((1, n), np.int8)
    L = oracle.lib()
    L.orc_classes2d(n, 1, 1, 1, ctypes.c_void_p(act.ctypes.data), ctypes.c_void_p(ci.ctypes.data),
                    ctypes.c_void_p(cj.ctypes.data))
    c = ci[0]
    assert list(c[10:14]) == [15] * 4
    assert list(c[14:18]) == [1, 2, 3, 4]
    assert list(c[6:10]) == [8, 7, 6, 5]
    # a run shorter than 8 points is turned into a hole
    act = np.ones((1, n), np.int8)
    act[0, 3] = 0
    act[0, 9] = 0
    L.orc_classes2d(n, 1, 1, 1, ctypes.c_void_p(act.ctypes.data), ctypes.c_void_p(ci.ctypes.data),
                    ctypes.c_void_p(cj.ctypes.data))
    assert act[0, 3:10].sum() == 0 and act[0, 10:].all() and act[0, :3].all()
