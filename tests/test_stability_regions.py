"""Stability regions of the scalar test equation (Sec. 3.2 and the appendix on plotting stability
regions) as the corner-penalty study uses them, pinned to closed forms.

* RK4: |R(x)| = 1 on the negative real axis at the real root of x^3 + 4x^2 + 12x + 24 = 0 and on
  the imaginary axis at y = 2 sqrt(2) (|R(iy)|^2 = 1 - y^6/72 + y^8/576).
* AB3: the library's weights are (5, -16, 23)/12; the real interval is (-6/11, 0) (the boundary
  locus at zeta = -1); the imaginary bound is the boundary locus's first crossing of the axis.
* AB34 (min-norm weights on four nodes, Sec. 3.2 eq. (ext_ab)): reaches further along the
  negative real axis than AB3 and less far along the imaginary axis, as the paper states; its
  real bound is the boundary locus's first crossing of the negative real axis (from a complex pair
  of unit roots: zeta = -1 gives a crossing further out).
* The amplification bound 2^(1/100) is the appendix's marching test (y from 1, 100 steps, fail
  when |y| passes 2): for RK4, whose iterates are R(z)^n, the two decide alike on every ray.
* The mirror split of an operator gives the spectrum of the full operator.
"""
import math

import numpy as np
import pytest

import workloads as W
from paper_1805_06607_gb300 import HostTables
from paper_1805_06607_gb300.stability import (GROWTH_100, ab_amplification, largest_stable_step, mirror_blocks,
                                              rk4_amplification)


def _plan(hist_len):
    h = HostTables(W.corner_box_in_box(1.0, hist_len=hist_len))
    try:
        return h.plan()[0]
    finally:
        h.close()


def _locus(ab, theta):
    """Boundary locus z(theta) of an AB step (weights oldest first): zeta = e^{i theta} solves
    zeta^m - zeta^(m-1) = z sum_j ab[j] zeta^j."""
    zeta = np.exp(1j * np.asarray(theta))
    m = len(ab)
    den = sum(ab[j] * zeta ** j for j in range(m))
    return (zeta ** m - zeta ** (m - 1)) / den


def _imag_bound(ab):
    th = np.linspace(0.05, np.pi, 200001)
    z = _locus(ab, th)
    s = np.sign(z.real)
    idx = np.nonzero(s[1:] != s[:-1])[0]
    return float(np.min(np.abs(z.imag[idx])))


def _real_bound(ab):
    """|z| of the boundary locus's first crossing of the negative real axis (a crossing may come
    from a complex pair of roots on the unit circle, not only from zeta = -1)."""
    th = np.linspace(0.05, np.pi, 400001)
    z = _locus(ab, th)
    im = np.where(np.abs(z.imag) < 1e-12, 0.0, z.imag)
    idx = np.nonzero((np.sign(im[1:]) != np.sign(im[:-1])) | (im[1:] == 0.0))[0]
    xs = []
    for i in idx:
        a, b = z[i], z[i + 1]
        t = 0.0 if b.imag == a.imag else a.imag / (a.imag - b.imag)
        xs.append(a.real + t * (b.real - a.real))
    xs = [x for x in xs if x < 0.0]
    return float(min(-x for x in xs))


def test_rk4_real_and_imaginary_bounds():
    x = np.roots([1.0, 4.0, 12.0, 24.0])
    xr = float(x[np.abs(x.imag) < 1e-12].real[0])
    dt, lim = largest_stable_step(rk4_amplification, [-1.0], 5.0, growth=1.0 + 1e-13, rel_tol=1e-12)
    assert abs(dt - (-xr)) < 1e-9 and lim == -1.0
    dt, _ = largest_stable_step(rk4_amplification, [1j], 5.0, growth=1.0 + 1e-13, rel_tol=1e-12)
    assert abs(dt - 2.0 * math.sqrt(2.0)) < 1e-6


def test_ab3_weights_and_bounds():
    ab = _plan(3)
    assert np.allclose(ab, np.array([5.0, -16.0, 23.0]) / 12.0, rtol=0, atol=1e-14)
    dt, _ = largest_stable_step(lambda z: ab_amplification(ab, z), [-1.0], 2.0, growth=1.0 + 1e-12, rel_tol=1e-12)
    assert abs(dt - 6.0 / 11.0) < 1e-9
    assert abs(float(_locus(ab, np.pi).real) + 6.0 / 11.0) < 1e-14
    yb = _imag_bound(ab)
    dt, _ = largest_stable_step(lambda z: ab_amplification(ab, z), [1j], 2.0, growth=1.0 + 1e-9, rel_tol=1e-10)
    assert abs(dt - yb) < 1e-4 and abs(yb - 0.7236) < 1e-3


def test_ab34_reaches_further_along_the_negative_real_axis():
    a3, a4 = _plan(3), _plan(4)
    assert a4.size == 4 and abs(a4.sum() - 1.0) < 1e-14
    real = {}
    for name, ab in (("ab3", a3), ("ab34", a4)):
        real[name], _ = largest_stable_step(lambda z: ab_amplification(ab, z), [-1.0], 4.0, growth=1.0 + 1e-12,
                                            rel_tol=1e-12)
    assert abs(real["ab34"] - _real_bound(a4)) < 1e-6
    assert abs(real["ab3"] - _real_bound(a3)) < 1e-6
    assert real["ab34"] > 1.2 * real["ab3"]
    assert _imag_bound(a4) < _imag_bound(a3)


@pytest.mark.parametrize("theta", [0.5 * math.pi + 0.05, 0.75 * math.pi, math.pi, 1.2 * math.pi])
def test_growth_bound_is_the_marching_test(theta):
    """Ray from the point -0.3 (inside every region used): the largest radius the appendix's marching
    test accepts equals the one the amplification bound accepts."""
    c = -0.3
    d = np.exp(1j * theta)

    def marches(r):
        z = c + r * d
        y = 1.0 + 0.0j
        R = 1.0 + z * (1.0 + z * (0.5 + z * (1.0 / 6.0 + z / 24.0)))
        for _ in range(100):
            y *= R
            if abs(y) > 2.0:
                return False
        return True

    def bound(ok):
        lo, hi = 0.0, 8.0
        while hi - lo > 1e-12:
            mid = 0.5 * (lo + hi)
            lo, hi = (mid, hi) if ok(mid) else (lo, mid)
        return lo

    r_march = bound(marches)
    r_amp = bound(lambda r: rk4_amplification(c + r * d)[0] <= GROWTH_100)
    assert abs(r_march - r_amp) < 1e-9


def test_limiting_eigenvalue_and_non_star_region():
    ab = _plan(3)
    lam = np.array([-1.0, 20j, -0.1 + 1j])
    dt, lim = largest_stable_step(lambda z: ab_amplification(ab, z), lam, 1.0, growth=1.0 + 1e-9)
    assert lim == 20j and abs(dt - _imag_bound(ab) / 20.0) < 1e-5
    # a region with a gap: stable below 1, unstable on [1, 2), stable again above; the scan finds 1
    amp = lambda z: np.where((np.abs(z) >= 1.0) & (np.abs(z) < 2.0), 2.0, 0.5)  # noqa: E731
    dt, _ = largest_stable_step(amp, [1.0], 4.0, growth=1.0)
    assert abs(dt - 1.0) < 1e-6


def test_mirror_blocks_keep_the_spectrum():
    rng = np.random.default_rng(3)
    n = 41
    perm = np.arange(n)
    perm[:20], perm[20:40] = np.arange(20, 40), np.arange(20)  # pairs (a, a + 20); 40 is fixed
    sign = np.ones(n)
    sign[[5, 25]] = -1.0
    B = rng.standard_normal((n, n))
    R = np.zeros((n, n))
    R[perm, np.arange(n)] = sign
    A = 0.5 * (B + R @ B @ R.T)  # commutes with R
    blocks = mirror_blocks(A, perm, sign)
    assert blocks is not None and sum(b.shape[0] for b in blocks) == n
    got = np.sort_complex(np.concatenate([np.linalg.eigvals(b) for b in blocks]))
    want = np.sort_complex(np.linalg.eigvals(A))
    assert np.abs(got - want).max() < 1e-10
    assert mirror_blocks(B, perm, sign) is None
