"""Pins of the oracle's MRAB with any number of rates (the extension Sec. 3.3 mentions): for two
rates it is the two-rate macro step bit for bit, with every step ratio 1 it is single-rate
Adams-Bashforth bit for bit, it integrates a coupled chain with right-hand sides of degree <= 2
along the exact solution exactly for three and four rates (only with the right extrapolation
interval at every level), and it reaches third order on a three-component linear ODE whose
components evolve on time scales 30 : 3 : 1."""
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import ab_coefficients, mrab_macro_step, mrab_macro_step_multirate, srab_step


def _linear(A):
    return lambda r, vals: A[r] @ np.array([float(v) for v in vals])


def test_two_rates_equal_the_two_rate_macro_step():
    rng = np.random.default_rng(3)
    A = np.array([[-1.0, 0.4], [0.3, -8.0]])          # component 0 slow, 1 fast
    for sr in (1, 2, 3, 5):
        for m, order in ((3, 3), (4, 3), (4, 4)):
            hs = list(rng.normal(size=m))
            hf = list(rng.normal(size=m))
            s, f = 0.7, -0.2
            H = 0.05
            ys, hists = [s, f], [hs, hf]
            f2, s2, hf2, hs2 = f, s, hf, hs
            for _ in range(4):
                ys, hists = mrab_macro_step_multirate(ys, hists, H, [sr], order, _linear(A))
                f2, s2, hf2, hs2 = mrab_macro_step(f2, s2, hf2, hs2, H, sr, order,
                                                   rhs_fast=lambda ff, ss: A[1] @ np.array([ss, ff]),
                                                   rhs_slow=lambda ss, ff: A[0] @ np.array([ss, ff]))
            assert ys[0] == s2 and ys[1] == f2, (sr, m, order)
            assert hists[0] == hs2 and hists[1] == hf2


def test_unit_ratios_equal_single_rate_ab():
    rng = np.random.default_rng(4)
    A = rng.normal(size=(3, 3)) - 2 * np.eye(3)
    m, H = 3, 0.03
    hist = [list(rng.normal(size=3)) for _ in range(m)]      # hist[k][c]
    y = list(rng.normal(size=3))
    ys, hists = list(y), [[hist[k][c] for k in range(m)] for c in range(3)]
    z, hz = [np.array(v) for v in y], [[np.array(v) for v in hk] for hk in hist]
    rhs_all = lambda yy: [np.array(A[c] @ np.array([float(v) for v in yy])) for c in range(3)]  # noqa: E731
    for _ in range(5):
        ys, hists = mrab_macro_step_multirate(ys, hists, H, [1, 1], 3, _linear(A))
        z, hz = srab_step(z, hz, H, 3, rhs_all)
    for c in range(3):
        assert float(ys[c]) == float(z[c])


def _chain(R):
    """y0' = 1, y1' = y0, y2' = y1, y3' = y1 - y0^2 / 2 from y = 0 at t = 0: y0 = t, y1 = t^2/2,
    y2 = t^3/6, y3 = 0. Along the exact solution every right-hand side is a polynomial of degree
    <= 2 in time; y3's vanishes only if y0 and y1 reach the fastest level exactly."""
    ex = [lambda t: t, lambda t: t * t / 2, lambda t: t ** 3 / 6, lambda t: 0.0][:R]

    def rhs(r, v):
        v = [float(x) for x in v]
        return [1.0, v[0] if R > 1 else 0.0, v[1] if R > 2 else 0.0,
                (v[1] - 0.5 * v[0] * v[0]) if R > 3 else 0.0][r]
    return ex, rhs


@pytest.mark.parametrize("ratios", [[3, 2], [2, 2, 3], [4, 1], [1, 3]])
def test_exact_on_polynomial_chain(ratios):
    """Right-hand sides of degree <= 2 in time along the exact solution: third-order MRAB
    integrates them exactly at every level, which holds only if each level extrapolates the
    slower ones over the right interval (the start of their current step to the evaluation
    time) and takes the faster ones' states at that time."""
    R = len(ratios) + 1
    ex, rhs = _chain(R)
    H, t0, m = 0.1, 0.3, 3
    h = [H]
    for q in ratios:
        h.append(h[-1] / q)
    der = [lambda t: 1.0, lambda t: t, lambda t: t * t / 2, lambda t: 0.0]   # the exact right-hand sides
    hists = [[der[r](t0 - k * h[r]) for k in (2, 1, 0)] for r in range(R)]
    ys = [ex[r](t0) for r in range(R)]
    n = 5
    for _ in range(n):
        ys, hists = mrab_macro_step_multirate(ys, hists, H, ratios, 3, rhs)
    T = t0 + n * H
    for r in range(R):
        assert abs(ys[r] - ex[r](T)) < 1e-13, (r, ys[r], ex[r](T))


def test_third_order_on_three_component_linear_ode():
    A = np.array([[-1.0, 0.3, 0.0], [0.2, -3.0, 0.4], [0.0, 0.5, -30.0]])   # slow, medium, fast
    y0 = np.array([1.0, 0.5, -0.3])
    ratios = [3, 4]
    T = 1.0
    ex = lambda t: scipy.linalg.expm(A * t) @ y0  # noqa: E731
    errs = []
    for n in (100, 200, 400):
        H = T / n
        h = [H, H / 3, H / 12]
        hists = [[float(A[r] @ ex(-k * h[r])) for k in (2, 1, 0)] for r in range(3)]
        ys = list(y0)
        for _ in range(n):
            ys, hists = mrab_macro_step_multirate(ys, hists, H, ratios, 3, _linear(A))
        errs.append(float(np.linalg.norm(np.array(ys, dtype=float) - ex(T))))
    eocs = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert all(2.85 < e < 3.2 for e in eocs), eocs


def test_extrapolation_interval_matters():
    """Planted mistake: extrapolating the slower components over the whole slow step instead of
    up to the evaluation time breaks exactness on the chain (the check is not vacuous)."""
    ratios = [3, 2]
    ex, rhs = _chain(3)
    H, t0 = 0.1, 0.3
    h = [H, H / 3, H / 6]
    der = [lambda t: 1.0, lambda t: t, lambda t: t * t / 2]
    hists = [[der[r](t0 - k * h[r]) for k in (2, 1, 0)] for r in range(3)]
    ys = [ex[r](t0) for r in range(3)]
    nodes = np.arange(-2, 1.0)
    # a wrong medium component: its right-hand side at every micro step sees y0 extrapolated to
    # the end of the slow step
    wrong = lambda r, v: rhs(r, [v[0] + (ab_coefficients(nodes, 0, 1, 3) @ np.array(hists[0]) * H  # noqa: E731
                                         if r > 0 else 0.0)] + list(v[1:]))
    ys2, _ = mrab_macro_step_multirate(list(ys), [list(x) for x in hists], H, ratios, 3, wrong)
    ys1, _ = mrab_macro_step_multirate(list(ys), [list(x) for x in hists], H, ratios, 3, rhs)
    assert abs(ys1[1] - ex[1](t0 + H)) < 1e-13
    assert abs(ys2[1] - ex[1](t0 + H)) > 1e-6
