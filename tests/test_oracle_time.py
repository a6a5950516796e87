"""Pins of the oracle's time integrators: textbook Adams-Bashforth weights (Sec. 3.1), the
minimum-norm property of the extended-history weights (Sec. 3.2), the AB3 real stability
bound 6/11, the identity MRAB(SR=1) == single-rate AB (Sec. 5.2), MRAB design order on a
two-component linear ODE (Sec. 3.3), and the performance model of Sec. 6.1."""
import math

import numpy as np
import pytest
import scipy.linalg

import workloads as W
from conftest import golden
from oracle import (OracleSystem, ab_coefficients, mrab_macro_step, mrab_macro_step_slowest_first,
                    mrab_macro_step_var, rk3_heun_step, rk4_step, srab_step)


def test_ab_textbook():
    n3 = np.arange(-2, 1.0)
    assert np.allclose(ab_coefficients(n3, 0, 1, 3), np.array([5, -16, 23]) / 12, atol=1e-15)
    n4 = np.arange(-3, 1.0)
    assert np.allclose(ab_coefficients(n4, 0, 1, 4), np.array([-9, 37, -59, 55]) / 24, atol=1e-14)
    # scale invariance: nodes and interval in another unit
    assert np.allclose(ab_coefficients(0.1 * n3, 0, 0.1, 3), 0.1 * np.array([5, -16, 23]) / 12, atol=1e-15)


def test_extended_history_min_norm():
    nodes = np.arange(-3, 1.0)
    a = ab_coefficients(nodes, 0, 1, 3)
    # moment conditions hold
    for i in range(3):
        assert abs(np.sum(a * nodes ** i) - 1.0 / (i + 1)) < 1e-14
    # minimum norm <=> orthogonal to the null space of V^T, spanned here by the third
    # difference (-1, 3, -3, 1) (which annihilates quadratics)
    z = np.array([-1.0, 3.0, -3.0, 1.0])
    assert abs(a @ z) < 1e-14
    assert abs(np.sum(z * nodes ** 2)) < 1e-14


def _max_root(alpha, z):
    # y_{n+1} = y_n + z sum_k alpha_k y_{n-m+1+k}; characteristic polynomial in zeta
    m = len(alpha)
    c = np.zeros(m + 1)
    c[0] = 1.0
    c[1] = -1.0
    for k in range(m):
        c[m - k] -= z * alpha[k]
    return np.abs(np.roots(c)).max()


def test_ab3_real_stability_bound():
    a = ab_coefficients(np.arange(-2, 1.0), 0, 1, 3)
    assert abs(_max_root(a, -6.0 / 11.0) - 1.0) < 1e-9
    assert _max_root(a, -0.54) < 1.0
    assert _max_root(a, -0.55) > 1.0
    # extended history stretches the negative-real bound (Sec. 3.2)
    a34 = ab_coefficients(np.arange(-3, 1.0), 0, 1, 3)
    assert _max_root(a34, -0.85) < 1.0


def test_mrab_sr1_equals_srab():
    wl = W.vortex_box_in_box(seed=4, n_bg=32, n_fine=21, step_ratio=1)
    S = OracleSystem(wl)
    H = S.macro_step_size(wl["q0"])
    y, hf, hs = S.bootstrap(wl["q0"], H)
    out, _, _ = S.mrab(y, hf, hs, H, 3)
    hist = [[hs[k], hf[k]] for k in range(3)]
    z = [y[0], y[1]]
    for _ in range(3):
        z, hist = srab_step(z, hist, H, 3, S.rhs_all)
    assert np.array_equal(out[0], z[0]) and np.array_equal(out[1], z[1])


def test_mrab_order_linear_ode():
    lf, ls, c = 10.0, 1.0, 0.5
    A = np.array([[-lf, c], [c, -ls]])
    y0 = np.array([1.0, 0.5])
    T = 1.0
    errs = []
    for n in (80, 160, 320):
        H = T / n
        sr = 3
        h = H / sr
        # exact histories at t = 0: fast at -2h,-h,0, slow at -2H,-H,0
        ex = lambda t: scipy.linalg.expm(A * t) @ y0
        hf = [A[0] @ ex(-k * h) for k in (2, 1, 0)]
        hs = [A[1] @ ex(-k * H) for k in (2, 1, 0)]
        f, s = y0[0], y0[1]
        for _ in range(n):
            f, s, hf, hs = mrab_macro_step(f, s, hf, hs, H, sr, 3,
                                           rhs_fast=lambda ff, ss: A[0, 0] * ff + A[0, 1] * ss,
                                           rhs_slow=lambda ss, ff: A[1, 0] * ff + A[1, 1] * ss)
        e = ex(T)
        errs.append(math.hypot(f - e[0], s - e[1]))
    eocs = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert all(2.9 < e < 3.15 for e in eocs), eocs


@pytest.mark.parametrize("reextrapolate", [False, True])
def test_slowest_first_sr1_equals_srab(reextrapolate):
    """At step ratio 1 the extrapolated fast state is the fast update itself, so both
    slowest-first variants reduce to single-rate AB, bit for bit."""
    wl = W.vortex_box_in_box(seed=4, n_bg=32, n_fine=21, step_ratio=1)
    S = OracleSystem(wl)
    H = S.macro_step_size(wl["q0"])
    y, hf, hs = S.bootstrap(wl["q0"], H)
    scheme = "slowest_first_reextrapolate" if reextrapolate else "slowest_first"
    out, _, _ = S.mrab(y, hf, hs, H, 3, scheme=scheme)
    hist = [[hs[k], hf[k]] for k in range(3)]
    z = [y[0], y[1]]
    for _ in range(3):
        z, hist = srab_step(z, hist, H, 3, S.rhs_all)
    assert np.array_equal(out[0], z[0]) and np.array_equal(out[1], z[1])


@pytest.mark.parametrize("scheme", ["fastest_first", "slowest_first", "slowest_first_reextrapolate"])
def test_mrab_variants_exact_on_polynomial_chain(scheme):
    """A coupled chain whose right-hand sides are polynomials of degree <= 2 in time along the
    exact solution: s1' = 1, s2' = s1, s4' = s2, f' = s2, s3' = f - s4, from zero (s1 = t,
    s2 = t^2/2, s4 = f = t^3/6, s3 = 0). Third-order MRAB integrates it exactly in every
    variant, but only with the right extrapolation weights: the fast micro steps need the slow
    extrapolant (or re-extrapolant) of s2 at the micro times, and s3 stays 0 only if the
    extrapolated fast state at t+H (slowest-first) or the fast state itself is exact."""
    sr, H = 3, 0.1
    h = H / sr
    ex_s = lambda t: np.array([t, t * t / 2, 0.0, t ** 3 / 6])  # noqa: E731
    ex_f = lambda t: np.array([t ** 3 / 6])  # noqa: E731
    rhs_s = lambda ss, ff: np.array([1.0, ss[0], ff[0] - ss[3], ss[1]])  # noqa: E731
    rhs_f = lambda ff, ss: np.array([ss[1]])  # noqa: E731
    t0 = 0.4
    hf = [rhs_f(ex_f(t0 - k * h), ex_s(t0 - k * h)) for k in (2, 1, 0)]
    hs = [rhs_s(ex_s(t0 - k * H), ex_f(t0 - k * H)) for k in (2, 1, 0)]
    f, s = ex_f(t0), ex_s(t0)
    n = 7
    for _ in range(n):
        if scheme == "fastest_first":
            f, s, hf, hs = mrab_macro_step(f, s, hf, hs, H, sr, 3, rhs_fast=rhs_f, rhs_slow=rhs_s)
        else:
            f, s, hf, hs = mrab_macro_step_slowest_first(f, s, hf, hs, H, sr, 3, rhs_fast=rhs_f, rhs_slow=rhs_s,
                                                         reextrapolate=scheme.endswith("reextrapolate"))
    T = t0 + n * H
    assert np.abs(f - ex_f(T)).max() < 1e-13
    assert np.abs(s - ex_s(T)).max() < 1e-13


def _chain():
    ex_s = lambda t: np.array([t, t * t / 2, 0.0, t ** 3 / 6])  # noqa: E731
    ex_f = lambda t: np.array([t ** 3 / 6])  # noqa: E731
    rhs_s = lambda ss, ff: np.array([1.0, ss[0], ff[0] - ss[3], ss[1]])  # noqa: E731
    rhs_f = lambda ff, ss: np.array([ss[1]])  # noqa: E731
    return ex_s, ex_f, rhs_s, rhs_f


def test_variable_macro_step_exact_on_polynomial_chain():
    """Changing H between macro steps (Sec. 3.3 Step 1): with the weights solved on the actual
    node times, third-order MRAB stays exact on the polynomial chain for any step sequence."""
    ex_s, ex_f, rhs_s, rhs_f = _chain()
    sr, H0, t = 3, 0.1, 0.4
    h0 = H0 / sr
    tf = np.array([t - 2 * h0, t - h0, t])
    ts = np.array([t - 2 * H0, t - H0, t])
    hf = [rhs_f(ex_f(x), ex_s(x)) for x in tf]
    hs = [rhs_s(ex_s(x), ex_f(x)) for x in ts]
    f, s = ex_f(t), ex_s(t)
    for H in (0.1, 0.07, 0.07, 0.13, 0.05, 0.1, 0.1):
        f, s, hf, tf, hs, ts = mrab_macro_step_var(f, s, hf, tf, hs, ts, t, H, sr, 3, rhs_fast=rhs_f, rhs_slow=rhs_s)
        t += H
    assert np.abs(f - ex_f(t)).max() < 1e-13
    assert np.abs(s - ex_s(t)).max() < 1e-13


def test_variable_macro_step_uniform_equals_fixed():
    """With a constant H the variable-step weights are the fixed-step ones: the same states to
    rounding of the node offsets."""
    wl = W.vortex_box_in_box(seed=5, n_bg=32, n_fine=21)
    S = OracleSystem(wl)
    H = S.macro_step_size(wl["q0"])
    y, hf, hs = S.bootstrap(wl["q0"], H)
    a, _, _ = S.mrab(y, hf, hs, H, 3)
    b = S.mrab_var(y, hf, hs, H, [H, H, H])
    for k in range(2):
        assert np.abs(a[k] - b[k]).max() <= 1e-13 * np.abs(a[k]).max()


def test_variable_macro_step_order_linear_ode():
    """Third order on the two-component linear ODE with macro steps alternating between H and
    0.6 H."""
    lf, ls, c = 10.0, 1.0, 0.5
    A = np.array([[-lf, c], [c, -ls]])
    y0 = np.array([1.0, 0.5])
    errs = []
    for n in (80, 160, 320):
        H = 1.0 / n
        sr = 3
        h = H / sr
        ex = lambda t: scipy.linalg.expm(A * t) @ y0  # noqa: E731
        tf = np.array([-2 * h, -h, 0.0])
        ts = np.array([-2 * H, -H, 0.0])
        hf = [A[0] @ ex(x) for x in tf]
        hs = [A[1] @ ex(x) for x in ts]
        f, s, t = y0[0], y0[1], 0.0
        for i in range(n):
            Hi = H if i % 2 == 0 else 0.6 * H
            f, s, hf, tf, hs, ts = mrab_macro_step_var(
                f, s, hf, tf, hs, ts, t, Hi, sr, 3, rhs_fast=lambda ff, ss: A[0, 0] * ff + A[0, 1] * ss,
                rhs_slow=lambda ss, ff: A[1, 0] * ff + A[1, 1] * ss)
            t += Hi
        e = ex(t)
        errs.append(math.hypot(f - e[0], s - e[1]))
    eocs = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert all(2.85 < e < 3.2 for e in eocs), eocs


@pytest.mark.parametrize("reextrapolate", [False, True])
def test_slowest_first_order_linear_ode(reextrapolate):
    lf, ls, c = 10.0, 1.0, 0.5
    A = np.array([[-lf, c], [c, -ls]])
    y0 = np.array([1.0, 0.5])
    T = 1.0
    errs = []
    for n in (80, 160, 320):
        H = T / n
        sr = 3
        h = H / sr
        ex = lambda t: scipy.linalg.expm(A * t) @ y0  # noqa: E731
        hf = [A[0] @ ex(-k * h) for k in (2, 1, 0)]
        hs = [A[1] @ ex(-k * H) for k in (2, 1, 0)]
        f, s = y0[0], y0[1]
        for _ in range(n):
            f, s, hf, hs = mrab_macro_step_slowest_first(
                f, s, hf, hs, H, sr, 3, rhs_fast=lambda ff, ss: A[0, 0] * ff + A[0, 1] * ss,
                rhs_slow=lambda ss, ff: A[1, 0] * ff + A[1, 1] * ss, reextrapolate=reextrapolate)
        e = ex(T)
        errs.append(math.hypot(f - e[0], s - e[1]))
    eocs = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert all(2.85 < e < 3.2 for e in eocs), eocs


def test_rk3_order():
    lam = -1.3
    errs = []
    for n in (20, 40):
        y = [np.array(1.0)]
        for _ in range(n):
            y, _ = rk3_heun_step(y, 1.0 / n, lambda z: [lam * z[0]])
        errs.append(abs(float(y[0]) - math.exp(lam)))
    assert 2.9 < math.log2(errs[0] / errs[1]) < 3.1


def test_rk4_order():
    lam = -1.3
    errs = []
    for n in (10, 20):
        y = [np.array(1.0)]
        for _ in range(n):
            y = rk4_step(y, 1.0 / n, lambda z: [lam * z[0]])
        errs.append(abs(float(y[0]) - math.exp(lam)))
    assert 3.9 < math.log2(errs[0] / errs[1]) < 4.1


def test_rk4_amplification_is_the_degree_4_taylor_polynomial():
    """One step on y' = z y multiplies y by 1 + z + z^2/2 + z^3/6 + z^4/24 (complex z): every
    stage weight and node enters a different power."""
    for z in (0.3 + 0.0j, -1.7 + 0.4j, 2.1j, -0.5 - 2.6j):
        y = rk4_step([np.array(1.0 + 0.0j)], 1.0, lambda v, z=z: [z * v[0]])
        assert abs(complex(y[0]) - (1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24)) < 1e-14


def test_performance_model_rk4_total():
    g = {r[0]: int(r[1]) for r in golden("perf_model.txt")}
    # eq. (perf_RK4) with t = dt_RK4
    assert 4 * (g["n_fast"] + g["n_slow"]) == g["rk4_total"]
