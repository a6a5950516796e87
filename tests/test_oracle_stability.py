"""Step-matrix stability (Sec. 4.3) of the oracle's MRAB step, pinned to theory.

On a uniform flow the linearised semi-discretisation is the periodic SBP operator (spectral
radius 1.3722 / dx on the imaginary axis, Sec. 4.4) times the wave speeds, so single-rate AB3
at the fast mesh's micro step is stable up to (AB3 imaginary-axis bound) / 1.3722 of the
Sec. 4.1 step estimate. The AB3 bound is computed here from the AB3 weights by the boundary
locus. MRAB with step ratio 2 on the vortex geometry, where the fine patch sets the limit,
must reach that bound (the paper's ~100 % efficiency below the spacing ratio).
"""
import ctypes
import math

import numpy as np

import oracle
import workloads as W
from conftest import golden
from oracle import OracleSystem, ab_coefficients, rk4_step


def _arnoldi_radius(matvec, n, kdim=60, seed=0):
    V = np.zeros((kdim + 1, n))
    Hm = np.zeros((kdim + 1, kdim))
    v = np.random.default_rng(seed).standard_normal(n)
    V[0] = v / np.linalg.norm(v)
    for j in range(kdim):
        w = matvec(V[j])
        for _ in range(2):
            for i in range(j + 1):
                c = V[i] @ w
                Hm[i, j] += c
                w -= c * V[i]
        Hm[j + 1, j] = np.linalg.norm(w)
        V[j + 1] = w / Hm[j + 1, j]
    return float(np.abs(np.linalg.eigvals(Hm[:kdim, :kdim])).max())


def _ab3_imaginary_bound():
    """Largest y with AB3 stable at lambda dt = i y: boundary locus z = e^{i theta},
    lambda dt = (z^3 - z^2) / sum_k alpha_k z^k, first crossing of the imaginary axis."""
    a = ab_coefficients(np.array([-2.0, -1.0, 0.0]), 0.0, 1.0, 3)  # oldest first
    th = np.linspace(0.05, np.pi, 200001)  # away from the tangency at the origin
    z = np.exp(1j * th)
    mu = (z ** 3 - z ** 2) / (a[0] + a[1] * z + a[2] * z ** 2)
    s = np.sign(mu.real)
    idx = np.nonzero(s[1:] != s[:-1])[0]
    return float(np.min(np.abs(mu.imag[idx])))


def test_arnoldi_radius_finds_outlier():
    rng = np.random.default_rng(1)
    n = 300
    Q = np.linalg.qr(rng.standard_normal((n, n)))[0]
    ev = np.concatenate([[1.3], 0.9 * np.exp(2j * np.pi * rng.uniform(size=n - 1)).real])
    A = Q @ np.diag(ev) @ Q.T
    assert abs(_arnoldi_radius(lambda v: A @ v, n) - 1.3) < 1e-8


def test_ab3_imaginary_axis_bound():
    assert abs(_ab3_imaginary_bound() - 0.7236) < 1e-3


def test_mrab_uniform_flow_stability_limit_matches_theory():
    wl = W.vortex_box_in_box(seed=51, n_bg=32, n_fine=21)
    o = OracleSystem(wl)
    qinf = np.asarray(wl["params"]["qinf"])
    uni = [np.broadcast_to(qinf[:, None, None], (4, m["n"][1], m["n"][0])).copy() for m in wl["meshes"]]
    m = wl["params"]["hist_len"]
    sr = wl["params"]["step_ratio"]
    F, Sl = o.fast, o.slow
    act = [o.iblank[k] != 0 for k in range(2)]
    spectral = float(golden("periodic_spectrum.txt")[0][0])
    f_star = _ab3_imaginary_bound() / spectral
    dt_fast = o.dt_mesh(F, uni[F])

    def pack(hs):
        return np.concatenate([x for k, (q, h) in enumerate(hs)
                               for x in (q[:, act[k]].reshape(-1), h[:, :, act[k]].reshape(-1))])

    def unpack(vec, like):
        out, o_ = [], 0
        for k, (q, h) in enumerate(like):
            q, h = q.copy(), h.copy()
            n = int(act[k].sum()) * 4
            q[:, act[k]] = vec[o_:o_ + n].reshape(4, -1)
            o_ += n
            nh = n * (m - 1)
            h[:, :, act[k]] = vec[o_:o_ + nh].reshape(m - 1, 4, -1)
            o_ += nh
            out.append((q, h))
        return out

    def rho(H):
        qs, hf, hs = o.bootstrap(uni, H)
        base = [None, None]
        base[F] = (qs[F], np.stack(hf[:-1]))
        base[Sl] = (qs[Sl], np.stack(hs[:-1]))

        def step(state):
            q = [state[0][0], state[1][0]]
            hist_f = list(state[F][1]) + [o.coupled_rhs(F, q[F], q[Sl])]
            hist_s = list(state[Sl][1]) + [o.coupled_rhs(Sl, q[Sl], q[F])]
            qn, a, b = o.mrab(q, hist_f, hist_s, H, 1)
            out = [None, None]
            out[F] = (qn[F], np.stack(a[:-1]))
            out[Sl] = (qn[Sl], np.stack(b[:-1]))
            return pack(out)

        b0 = pack(base)
        y0 = step(base)

        def mv(v):
            nv = np.linalg.norm(v)
            return (step(unpack(b0 + 1e-7 * v / nv, base)) - y0) * (nv / 1e-7)

        return _arnoldi_radius(mv, b0.size)

    assert rho(0.95 * f_star * sr * dt_fast) <= 1.0 + 1e-3
    assert rho(1.05 * f_star * sr * dt_fast) > 1.0 + 1e-3


def _e2_case():
    g = {r[0]: float(r[1]) for r in golden("rk4_advection_stability.txt")}
    n = int(g["n_points"])
    dx = g["length"] / n  # periodic: the point at x = length is the point at x = 0
    L = oracle.lib()
    cls = np.zeros(n, np.int8)  # periodic line: the interior row everywhere
    D = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        out = np.zeros(n)
        L.orc_apply_d1(n, ctypes.c_void_p(cls.ctypes.data), ctypes.c_void_p(e.ctypes.data),
                       ctypes.c_void_p(out.ctypes.data))
        D[:, k] = out
    return g, n, dx, D


def _step_matrix_radius(step, base, eps=1e-7):
    """The step matrix of Sec. 4.3 built column by column as the paper does (perturb one entry
    of the integrator state by eps, eq. (sm_form)), and its spectral radius from a dense
    eigen-decomposition (in place of SLEPc's Krylov-Schur solver)."""
    n = base.size
    y0 = step(base)
    G = np.empty((n, n))
    for j in range(n):
        ph = base.copy()
        ph[j] += eps
        G[:, j] = (step(ph) - y0) / eps
    return float(np.abs(np.linalg.eigvals(G)).max())


def test_rk4_advection_step_matrix_reproduces_sec44():
    """Sec. 4.4: RK4 on 1D periodic advection (61 points on [0, 1.01666]); the step-matrix
    procedure finds the largest stable step between 0.03 and 0.035, consistent with the
    estimate (RK4 imaginary-axis bound) / (lambda_max dx) * dx. Here the bound is the exact
    2 sqrt(2) of the RK4 amplification polynomial and lambda_max is this grid's own largest
    eigenvalue of D, so the bisection must land on that closed form."""
    g, n, dx, D = _e2_case()
    x = np.arange(n) * dx
    base = np.sin(2.0 * math.pi * x / g["length"]) + 0.3 * np.cos(6.0 * math.pi * x / g["length"])

    def radius(dt):
        return _step_matrix_radius(lambda u: rk4_step([u], dt, lambda v: [-(D @ v[0]) / dx])[0], base)

    assert radius(g["dt_stable"]) <= 1.0 + 1e-6
    assert radius(g["dt_unstable"]) > 1.0 + 1e-6
    lo, hi = g["dt_stable"], g["dt_unstable"]
    while hi - lo > 1e-7:
        mid = 0.5 * (lo + hi)
        if radius(mid) <= 1.0 + 1e-6:
            lo = mid
        else:
            hi = mid
    lam_dx = float(np.abs(np.linalg.eigvals(D)).max())
    # 61 discrete wave numbers sample the continuous maximum 1.3722 (1.3705 here)
    assert abs(lam_dx - float(golden("periodic_spectrum.txt")[0][0])) < 2e-3
    closed = 2.0 * math.sqrt(2.0) / lam_dx * dx
    assert abs(lo - closed) < 2e-6 * closed, (lo, closed)
    # the paper's estimate from its approximate imaginary-axis bound lies in the same bracket
    est = g["rk4_imag_bound_approx"] / float(golden("periodic_spectrum.txt")[0][0]) * dx
    assert abs(est - g["dt_estimate"]) < 2e-5
    assert g["dt_stable"] < est < lo < g["dt_unstable"]
