"""Host logic of the library's step-matrix stability tool (Sec. 4.3), without a GPU: the
Krylov spectral-radius estimate and the bisection on the step reproduce the paper's Sec. 4.4
validation (RK4 on 1D periodic advection, 61 points on [0, 1.01666]: largest stable step
between 0.03 and 0.035) when the step is applied matrix-free by finite differences, as the
library applies it to its GPU steps."""
import ctypes
import math

import numpy as np

import oracle
from conftest import build_library, golden


def _advection():
    g = {r[0]: float(r[1]) for r in golden("rk4_advection_stability.txt")}
    n = int(g["n_points"])
    dx = g["length"] / n
    L = oracle.lib()
    cls = np.zeros(n, np.int8)
    D = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        out = np.zeros(n)
        L.orc_apply_d1(n, ctypes.c_void_p(cls.ctypes.data), ctypes.c_void_p(e.ctypes.data),
                       ctypes.c_void_p(out.ctypes.data))
        D[:, k] = out
    return g, n, dx, D


def test_krylov_bisection_reproduces_sec44_bracket():
    build_library()
    from paper_1805_06607_gb300.stability import arnoldi_radius, bisect_stable_step
    g, n, dx, D = _advection()
    base = np.cos(2.0 * math.pi * np.arange(n) / n)

    def radius(dt):
        def step(u):
            return oracle.rk4_step([u], dt, lambda v: [-(D @ v[0]) / dx])[0]

        y0 = step(base)
        eps = 1e-7

        def mv(v):
            nv = np.linalg.norm(v)
            return (step(base + eps * v / nv) - y0) * (nv / eps)

        # a Krylov space of the full dimension: the Ritz values are the eigenvalues
        return arnoldi_radius(mv, n, kdim=n)

    H, evals = bisect_stable_step(radius, 0.02, 0.05, rel_tol=1e-5, slack=1e-6)
    assert g["dt_stable"] < H < g["dt_unstable"]
    lam_dx = float(np.abs(np.linalg.eigvals(D)).max())
    assert abs(H - 2.0 * math.sqrt(2.0) / lam_dx * dx) < 2e-5 * H
    assert len(evals) > 5
