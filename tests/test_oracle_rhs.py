"""Pins of the oracle's right-hand side (Sec. 2.2 eq. (int); App. C.1) against what the paper and
the mathematics fix: the convergence orders the paper prints for manufactured solutions,
free-stream preservation on a curvilinear mesh, the penalty matrix against a library
eigen-decomposition, telescoping of the SBP flux sum on a periodic mesh, and the closed-form
time step on a uniform state."""
import ctypes
import math

import numpy as np
import pytest

import oracle
import workloads as W
from conftest import golden
from oracle import OracleSystem, l2_norm


def _mms_error(n, kind):
    wl = W.mms_box_in_box(n, kind)
    S = OracleSystem(wl)
    r = S.rhs_all(wl["q0"])
    errs = []
    for k, m in enumerate(wl["meshes"]):
        if kind == "inviscid":   # d rho/dt = -d(rho u)/dx
            e = r[k][0] + 2 * math.pi * np.cos(2 * math.pi * (m["x"] - 0.5))
        else:                    # d(rho u)/dt = mu d2u/dy2
            e = r[k][1] + 4 * math.pi ** 2 * np.sin(2 * math.pi * (m["y"] - 0.5))
        errs.append(np.where(S.iblank[k] != 0, e, 0.0))
    return l2_norm(errs, S.cell_sizes())


@pytest.mark.parametrize("kind,fixture", [("inviscid", "mms_rhs_inviscid.txt"),
                                          ("viscous", "mms_rhs_viscous.txt")])
def test_mms_orders_match_paper(kind, fixture):
    rows = golden(fixture)
    errs = [_mms_error(int(r[0]), kind) for r in rows]
    for k in range(1, len(rows)):
        eoc = math.log(errs[k - 1] / errs[k]) / math.log(int(rows[k][0]) / int(rows[k - 1][0]))
        # orders (not absolute errors, which depend on unstated parameters) are the pin
        assert abs(eoc - float(rows[k][2])) < 0.03, (kind, rows[k], eoc)


def _uniform(wl, q):
    return [np.broadcast_to(q[:, None, None], (4,) + m["x"].shape).copy() for m in wl["meshes"]]


def test_freestream_preserved_on_ogrid():
    wl = W.cylinder_small(seed=3)
    wl["meshes"][1]["bc"] = ("periodic", "periodic", "farfield", "interface")
    S = OracleSystem(wl)
    qs = _uniform(wl, wl["params"]["qinf"])
    r = S.rhs_all(qs)
    scale = max(np.abs(S.met[1][4]).max(), 1.0)
    assert np.abs(r[1]).max() < 1e-13 * scale
    assert np.abs(r[0]).max() < 1e-12
    # the wall penalty is the only term a uniform flow excites once the wall is restored
    wl["meshes"][1]["bc"] = ("periodic", "periodic", "wall", "interface")
    S = OracleSystem(wl)
    r = S.rhs_all(qs)
    assert np.abs(r[1][:, 1:, :]).max() < 1e-13 * scale
    assert np.abs(r[1][:, 0, :]).max() > 1.0


def test_penalty_matrix_against_eig():
    L = oracle.lib()
    rng = np.random.default_rng(5)
    g = 1.4
    for _ in range(20):
        rho = rng.uniform(0.5, 2.0)
        u, v = rng.uniform(-0.8, 0.8, 2)
        p = rng.uniform(0.3, 2.0)
        q = np.array([rho, rho * u, rho * v, p / (g - 1) + 0.5 * rho * (u * u + v * v)])
        kx, ky = rng.uniform(-3, 3, 2)
        # Jacobian by central differences of the flux k.(F, G) (independent of the oracle's form)
        def flux(qq):
            r_, u_, v_ = qq[0], qq[1] / qq[0], qq[2] / qq[0]
            p_ = (g - 1) * (qq[3] - 0.5 * r_ * (u_ * u_ + v_ * v_))
            U = kx * u_ + ky * v_
            return np.array([r_ * U, qq[1] * U + kx * p_, qq[2] * U + ky * p_, (qq[3] + p_) * U])
        A = np.zeros((4, 4))
        for c in range(4):
            e = np.zeros(4)
            e[c] = 1e-6
            A[:, c] = (flux(q + e) - flux(q - e)) / 2e-6
        lam, T = np.linalg.eig(A)
        Ti = np.linalg.inv(T)
        for side in (1, -1):
            K = np.zeros((4, 4))
            L.orc_penalty_matrix2d(ctypes.c_void_p(q.ctypes.data), g, kx, ky, side,
                                   ctypes.c_void_p(K.ctypes.data))
            ref = (T @ np.diag(0.5 * (np.abs(lam.real) + side * lam.real)) @ Ti).real
            assert np.allclose(K, ref, atol=1e-7 * np.abs(A).max())


def test_periodic_flux_sum_telescopes():
    """On a periodic hole-free mesh sum_p J^-1 dq/dt = 0 (1^T D = 0 for the periodic operator)."""
    wl = W.vortex_box_in_box(seed=2)
    m = wl["meshes"][0]
    S = OracleSystem(wl)
    ci = np.zeros_like(S.ci[0])
    cj = np.zeros_like(S.cj[0])
    ni, nj = m["n"]
    q = np.ascontiguousarray(wl["q0"][0])
    out = np.zeros_like(q)
    L = oracle.lib()
    z = np.zeros(1, np.int32)
    zf = np.zeros(1)
    P = lambda a: ctypes.c_void_p(a.ctypes.data)
    L.orc_rhs2d(ni, nj, 1, 1, P(ci), P(cj), P(S.met[0]), P(q), 0, 1.4, 0.0, 0.72, 0, P(z), P(z), P(z), P(z),
                P(z), P(zf), 0, P(zf), None, P(wl["params"]["qinf"]), 1.0, 0.5, 1.0, P(out))
    vol = 1.0 / S.met[0][4]
    for v in range(4):
        assert abs((out[v] * vol).sum()) < 1e-12 * np.abs(out[v] * vol).sum()


def test_timestep_closed_form():
    wl = W.vortex_box_in_box(seed=0)
    S = OracleSystem(wl)
    q = _uniform(wl, wl["params"]["qinf"])[0]
    h = wl["meshes"][0]["h"][0]
    u = wl["params"]["qinf"][1]
    c = math.sqrt(1.4 * (1.4 - 1) * (wl["params"]["qinf"][3] - 0.5 * u * u))
    expect = 1.0 / (abs(u) / h + c * math.sqrt(2.0) / h)
    assert abs(S.dt_mesh(0, q) - expect) < 1e-14 * expect
