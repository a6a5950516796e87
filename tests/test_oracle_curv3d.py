"""Pins of the 3D curvilinear oracle (oracle.curv3d):

* free-stream preservation: a uniform state has zero flux divergence on a warped mesh, exactly
  up to rounding, because the Thomas-Lombard metric terms satisfy the discrete metric identity;
  the same metrics taken as plain cofactors of the coordinate derivatives do not (a planted
  mistake that the pin catches);
* on a uniform Cartesian mesh it is the pinned Cartesian 3D oracle's flux divergence (orc_rhs3d
  without SAT terms), inviscid and viscous;
* on a warped mesh it converges to the exact divergence of the Euler and Navier-Stokes fluxes
  of a smooth manufactured state at fourth order away from the boundary closures;
* the far-field SAT on a rotated uniform mesh is the Cartesian oracle's far-field SAT turned
  by the same rotation, and it vanishes at the free stream;
* interface SAT terms (with donor values and donor viscous fluxes) on a rotated uniform mesh are
  the Cartesian oracle's interface terms turned by the same rotation."""
import ctypes

import numpy as np
import pytest

import oracle
from oracle.curv3d import Curvilinear3D

GAMMA = 1.4


def _grid(n, eps=0.03, waves=2):
    """The unit cube, each coordinate displaced by eps sin(waves pi .) sin(waves pi .) of the
    other two."""
    t = np.linspace(0.0, 1.0, n)
    Z, Y, X = np.meshgrid(t, t, t, indexing="ij")
    s = waves * np.pi
    x = X + eps * np.sin(s * Y) * np.sin(s * Z)
    y = Y + eps * np.sin(s * X) * np.sin(s * Z)
    z = Z + eps * np.sin(s * X) * np.sin(s * Y)
    return x, y, z


def _uniform_state(shape):
    rho, u, v, w, p = 1.1, 0.3, -0.2, 0.15, 0.9
    E = p / (GAMMA - 1) + 0.5 * rho * (u * u + v * v + w * w)
    return np.array([np.full(shape, c) for c in (rho, rho * u, rho * v, rho * w, E)])


@pytest.mark.parametrize("mu", [0.0, 0.01])
def test_free_stream_preserved_on_warped_mesh(mu):
    x, y, z = _grid(20)
    g = Curvilinear3D(x, y, z)
    assert g.Jinv.min() > 0
    q = _uniform_state(x.shape)
    r = g.rhs(q, GAMMA, mu)
    # the divergence scales like |F| / h ~ 20: rounding level
    assert np.abs(r).max() < 2e-12, np.abs(r).max()
    # metric identity itself
    for j in range(3):
        s = sum(g.deriv(g.M[m][j], m) for m in range(3))
        assert np.abs(s).max() < 1e-14


def test_plain_cofactor_metrics_break_free_stream():
    """Planted mistake: metrics as cofactors of the coordinate derivatives (not conservative)."""
    x, y, z = _grid(20)
    g = Curvilinear3D(x, y, z)
    dX = [[g.deriv(c, a) for a in range(3)] for c in (x, y, z)]
    cyc = [(0, 1, 2), (1, 2, 0), (2, 0, 1)]
    for m, a, b in cyc:
        for j, c, e in cyc:
            g.M[m][j] = dX[c][a] * dX[e][b] - dX[c][b] * dX[e][a]
    r = g.rhs(_uniform_state(x.shape), GAMMA)
    assert np.abs(r).max() > 1e-6


@pytest.mark.parametrize("mu", [0.0, 0.02])
def test_uniform_mesh_equals_cartesian_oracle(mu):
    ni, nj, nk = 12, 10, 9
    h = (0.1, 0.07, 0.13)
    Z, Y, X = np.meshgrid(np.arange(nk) * h[2], np.arange(nj) * h[1], np.arange(ni) * h[0], indexing="ij")
    g = Curvilinear3D(X, Y, Z)
    rng = np.random.default_rng(5)
    q = _uniform_state(X.shape) * (1.0 + 0.05 * rng.standard_normal((5,) + X.shape))
    got = g.rhs(q, GAMMA, mu)
    L = oracle.lib()
    iblank = np.ones((nk, nj, ni), np.int8)
    ci, cj, ck = (np.zeros((nk, nj, ni), np.int8) for _ in range(3))
    p = lambda a: ctypes.c_void_p(a.ctypes.data) if a is not None else None  # noqa: E731
    assert L.orc_classes3d(ni, nj, nk, 0, 0, 0, p(iblank), p(ci), p(cj), p(ck)) >= 0
    want = np.zeros((5, nk, nj, ni))
    qc = np.ascontiguousarray(q)
    qinf = np.zeros(5)
    rc = L.orc_rhs3d(ni, nj, nk, p(ci), p(cj), p(ck), ctypes.c_double(h[0]), ctypes.c_double(h[1]),
                     ctypes.c_double(h[2]), p(qc), int(mu > 0), ctypes.c_double(GAMMA), ctypes.c_double(mu),
                     ctypes.c_double(0.72), 0, None, None, None, None, None, None, 0, None, None, p(qinf),
                     ctypes.c_double(0.5), ctypes.c_double(1.0), p(want))
    assert rc == 0
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert err < 1e-13, err


def _manufactured(mu):
    """Exact -div(F - F^V) of a smooth state, by symbolic differentiation."""
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z")
    s = 2 * sp.pi
    rho = 1 + sp.Rational(1, 10) * sp.sin(s * x) * sp.cos(s * y) * sp.sin(s * z)
    u = sp.Rational(3, 10) + sp.Rational(1, 10) * sp.cos(s * x) * sp.sin(s * z)
    v = -sp.Rational(1, 5) + sp.Rational(1, 10) * sp.sin(s * y) * sp.cos(s * x)
    w = sp.Rational(1, 10) * sp.sin(s * x) * sp.sin(s * y)
    p = sp.Rational(9, 10) + sp.Rational(1, 20) * sp.cos(s * x) * sp.cos(s * y) * sp.cos(s * z)
    g = sp.Rational(7, 5)
    E = p / (g - 1) + rho * (u * u + v * v + w * w) / 2
    X = (x, y, z)
    vel = (u, v, w)
    T = g * p / rho
    F = [[rho * vel[d]] + [rho * vel[d] * vel[c] + (p if c == d else 0) for c in range(3)] + [(E + p) * vel[d]]
         for d in range(3)]
    if mu:
        mu_s = sp.nsimplify(mu)
        lam, kap = -sp.Rational(2, 3) * mu_s, mu_s / (sp.Rational(18, 25) * (g - 1))
        div = sum(sp.diff(vel[c], X[c]) for c in range(3))
        for d in range(3):
            tau = [mu_s * (sp.diff(vel[d], X[c]) + sp.diff(vel[c], X[d])) + (lam * div if c == d else 0)
                   for c in range(3)]
            for c in range(3):
                F[d][1 + c] = F[d][1 + c] - tau[c]
            F[d][4] = F[d][4] - (sum(vel[c] * tau[c] for c in range(3)) + kap * sp.diff(T, X[d]))
    res = [-sum(sp.diff(F[d][k], X[d]) for d in range(3)) for k in range(5)]
    state = [rho, rho * u, rho * v, rho * w, E]
    return sp.lambdify(X, state, "numpy"), sp.lambdify(X, res, "numpy")


@pytest.mark.parametrize("mu", [0.0, 0.05])
def test_fourth_order_on_warped_mesh(mu):
    qf, rf = _manufactured(mu)
    errs = []
    ns = (33, 49, 65)
    for n in ns:
        x, y, z = _grid(n, waves=1)
        g = Curvilinear3D(x, y, z)
        q = np.array([np.broadcast_to(c, x.shape) for c in qf(x, y, z)], dtype=float)
        got = g.rhs(q, GAMMA, mu, pr=0.72)
        want = np.array([np.broadcast_to(c, x.shape) for c in rf(x, y, z)], dtype=float)
        # away from the closures: the metric terms apply D twice to the coordinates and the
        # divergence once more to their products
        sl = (slice(None),) + (slice(8, -8),) * 3
        errs.append(np.abs(got[sl] - want[sl]).max())
    hs = [1.0 / (n - 1) for n in ns]
    eocs = [np.log(errs[k] / errs[k + 1]) / np.log(hs[k] / hs[k + 1]) for k in range(2)]
    assert all(3.5 < e < 4.5 for e in eocs), (errs, eocs)


def _cartesian_farfield(q, h, mu, qinf, sigma):
    """orc_rhs3d on a Cartesian mesh with far-field terms on every face point (edges and corners
    carry one term per face they lie on)."""
    _, nk, nj, ni = q.shape
    L = oracle.lib()
    p = lambda a: ctypes.c_void_p(a.ctypes.data) if a is not None else None  # noqa: E731
    iblank = np.ones((nk, nj, ni), np.int8)
    ci, cj, ck = (np.zeros((nk, nj, ni), np.int8) for _ in range(3))
    assert L.orc_classes3d(ni, nj, nk, 0, 0, 0, p(iblank), p(ci), p(cj), p(ck)) >= 0
    pts, dirs, sides = [], [], []
    n = (ni, nj, nk)
    for k in range(nk):
        for j in range(nj):
            for i in range(ni):
                c = (i, j, k)
                for d in range(3):
                    for side, at in ((1, 0), (-1, n[d] - 1)):
                        if c[d] == at:
                            pts.append((k * nj + j) * ni + i)
                            dirs.append(d)
                            sides.append(side)
    m = len(pts)
    t_pt = np.array(pts, np.int64)
    t_dir, t_side = np.array(dirs, np.int32), np.array(sides, np.int32)
    t_kind, t_recv = np.full(m, 2, np.int32), np.full(m, -1, np.int32)
    t_scale = np.ones(m)
    want = np.zeros((5, nk, nj, ni))
    qc = np.ascontiguousarray(q)
    qi = np.ascontiguousarray(qinf, dtype=np.float64)
    rc = L.orc_rhs3d(ni, nj, nk, p(ci), p(cj), p(ck), ctypes.c_double(h[0]), ctypes.c_double(h[1]),
                     ctypes.c_double(h[2]), p(qc), int(mu > 0), ctypes.c_double(GAMMA), ctypes.c_double(mu),
                     ctypes.c_double(0.72), m, p(t_pt), p(t_dir), p(t_side), p(t_kind), p(t_recv), p(t_scale),
                     0, None, None, p(qi), ctypes.c_double(0.5), ctypes.c_double(sigma), p(want))
    assert rc == 0
    return want


def _rotation():
    a, b = 0.4, -0.7
    Rz = np.array([[np.cos(a), -np.sin(a), 0], [np.sin(a), np.cos(a), 0], [0, 0, 1]])
    Rx = np.array([[1, 0, 0], [0, np.cos(b), -np.sin(b)], [0, np.sin(b), np.cos(b)]])
    return Rz @ Rx


@pytest.mark.parametrize("mu", [0.0, 0.02])
def test_farfield_sat_on_rotated_mesh_equals_cartesian_oracle(mu):
    """Far-field SAT on all six faces: a uniform mesh turned by a rotation R, with the state's
    momentum and the free stream's turned alike, gives the Cartesian oracle's right-hand side
    (its far-field term lists on every face) with the momentum of the result turned by R. The
    normal k = J M[m][:] becomes R e_m / h_m here, so a transposed metric index, a wrong face
    side or a dropped edge term fails."""
    ni, nj, nk = 11, 9, 10
    h = (0.1, 0.07, 0.13)
    R = _rotation()
    Z, Y, X = np.meshgrid(np.arange(nk) * h[2], np.arange(nj) * h[1], np.arange(ni) * h[0], indexing="ij")
    P = np.stack([X, Y, Z])
    Xr = np.einsum("ab,b...->a...", R, P)
    g = Curvilinear3D(*Xr)
    rng = np.random.default_rng(11)
    q = _uniform_state(X.shape) * (1.0 + 0.05 * rng.standard_normal((5,) + X.shape))
    qinf = np.array([1.0, 0.35, -0.1, 0.05, 2.4])
    sigma = 1.3
    want = _cartesian_farfield(q, h, mu, qinf, sigma)
    qr = q.copy()
    qr[1:4] = np.einsum("ab,b...->a...", R, q[1:4])
    qinf_r = qinf.copy()
    qinf_r[1:4] = R @ qinf[1:4]
    got = g.rhs(qr, GAMMA, mu, qinf=qinf_r, sigma=sigma)
    got[1:4] = np.einsum("ba,b...->a...", R, got[1:4])
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert err < 1e-12, err
    # the penalty itself is a sizeable part of the result here
    plain = _cartesian_farfield(q, h, mu, qinf, 0.0)
    assert np.linalg.norm(want - plain) > 0.1 * np.linalg.norm(want)


def test_farfield_sat_vanishes_at_free_stream_and_damps_deviation():
    """On a warped mesh a uniform state equal to the free stream has zero right-hand side with
    the SAT on; a perturbed state's SAT changes boundary points only."""
    x, y, z = _grid(14)
    g = Curvilinear3D(x, y, z)
    q0 = _uniform_state(x.shape)
    qinf = q0[:, 0, 0, 0].copy()
    assert np.abs(g.rhs(q0, GAMMA, 0.01, qinf=qinf)).max() < 2e-12
    rng = np.random.default_rng(3)
    q = q0 * (1.0 + 0.01 * rng.standard_normal(q0.shape))
    sat = g.rhs(q, GAMMA, qinf=qinf) - g.rhs(q, GAMMA)
    assert np.abs(sat[:, 1:-1, 1:-1, 1:-1]).max() == 0.0
    assert np.abs(sat).max() > 1e-3


@pytest.mark.parametrize("mu", [0.0, 0.02])
def test_interface_sat_on_rotated_mesh_equals_cartesian_oracle(mu):
    """Interface SAT terms (receiver points on faces, edges and a corner, with donor values and,
    for Navier-Stokes, donor viscous fluxes) on a uniform mesh turned by R equal the Cartesian
    oracle's interface terms (kind 1 of orc_rhs3d) with every vector and the viscous-flux tensor
    turned alike, the result's momentum turned back. A wrong face side, a transposed metric
    index or a dropped viscous-flux jump fails it."""
    ni, nj, nk = 11, 9, 10
    h = (0.1, 0.07, 0.13)
    R = _rotation()
    Z, Y, X = np.meshgrid(np.arange(nk) * h[2], np.arange(nj) * h[1], np.arange(ni) * h[0], indexing="ij")
    g = Curvilinear3D(*np.einsum("ab,b...->a...", R, np.stack([X, Y, Z])))
    rng = np.random.default_rng(17)
    q = _uniform_state(X.shape) * (1.0 + 0.05 * rng.standard_normal((5,) + X.shape))
    # (i, j, k, normal direction, side, receiver column, scale)
    terms = [(0, 3, 4, 0, 1, 0, 1.0), (ni - 1, 5, 2, 0, -1, 1, 1.0), (4, 0, 6, 1, 1, 2, 1.0),
             (6, nj - 1, 3, 1, -1, 3, 1.0), (5, 4, 0, 2, 1, 4, 1.0), (3, 2, nk - 1, 2, -1, 5, 1.0),
             (0, 0, 5, 0, 1, 6, 0.7), (0, 0, 5, 1, 1, 6, 0.7),                      # an edge, weighted
             (ni - 1, nj - 1, nk - 1, 0, -1, 7, 1.0), (ni - 1, nj - 1, nk - 1, 2, -1, 7, 1.0)]
    nrecv = 8
    qhat = np.array([q[:, t[2], t[1], t[0]] for t in sorted({(x[0], x[1], x[2], x[5]) for x in terms},
                                                             key=lambda x: x[3])]).T
    qhat = qhat * (1.0 + 0.03 * rng.standard_normal(qhat.shape))
    fvhat = 0.05 * rng.standard_normal((12, nrecv))
    sigma = 0.5
    # Cartesian oracle
    L = oracle.lib()
    p = lambda a: ctypes.c_void_p(a.ctypes.data) if a is not None else None  # noqa: E731
    iblank = np.ones((nk, nj, ni), np.int8)
    ci, cj, ck = (np.zeros((nk, nj, ni), np.int8) for _ in range(3))
    assert L.orc_classes3d(ni, nj, nk, 0, 0, 0, p(iblank), p(ci), p(cj), p(ck)) >= 0
    t_pt = np.array([(t[2] * nj + t[1]) * ni + t[0] for t in terms], np.int64)
    t_dir = np.array([t[3] for t in terms], np.int32)
    t_side = np.array([t[4] for t in terms], np.int32)
    t_kind = np.ones(len(terms), np.int32)
    t_recv = np.array([t[5] for t in terms], np.int32)
    t_scale = np.array([t[6] for t in terms])
    want = np.zeros((5, nk, nj, ni))
    qc, qh, fh = (np.ascontiguousarray(a) for a in (q, qhat, fvhat))
    rc = L.orc_rhs3d(ni, nj, nk, p(ci), p(cj), p(ck), ctypes.c_double(h[0]), ctypes.c_double(h[1]),
                     ctypes.c_double(h[2]), p(qc), int(mu > 0), ctypes.c_double(GAMMA), ctypes.c_double(mu),
                     ctypes.c_double(0.72), len(terms), p(t_pt), p(t_dir), p(t_side), p(t_kind), p(t_recv),
                     p(t_scale), nrecv, p(qh), p(fh) if mu > 0 else None, p(np.zeros(5)), ctypes.c_double(sigma),
                     ctypes.c_double(1.0), p(want))
    assert rc == 0
    # the same terms on the turned mesh
    turn = lambda a: np.einsum("ab,b...->a...", R, a)  # noqa: E731
    qr, qhr = q.copy(), qhat.copy()
    qr[1:4], qhr[1:4] = turn(q[1:4]), turn(qhat[1:4])
    F = fvhat.reshape(3, 4, nrecv)                       # F[d][c]
    Fr = np.empty_like(F)
    Fr[:, :3] = np.einsum("da,cb,abr->dcr", R, R, F[:, :3])
    Fr[:, 3] = turn(F[:, 3])
    got = g.rhs(qr, GAMMA, mu, interface=dict(terms=terms, qhat=qhr, fvhat=Fr.reshape(12, nrecv), sigma=sigma))
    got[1:4] = np.einsum("ba,b...->a...", R, got[1:4])
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert err < 1e-12, err
    plain = g.rhs(qr, GAMMA, mu)
    plain[1:4] = np.einsum("ba,b...->a...", R, plain[1:4])
    assert np.linalg.norm(got - plain) > 1e-3 * np.linalg.norm(want)
