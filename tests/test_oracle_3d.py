"""Pins of the 3D Cartesian oracle (oracle/orc3d.c, oracle/system3d.py).

- Reduction to 2D: a pinned 2D workload extruded along a new periodic direction (velocity 0
  along it) is a solution whose 3D right-hand side must equal the 2D oracle's, slice by slice,
  with zero momentum along the extruded direction. Extruding along z exercises the i/j code
  paths, extruding along y (the 2D plane in (x, z)) the k paths: stencil classes, derivatives,
  SAT terms, donors and interpolation along k, and the w terms of the viscous stress.
- K^{+/-} of the 3D flux Jacobian against numpy's eigen-decomposition of a finite-difference
  Jacobian of k . (F, G, H).
- A uniform state is steady (free-stream preservation, interface jumps zero).
- Tensor-product Lagrange interpolation reproduces tricubic fields; the time step matches its
  closed form on a uniform state.
- The sponge layer reduces to the pinned 2D one on an extruded pair with far-field faces.
"""
import ctypes

import numpy as np
import pytest

import oracle
import workloads as W
from oracle import OracleSystem, OracleSystem3D


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


# (workload, hole margin in background spacings chosen so that no background point sits
# exactly at the margin, where the 2D polygon-distance test and the 3D box test may round
# differently)
CASES_2D = {
    "vortex_euler": (lambda: W.vortex_box_in_box(seed=3, n_bg=40, n_fine=25), 2.5),
    "mms_viscous": (lambda: W.mms_box_in_box(40, "viscous"), 3.7),
}


@pytest.mark.parametrize("case", sorted(CASES_2D))
@pytest.mark.parametrize("axis", [2, 1])
def test_extruded_rhs_equals_2d(case, axis):
    mk, hole_cells = CASES_2D[case]
    wl2 = mk()
    o2 = OracleSystem(wl2, hole_cells=hole_cells)
    assert (o2.iblank[0] == 0).any()
    r2 = o2.rhs_all(wl2["q0"])
    # extruded spacing = the background's (the hole margin counts background spacings)
    wl3 = W.extrude_to_3d(wl2, nk=6, lz=6 * max(wl2["meshes"][0]["h"]), axis=axis)
    o3 = OracleSystem3D(wl3, hole_cells=hole_cells)
    for k in range(2):
        assert o3.recv_pts[k].size == o2.recv_pts[k].size * 6
    r3 = o3.rhs_all(wl3["q0"])
    for k in range(2):
        got = r3[k]
        if axis == 2:
            want = np.stack([r2[k][0], r2[k][1], r2[k][2], np.zeros_like(r2[k][0]), r2[k][3]])
            for s in range(6):
                assert _rel(got[:, s], want) < 1e-12, (k, s)
        else:
            want = np.stack([r2[k][0], r2[k][1], np.zeros_like(r2[k][0]), r2[k][2], r2[k][3]])
            for s in range(6):
                assert _rel(got[:, :, s, :], want) < 1e-12, (k, s)


def test_penalty_matrix3d_against_eig():
    L = oracle.lib()
    rng = np.random.default_rng(7)
    g = 1.4
    for _ in range(20):
        rho = rng.uniform(0.5, 2.0)
        u = rng.uniform(-0.8, 0.8, 3)
        p = rng.uniform(0.3, 2.0)
        q = np.array([rho, *(rho * u), p / (g - 1) + 0.5 * rho * u @ u])
        kv = rng.uniform(-3, 3, 3)

        def flux(qq):
            r_, vel = qq[0], qq[1:4] / qq[0]
            p_ = (g - 1) * (qq[4] - 0.5 * r_ * vel @ vel)
            U = kv @ vel
            return np.array([r_ * U, *(qq[1:4] * U + kv * p_), (qq[4] + p_) * U])

        A = np.zeros((5, 5))
        for c in range(5):
            e = np.zeros(5)
            e[c] = 1e-6
            A[:, c] = (flux(q + e) - flux(q - e)) / 2e-6
        lam, T = np.linalg.eig(A)
        Ti = np.linalg.inv(T)
        for side in (1, -1):
            K = np.zeros((5, 5))
            L.orc_penalty_matrix3d(ctypes.c_void_p(q.ctypes.data), g, *kv, side, ctypes.c_void_p(K.ctypes.data))
            ref = (T @ np.diag(0.5 * (np.abs(lam.real) + side * lam.real)) @ Ti).real
            assert np.allclose(K, ref, atol=1e-7 * np.abs(A).max())


def test_uniform_state_is_steady():
    wl = W.taylor_green_small(seed=2)
    qinf = W.freestream3d(0.3)
    wl["params"] = dict(wl["params"], qinf=qinf)
    q = [np.broadcast_to(qinf[:, None, None, None], (5,) + o.shape).copy()
         for o in (np.zeros((m["n"][2], m["n"][1], m["n"][0])) for m in wl["meshes"])]
    o = OracleSystem3D(wl)
    for r in o.rhs_all(q):
        assert np.abs(r).max() < 1e-13


def test_interp3d_reproduces_tricubics():
    wl = W.taylor_green_small(seed=4)
    o = OracleSystem3D(wl)
    rng = np.random.default_rng(9)
    c = rng.standard_normal((4, 4, 4)) * 0.1
    bg, fine = wl["meshes"]

    def P(x, y, z):
        return sum(c[a, b, d] * x ** a * y ** b * z ** d for a in range(4) for b in range(4) for d in range(4))

    x, y, z = W.axes3d(bg)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    field = P(X, Y, Z)[None]
    got = o.interp(1, field)[0]
    pts = o.recv_pts[1]
    ni, nj = fine["n"][0], fine["n"][1]
    fx, fy, fz = W.axes3d(fine)
    want = P(fx[pts % ni], fy[(pts // ni) % nj], fz[pts // (ni * nj)])
    assert np.abs(got - want).max() < 1e-11 * np.abs(want).max()


def test_dt3d_closed_form():
    wl = W.taylor_green_small(seed=5)
    o = OracleSystem3D(wl)
    g, mu, pr = 1.4, wl["params"]["mu"], wl["params"]["pr"]
    rho, vel, p = 1.3, np.array([0.2, -0.1, 0.3]), 0.9
    q = np.array([rho, *(rho * vel), p / (g - 1) + 0.5 * rho * vel @ vel])
    m = wl["meshes"][0]
    state = np.broadcast_to(q[:, None, None, None], (5, m["n"][2], m["n"][1], m["n"][0])).copy()
    h = np.array(m["h"])
    c = np.sqrt(g * p / rho)
    inv = np.sum(np.abs(vel) / h) + c * np.sqrt(np.sum(1 / h ** 2))
    nu = max(mu, g * mu / pr) / rho
    want = 1.0 / (inv + 2 * nu * np.sum(1 / h ** 2))
    assert abs(o.dt_mesh(0, state) - want) < 1e-14 * want


def _sponge_vortex():
    """The vortex pair with a far-field background (not periodic) and a sponge six points deep."""
    wl = W.vortex_box_in_box(seed=3, n_bg=40, n_fine=25)
    bg = wl["meshes"][0]
    far = W.cartesian_mesh("background", bg["n"], bg["lo"], bg["h"], ("farfield",) * 4)
    params = dict(wl["params"], sponge_cells=6, sponge_strength=2.0)
    return dict(wl, meshes=[far, wl["meshes"][1]], params=params)


@pytest.mark.parametrize("axis", [2, 1])
def test_extruded_sponge_equals_2d(axis):
    """The sponge layer (Sec. 5.1) in three directions reduces to the pinned 2D one: on the vortex
    pair with far-field background faces extruded along a periodic direction (no far-field face
    there), the 3D right-hand side equals the 2D oracle's slice by slice, and without the sponge
    it does not."""
    wl2 = _sponge_vortex()
    o2 = OracleSystem(wl2, hole_cells=2.5)
    r2 = o2.rhs_all(wl2["q0"])
    wl3 = W.extrude_to_3d(wl2, nk=6, lz=6 * max(wl2["meshes"][0]["h"]), axis=axis)
    o3 = OracleSystem3D(wl3, hole_cells=2.5)
    r3 = o3.rhs_all(wl3["q0"])
    plain = OracleSystem3D(dict(wl3, params=dict(wl3["params"], sponge_cells=0)), hole_cells=2.5)
    r3p = plain.rhs_all(wl3["q0"])
    for s in range(6):
        if axis == 2:
            want = np.stack([r2[0][0], r2[0][1], r2[0][2], np.zeros_like(r2[0][0]), r2[0][3]])
            got, nosp = r3[0][:, s], r3p[0][:, s]
        else:
            want = np.stack([r2[0][0], r2[0][1], np.zeros_like(r2[0][0]), r2[0][2], r2[0][3]])
            got, nosp = r3[0][:, :, s, :], r3p[0][:, :, s, :]
        assert _rel(got, want) < 1e-12, s
        assert _rel(nosp, want) > 1e-3, s
    assert np.abs(o3.sponge_strength(1)).max() == 0.0  # the fine box has no far-field face
