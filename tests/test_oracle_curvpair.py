"""Pins of the curvilinear overset pair oracle (oracle.curvpair):

* turned Cartesian pair: two uniform Cartesian meshes (far-field background, overset fine box)
  turned by one rotation and handed to the curvilinear pair are the pinned Cartesian 3D system
  (oracle.system3d) turned by the same rotation: the same holes, receivers and donor stencils,
  weights to rounding, coupled right-hand sides of both meshes (momentum turned back) and time
  steps to 1e-12, and the states after the bootstrap and two MRAB macro steps; Euler and
  Navier-Stokes, with a corner weight Omega != 1;
* free stream: a uniform state equal to the far-field state has zero coupled right-hand side on
  a pair whose overset mesh is warped and turned (the background Cartesian, so that its hole
  segments keep the metric identity);
* planted mistakes in the pair's assembly fail those pins: the side of the hole-boundary
  terms flipped, a direction dropped from the time step, the donor viscous fluxes dropped;
* on a warped background with holes and a warped, turned overset mesh, the coupled right-hand
  sides converge to the exact divergence of a smooth Euler state (EOC 2.4 under refinement by
  1.5, the 4-2 operator's closures showing in the L2 norm); with the donor weights of one
  direction applied in reverse (planted) they do not;
* sponge layer (Sec. 5.1, six points deep) on the background: on a uniform state offset from the
  free stream it adds -sigma (q - qinf) alone, at one rate for all five variables, decaying away
  from the faces to zero at the sixth point, zero at holes and on the overset mesh (its profile
  inside the layer is a reading: parity unpinned for its shape)."""
import numpy as np
import pytest

import workloads as W
from conftest import planted_oracle, run_with_oracle
from oracle.curvpair import OracleCurvPair
from oracle.system3d import OracleSystem3D

ANGLES = (0.3, -0.2, 0.4)


def cartesian_pair(physics="euler", n=22, nf=21):
    """Background n^3 over [-1, 1]^3 (far field), fine box nf^3 at half the spacing (interface),
    offset from the background nodes by 0.3 fine spacings so that no node of one mesh lies on
    a node plane of the other; a smooth state with a pulse and a swirl."""
    h = 2.0 / (n - 1)
    hf = h / 2.0
    lo_f = -0.5 * (nf - 1) * hf + 0.3 * hf
    bg = W.cartesian_mesh3d("background", (n,) * 3, (-1.0,) * 3, (h,) * 3, ("farfield",) * 6)
    fine = W.cartesian_mesh3d("fine", (nf,) * 3, (lo_f,) * 3, (hf,) * 3, ("interface",) * 6)
    qs = []
    for m in (bg, fine):
        x, y, z = W.axes3d(m)
        Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
        G = np.exp(-(X ** 2 + Y ** 2 + Z ** 2) / 0.1)
        rho = 1.0 + 0.03 * G
        u, v, w = 0.2 - 0.05 * Y * G, -0.1 + 0.05 * X * G, 0.15 + 0.02 * np.sin(2 * X)
        p = (1.0 + 0.05 * G) / 1.4
        E = p / 0.4 + 0.5 * rho * (u * u + v * v + w * w)
        qs.append(np.stack([rho, rho * u, rho * v, rho * w, E]))
    qinf = np.array([1.0, 0.2, -0.1, 0.15, 1.0 / (1.4 * 0.4) + 0.5 * (0.04 + 0.01 + 0.0225)])
    params = dict(physics=physics, gamma=1.4, mu=(0.02 if physics == "ns" else 0.0), pr=0.72, order=3, hist_len=3,
                  step_ratio=2, fast_mesh=1, cfl=0.5, qinf=qinf, twall=1.0, omega_corner=0.7)
    return {"meshes": [bg, fine], "q0": qs, "params": params}


def turn(wl, R):
    """The curvilinear pair of a Cartesian pair workload turned by R about the origin: node
    coordinates, momenta and the far-field state's momentum turned; the hole margin of 3
    background spacings becomes 6 index units of the fine mesh."""
    meshes, qs = [], []
    for m, q in zip(wl["meshes"], wl["q0"]):
        x, y, z = W.axes3d(m)
        Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
        P = [sum(R[a, b] * c for b, c in enumerate((X, Y, Z))) for a in range(3)]
        meshes.append(W.curvilinear_mesh3d(m["name"], *P))
        qs.append(turn_state(q, R))
    p = dict(wl["params"])
    p["qinf"] = turn_state(np.asarray(p["qinf"], dtype=np.float64), R)
    p["hole_cells"] = 6
    return {"meshes": meshes, "q0": qs, "params": p}


def turn_state(q, R):
    q = np.asarray(q, dtype=np.float64)
    m = np.tensordot(R, q[1:4], axes=(1, 0))
    return np.concatenate([q[:1], m, q[4:]])


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module", params=["euler", "ns"])
def pair(request):
    R = W.rotation3d(ANGLES)
    wl = cartesian_pair(request.param)
    wc = turn(wl, R)
    return R, wl, wc, OracleSystem3D(wl, hole_cells=3), OracleCurvPair(wc)


def test_tables_equal_cartesian_system(pair):
    R, wl, wc, o3, oc = pair
    assert (oc.iblank[0] == 0).sum() > 20
    for k in range(2):
        assert np.array_equal(oc.iblank[k] != 0, o3.iblank[k] != 0), k
        assert np.array_equal(oc.recv_pts[k], o3.recv_pts[k]), k
        assert np.array_equal(oc.base[k], o3.base[k]), k
        assert np.abs(oc.w[k] - o3.w[k]).max() < 1e-12, k
        assert len(oc.terms[k]) == o3.terms[k]["pt"].size - (0 if k else int((o3.terms[k]["kind"] == 2).sum()))


def test_coupled_rhs_and_dt_equal_cartesian_system(pair):
    R, wl, wc, o3, oc = pair
    for k in range(2):
        want = o3.coupled_rhs(k, wl["q0"][k], wl["q0"][1 - k])
        got = turn_state(oc.coupled_rhs(k, wc["q0"][k], wc["q0"][1 - k]), R.T)
        assert rel(got, want) < 1e-12, (k, rel(got, want))
        d3, dc = o3.dt_mesh(k, wl["q0"][k]), oc.dt_mesh(k, wc["q0"][k])
        # |k_m|^2 from metric terms computed by D carries a few ulps more than 1 / h^2
        assert abs(dc - d3) <= 1e-13 * d3, (k, dc, d3)


def test_mrab_equals_cartesian_system(pair):
    R, wl, wc, o3, oc = pair
    H = o3.macro_step_size(wl["q0"])
    assert abs(oc.macro_step_size(wc["q0"]) - H) <= 1e-13 * H
    y3, hf3, hs3 = o3.bootstrap(wl["q0"], H)
    yc, hfc, hsc = oc.bootstrap(wc["q0"], H)
    y3, _, _ = o3.mrab(y3, hf3, hs3, H, 2)
    yc, _, _ = oc.mrab(yc, hfc, hsc, H, 2)
    for k in range(2):
        d_want = y3[k] - wl["q0"][k]
        d_got = turn_state(yc[k], R.T) - wl["q0"][k]
        assert rel(d_got, d_want) < 1e-11, (k, rel(d_got, d_want))


def test_free_stream_preserved():
    wl = W.curvilinear_pair(eps_bg=0.0)
    qinf = np.asarray(wl["params"]["qinf"])
    o = OracleCurvPair(wl)
    qs = [np.broadcast_to(qinf[:, None, None, None], (5,) + m["x"].shape).copy() for m in wl["meshes"]]
    for k in range(2):
        r = o.coupled_rhs(k, qs[k], qs[1 - k])
        assert np.abs(r).max() < 1e-11, (k, np.abs(r).max())


PLANTS = {
    "hole_side": ("for side, off in ((1, -1), (-1, 1)):", "for side, off in ((-1, -1), (1, 1)):", "euler", "rhs"),
    "dt_direction": ("        for m in range(3):\n            kv = [op.J", "        for m in range(2):\n            kv = [op.J",
                     "euler", "dt"),
    "donor_viscous_fluxes": ("iface = dict(terms=self.terms[k], qhat=np.asarray(qhat), fvhat=fvhat,",
                             "iface = dict(terms=self.terms[k], qhat=np.asarray(qhat), fvhat=0 * fvhat,", "ns", "rhs"),
}


@pytest.mark.parametrize("plant", sorted(PLANTS))
def test_planted_mistakes_fail(tmp_path, plant):
    old, new, phys, what = PLANTS[plant]
    root = planted_oracle(tmp_path, "curvpair.py", old, new)
    code = ("import numpy as np, workloads as W\n"
            "import test_oracle_curvpair as T\n"
            "from oracle.curvpair import OracleCurvPair\n"
            "from oracle.system3d import OracleSystem3D\n"
            "R = W.rotation3d(T.ANGLES)\n"
            "wl = T.cartesian_pair(%r)\n"
            "wc = T.turn(wl, R)\n"
            "o3, oc = OracleSystem3D(wl, hole_cells=3), OracleCurvPair(wc)\n"
            "if %r == 'dt':\n"
            "    print(max(abs(oc.dt_mesh(k, wc['q0'][k]) / o3.dt_mesh(k, wl['q0'][k]) - 1) for k in range(2)))\n"
            "else:\n"
            "    print(max(T.rel(T.turn_state(oc.coupled_rhs(k, wc['q0'][k], wc['q0'][1 - k]), R.T),\n"
            "                    o3.coupled_rhs(k, wl['q0'][k], wl['q0'][1 - k])) for k in range(2)))\n" % (phys, what))
    assert float(run_with_oracle(root, code)) > 1e-6


def _field(x, y, z):
    """A smooth state (rho, rho u, rho v, rho w, rho E) at the given coordinates."""
    rho = 1.0 + 0.1 * np.sin(2 * x + y) * np.cos(z)
    u = 0.3 + 0.1 * np.cos(x + 2 * z)
    v = -0.2 + 0.1 * np.sin(y)
    w = 0.1 * np.cos(x + y)
    p = 0.9 + 0.05 * np.sin(x + y + z)
    return np.stack([rho, rho * u, rho * v, rho * w, p / 0.4 + 0.5 * rho * (u * u + v * v + w * w)])


def _exact_rhs(x, y, z, h=1e-5):
    """-div F of the Euler fluxes of _field, by central differences of the analytic field."""
    def flux(X, d):
        q = _field(*X)
        rho, vel = q[0], q[1:4] / q[0]
        p = 0.4 * (q[4] - 0.5 * rho * (vel ** 2).sum(axis=0))
        return np.stack([q[1 + d], *(q[1 + c] * vel[d] + (p if c == d else 0.0) for c in range(3)),
                         (q[4] + p) * vel[d]])
    out = 0.0
    for d in range(3):
        Xp = [x, y, z]
        Xm = [x, y, z]
        Xp = [c + (h if a == d else 0.0) for a, c in enumerate(Xp)]
        Xm = [c - (h if a == d else 0.0) for a, c in enumerate(Xm)]
        out = out - (flux(Xp, d) - flux(Xm, d)) / (2 * h)
    return out


def coupled_rhs_error(n_bg, n_fine, hole_cells):
    """L2 error of the coupled right-hand sides of both meshes of a warped, turned pair against the
    exact divergence of a smooth Euler state (background face points excluded: the far-field
    SAT pulls them toward a constant state); cell-volume weighted."""
    wl = W.curvilinear_pair(seed=1, n_bg=n_bg, n_fine=n_fine, hole_cells=hole_cells)
    o = OracleCurvPair(wl)
    qs = [_field(m["x"], m["y"], m["z"]) for m in wl["meshes"]]
    vols = o.cell_sizes()
    err, ref = 0.0, 0.0
    for k, m in enumerate(wl["meshes"]):
        r = o.coupled_rhs(k, qs[k], qs[1 - k])
        ex = _exact_rhs(m["x"], m["y"], m["z"])
        mask = o.iblank[k] != 0
        if k == 0:
            mask = mask.copy()
            mask[0, :, :] = mask[-1, :, :] = mask[:, 0, :] = mask[:, -1, :] = mask[:, :, 0] = mask[:, :, -1] = False
        err += float(((r - ex) ** 2 * vols[k])[:, mask].sum())
        ref += float((ex ** 2 * vols[k])[:, mask].sum())
    return (err / ref) ** 0.5


def test_coupled_rhs_converges_on_warped_pair():
    """The whole coupled right-hand side of a warped background with holes and a warped, turned
    overset mesh (segment derivatives next to holes, metric terms on whole lines, interface terms
    at the overset faces and the hole boundary, Lagrange donors) converges to the exact divergence
    of a smooth state under refinement by 1.5: the closures' second order shows in the L2 norm
    (the paper's 4-2 operator, Sec. 2.1)."""
    e0 = coupled_rhs_error(24, 25, 7.0)
    e1 = coupled_rhs_error(36, 37, 10.5)
    eoc = np.log(e0 / e1) / np.log(35.0 / 23.0)
    assert e1 < e0 and eoc > 1.8, (e0, e1, eoc)


def test_convergence_fails_planted_donor_weight_order(tmp_path):
    # the i-direction Lagrange weights applied in reverse order: the receivers' donor values are
    # first-order wrong and the interface terms stop converging
    root = planted_oracle(tmp_path, "curvpair.py",
                          "return interpolate(np.asarray(field, dtype=np.float64), self.base[k], self.w[k])",
                          "return interpolate(np.asarray(field, dtype=np.float64), self.base[k], "
                          "self.w[k][:, [3, 2, 1, 0] + list(range(4, 12))])")
    out = run_with_oracle(root, "import numpy as np, test_oracle_curvpair as T\n"
                                "e0 = T.coupled_rhs_error(24, 25, 7.0)\n"
                                "e1 = T.coupled_rhs_error(36, 37, 10.5)\n"
                                "print(np.log(e0 / e1) / np.log(35.0 / 23.0))\n")
    assert float(out) < 1.0


def test_sponge_layer_on_the_background():
    """Sec. 5.1's sponge (six points deep) on the pair's background, on a uniform state offset from
    the free stream: it adds -sigma (q - qinf) and nothing else, with the same rate for every
    variable, zero from the sixth point inside the faces on, at holes and on the overset mesh, and a
    rate that decreases away from the faces (the background Cartesian, as in the free-stream pin, so
    that the uniform state's flux divergence vanishes on its hole segments too)."""
    base = dict(eps_bg=0.0)
    wl = W.curvilinear_pair(sponge_cells=6, sponge_strength=2.0, **base)
    qinf = np.asarray(wl["params"]["qinf"])
    off = np.array([0.01, 0.02, -0.01, 0.015, 0.03])
    qs = [np.broadcast_to((qinf + off)[:, None, None, None], (5,) + m["x"].shape).copy() for m in wl["meshes"]]
    o = OracleCurvPair(wl)
    plain = OracleCurvPair(W.curvilinear_pair(**base))
    sig = o.sponge_strength(0)
    r = [o.coupled_rhs(k, qs[k], qs[1 - k]) for k in range(2)]
    p = [plain.coupled_rhs(k, qs[k], qs[1 - k]) for k in range(2)]
    scale = np.abs(p[0]).max()
    assert np.abs((r[0] - p[0]) + sig[None] * off[:, None, None, None]).max() <= 1e-13 * scale
    assert np.array_equal(r[1], p[1])
    nk, nj, ni = sig.shape
    kk, jj, ii = np.meshgrid(np.arange(nk), np.arange(nj), np.arange(ni), indexing="ij")
    d = np.minimum.reduce([ii, ni - 1 - ii, jj, nj - 1 - jj, kk, nk - 1 - kk])
    act = o.iblank[0] != 0
    assert np.all(sig[d >= 6] == 0.0) and np.all(sig[~act] == 0.0)
    assert np.all(sig[(d < 6) & act] > 0.0)
    prof = [sig[(d == e) & act].max() for e in range(6)]
    assert all(prof[e] == sig[(d == e) & act].min() for e in range(6))  # a function of d alone
    assert all(prof[e + 1] < prof[e] for e in range(5))
    # away from the faces the uniform state's right-hand side is the sponge term alone
    inner = (d >= 1) & (d < 6) & act
    rate = -r[0][:, inner] / off[:, None]
    assert np.abs(rate - sig[inner][None]).max() <= 1e-9 * prof[0]
