"""Pins of the oracle's probe-pressure objective (the objective of the discrete adjoint).

- The probe stencil is a 4 x 4 Lagrange interpolation (the stencil kind of Sec. 2.2): it
  reproduces every bicubic polynomial exactly, in the interior and at clamped edges.
- A uniform state is a steady solution of the discretisation on a periodic box-in-box pair
  (SBP derivatives of constants vanish and the interface penalties see zero jumps), so the
  objective of a run from it is H * n_steps * n_probes * p_inf^2 exactly up to rounding.
"""
import numpy as np

import workloads as W
from oracle import OracleSystem
from oracle.system import probe_objective, probe_pressure, probe_stencil

GAMMA = 1.4


def _pressure_state(mesh, P):
    """State with rho = 1, zero momentum and pressure field P (so p(q) = P)."""
    x, y = mesh["x"], mesh["y"]
    p = P(x, y)
    return np.stack([np.ones_like(x), np.zeros_like(x), np.zeros_like(x), p / (GAMMA - 1.0)])


def test_probe_stencil_reproduces_bicubics():
    rng = np.random.default_rng(5)
    mesh = W.cartesian_mesh("bg", (23, 17), (-1.0, -0.5), (0.13, 0.11), ("farfield",) * 4)
    c = rng.standard_normal((4, 4))

    def P(x, y):
        return 2.0 + sum(c[a, b] * x ** a * y ** b for a in range(4) for b in range(4)) * 0.01

    q = _pressure_state(mesh, P)
    lo, hi = np.array(mesh["lo"]), np.array(mesh["lo"]) + (np.array(mesh["n"]) - 1) * np.array(mesh["h"])
    pts = rng.uniform(lo, hi, size=(40, 2))
    pts = np.vstack([pts, lo, hi, [lo[0], hi[1]], lo + 0.5 * np.array(mesh["h"])])  # corners and edges
    for xy in pts:
        st = probe_stencil(mesh, xy)
        assert 0 <= st[0][0] <= mesh["n"][0] - 4 and 0 <= st[0][1] <= mesh["n"][1] - 4
        assert abs(probe_pressure(mesh, q, st, GAMMA) - P(*xy)) < 1e-12


def test_probe_stencil_weights_partition_unity_and_node_values():
    mesh = W.cartesian_mesh("bg", (12, 12), (0.0, 0.0), (1.0, 1.0), ("farfield",) * 4)
    for xy in [(3.0, 5.0), (4.25, 7.5), (0.0, 11.0)]:
        (i0, j0), (wi, wj) = probe_stencil(mesh, xy)
        assert abs(wi.sum() - 1.0) < 1e-14 and abs(wj.sum() - 1.0) < 1e-14
        if float(xy[0]).is_integer():
            # at a node the stencil picks that node alone
            e = np.zeros(4)
            e[int(xy[0]) - i0] = 1.0
            assert np.allclose(wi, e, atol=1e-15)


def test_probe_objective_uniform_flow_closed_form():
    wl = W.mms_box_in_box(24, "inviscid")
    qinf = W.freestream(0.3)
    q0 = [np.broadcast_to(qinf[:, None, None], (4, m["n"][1], m["n"][0])).copy() for m in wl["meshes"]]
    wl["params"] = dict(wl["params"], qinf=qinf, step_ratio=2)
    o = OracleSystem(wl)
    H = 0.5 * o.macro_step_size(q0)
    probes = np.array([[0.71, 0.6], [-0.8, -0.73], [0.66, -0.9]])
    n_steps = 3
    J, pr = probe_objective(o, q0, probes, n_steps, H)
    p_inf = 1.0 / GAMMA
    assert np.allclose(pr, p_inf, rtol=0, atol=1e-13)
    assert abs(J - H * n_steps * len(probes) * p_inf ** 2) < 1e-13
