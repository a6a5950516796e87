"""Pins of the oracle's own derivative (oracle.adjoint: the oracle's arithmetic on dual numbers),
the reference for the GPU's discrete adjoint:

* the values it carries are the plain oracle's, bit for bit (right-hand sides and the probe
  objective);
* its derivatives agree with central differences of the plain oracle (the definition of the
  derivative) to the differences' own accuracy, along random directions of both states and of
  the far-field state, for Euler and Navier-Stokes meshes; a planted mistake in one rule of
  differentiation (the square root's) fails that;
* the vector-Jacobian product assembled from its columns satisfies <lam, J v> = <J^T lam, v>."""
import numpy as np
import pytest

import workloads as W
from conftest import planted_oracle, run_with_oracle
from oracle import OracleSystem
from oracle.adjoint import coupled_rhs_jvp, probe_objective_jvp, rhs_vjp
from oracle.system import probe_objective


def tiny_vortex():
    return W.vortex_box_in_box(seed=5, n_bg=24, n_fine=13, bg_half=3.0, fine_half=1.25), 2


def tiny_cylinder(**kw):
    return W.cylinder_small(seed=6, n_theta=40, n_r=12, bg_n=(40, 30), s_bg=0.15, bg_lo=(-3.0, -2.25),
                            stretch=1.12, **kw), 4


CASES = {"vortex": tiny_vortex, "cylinder": tiny_cylinder,
         "cylinder_sponge": lambda: tiny_cylinder(sponge_cells=6, sponge_strength=2.0)}


@pytest.mark.parametrize("case", sorted(CASES))
def test_values_are_the_plain_oracle(case):
    wl, hc = CASES[case]()
    o = OracleSystem(wl, hole_cells=hc)
    for k in range(2):
        v, _ = coupled_rhs_jvp(o, k, wl["q0"][k], wl["q0"][1 - k])
        assert np.array_equal(v, o.coupled_rhs(k, wl["q0"][k], wl["q0"][1 - k]))


def directional_errors(wl, hc, seed=0, h=1e-6):
    """Relative errors of the dual derivative against central differences of the plain oracle,
    per mesh, along a random direction of both states and of the far-field state."""
    o = OracleSystem(wl, hole_cells=hc)
    rng = np.random.default_rng(seed)
    q = wl["q0"]
    dq = [rng.standard_normal(np.shape(x)) * 1e-2 for x in q]
    dqi = rng.standard_normal(4) * 1e-2
    qinf = np.asarray(wl["params"]["qinf"], dtype=np.float64)
    errs = []
    for k in range(2):
        _, d = coupled_rhs_jvp(o, k, q[k], q[1 - k], dq[k], dq[1 - k], dqi)
        rs = []
        for s in (1.0, -1.0):
            o.p["qinf"] = qinf + s * h * dqi
            rs.append(o.coupled_rhs(k, q[k] + s * h * dq[k], q[1 - k] + s * h * dq[1 - k]))
        o.p["qinf"] = qinf
        fd = (rs[0] - rs[1]) / (2.0 * h)
        act = o.iblank[k] != 0
        errs.append(float(np.linalg.norm((d - fd)[:, act]) / np.linalg.norm(fd[:, act])))
    return errs


@pytest.mark.parametrize("case", sorted(CASES))
def test_derivative_matches_central_differences(case):
    wl, hc = CASES[case]()
    errs = directional_errors(wl, hc)
    assert max(errs) < 1e-6, errs


def test_planted_square_root_rule_fails(tmp_path):
    root = planted_oracle(tmp_path, "dual.cpp", "return dual(r, a.d / (2.0 * r));", "return dual(r, a.d / r);")
    out = run_with_oracle(root, "import test_oracle_adjoint as T\n"
                                "wl, hc = T.tiny_cylinder()\n"
                                "print(max(T.directional_errors(wl, hc)))\n")
    assert float(out) > 1e-4


def test_vjp_columns_satisfy_the_dot_product_identity():
    wl, hc = tiny_vortex()
    o = OracleSystem(wl, hole_cells=hc)
    rng = np.random.default_rng(3)
    q = wl["q0"]
    for k in range(2):
        lam = rng.standard_normal(np.shape(q[k]))
        gs, go, gi = rhs_vjp(o, k, q[k], q[1 - k], lam)
        v = [rng.standard_normal(np.shape(x)) for x in q]
        vi = rng.standard_normal(4)
        _, d = coupled_rhs_jvp(o, k, q[k], q[1 - k], v[k], v[1 - k], vi)
        lhs = float(np.sum(lam * d))
        rhs = float(np.sum(gs * v[k]) + np.sum(go * v[1 - k]) + gi @ vi)
        assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1e-300) * 1e2


def test_probe_objective_value_and_derivative():
    wl, hc = tiny_cylinder()
    o = OracleSystem(wl, hole_cells=hc)
    q0 = wl["q0"]
    H = o.macro_step_size(q0)
    probes = [(1.2, 0.3), (2.0, -0.4), (-2.6, 1.8)]
    n = 4
    J, _ = probe_objective(o, q0, probes, n, H)
    rng = np.random.default_rng(4)
    dq = [rng.standard_normal(np.shape(x)) * 1e-2 for x in q0]
    dqi = rng.standard_normal(4) * 1e-2
    Jd, dJ = probe_objective_jvp(o, q0, probes, n, H, dq, dqi)
    assert Jd == J
    h = 1e-6
    qinf = np.asarray(wl["params"]["qinf"], dtype=np.float64)
    Js = []
    for s in (1.0, -1.0):
        o.p["qinf"] = qinf + s * h * dqi
        Js.append(probe_objective(o, [x + s * h * d for x, d in zip(q0, dq)], probes, n, H)[0])
    o.p["qinf"] = qinf
    fd = (Js[0] - Js[1]) / (2 * h)
    assert abs(dJ - fd) < 1e-6 * abs(fd) + 4 * np.finfo(float).eps * abs(J) / h
