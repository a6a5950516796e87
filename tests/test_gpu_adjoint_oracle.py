"""The GPU's discrete adjoint against the oracle's own derivative (oracle.adjoint: the oracle's
arithmetic on dual numbers, exact up to rounding):

* sbp_rhs_eval_vjp element by element against the oracle's vector-Jacobian product on a tiny
  Euler pair (every column of the oracle's Jacobian), to 1e-12 relative;
* on Navier-Stokes meshes, <J^T lam, v> from the GPU against <lam, J v> from the oracle's
  derivative along random directions of both states and the far-field state, to 1e-12;
* the probe objective's gradient (sbp_adjoint_probe) against the oracle's derivative of the same
  objective along random directions of the initial states and of the far-field state, to
  1e-10 relative (bootstrap + MRAB macro steps: a longer chain of roundings)."""
import numpy as np
import pytest

from conftest import build_library
from oracle import OracleSystem
from oracle.adjoint import coupled_rhs_jvp, probe_objective_jvp, rhs_vjp
from test_oracle_adjoint import tiny_cylinder, tiny_vortex
from tolerances import rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sbp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build_library()
    import paper_1805_06607_gb300 as mod
    return mod


def test_rhs_vjp_element_by_element(sbp):
    wl, hc = tiny_vortex()
    o = OracleSystem(wl, hole_cells=hc)
    g = sbp.System(wl, hole_cells=hc)
    q = wl["q0"]
    qd = [g.to_device(k, q[k]) for k in range(2)]
    rng = np.random.default_rng(11)
    for k in range(2):
        lam = rng.standard_normal(np.shape(q[k]))
        want_s, want_o, want_i = rhs_vjp(o, k, q[k], q[1 - k], lam)
        gs, go, gi = g.rhs_eval_vjp(k, qd[k], qd[1 - k], g.to_device(k, lam))
        assert rel(g.to_host(k, gs), want_s) < 1e-12
        assert rel(g.to_host(1 - k, go), want_o) < 1e-12
        assert rel(gi, want_i) < 1e-12 or np.abs(gi - want_i).max() < 1e-12 * np.abs(want_s).max()
    g.close()


@pytest.mark.parametrize("make", [tiny_vortex, tiny_cylinder], ids=["euler", "navier_stokes"])
def test_rhs_vjp_against_oracle_derivative(sbp, make):
    wl, hc = make()
    o = OracleSystem(wl, hole_cells=hc)
    g = sbp.System(wl, hole_cells=hc)
    q = wl["q0"]
    qd = [g.to_device(k, q[k]) for k in range(2)]
    rng = np.random.default_rng(12)
    for k in range(2):
        lam = rng.standard_normal(np.shape(q[k]))
        gs, go, gi = g.rhs_eval_vjp(k, qd[k], qd[1 - k], g.to_device(k, lam))
        gs, go = g.to_host(k, gs), g.to_host(1 - k, go)
        for _ in range(3):
            v = [rng.standard_normal(np.shape(x)) for x in q]
            vi = rng.standard_normal(4)
            _, d = coupled_rhs_jvp(o, k, q[k], q[1 - k], v[k], v[1 - k], vi)
            want = float(np.sum(lam * d))
            got = float(np.sum(gs * v[k]) + np.sum(go * v[1 - k]) + gi @ vi)
            assert abs(got - want) <= 1e-12 * abs(want), (k, got, want)
    g.close()


def test_probe_gradient_against_oracle_derivative(sbp):
    wl, hc = tiny_cylinder()
    o = OracleSystem(wl, hole_cells=hc)
    g = sbp.System(wl, hole_cells=hc)
    q0 = wl["q0"]
    qd = [g.to_device(k, q0[k]) for k in range(2)]
    _, H = g.timestep(qd[0], qd[1])
    assert abs(H - o.macro_step_size(q0)) <= 1e-14 * H
    probes = [(1.2, 0.3), (2.0, -0.4), (-2.6, 1.8)]
    n = 4
    r = g.adjoint_probe(qd, probes, n, H)
    grad = [g.to_host(k, r["dq0"][k]) for k in range(2)]
    rng = np.random.default_rng(13)
    for trial in range(3):
        dq = [rng.standard_normal(np.shape(x)) for x in q0]
        dqi = rng.standard_normal(4) if trial else np.zeros(4)
        J, dJ = probe_objective_jvp(o, q0, probes, n, H, dq, dqi)
        assert abs(r["J"] - J) <= 1e-12 * abs(J)
        got = float(sum(np.sum(gr * d) for gr, d in zip(grad, dq)) + r["dqinf"] @ dqi)
        assert abs(got - dJ) <= 1e-10 * abs(dJ), (trial, got, dJ)
    g.close()
