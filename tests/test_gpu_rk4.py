"""The classical Runge-Kutta baseline integrator (Sec. 4.4, 6.1) on the GPU path.

- sbp_rk4_step against the oracle's RK4 on the same two-mesh systems (every stage coupled
  through the interface), on the increments over the steps: 1e-12 relative in FP64; in FP32 the
  states within 1e-5 and the increments within the derived FP32 right-hand-side bound.
- CUDA-graph replay gives the same bits as kernel-by-kernel launches.
- The step-matrix tool on RK4 steps: on uniform flow the largest stable step is the RK4
  imaginary-axis bound 2 sqrt(2) over the periodic operator's 1.3722, in units of the Sec. 4.1
  step estimate of the fine mesh (which sets the limit at one rate).
"""
import math

import numpy as np
import pytest

import workloads as W
from conftest import build_library, golden
from oracle import OracleSystem
from tolerances import U32, U64, fp32_rhs_tol, increment_tol, rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sbp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build_library()
    import paper_1805_06607_gb300 as mod
    return mod


CASES = {
    "vortex": lambda: W.vortex_box_in_box(seed=21, n_bg=48, n_fine=33),
    "cylinder": lambda: W.cylinder_small(seed=22),
}


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("case", sorted(CASES))
def test_rk4_matches_oracle(sbp, case, dtype):
    wl = CASES[case]()
    ref = OracleSystem(wl)
    g = sbp.System(wl, dtype=dtype)
    g.bind(wl["q0"])
    dts, _ = g.timestep(g.current_state(0), g.current_state(1))
    h = 0.8 * min(dts)
    n = 3
    want = ref.rk4(wl["q0"], h, n)
    g.rk4_step(n, h)
    g.check()
    q0 = wl["q0"]
    for k in range(2):
        act = ref.iblank[k] != 0
        got = g.to_host(k, g.current_state(k))[:, act]
        e = rel(got, want[k][:, act])
        assert e < (1e-12 if dtype == "f64" else 1e-5), (k, e)
        if dtype == "f64":
            bar, unit = 1e-12, U64
        else:
            bar = max(fp32_rhs_tol(ref.met[j], q0[j], ref.iblank[j] != 0, ref.coupled_rhs(j, q0[j], q0[1 - j]),
                               ref.mu, ref.pr)
                      for j in range(2))
            unit = U32
        ei = rel(got - q0[k][:, act], want[k][:, act] - q0[k][:, act])
        tol = increment_tol(bar, q0[k][:, act], want[k][:, act], 4 * n, unit)
        assert ei < tol, (k, ei, tol)
    _, t = g.mrab_time()
    assert t == pytest.approx(n * h)
    # the MRAB history is stale after Runge-Kutta steps
    with pytest.raises(RuntimeError):
        g.mrab_step(1)
    g.close()


def test_rk4_graph_matches_eager(sbp):
    wl = CASES["cylinder"]()
    out = []
    for graphs in (False, True):
        g = sbp.System(wl)
        g.use_graphs(graphs)
        g.bind(wl["q0"])
        dts, _ = g.timestep(g.current_state(0), g.current_state(1))
        g.rk4_step(5, 0.5 * min(dts))
        g.check()
        out.append([g.to_host(k, g.current_state(k)) for k in range(2)])
        g.close()
    for k in range(2):
        assert np.array_equal(out[0][k], out[1][k])


def test_rk4_then_mrab(sbp):
    """Runge-Kutta steps, then a fresh MRAB bootstrap from the state they reached, equal the
    oracle doing the same."""
    wl = CASES["vortex"]()
    ref = OracleSystem(wl)
    g = sbp.System(wl)
    g.bind(wl["q0"])
    dts, H = g.timestep(g.current_state(0), g.current_state(1))
    h = 0.5 * min(dts)
    g.rk4_step(2, h)
    g.mrab_init(H)
    g.mrab_step(2)
    g.check()
    y = ref.rk4(wl["q0"], h, 2)
    y, hf, hs = ref.bootstrap(y, H)
    want, _, _ = ref.mrab(y, hf, hs, H, 2)
    for k in range(2):
        got = g.to_host(k, g.current_state(k))
        assert rel(got, want[k]) < 1e-12
        tol = increment_tol(1e-12, wl["q0"][k], want[k], 30, U64)
        assert rel(got - wl["q0"][k], want[k] - wl["q0"][k]) < tol
    g.close()


@pytest.mark.timeout(900)
def test_rk4_stability_limit_matches_theory(sbp):
    from paper_1805_06607_gb300.stability import StepMatrix
    wl = W.vortex_box_in_box(seed=51, n_bg=32, n_fine=21)
    qinf = np.asarray(wl["params"]["qinf"], dtype=np.float64)
    uni = [np.broadcast_to(qinf[:, None, None], (4, m["n"][1], m["n"][0])).copy() for m in wl["meshes"]]
    spectral = float(golden("periodic_spectrum.txt")[0][0])
    f_star = 2.0 * math.sqrt(2.0) / spectral
    rho = {}
    for f in (0.9, 1.1):
        g = sbp.System(wl)
        g.bind(uni)
        dts, _ = g.timestep(g.current_state(0), g.current_state(1))
        rho[f] = StepMatrix(g, f * f_star * dts[1], integrator="rk4").spectral_radius()
        g.close()
    assert rho[0.9] <= 1.0 + 0.02, rho
    assert rho[1.1] > 1.05, rho
