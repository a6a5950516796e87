"""The 3D curvilinear overset pair on the GPU (sbp3c_system_*) against its oracle
(oracle.curvpair), on the seeded curvilinear_pair workload (a warped 24^3 background with 125
holes, a warped and turned 25^3 overset box), Euler and Navier-Stokes:

* setup tables: holes after growth, receivers and donor stencils bit-exact, weights to 1e-13;
* right-hand sides of both meshes (0 at holes): FP64 to 1e-12 or, where the stream's flux
  differences cancel, to the same derived rounding bound in FP64 (tolerances.fp32_rhs_tol_curv
  with u64: 1.1e-11 on this background), FP32 to the derived FP32 bound; donor states at the
  receivers: FP64 to 1e-12; donor viscous fluxes: FP64 to 1e-12 of their largest value plus
  their derived absolute rounding (they nearly vanish where the stream is uniform);
* the time step of each mesh and the macro step: FP64 to 1e-13;
* bootstrap + 3 MRAB macro steps: increments over the 3 macro steps to the FP64 bar above and
  to the derived FP32 right-hand-side bound (FP32), each with the stored state's rounding floor;
* a non-finite state planted on the host is reported by the step's check as SBP_ERR_NONFINITE;
* with the sponge layer on the background (Navier-Stokes, six points deep, strength 2) the same
  right-hand-side and MRAB bars, and a depth beyond 16 refused."""
import numpy as np
import pytest

import workloads as W
from conftest import build_library
from oracle.curvpair import OracleCurvPair
from tolerances import U32, U64, fp32_rhs_tol_curv, increment_tol, rel, viscous_flux_rounding_curv

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

_CACHE = {}


@pytest.fixture(scope="module")
def sbp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build_library()
    import paper_1805_06607_gb300 as mod
    return mod


def case(phys):
    if phys not in _CACHE:
        if phys == "ns_sponge":
            wl = W.curvilinear_pair(seed=3, physics="ns", sponge_cells=6, sponge_strength=2.0)
        else:
            wl = W.curvilinear_pair(seed=3, physics=phys)
        _CACHE[phys] = (wl, OracleCurvPair(wl))
    return _CACHE[phys]


@pytest.mark.parametrize("phys", ["euler", "ns"])
def test_tables(sbp, phys):
    wl, o = case(phys)
    g = sbp.CurvilinearPair(wl)
    assert g.info[0].n_holes == int((o.iblank[0] == 0).sum()) > 100
    for k in range(2):
        t = g.tables(k)
        assert np.array_equal(t["iblank"] != 0, o.iblank[k] != 0), k
        assert np.array_equal(t["receivers"], o.recv_pts[k]), k
        assert np.array_equal(t["base"], o.base[k]), k
        assert np.abs(t["w"] - o.w[k]).max() < 1e-13, k
    g.close()


@pytest.mark.parametrize("phys", ["euler", "ns", "ns_sponge"])
def test_rhs_and_donor_values(sbp, phys):
    wl, o = case(phys)
    q = wl["q0"]
    mu = wl["params"]["mu"]
    for dtype in ("f64", "f32"):
        g = sbp.CurvilinearPair(wl, dtype=dtype)
        qd = [g.to_device(k, q[k]) for k in range(2)]
        for k in range(2):
            act = o.iblank[k] != 0
            want = o.coupled_rhs(k, q[k], q[1 - k])
            got = g.to_host(k, g.rhs_eval(k, qd[k], qd[1 - k]))
            tol = fp32_rhs_tol_curv(q[k], o.ops[k], act, want, mu, unit=U32 if dtype == "f32" else U64)
            tol = tol if dtype == "f32" else max(1e-12, tol)
            assert rel(got[:, act], want[:, act]) < tol, (dtype, k, rel(got[:, act], want[:, act]), tol)
            assert np.all(got[:, ~act] == 0.0)
            if dtype == "f64":
                qh, fh = g.overset_interp(k, qd[1 - k])
                assert rel(qh.cpu().numpy(), o.interp(k, q[1 - k])) < 1e-12, k
                if phys != "euler":
                    # the donor mesh's viscous fluxes are small where its stream is nearly
                    # uniform: 1e-12 relative, or their derived absolute rounding
                    fw = o.interp(k, o.viscflux(1 - k, q[1 - k]))
                    floor = viscous_flux_rounding_curv(q[1 - k], o.ops[1 - k], o.iblank[1 - k] != 0, mu)
                    err = np.abs(fh.cpu().numpy() - fw).max()
                    assert err < 1e-12 * np.abs(fw).max() + floor, (k, err, floor, np.abs(fw).max())
        g.close()


def test_timestep(sbp):
    wl, o = case("ns")
    g = sbp.CurvilinearPair(wl)
    q = [g.to_device(k, wl["q0"][k]) for k in range(2)]
    dts, H = g.timestep(q[0], q[1])
    for k in range(2):
        want = o.dt_mesh(k, wl["q0"][k])
        assert abs(dts[k] - want) < 1e-13 * want, (k, dts[k], want)
    assert abs(H - o.macro_step_size(wl["q0"])) < 1e-13 * H
    g.close()


@pytest.mark.parametrize("phys", ["euler", "ns", "ns_sponge"])
def test_mrab(sbp, phys):
    """Bootstrap + 3 macro steps: increments over the 3 macro steps, each side from its own
    start."""
    wl, o = case(phys)
    q0 = wl["q0"]
    mu = wl["params"]["mu"]
    H = o.macro_step_size(q0)
    n = 3
    y, hf, hs = o.bootstrap(q0, H)
    want, _, _ = o.mrab(y, hf, hs, H, n)
    sr = wl["params"]["step_ratio"]
    bars = {u: max(fp32_rhs_tol_curv(q0[j], o.ops[j], o.iblank[j] != 0, o.coupled_rhs(j, q0[j], q0[1 - j]), mu,
                                     unit=u) for j in range(2)) for u in (U32, U64)}
    fp64_bar = max(1e-12, bars[U64])
    for dtype in ("f64", "f32"):
        g = sbp.CurvilinearPair(wl, dtype=dtype)
        g.bind(q0)
        g.mrab_init(H)
        start = [g.to_host(k, g.current_state(k)) for k in range(2)]
        g.mrab_step(n)
        g.check()
        assert g.mrab_time() == (H, pytest.approx(n * H))
        for k in range(2):
            act = o.iblank[k] != 0
            got = g.to_host(k, g.current_state(k))
            if dtype == "f64":
                assert rel(start[k][:, act] - q0[k][:, act], y[k][:, act] - q0[k][:, act]) < fp64_bar, k
            ei = rel(got[:, act] - start[k][:, act], want[k][:, act] - y[k][:, act])
            itol = increment_tol(fp64_bar if dtype == "f64" else bars[U32], y[k][:, act], want[k][:, act], n * sr,
                                 U64 if dtype == "f64" else U32)
            assert ei < itol, (dtype, k, ei, itol)
        g.close()


def test_nonfinite_state_reported(sbp):
    wl, o = case("euler")
    q = [np.array(x) for x in wl["q0"]]
    q[1][4, 12, 12, 12] = np.nan
    g = sbp.CurvilinearPair(wl)
    g.bind(q)
    g.mrab_init(o.macro_step_size(wl["q0"]))
    g.mrab_step(1)
    with pytest.raises(sbp.SbpError) as e:
        g.check()
    assert e.value.status == -5
    g.close()


def test_sponge_changes_the_background_and_bad_depth_is_refused(sbp):
    wl, o = case("ns_sponge")
    wl0, _ = case("ns")
    g, g0 = sbp.CurvilinearPair(wl), sbp.CurvilinearPair(wl0)
    q = [g.to_device(k, wl["q0"][k]) for k in range(2)]
    r = [g.to_host(k, g.rhs_eval(k, q[k], q[1 - k])) for k in range(2)]
    r0 = [g0.to_host(k, g0.rhs_eval(k, q[k], q[1 - k])) for k in range(2)]
    sig = o.sponge_strength(0)
    qinf = np.asarray(wl["params"]["qinf"])
    want = -sig[None] * (wl["q0"][0] - qinf[:, None, None, None])
    assert np.abs((r[0] - r0[0]) - want).max() <= 1e-12 * np.abs(r0[0]).max()
    assert np.array_equal(r[1], r0[1])
    g.close()
    g0.close()
    bad = dict(wl, params=dict(wl["params"], sponge_cells=17))
    with pytest.raises(sbp.SbpError):
        sbp.CurvilinearPair(bad)
