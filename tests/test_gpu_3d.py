"""3D Cartesian GPU path against the 3D oracle through the C ABI (sbp3_*).

FP64: setup tables exact (hole cut, receivers) or to rounding (donor weights), right-hand side,
interpolation and whole MRAB runs to 1e-12 relative L2 (states and increments); FP32 state with
FP64 update arithmetic within 1e-5 of the FP64 oracle after the bootstrap and several macro
steps, its increments within the derived FP32 bound."""
import numpy as np
import pytest

import workloads as W
from conftest import build_library
from oracle import OracleSystem3D
from tolerances import U32, U64, fp32_rhs_tol_3d, increment_tol, rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sbp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build_library()
    import paper_1805_06607_gb300 as mod
    return mod


_rel = rel


def _sponge_vortex_y():
    """The vortex pair with far-field background faces and a sponge six points deep, extruded
    along y (the far-field faces along i and k)."""
    wl = W.vortex_box_in_box(seed=45, n_bg=40, n_fine=25)
    bg = wl["meshes"][0]
    far = W.cartesian_mesh("background", bg["n"], bg["lo"], bg["h"], ("farfield",) * 4)
    wl = dict(wl, meshes=[far, wl["meshes"][1]], params=dict(wl["params"], sponge_cells=6, sponge_strength=2.0))
    return W.extrude_to_3d(wl, 8, 8 * bg["h"][0], axis=1)


CASES = {
    "tg_ns": (lambda: W.taylor_green_small(seed=41), 4),
    "extruded_y_sponge": (_sponge_vortex_y, 2.5),
    "tg_euler": (lambda: W.taylor_green_small(seed=42, physics="euler", n_bg=20, n_fine=17), 4),
    "tg_sr3_ab34": (lambda: W.taylor_green_small(seed=43, step_ratio=3, hist_len=4, n_bg=20, n_fine=19), 4),
    "extruded_z_vortex": (lambda: W.extrude_to_3d(W.vortex_box_in_box(seed=44, n_bg=40, n_fine=25), 8, 2.0, axis=2),
                          2.5),
    "extruded_y_mms": (lambda: W.extrude_to_3d(W.mms_box_in_box(40, "viscous"), 8, 0.4, axis=1), 3.7),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_setup_tables_3d(sbp, case):
    mk, hc = CASES[case]
    wl = mk()
    o = OracleSystem3D(wl, hole_cells=hc)
    g = sbp.System3D(wl, hole_cells=hc)
    for k in range(2):
        t = g.tables(k)
        assert np.array_equal(t["iblank"], o.iblank[k])
        assert np.array_equal(t["receivers"], o.recv_pts[k])
        if o.recv_pts[k].size:
            assert np.array_equal(t["base"], o.base[k])
            assert np.abs(t["w"] - o.w[k]).max() < 1e-13


@pytest.mark.parametrize("case", sorted(CASES))
def test_rhs_and_interp_3d_fp64(sbp, case):
    mk, hc = CASES[case]
    wl = mk()
    o = OracleSystem3D(wl, hole_cells=hc)
    g = sbp.System3D(wl, hole_cells=hc)
    q = [g.to_device(k, wl["q0"][k]) for k in range(2)]
    for k in range(2):
        got = g.to_host(k, g.rhs_eval(k, q[k], q[1 - k]))
        want = o.coupled_rhs(k, wl["q0"][k], wl["q0"][1 - k])
        act = o.iblank[k] != 0
        assert _rel(got[:, act], want[:, act]) < 1e-12, k
        assert np.abs(got[:, ~act]).max(initial=0.0) == 0.0
        nr = o.recv_pts[k].size
        if nr:
            qh, fh = g.overset_interp(k, q[1 - k])
            assert _rel(qh.cpu().numpy(), o.interp(k, wl["q0"][1 - k])) < 1e-13
            if o.viscous:
                assert _rel(fh.cpu().numpy(), o.interp(k, o.viscflux(1 - k, wl["q0"][1 - k]))) < 1e-12


@pytest.mark.parametrize("case", ["tg_ns", "tg_sr3_ab34", "extruded_y_mms", "extruded_y_sponge"])
def test_mrab_3d(sbp, case):
    """Bootstrap + 3 macro steps against the oracle: the states (FP64 1e-12, FP32 1e-5) and the
    increments over the 3 macro steps, each side from its own start (FP64 1e-12; FP32 the
    derived FP32 right-hand-side bound), with the stored state's rounding floor added."""
    mk, hc = CASES[case]
    wl = mk()
    o = OracleSystem3D(wl, hole_cells=hc)
    H = o.macro_step_size(wl["q0"])
    n = 3
    y, hf, hs = o.bootstrap(wl["q0"], H)
    want, _, _ = o.mrab(y, hf, hs, H, n)
    sr = wl["params"]["step_ratio"]
    q0 = wl["q0"]
    fp32_bar = max(fp32_rhs_tol_3d(q0[j], wl["meshes"][j]["h"], o.iblank[j] != 0,
                                   o.coupled_rhs(j, q0[j], q0[1 - j])) for j in range(2))
    for dtype, tol in (("f64", 1e-12), ("f32", 1e-5)):
        g = sbp.System3D(wl, dtype=dtype, hole_cells=hc)
        g.bind(wl["q0"])
        g.mrab_init(H)
        start = [g.to_host(k, g.current_state(k)) for k in range(2)]
        g.mrab_step(n)
        g.check()
        for k in range(2):
            got = g.to_host(k, g.current_state(k))
            act = o.iblank[k] != 0
            err = _rel(got[:, act], want[k][:, act])
            assert err < tol, (dtype, k, err)
            ei = _rel(got[:, act] - start[k][:, act], want[k][:, act] - y[k][:, act])
            itol = increment_tol(1e-12 if dtype == "f64" else fp32_bar, y[k][:, act], want[k][:, act], n * sr,
                                 U64 if dtype == "f64" else U32)
            assert ei < itol, (dtype, k, ei, itol)
        g.close()


def test_timestep_3d(sbp):
    wl = W.taylor_green_small(seed=45)
    o = OracleSystem3D(wl)
    g = sbp.System3D(wl)
    q = [g.to_device(k, wl["q0"][k]) for k in range(2)]
    dts, H = g.timestep(q[0], q[1])
    for k in range(2):
        assert abs(dts[k] - o.dt_mesh(k, wl["q0"][k])) < 1e-13 * dts[k]
    assert abs(H - o.macro_step_size(wl["q0"])) < 1e-13 * H


def _designs_run(sbp, wl, hc, dtype, kchunk, steps):
    g = sbp.System3D(wl, dtype=dtype, hole_cells=hc)
    for k in range(2):
        g.set_rhs_kernel(k, kchunk)
    q = [g.to_device(k, wl["q0"][k]) for k in range(2)]
    rhs = [g.to_host(k, g.rhs_eval(k, q[k], q[1 - k])) for k in range(2)]
    states = None
    if steps:
        g.bind(wl["q0"])
        g.mrab_init()
        g.mrab_step(steps)
        states = [g.to_host(k, g.current_state(k)) for k in range(2)]
    g.check()
    g.close()
    return rhs, states


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("case", sorted(CASES))
def test_rhs_designs_3d_bit_identical(sbp, case, dtype):
    """The k-marching right-hand side (chunks of 5 planes with a ragged last chunk, and of 32) and
    the per-point kernels give the same bits: right-hand sides and states after MRAB steps."""
    mk, hc = CASES[case]
    wl = mk()
    ref_rhs, ref_q = _designs_run(sbp, wl, hc, dtype, 0, 2)
    for kc in (5, 32):
        rhs, qs = _designs_run(sbp, wl, hc, dtype, kc, 2)
        for k in range(2):
            assert np.array_equal(rhs[k], ref_rhs[k]), (kc, k)
            assert np.array_equal(qs[k], ref_q[k]), (kc, k)


def test_rhs_designs_3d_full_size_fp32(sbp):
    """At the Taylor-Green workload's full size (256^3 background + 192^3 box, FP32) the
    marching right-hand side of both meshes equals the per-point kernels' bit for bit; the
    per-point kernels are the ones checked against the oracle above."""
    wl = W.taylor_green_box(seed=3)
    a, _ = _designs_run(sbp, wl, 4, "f32", 32, 0)
    b, _ = _designs_run(sbp, wl, 4, "f32", 0, 0)
    for k in range(2):
        assert np.isfinite(a[k]).all()
        assert np.array_equal(a[k], b[k]), k
