"""GPU path against the oracle, element by element, through the C ABI.

FP64 bar: 1e-12 relative L2 (setup tables bit-exact where the computation is integer or
follows the same operation order); time steps are compared on their increments (the state at
the end minus the state at the start of the tested steps, on each side), with the stored
state's own rounding added where it is a larger fraction of the increment. FP32: states after
time steps within 1e-5 relative L2 of the FP64 oracle's; right-hand sides and increments within
the bound derived from FP32 rounding and the cancellation in the flux differences
(tests/tolerances.py)."""
import numpy as np
import pytest

import workloads as W
from conftest import build_library
from oracle import OracleSystem
from tolerances import U32, U64, fp32_rhs_tol, increment_tol, rel, rel_increment

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sbp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build_library()
    import paper_1805_06607_gb300 as mod
    return mod


def _omega(wl, omega):
    wl["params"]["omega_corner"] = omega
    return wl


CASES = {
    "vortex": lambda: W.vortex_box_in_box(seed=11),
    "vortex_sr3_ab34": lambda: W.vortex_box_in_box(seed=12, n_bg=48, n_fine=33, step_ratio=3, hist_len=4),
    "vortex_sr1": lambda: W.vortex_box_in_box(seed=13, n_bg=40, n_fine=25, step_ratio=1),
    "cylinder": lambda: W.cylinder_small(seed=14),
    "cylinder_ab34": lambda: W.cylinder_small(seed=15, n_theta=72, n_r=20, bg_n=(90, 50), hist_len=4),
    "mms_viscous": lambda: W.mms_box_in_box(52, "viscous"),
    # far-field sponge layer six points deep (Sec. 5.1)
    "cylinder_sponge": lambda: W.cylinder_small(seed=20, sponge_cells=6, sponge_strength=2.0),
    # corner interface points weighted by Omega = 1/2 (Sec. 4.2 eq. (penalty_interp))
    "vortex_omega": lambda: _omega(W.vortex_box_in_box(seed=21, n_bg=48, n_fine=33), 0.5),
}

# The extended-history Adams-Bashforth family of Sec. 3.2 inside MRAB (order n, history m:
# ABnm), on small geometries: the interface and operator paths are those of CASES.
AB_CASES = {
    "vortex_ab45": lambda: W.vortex_box_in_box(seed=16, n_bg=40, n_fine=25, step_ratio=2, order=4, hist_len=5),
    "vortex_ab35_sr3": lambda: W.vortex_box_in_box(seed=17, n_bg=40, n_fine=25, step_ratio=3, order=3, hist_len=5),
    "vortex_ab44_sr4": lambda: W.vortex_box_in_box(seed=18, n_bg=40, n_fine=25, step_ratio=4, order=4, hist_len=4),
    "cylinder_ab46": lambda: W.cylinder_small(seed=19, n_theta=72, n_r=20, bg_n=(90, 50), order=4, hist_len=6,
                                              step_ratio=2),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_setup_tables(sbp, case):
    wl = CASES[case]()
    ref = OracleSystem(wl)
    g = sbp.System(wl)
    for k, m in enumerate(wl["meshes"]):
        t = g.tables(k)
        assert np.array_equal(t["iblank"], ref.iblank[k]), "hole cut differs"
        assert np.array_equal(t["receivers"], ref.recv_pts[k]), "receiver set differs"
        ni, nj = wl["meshes"][1 - k]["n"]
        nr = ref.recv_pts[k].size
        if nr:
            # the donor coordinates are unique; the stencil start is not when a receiver sits on
            # a donor node (both 4-point stencils then interpolate the same value)
            lin = np.arange(4.0)
            s_got = t["base"][:, 0] + t["w"][:, :4] @ lin
            r_got = t["base"][:, 1] + t["w"][:, 4:] @ lin
            ds = (s_got - ref.xe[k][:, 0] + ni / 2) % ni - ni / 2
            dr = (r_got - ref.xe[k][:, 1] + nj / 2) % nj - nj / 2
            assert np.abs(ds).max() < 1e-10 and np.abs(dr).max() < 1e-10
            same = np.all((t["base"] - ref.base[k]) % [ni, nj] == 0, axis=1)
            assert same.mean() > 0.5
            assert np.abs(t["w"][same] - ref.w[k][same]).max() < 1e-12
            node = ~same
            assert np.all(np.minimum(np.abs(ds[node] + ref.xe[k][node, 0] - np.round(ref.xe[k][node, 0])),
                                     np.abs(dr[node] + ref.xe[k][node, 1] - np.round(ref.xe[k][node, 1]))) < 1e-9)
        act = ref.iblank[k] != 0
        for c in range(5):
            a, b = t["metrics"][c][act], ref.met[k][c][act]
            assert np.array_equal(a, b) or rel(a, b) < 1e-15, ("metric", c)
    g.close()


@pytest.mark.parametrize("case", sorted(CASES))
def test_interp_and_rhs_fp64(sbp, case):
    wl = CASES[case]()
    ref = OracleSystem(wl)
    g = sbp.System(wl)
    qd = [g.to_device(k, wl["q0"][k]) for k in range(2)]
    for k in range(2):
        qhat, fvhat = g.overset_interp(k, qd[1 - k])
        want = ref.interp(k, wl["q0"][1 - k])
        assert rel(qhat.cpu().numpy(), want) < 1e-13
        if ref.viscous:
            want_fv = ref.interp(k, ref.viscflux(1 - k, wl["q0"][1 - k]))
            assert rel(fvhat.cpu().numpy(), want_fv) < 1e-12
        got = g.to_host(k, g.rhs_eval(k, qd[k], qd[1 - k]))
        want = ref.coupled_rhs(k, wl["q0"][k], wl["q0"][1 - k])
        assert rel(got, want) < 1e-12, (k, rel(got, want))
        assert np.all(got[:, ref.iblank[k] == 0] == 0.0)
    g.close()


@pytest.mark.parametrize("case", ["vortex", "cylinder", "vortex_sr3_ab34", "cylinder_ab34", "vortex_sr1",
                                  "cylinder_sponge", "vortex_omega"] + sorted(AB_CASES))
def test_mrab_fp64(sbp, case):
    wl = {**CASES, **AB_CASES}[case]()
    ref = OracleSystem(wl)
    g = sbp.System(wl)
    qd = [g.to_device(k, wl["q0"][k]) for k in range(2)]
    dts, H = g.timestep(qd[0], qd[1])
    H_ref = ref.macro_step_size(wl["q0"])
    assert abs(H - H_ref) <= 1e-14 * H_ref
    for k in range(2):
        want = ref.dt_mesh(k, wl["q0"][k])
        assert abs(dts[k] - want) <= 1e-14 * want
    y, hf, hs = ref.bootstrap(wl["q0"], H_ref)
    g.bind(wl["q0"])
    g.mrab_init()
    sr, m = wl["params"]["step_ratio"], wl["params"]["hist_len"]
    start = []
    for k in range(2):
        got = g.to_host(k, g.current_state(k))
        tol = increment_tol(1e-12, wl["q0"][k], y[k], (m - 1) * sr, U64)
        assert rel_increment(got, y[k], wl["q0"][k]) < tol, "bootstrap increment"
        start.append(got)
    nsteps = 3
    want, _, _ = ref.mrab(y, hf, hs, H_ref, nsteps)
    g.mrab_step(nsteps)
    g.check()
    for k in range(2):
        got = g.to_host(k, g.current_state(k))
        assert rel(got, want[k]) < 1e-12, (k, rel(got, want[k]))
        # the increment over the tested steps, each side from its own start
        e = rel(got - start[k], want[k] - y[k])
        tol = increment_tol(1e-12, y[k], want[k], nsteps * sr, U64)
        assert e < tol, (k, e, tol)
    Hg, t = g.mrab_time()
    assert t == pytest.approx(nsteps * Hg)
    g.close()


@pytest.mark.parametrize("case", ["cylinder", "vortex_sr3_ab34"])
def test_graph_replay_matches_eager(sbp, case):
    """CUDA-graph macro steps (slow RHS and first micro step on parallel branches) give the
    same states as kernel-by-kernel launches, over more steps than the ring/buffer period."""
    wl = CASES[case]()
    out = []
    for graphs in (False, True):
        g = sbp.System(wl)
        g.use_graphs(graphs)
        g.bind(wl["q0"])
        g.mrab_init()
        g.mrab_step(7)
        g.check()
        out.append([g.to_host(k, g.current_state(k)) for k in range(2)])
        g.close()
    for k in range(2):
        assert np.array_equal(out[0][k], out[1][k])


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_graph_replay_matches_eager_full_size(sbp, dtype):
    """On the full-size cylinder the captured macro step also splits the slow right-hand side:
    the tiles around the fast receivers' donor points first, the rest of the background beside
    the fast micro steps. The states stay bit-identical to kernel-by-kernel launches."""
    wl = W.cylinder_overset(seed=3)
    out = []
    for graphs in (False, True):
        g = sbp.System(wl, dtype=dtype)
        g.use_graphs(graphs)
        g.bind(wl["q0"])
        g.mrab_init()
        g.mrab_step(8)
        g.check()
        out.append([g.to_host(k, g.current_state(k)) for k in range(2)])
        # donor values 3, the O-grid's 4 micro steps 2 each, the background's right-hand side 2 x 2
        assert g.graph_launches() == (15 if graphs else 0)
        g.close()
    for k in range(2):
        assert np.array_equal(out[0][k], out[1][k])


def test_zero_steps_is_noop(sbp):
    wl = CASES["vortex_sr1"]()
    g = sbp.System(wl)
    g.bind(wl["q0"])
    g.mrab_init()
    before = [g.to_host(k, g.current_state(k)) for k in range(2)]
    g.mrab_step(0)
    for k in range(2):
        assert np.array_equal(g.to_host(k, g.current_state(k)), before[k])
    g.close()


def test_sponge_changes_the_state_and_is_refused_by_the_adjoint(sbp):
    wl = CASES["cylinder_sponge"]()
    wl0 = W.cylinder_small(seed=20)
    g, g0 = sbp.System(wl), sbp.System(wl0)
    qd = [g.to_device(k, wl["q0"][k]) for k in range(2)]
    r = g.to_host(0, g.rhs_eval(0, qd[0], qd[1]))
    r0 = g0.to_host(0, g0.rhs_eval(0, qd[0], qd[1]))
    assert rel(r, r0) > 1e-3
    lam = torch.zeros_like(qd[0])
    with pytest.raises(sbp.SbpError):
        g.rhs_eval_vjp(0, qd[0], qd[1], lam)
    g.close()
    g0.close()


@pytest.mark.parametrize("case", ["vortex", "cylinder", "cylinder_sponge", "vortex_omega"])
def test_fp32(sbp, case):
    """FP32 state and right-hand side with FP64 MRAB accumulation, against the FP64 oracle."""
    wl = CASES[case]()
    ref = OracleSystem(wl)
    g = sbp.System(wl, dtype="f32")
    qd = [g.to_device(k, wl["q0"][k]) for k in range(2)]
    rhs_tol = []
    for k in range(2):
        act = ref.iblank[k] != 0
        got = g.to_host(k, g.rhs_eval(k, qd[k], qd[1 - k]))
        want = ref.coupled_rhs(k, wl["q0"][k], wl["q0"][1 - k])
        tol = fp32_rhs_tol(ref.met[k], wl["q0"][k], act, want, ref.mu, ref.pr)
        e = rel(got[:, act], want[:, act])
        print("fp32 rhs", case, k, "error %.3e bound %.3e" % (e, tol))
        assert e < tol, (k, e, tol)
        rhs_tol.append(tol)
    H_ref = ref.macro_step_size(wl["q0"])
    y, hf, hs = ref.bootstrap(wl["q0"], H_ref)
    nsteps = 3
    want, _, _ = ref.mrab(y, hf, hs, H_ref, nsteps)
    g.bind(wl["q0"])
    g.mrab_init()
    start = [g.to_host(k, g.current_state(k)) for k in range(2)]
    g.mrab_step(nsteps)
    g.check()
    sr = wl["params"]["step_ratio"]
    for k in range(2):
        act = ref.iblank[k] != 0
        got = g.to_host(k, g.current_state(k))
        e = rel(got[:, act], want[k][:, act])
        assert e < 1e-5, (k, e)
        # the increment is as accurate as the FP32 right-hand sides it integrates
        ei = rel(got[:, act] - start[k][:, act], want[k][:, act] - y[k][:, act])
        tol = increment_tol(max(rhs_tol), y[k][:, act], want[k][:, act], nsteps * sr, U32)
        print("fp32 increment", case, k, "error %.3e bound %.3e" % (ei, tol))
        assert ei < tol, (k, ei, tol)
    g.close()


def test_full_size_cylinder_rhs(sbp):
    """The benchmark's workload at full size (O-grid 512x128, background 1024x512): FP64 within
    1e-12, FP32 within its derived bound."""
    wl = W.cylinder_overset(seed=0)
    ref = OracleSystem(wl)
    want = [ref.coupled_rhs(k, wl["q0"][k], wl["q0"][1 - k]) for k in range(2)]
    for dtype in ("f64", "f32"):
        g = sbp.System(wl, dtype=dtype)
        qd = [g.to_device(k, wl["q0"][k]) for k in range(2)]
        for k in range(2):
            act = ref.iblank[k] != 0
            got = g.to_host(k, g.rhs_eval(k, qd[k], qd[1 - k]))
            tol = 1e-12 if dtype == "f64" else fp32_rhs_tol(ref.met[k], wl["q0"][k], act, want[k],
                                                                 ref.mu, ref.pr)
            e = rel(got[:, act], want[k][:, act])
            print("full-size rhs", dtype, k, "error %.3e bound %.3e" % (e, tol))
            assert e < tol, (dtype, k, e, tol)
        g.close()


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_full_size_cylinder_mrab(sbp, dtype, tol):
    """The benchmark's step at full size and in its launch configuration (autotuned kernel
    shapes, CUDA-graph macro steps): the Runge-Kutta bootstrap and two MRAB macro steps against
    the oracle's, on the states and on the increments over the two macro steps. In FP32 the
    background's increment over two macro steps (4e-7 of the state) is below the FP32 state's
    own rounding, so only the O-grid's increment is compared there; the full-size FP32
    right-hand side is checked in test_full_size_cylinder_rhs."""
    wl = W.cylinder_overset(seed=1)
    ref = OracleSystem(wl)
    H = ref.macro_step_size(wl["q0"])
    y, hf, hs = ref.bootstrap(wl["q0"], H)
    want, _, _ = ref.mrab(y, hf, hs, H, 2)
    g = sbp.System(wl, dtype=dtype)
    g.bind(wl["q0"])
    g.mrab_init()
    start = [g.to_host(k, g.current_state(k)) for k in range(2)]
    g.mrab_step(2)
    g.check()
    sr = wl["params"]["step_ratio"]
    for k in range(2):
        act = ref.iblank[k] != 0
        got = g.to_host(k, g.current_state(k))
        e = rel(got[:, act], want[k][:, act])
        assert e < tol, (dtype, k, e)
        if dtype == "f32" and k == 0:
            continue
        bar = tol if dtype == "f64" else fp32_rhs_tol(ref.met[k], y[k], act, hs[-1] if k == ref.slow else hf[-1],
                                                              ref.mu, ref.pr)
        itol = increment_tol(bar, y[k][:, act], want[k][:, act], 2 * sr, U64 if dtype == "f64" else U32)
        ei = rel(got[:, act] - start[k][:, act], want[k][:, act] - y[k][:, act])
        print("full-size increment", dtype, k, "error %.3e bound %.3e" % (ei, itol))
        assert ei < itol, (dtype, k, ei, itol)
    g.close()


@pytest.mark.parametrize("n", [(7, 40), (40, 7), (65536, 8), (8, 65536)])
def test_mesh_size_limits_rejected(sbp, n):
    """Meshes below the closures' 8 points or above the 16-bit point tables' 65535 points per
    direction are refused at creation (the fine patch is the same small one every time)."""
    bg = W.cartesian_mesh("background", n, (-1.0, -1.0), (2.0 / n[0], 2.0 / n[1]), ("farfield",) * 4)
    fine = W.cartesian_mesh("fine", (25, 25), (-0.2, -0.2), (0.4 / 24, 0.4 / 24), ("interface",) * 4)
    wl = W.vortex_box_in_box(seed=1, n_bg=40, n_fine=25)
    wl = dict(wl, meshes=[bg, fine], q0=[np.ones((4, n[1], n[0])), np.ones((4, 25, 25))])
    with pytest.raises(sbp.SbpError):
        sbp.System(wl)
