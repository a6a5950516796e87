"""Discrete adjoint (FP64) through the C ABI.

- Tangent of the right-hand side (sbp_rhs_eval_jvp) against central differences of the GPU
  right-hand side; vector-Jacobian products (sbp_rhs_eval_vjp, sbp_overset_interp_vjp)
  against the tangent by the dot-product identity <w, J v> = <J^T w, v> (to 1e-12: the two
  share only point-wise formulas, the stencils enter forward in one and transposed in the
  other).
- The probe objective's forward equals the library's own MRAB run (sbp_mrab_init +
  sbp_mrab_step) and the oracle's; its gradient w.r.t. the initial states and the far-field
  Mach number matches central differences (h = 1e-6) of the GPU forward and of the oracle
  forward within 1e-6 relative.
- Checkpoint schedules change the recomputation count, never the bits of the gradient.
"""
import numpy as np
import pytest

import workloads as W
from conftest import build_library
from oracle import OracleSystem
from oracle.system import probe_objective, probe_pressure, probe_stencil

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sbp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build_library()
    import paper_1805_06607_gb300 as mod
    return mod


RHS_CASES = {
    "cylinder_ns": lambda: W.cylinder_small(seed=21),
    "vortex_euler": lambda: W.vortex_box_in_box(seed=22, n_bg=40, n_fine=25),
    "mms_viscous": lambda: W.mms_box_in_box(40, "viscous"),
}


def _rand_state(g, k, rng, scale=1.0):
    inf = g.info[k]
    v = rng.standard_normal((4, inf.nj, inf.ni)) * scale
    return g.to_device(k, v)


def _dot(a, b):
    return float((a * b).sum())


def _active(g, k):
    ib = torch.from_numpy(g.tables(k)["iblank"].astype(np.float64)).cuda()
    inf = g.info[k]
    m = torch.zeros((inf.nj, inf.pitch), dtype=torch.float64, device="cuda")
    m[:, :inf.ni] = ib
    return m


@pytest.mark.parametrize("case", sorted(RHS_CASES))
@pytest.mark.parametrize("k", [0, 1])
def test_rhs_jvp_matches_central_differences(sbp, case, k):
    wl = RHS_CASES[case]()
    g = sbp.System(wl)
    rng = np.random.default_rng(31 + k)
    q = [g.to_device(m, wl["q0"][m]) for m in range(2)]
    v = [_rand_state(g, m, rng, 1e-2) for m in range(2)]
    dqinf = rng.standard_normal(4) * 1e-2
    qinf = np.asarray(wl["params"]["qinf"], dtype=np.float64)
    tan = g.rhs_eval_jvp(k, q[k], q[1 - k], v[k], v[1 - k], dqinf)
    eps = 1e-6
    g.set_freestream(qinf + eps * dqinf)
    rp = g.rhs_eval(k, q[k] + eps * v[k], q[1 - k] + eps * v[1 - k]).clone()
    g.set_freestream(qinf - eps * dqinf)
    rm = g.rhs_eval(k, q[k] - eps * v[k], q[1 - k] - eps * v[1 - k]).clone()
    g.set_freestream(qinf)
    fd = (rp - rm) / (2 * eps)
    act = _active(g, k)
    err = float(((tan - fd) * act).norm() / (fd * act).norm())
    assert err < 1e-6, err
    assert float((tan * (1 - act)).abs().max()) == 0.0


@pytest.mark.parametrize("case", sorted(RHS_CASES))
@pytest.mark.parametrize("k", [0, 1])
def test_rhs_vjp_dot_product(sbp, case, k):
    wl = RHS_CASES[case]()
    g = sbp.System(wl)
    rng = np.random.default_rng(41 + k)
    q = [g.to_device(m, wl["q0"][m]) for m in range(2)]
    v = [_rand_state(g, m, rng) for m in range(2)]
    dqinf = rng.standard_normal(4)
    w = _rand_state(g, k, rng) * _active(g, k)
    jv = g.rhs_eval_jvp(k, q[k], q[1 - k], v[k], v[1 - k], dqinf)
    ls, lo, lqinf = g.rhs_eval_vjp(k, q[k], q[1 - k], w)
    lhs = _dot(w, jv)
    rhs = _dot(ls, v[k]) + _dot(lo, v[1 - k]) + float(lqinf @ dqinf)
    scale = float(w.norm() * jv.norm())
    assert abs(lhs - rhs) <= 1e-12 * scale, (lhs, rhs, scale)
    # deterministic: a second call gives the same bits
    ls2, lo2, lqinf2 = g.rhs_eval_vjp(k, q[k], q[1 - k], w)
    assert torch.equal(ls, ls2) and torch.equal(lo, lo2) and np.array_equal(lqinf, lqinf2)


@pytest.mark.parametrize("case", sorted(RHS_CASES))
@pytest.mark.parametrize("recv", [0, 1])
def test_interp_vjp(sbp, case, recv):
    wl = RHS_CASES[case]()
    g = sbp.System(wl)
    nr = g.info[recv].n_receivers
    if nr == 0:
        pytest.skip("no receivers")
    rng = np.random.default_rng(51 + recv)
    don = 1 - recv
    qd = g.to_device(don, wl["q0"][don])
    v = _rand_state(g, don, rng, 1e-2)
    lq = torch.from_numpy(rng.standard_normal((4, nr))).cuda()
    # the state part is linear: exact dot-product identity
    iv, _ = g.overset_interp(recv, v, viscous_fluxes=False)
    back = g.overset_interp_vjp(recv, qd, lq)
    assert abs(_dot(lq, iv) - _dot(back, v)) <= 1e-13 * float(lq.norm() * iv.norm())
    if wl["params"]["physics"] == "ns":
        lfv = torch.from_numpy(rng.standard_normal((6, nr))).cuda()
        eps = 1e-6
        qp, fp = g.overset_interp(recv, qd + eps * v)
        qp, fp = qp.clone(), fp.clone()
        qm, fm = g.overset_interp(recv, qd - eps * v)
        lin = (_dot(lq, qp - qm) + _dot(lfv, fp - fm)) / (2 * eps)
        back = g.overset_interp_vjp(recv, qd, lq, lfv)
        assert abs(lin - _dot(back, v)) <= 1e-6 * abs(lin)


# ---------------------------------------------------------------------------------------------
def _probe_case(seed=61, **kw):
    """Small cylinder with 6 wake probes and 2 probes half a unit inside the far-field faces
    (so that the far-field state reaches the objective within a few steps)."""
    wl = W.cylinder_small(seed=seed, **kw)
    bg = wl["meshes"][0]
    hi = [bg["lo"][d] + (bg["n"][d] - 1) * bg["h"][d] for d in range(2)]
    probes = np.vstack([W.wake_probes(seed, 6), [[hi[0] - 0.5, 0.0], [0.3, hi[1] - 0.5]]])
    return wl, probes


def _q0(g, wl):
    return [g.to_device(k, wl["q0"][k]) for k in range(2)]


def test_probe_forward_matches_library_run_and_oracle(sbp):
    wl, probes = _probe_case()
    g = sbp.System(wl)
    q0 = _q0(g, wl)
    _, H = g.timestep(q0[0], q0[1])
    n = 6
    r = g.adjoint_probe(q0, probes, n, H, grad=False)
    assert r["forward_steps"] == n
    # the library's own run (graphs), pressures read back on the host
    g.bind(wl["q0"])
    g.mrab_init(H)
    st = [probe_stencil(wl["meshes"][0], xy) for xy in probes]
    pr = np.zeros((n, len(probes)))
    for i in range(n):
        g.mrab_step(1)
        qb = g.to_host(0, g.current_state(0))
        pr[i] = [probe_pressure(wl["meshes"][0], qb, s, 1.4) for s in st]
    assert np.abs(r["p"] - pr).max() < 1e-13
    Jo, po = probe_objective(OracleSystem(wl), wl["q0"], probes, n, H)
    assert np.abs(r["p"] - po).max() < 1e-11
    assert abs(r["J"] - Jo) < 1e-11 * Jo


def _fd_J(g, q0, probes, n, H, dirs, h):
    jp = g.adjoint_probe([q0[k] + h * dirs[k] for k in range(2)], probes, n, H, grad=False)["J"]
    jm = g.adjoint_probe([q0[k] - h * dirs[k] for k in range(2)], probes, n, H, grad=False)["J"]
    return (jp - jm) / (2 * h)


@pytest.mark.parametrize("snapshots", [None, 2])
def test_probe_gradient_matches_central_differences(sbp, snapshots):
    wl, probes = _probe_case()
    g = sbp.System(wl)
    q0 = _q0(g, wl)
    _, H = g.timestep(q0[0], q0[1])
    n = 8
    r = g.adjoint_probe(q0, probes, n, H, n_snapshots=snapshots)
    rng = np.random.default_rng(71)
    for trial in range(2):
        dirs = [_rand_state(g, k, rng) * _active(g, k) for k in range(2)]
        fd = _fd_J(g, q0, probes, n, H, dirs, 1e-6)
        ad = _dot(r["dq0"][0], dirs[0]) + _dot(r["dq0"][1], dirs[1])
        assert abs(ad - fd) <= 1e-6 * abs(fd), (trial, ad, fd)
    # far-field Mach number (initial states held fixed)
    from paper_1805_06607_gb300.adjoint import freestream_state
    mach, h = 0.2, 1e-6
    dq_dm = np.array([0.0, 1.0, 0.0, mach])
    js = []
    for mm in (mach + h, mach - h):
        g.set_freestream(freestream_state(mm, 1.4).numpy())
        js.append(g.adjoint_probe(q0, probes, n, H, grad=False)["J"])
    g.set_freestream(freestream_state(mach, 1.4).numpy())
    fd_m = (js[0] - js[1]) / (2 * h)
    ad_m = float(r["dqinf"] @ dq_dm)
    assert abs(ad_m - fd_m) <= 1e-6 * abs(fd_m), (ad_m, fd_m)


def test_probe_gradient_matches_oracle_differences(sbp):
    wl, probes = _probe_case(seed=62, n_theta=64, n_r=16, bg_n=(80, 50))
    g = sbp.System(wl)
    q0 = _q0(g, wl)
    _, H = g.timestep(q0[0], q0[1])
    n = 5
    r = g.adjoint_probe(q0, probes, n, H, n_snapshots=1)
    o = OracleSystem(wl)
    rng = np.random.default_rng(81)
    dirs_h = [rng.standard_normal(np.shape(q)) * o.iblank[k] for k, q in enumerate(wl["q0"])]
    h = 1e-6
    jp, _ = probe_objective(o, [wl["q0"][k] + h * dirs_h[k] for k in range(2)], probes, n, H)
    jm, _ = probe_objective(o, [wl["q0"][k] - h * dirs_h[k] for k in range(2)], probes, n, H)
    fd = (jp - jm) / (2 * h)
    ad = sum(float((g.to_host(k, r["dq0"][k]) * dirs_h[k]).sum()) for k in range(2))
    assert abs(ad - fd) <= 1e-6 * abs(fd), (ad, fd)
    # Mach number through the oracle's far-field state
    qinf0 = np.asarray(wl["params"]["qinf"], dtype=np.float64)
    mach = float(qinf0[1])
    js = []
    for mm in (mach + h, mach - h):
        o.p = dict(o.p, qinf=W.freestream(mm))
        js.append(probe_objective(o, wl["q0"], probes, n, H)[0])
    fd_m = (js[0] - js[1]) / (2 * h)
    ad_m = float(r["dqinf"] @ np.array([0.0, 1.0, 0.0, mach]))
    assert abs(ad_m - fd_m) <= 1e-6 * abs(fd_m), (ad_m, fd_m)


def test_checkpoint_schedules_bit_identical(sbp):
    wl, probes = _probe_case(seed=63, n_theta=64, n_r=16, bg_n=(80, 50))
    g = sbp.System(wl)
    q0 = _q0(g, wl)
    _, H = g.timestep(q0[0], q0[1])
    n = 7
    runs = {c: g.adjoint_probe(q0, probes, n, H, n_snapshots=c) for c in (n, 2, 0)}
    ref = runs[n]
    assert ref["forward_steps"] == 2 * n - 1
    assert runs[0]["forward_steps"] == n * (n + 1) // 2
    assert 2 * n - 1 <= runs[2]["forward_steps"] <= n * (n + 1) // 2
    for c, r in runs.items():
        assert r["J"] == ref["J"]
        assert np.array_equal(r["dqinf"], ref["dqinf"])
        for k in range(2):
            assert torch.equal(r["dq0"][k], ref["dq0"][k]), c


def test_autograd_functions(sbp):
    from paper_1805_06607_gb300.adjoint import RhsEval, freestream_state, probe_objective as pobj
    wl, probes = _probe_case(seed=64, n_theta=64, n_r=16, bg_n=(80, 50))
    g = sbp.System(wl)
    q0 = [q.clone().requires_grad_(True) for q in _q0(g, wl)]
    _, H = g.timestep(q0[0].detach(), q0[1].detach())
    mach = torch.tensor(0.2, dtype=torch.float64, requires_grad=True)
    J = pobj(g, q0, freestream_state(mach, 1.4), probes, 5, H, n_snapshots=2)
    J.backward()
    r = g.adjoint_probe([q.detach() for q in q0], probes, 5, H)
    assert abs(float(J.detach()) - r["J"]) == 0.0
    for k in range(2):
        assert torch.equal(q0[k].grad, r["dq0"][k])
    assert abs(float(mach.grad) - float(r["dqinf"] @ np.array([0.0, 1.0, 0.0, 0.2]))) <= 1e-14 * abs(float(mach.grad))
    # right-hand side: d/dq of <w, R(q)> along v against central differences
    rng = np.random.default_rng(91)
    qs = [q.detach().clone().requires_grad_(True) for q in _q0(g, wl)]
    qinf = torch.tensor(np.asarray(wl["params"]["qinf"], dtype=np.float64), requires_grad=True)
    w = _rand_state(g, 1, rng) * _active(g, 1)
    loss = (RhsEval.apply(g, 1, qs[1], qs[0], qinf) * w).sum()
    loss.backward()
    v = [_rand_state(g, m, rng, 1e-2) for m in range(2)]
    eps = 1e-6
    lp = float((g.rhs_eval(1, qs[1].detach() + eps * v[1], qs[0].detach() + eps * v[0]) * w).sum())
    lm = float((g.rhs_eval(1, qs[1].detach() - eps * v[1], qs[0].detach() - eps * v[0]) * w).sum())
    fd = (lp - lm) / (2 * eps)
    ad = _dot(qs[1].grad, v[1]) + _dot(qs[0].grad, v[0])
    assert abs(ad - fd) <= 1e-6 * abs(fd)
