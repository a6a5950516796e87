"""Chains of nested overset meshes at one rate per mesh (C ABI sbp_chain_*) against the chain
oracle (oracle.chain.OracleChain: Sec. 3.3's MRAB with more than two rates read as the nested
two-rate recursion, Sec. 2.2's coupling at every level).

* setup: hole cuts and receivers exactly, each receiver's donor mesh exactly, weights to 1e-12;
* right-hand sides of every mesh to 1e-12 (Euler and Navier-Stokes), the middle mesh fed from
  both neighbours;
* bootstrap + 3 macro steps for step-ratio sets (2, 2) and (3, 2): states and increments over
  the macro steps to 1e-12 in FP64; FP32 states to 1e-5 and increments within the derived FP32
  right-hand-side bound."""
import numpy as np
import pytest

import workloads as W
from conftest import build_library
from oracle.chain import OracleChain
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


def _ns(wl, mu=0.01):
    wl["params"] = dict(wl["params"], physics="ns", mu=mu)
    return wl


CASES = {
    "euler_22": lambda: W.vortex_chain(seed=31, ratios=(2, 2)),
    "euler_32": lambda: W.vortex_chain(seed=32, ratios=(3, 2)),
    "ns_22": lambda: _ns(W.vortex_chain(seed=33, ratios=(2, 2))),
    "euler_22_ab34": lambda: W.vortex_chain(seed=34, ratios=(2, 2), hist_len=4),
    "euler_four_levels": lambda: W.vortex_chain(seed=35, n_bg=40, ratios=(2, 2, 2), halves=(5.0, 2.6, 1.3, 0.6)),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_chain_tables(sbp, case):
    wl = CASES[case]()
    o = OracleChain(wl)
    c = sbp.Chain(wl)
    for k in range(o.R):
        t = c.tables(k)
        assert np.array_equal(t["iblank"], o.iblank[k])
        assert np.array_equal(t["receivers"], o.recv_pts[k])
        assert np.array_equal(t["donor_mesh"], o.recv_src[k])
        if t["w"].size:
            # the donor coordinates are unique; the stencil start is not where a receiver sits on
            # a donor node (both stencils then interpolate the same value)
            lin = np.arange(4.0)
            for d in range(2):
                got = t["base"][:, d] + t["w"][:, 4 * d:4 * d + 4] @ lin
                want = o.base[k][:, d] + o.w[k][:, 4 * d:4 * d + 4] @ lin
                assert np.abs(got - want).max() < 1e-10
            same = np.all(t["base"] == o.base[k], axis=1)
            assert same.mean() > 0.5 and np.abs(t["w"][same] - o.w[k][same]).max() < 1e-12
    assert set(o.recv_src[1].tolist()) == {0, 2}
    c.close()


@pytest.mark.parametrize("case", sorted(CASES))
def test_chain_rhs_fp64(sbp, case):
    wl = CASES[case]()
    o = OracleChain(wl)
    c = sbp.Chain(wl)
    qd = [c.to_device(k, wl["q0"][k]) for k in range(o.R)]
    want = o.rhs_all(wl["q0"])
    for k in range(o.R):
        got = c.to_host(k, c.rhs_eval(k, qd))
        act = o.iblank[k] != 0
        assert rel(got[:, act], want[k][:, act]) < 1e-12, (k, rel(got[:, act], want[k][:, act]))
        assert np.all(got[:, ~act] == 0.0)
    dts, H = c.timestep(qd)
    assert abs(H - o.macro_step_size(wl["q0"])) <= 1e-14 * H
    c.close()


@pytest.mark.parametrize("case", sorted(CASES))
def test_chain_mrab_fp64(sbp, case):
    wl = CASES[case]()
    o = OracleChain(wl)
    H = o.macro_step_size(wl["q0"])
    y, hists = o.bootstrap(wl["q0"], H)
    n = 3
    want, _ = o.mrab(y, hists, H, n)
    c = sbp.Chain(wl)
    c.bind(wl["q0"])
    c.mrab_init(H)
    start = [c.to_host(k, c.current_state(k)) for k in range(o.R)]
    ticks = o.ticks()
    m = int(wl["params"]["hist_len"])
    for k in range(o.R):
        tol = increment_tol(1e-12, wl["q0"][k], y[k], (m - 1) * ticks[0] // ticks[k], U64)
        assert rel(start[k] - wl["q0"][k], y[k] - wl["q0"][k]) < tol, ("bootstrap", k)
    c.mrab_step(n)
    c.check()
    Hg, t = c.mrab_time()
    assert Hg == H and t == pytest.approx(n * H)
    for k in range(o.R):
        got = c.to_host(k, c.current_state(k))
        act = o.iblank[k] != 0
        assert rel(got[:, act], want[k][:, act]) < 1e-12, k
        ei = rel(got[:, act] - start[k][:, act], want[k][:, act] - y[k][:, act])
        tol = increment_tol(1e-12, y[k][:, act], want[k][:, act], n * ticks[0] // ticks[k], U64)
        assert ei < tol, (k, ei, tol)
    c.close()


@pytest.mark.parametrize("case", ["euler_22", "euler_32"])
def test_chain_mrab_fp32(sbp, case):
    wl = CASES[case]()
    o = OracleChain(wl)
    c = sbp.Chain(wl, dtype="f32")
    qd = [c.to_device(k, wl["q0"][k]) for k in range(o.R)]
    _, H = c.timestep(qd)
    assert abs(H - o.macro_step_size(wl["q0"])) <= 1e-6 * H
    y, hists = o.bootstrap(wl["q0"], H)
    n = 3
    want, _ = o.mrab(y, hists, H, n)
    c.bind(wl["q0"])
    c.mrab_init(H)
    start = [c.to_host(k, c.current_state(k)) for k in range(o.R)]
    c.mrab_step(n)
    c.check()
    q0 = wl["q0"]
    rhs0 = o.rhs_all(q0)
    bar = max(fp32_rhs_tol(o.met[j], q0[j], o.iblank[j] != 0, rhs0[j]) for j in range(o.R))
    ticks = o.ticks()
    for k in range(o.R):
        act = o.iblank[k] != 0
        got = c.to_host(k, c.current_state(k))[:, act]
        assert rel(got, want[k][:, act]) < 1e-5, k
        ei = rel(got - start[k][:, act], want[k][:, act] - y[k][:, act])
        tol = increment_tol(bar, y[k][:, act], want[k][:, act], n * ticks[0] // ticks[k], U32)
        assert ei < tol, (k, ei, tol)
    c.close()


def test_two_mesh_chain_equals_the_two_mesh_system(sbp):
    """A chain of two meshes steps like the two-mesh system (same kernels; the donor values of
    both paths agree to rounding)."""
    wl = W.vortex_box_in_box(seed=36, n_bg=48, n_fine=33)
    wl["ratios"] = [wl["params"]["step_ratio"]]
    c, g = sbp.Chain(wl), sbp.System(wl)
    qd = [c.to_device(k, wl["q0"][k]) for k in range(2)]
    _, H = c.timestep(qd)
    for x in (c, g):
        x.bind(wl["q0"])
        x.mrab_init(H)
        x.mrab_step(4)
        x.check()
    for k in range(2):
        a, b = c.to_host(k, c.current_state(k)), g.to_host(k, g.current_state(k))
        assert rel(a, b) < 1e-13
    c.close()
    g.close()


def test_chain_refuses_bad_layouts(sbp):
    wl = W.vortex_chain(seed=37, ratios=(2, 2))
    bad = dict(wl, ratios=[2, 0])
    with pytest.raises(sbp.SbpError):
        sbp.Chain(bad)
    # the outermost mesh with interface faces has no mesh to feed them
    m0 = dict(wl["meshes"][0], bc=("interface",) * 4, periodic=(False, False))
    with pytest.raises(sbp.SbpError):
        sbp.Chain(dict(wl, meshes=[m0] + wl["meshes"][1:]))
