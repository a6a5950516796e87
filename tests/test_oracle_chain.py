"""Pins of the oracle's chain of nested overset meshes stepped at one rate per mesh (Sec. 3.3's
extension of MRAB to any number of rates; Sec. 2.2's coupling at every level):

* two meshes: OracleSystem's coupled right-hand sides, macro step, bootstrap and MRAB macro steps
  bit for bit (vortex, viscous cylinder, step ratio 3 with AB34);
* every step ratio 1: single-rate Adams-Bashforth of the whole three-mesh system bit for bit;
* a uniform flow stays uniform (zero right-hand side on every mesh, the middle mesh's receivers
  fed from both of its neighbours);
* third order in time on the three-mesh vortex chain (ratios (2, 2) and (3, 2)) against RK4 at a
  tenth of the finest step; a planted mistake (the bootstrap recording every mesh's history at
  the coarsest step) breaks it, and receivers fed from the wrong neighbour find no donor."""
import numpy as np
import pytest

import oracle
import workloads as W
from conftest import planted_oracle, run_with_oracle
from oracle import OracleSystem, srab_step
from oracle.chain import OracleChain

oracle.lib().orc_set_threads(0)


@pytest.mark.parametrize("make", [lambda: W.vortex_box_in_box(seed=3, n_bg=40, n_fine=25),
                                  lambda: W.cylinder_small(seed=4),
                                  lambda: W.vortex_box_in_box(seed=5, n_bg=40, n_fine=25, step_ratio=3, hist_len=4)],
                         ids=["vortex", "cylinder", "vortex_sr3_ab34"])
def test_two_meshes_equal_the_two_mesh_system(make):
    wl = make()
    wl["ratios"] = [wl["params"]["step_ratio"]]
    a, c = OracleSystem(wl), OracleChain(wl)
    for x, y in zip(a.rhs_all(wl["q0"]), c.rhs_all(wl["q0"])):
        assert np.array_equal(x, y)
    H = a.macro_step_size(wl["q0"])
    assert c.macro_step_size(wl["q0"]) == H
    y, hf, hs = a.bootstrap(wl["q0"], H)
    yc, hc = c.bootstrap(wl["q0"], H)
    assert all(np.array_equal(p, q) for p, q in zip(y, yc))
    assert all(np.array_equal(p, q) for p, q in zip(hs, hc[0])) and all(np.array_equal(p, q) for p, q in zip(hf, hc[1]))
    w1, _, _ = a.mrab(y, hf, hs, H, 2)
    w2, _ = c.mrab(yc, hc, H, 2)
    assert all(np.array_equal(p, q) for p, q in zip(w1, w2))


def test_unit_ratios_equal_single_rate_ab():
    wl = W.vortex_chain(seed=7, ratios=(1, 1))
    c = OracleChain(wl)
    H = c.macro_step_size(wl["q0"])
    y, hists = c.bootstrap(wl["q0"], H)
    got, _ = c.mrab(y, hists, H, 3)
    hist = [[hists[r][k] for r in range(3)] for k in range(len(hists[0]))]
    z = [np.array(v) for v in y]
    for _ in range(3):
        z, hist = srab_step(z, hist, H, 3, c.rhs_all)
    assert all(np.array_equal(p, q) for p, q in zip(got, z))


def test_uniform_flow_is_steady():
    wl = W.vortex_chain(seed=8, ratios=(2, 2))
    qinf = np.asarray(wl["params"]["qinf"], dtype=np.float64)
    c = OracleChain(wl)
    assert set(c.recv_src[1].tolist()) == {0, 2}      # the middle mesh is fed from both sides
    uni = [np.broadcast_to(qinf[:, None, None], (4, m["n"][1], m["n"][0])).copy() for m in wl["meshes"]]
    for k, r in enumerate(c.rhs_all(uni)):
        assert np.abs(r).max() < 1e-12 * np.abs(qinf).max() / min(wl["meshes"][k]["h"]), k


T_CHAIN = 0.064


def chain_time_errors(ratios, hist=3, Hs=(T_CHAIN / 8, T_CHAIN / 16, T_CHAIN / 32)):
    """Max-norm density errors of the chain's MRAB at macro steps Hs after T_CHAIN, against RK4
    at a tenth of the finest step of the smallest macro step."""
    wl = W.vortex_chain(seed=9, n_bg=32, ratios=ratios, hist_len=hist)
    c = OracleChain(wl)
    fine = Hs[-1] / c.ticks()[0] / 10.0
    n_ref = int(round(T_CHAIN / fine))
    from oracle import rk4_step
    ref = [np.array(q) for q in wl["q0"]]
    for _ in range(n_ref):
        ref = rk4_step(ref, T_CHAIN / n_ref, c.rhs_all)
    errs = []
    m = int(wl["params"]["hist_len"])
    for H in Hs:
        y, hists = c.bootstrap(wl["q0"], H)
        y, _ = c.mrab(y, hists, H, int(round(T_CHAIN / H)) - (m - 1))
        errs.append(max(float(np.abs(y[k][0] - ref[k][0]).max()) for k in range(c.R)))
    return list(Hs), errs


def fit_order(Hs, errs):
    return float(np.polyfit(np.log(Hs), np.log(errs), 1)[0])


@pytest.mark.parametrize("ratios", [(2, 2), (3, 2)])
def test_chain_temporal_order(ratios):
    Hs, errs = chain_time_errors(ratios)
    assert abs(fit_order(Hs, errs) - 3.0) < 0.3, errs


def test_chain_order_fails_planted_history_spacing(tmp_path):
    # the bootstrap records every mesh's right-hand side at the coarsest mesh's step
    root = planted_oracle(tmp_path, "chain.py",
                          "if step % t[r] == 0 and step >= nsteps - (m - 1) * t[r]:",
                          "if step % t[0] == 0 and step >= nsteps - (m - 1) * t[0]:")
    out = run_with_oracle(root, "import test_oracle_chain as T\n"
                                "Hs, e = T.chain_time_errors((2, 2))\n"
                                "print(T.fit_order(Hs, e), e[-1])\n")
    order, last = map(float, out.split())
    _, good = chain_time_errors((2, 2))
    assert abs(order - 3.0) > 0.3 or last > 100.0 * good[-1], (order, last, good[-1])


def test_planted_donor_side_finds_no_donor(tmp_path):
    # hole-side receivers of the middle mesh read the coarse mesh: they lie in its hole
    root = planted_oracle(tmp_path, "chain.py", 'add(p, d, side, KIND["interface"], k + 1)',
                          'add(p, d, side, KIND["interface"], k - 1 if k > 0 else k + 1)')
    with pytest.raises(AssertionError, match="no donor"):
        run_with_oracle(root, "import workloads as W\nfrom oracle.chain import OracleChain\n"
                              "OracleChain(W.vortex_chain(seed=9, ratios=(2, 2)))\nprint(0)\n")
