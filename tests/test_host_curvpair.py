"""The host setup of the 3D curvilinear overset pair (sbp3c_host_tables_*, no GPU) against its
oracle (oracle.curvpair): holes after growth, receivers and donor stencils bit-exact, weights to
1e-13, on the seeded curvilinear_pair workload and on a turned Cartesian pair; refusals of bad
arguments and of an overset mesh that pokes out of the background (no donors)."""
import numpy as np
import pytest

import workloads as W
from oracle.curvpair import OracleCurvPair
from test_oracle_curvpair import ANGLES, cartesian_pair, turn

sbp = pytest.importorskip("paper_1805_06607_gb300")


@pytest.mark.parametrize("make", [lambda: W.curvilinear_pair(seed=3),
                                  lambda: turn(cartesian_pair(), W.rotation3d(ANGLES))],
                         ids=["warped", "turned_cartesian"])
def test_tables_match_oracle(make):
    wl = make()
    o = OracleCurvPair(wl)
    T = sbp.HostTablesCurvilinearPair(wl)
    assert (o.iblank[0] == 0).sum() > 20
    for k in range(2):
        t = T.tables(k)
        assert np.array_equal(t["iblank"] != 0, o.iblank[k] != 0), k
        assert np.array_equal(t["receivers"], o.recv_pts[k]), k
        assert np.array_equal(t["base"], o.base[k]), k
        assert np.abs(t["w"] - o.w[k]).max() < 1e-13, k
    T.close()


def test_refusals():
    wl = W.curvilinear_pair()
    for key, val in (("fast_mesh", 2), ("step_ratio", 0), ("gamma", 1.0)):
        bad = dict(wl, params=dict(wl["params"], **{key: val}))
        with pytest.raises(sbp.SbpError):
            sbp.HostTablesCurvilinearPair(bad)
    small = dict(wl["meshes"][1])
    small.update(x=small["x"][:7], y=small["y"][:7], z=small["z"][:7], n=(25, 25, 7))
    with pytest.raises(sbp.SbpError):
        sbp.HostTablesCurvilinearPair(dict(wl, meshes=[wl["meshes"][0], small]))
    # an overset box wider than the background: its faces have no donors
    big = W.curvilinear_pair(n_fine=45, hole_cells=16)
    with pytest.raises(sbp.SbpError) as e:
        sbp.HostTablesCurvilinearPair(big)
    assert e.value.status == -6
