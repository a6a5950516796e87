"""The library's host setup (sbp_host_tables_*, the part of sbp_system_create that runs on the
CPU) against the oracle, without a GPU: hole cut and receiver sets bit for bit, donor stencils
and Lagrange weights to rounding (a receiver on a donor node may take either of two equivalent
stencil starts), and the Adams-Bashforth / MRAB coefficient plan (Sec. 3.1-3.3) against the
oracle's moment solution."""
import numpy as np
import pytest

import workloads as W
from conftest import build_library
from oracle import OracleSystem, ab_coefficients

CASES = {
    "vortex": lambda: W.vortex_box_in_box(seed=11),
    "vortex_sr3_ab34": lambda: W.vortex_box_in_box(seed=12, n_bg=48, n_fine=33, step_ratio=3, hist_len=4),
    "cylinder": lambda: W.cylinder_small(seed=14),
    "cylinder_ragged_ab34": lambda: W.cylinder_small(seed=15, n_theta=72, n_r=20, bg_n=(90, 50), hist_len=4),
    "cylinder_ab46_sr2": lambda: W.cylinder_small(seed=19, n_theta=72, n_r=20, bg_n=(90, 50), order=4, hist_len=6,
                                                 step_ratio=2),
    "mms_viscous": lambda: W.mms_box_in_box(52, "viscous"),
}


@pytest.fixture(scope="module")
def sbp():
    build_library()
    import paper_1805_06607_gb300 as mod
    return mod


@pytest.mark.parametrize("case", sorted(CASES))
def test_host_tables_match_oracle(sbp, case):
    wl = CASES[case]()
    ref = OracleSystem(wl)
    h = sbp.HostTables(wl)
    for k in range(2):
        t = h.tables(k)
        assert np.array_equal(t["iblank"], ref.iblank[k]), "hole cut differs"
        assert np.array_equal(t["receivers"], ref.recv_pts[k]), "receiver set differs"
        nr = ref.recv_pts[k].size
        if not nr:
            continue
        ni, nj = wl["meshes"][1 - k]["n"]
        lin = np.arange(4.0)
        s_got = t["base"][:, 0] + t["w"][:, :4] @ lin   # the donor coordinates the weights encode
        r_got = t["base"][:, 1] + t["w"][:, 4:] @ lin
        ds = (s_got - ref.xe[k][:, 0] + ni / 2) % ni - ni / 2
        dr = (r_got - ref.xe[k][:, 1] + nj / 2) % nj - nj / 2
        assert np.abs(ds).max() < 1e-10 and np.abs(dr).max() < 1e-10
        same = np.all((t["base"] - ref.base[k]) % [ni, nj] == 0, axis=1)
        assert same.mean() > 0.5
        assert np.abs(t["w"][same] - ref.w[k][same]).max() < 1e-12
        assert np.allclose(t["w"].reshape(nr, 2, 4).sum(axis=2), 1.0, atol=1e-13)
    h.close()


@pytest.mark.parametrize("order,m,sr", [(3, 3, 1), (3, 3, 2), (3, 3, 4), (3, 4, 3), (4, 4, 4), (3, 5, 2),
                                        (4, 6, 8), (2, 2, 16)])
def test_host_plan_matches_oracle(sbp, order, m, sr):
    wl = W.vortex_box_in_box(seed=1, n_bg=40, n_fine=25)
    wl = dict(wl, params=dict(wl["params"], order=order, hist_len=m, step_ratio=sr))
    h = sbp.HostTables(wl)
    ab, ext = h.plan()
    nodes = np.arange(m, dtype=float) - (m - 1)
    assert ab.shape == (m,) and ext.shape == (sr, m)
    # both solve the moment system (minimum norm for m > order) in FP64; the condition number of
    # the Vandermonde matrix on up to 6 nodes allows differences of a few hundred ulps
    assert np.abs(ab - ab_coefficients(nodes, 0.0, 1.0, order)).max() < 1e-12
    assert np.all(ext[0] == 0.0)
    for j in range(1, sr):
        assert np.abs(ext[j] - ab_coefficients(nodes, 0.0, j / sr, order)).max() < 1e-12
    h.close()


def test_host_tables_reject_bad_input(sbp):
    wl = W.vortex_box_in_box(seed=1, n_bg=40, n_fine=25)
    with pytest.raises(sbp.SbpError):
        sbp.HostTables(dict(wl, params=dict(wl["params"], hist_len=2, order=3)))
    bg = dict(wl["meshes"][0], n=(7, 40))
    with pytest.raises(sbp.SbpError):
        sbp.HostTables(dict(wl, meshes=[bg, wl["meshes"][1]]))


CASES_3D = {
    "tg_ns": (lambda: W.taylor_green_small(seed=41), 4),
    "tg_sr3_ab34": (lambda: W.taylor_green_small(seed=43, step_ratio=3, hist_len=4, n_bg=20, n_fine=19), 4),
    "extruded_z_vortex": (lambda: W.extrude_to_3d(W.vortex_box_in_box(seed=44, n_bg=40, n_fine=25), 8, 2.0, axis=2),
                          2.5),
    "extruded_y_mms": (lambda: W.extrude_to_3d(W.mms_box_in_box(40, "viscous"), 8, 0.4, axis=1), 3.7),
}


@pytest.mark.parametrize("case", sorted(CASES_3D))
def test_host_tables_3d_match_oracle(sbp, case):
    from oracle import OracleSystem3D
    mk, hc = CASES_3D[case]
    wl = mk()
    ref = OracleSystem3D(wl, hole_cells=hc)
    h = sbp.HostTables3D(wl, hole_cells=hc)
    for k in range(2):
        t = h.tables(k)
        assert np.array_equal(t["iblank"], ref.iblank[k])
        assert np.array_equal(t["receivers"], ref.recv_pts[k])
        if ref.recv_pts[k].size:
            assert np.array_equal(t["base"], ref.base[k])
            assert np.abs(t["w"] - ref.w[k]).max() < 1e-13
    h.close()
