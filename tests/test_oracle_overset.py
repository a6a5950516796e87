"""Pins of the oracle's overset setup (Sec. 2.2): hole cut against a brute-force geometric
check, donor search against the receiver coordinates, and Lagrange weights against
polynomial exactness."""
import math

import numpy as np

import workloads as W
from oracle import OracleSystem


def test_holecut_box_brute_force():
    wl = W.vortex_box_in_box(seed=0)
    S = OracleSystem(wl)
    bg = wl["meshes"][0]
    margin = 4 * bg["h"][0]
    # inside the square [-1,1]^2 and farther than margin from its edges
    expect = (np.maximum(np.abs(bg["x"]), np.abs(bg["y"])) < 1.0 - margin)
    assert np.array_equal(S.iblank[0] == 0, expect)
    # receivers: the four hole-edge rows of the background, the perimeter of the fine mesh
    assert S.recv_pts[0].size == 4 * int(math.isqrt(int(expect.sum())))
    assert S.recv_pts[1].size == 4 * (41 - 1)


def test_holecut_ogrid_geometry():
    wl = W.cylinder_small(seed=0)
    S = OracleSystem(wl)
    bg, og = wl["meshes"]
    r = np.hypot(bg["x"], bg["y"])
    r_out = og["r"][-1]
    margin = 4 * bg["h"][0]
    hole = S.iblank[0] == 0
    assert hole[r < r_out - margin - 0.02].all()
    assert not hole[r > r_out - margin + 0.02].any()


def test_donors_reproduce_receiver_coordinates():
    for wl in (W.vortex_box_in_box(seed=1), W.cylinder_small(seed=1)):
        S = OracleSystem(wl)
        for k, m in enumerate(wl["meshes"]):
            dm = wl["meshes"][1 - k]
            pts = S.recv_pts[k]
            xr = S.interp(k, np.stack([dm["x"], dm["y"]]))
            if dm["periodic"][0] and dm["cartesian"]:
                continue  # coordinates of a periodic Cartesian mesh jump at the wrap
            assert np.abs(xr[0] - m["x"].ravel()[pts]).max() < 1e-12
            assert np.abs(xr[1] - m["y"].ravel()[pts]).max() < 1e-12
            w = S.w[k]
            assert np.abs(w[:, :4].sum(1) - 1).max() < 1e-14
            assert np.abs(w[:, 4:].sum(1) - 1).max() < 1e-14


def test_interpolation_exact_for_cubics():
    wl = W.cylinder_small(seed=2)
    S = OracleSystem(wl)
    bg, og = wl["meshes"]
    # background receivers on the O-grid: a cubic in the radial index (the angular index is
    # periodic, so only periodic functions of it are smooth there)
    ni, nj = og["n"]
    I, J = np.meshgrid(np.arange(ni, dtype=float), np.arange(nj, dtype=float))
    f = 0.3 * J ** 3 - 0.1 * J * J + 0.7 * J - 2.0
    got = S.interp(0, f[None])[0]
    r = S.xe[0][:, 1]
    assert np.abs(got - (0.3 * r ** 3 - 0.1 * r * r + 0.7 * r - 2.0)).max() < 1e-9
    # O-grid receivers on the Cartesian background: a full tensor cubic in both indices
    ni, nj = bg["n"]
    I, J = np.meshgrid(np.arange(ni, dtype=float), np.arange(nj, dtype=float))
    cub = lambda a, b: 1e-4 * a ** 3 - 2e-3 * a * a * b + 0.1 * b * b * b * 1e-3 + 0.5 * a * b - b + 3.0
    got = S.interp(1, cub(I, J)[None])[0]
    s, r = S.xe[1][:, 0], S.xe[1][:, 1]
    assert np.abs(got - cub(s, r)).max() < 1e-9
