"""The library's curvilinear donor search (sbp3c_donor_search, host code, no GPU) against the
oracle's (oracle.curv3d.donors): stencil starts identical, computational coordinates and weights
to 1e-12, on warped meshes larger than the coarse start's stride and on a mesh of 8 points along
one direction; the same first failing point for points outside the mesh and for stencils over
inactive points."""
import numpy as np
import pytest

from conftest import build_library
from oracle.curv3d import DonorError, donors


@pytest.fixture(scope="module")
def sbp():
    build_library()
    import paper_1805_06607_gb300 as mod
    return mod


def _mesh(ni, nj, nk, eps=0.05):
    Z, Y, X = np.meshgrid(np.linspace(0, 1.3, nk), np.linspace(0, 0.9, nj), np.linspace(0, 1.1, ni), indexing="ij")
    s = 2 * np.pi
    return (X + eps * np.sin(s * Y) * np.sin(s * Z), Y + eps * np.sin(s * X) * np.sin(s * Z),
            Z + eps * np.sin(s * X) * np.sin(s * Y))


def _points(x, y, z, n, seed):
    """Points inside the mesh: a random trilinear mix of the corners of a random cell that
    touches no boundary face (on a face cell the mix can fall just outside the face of the
    cubic-interpolated map, where both searches rightly refuse it)."""
    rng = np.random.default_rng(seed)
    nk, nj, ni = x.shape
    out = []
    for _ in range(n):
        i, j, k = rng.integers(1, ni - 2), rng.integers(1, nj - 2), rng.integers(1, nk - 2)
        a, b, c = rng.uniform(0, 1, 3)
        p = np.zeros(3)
        for dk, wk in ((0, 1 - c), (1, c)):
            for dj, wj in ((0, 1 - b), (1, b)):
                for di, wi in ((0, 1 - a), (1, a)):
                    p += wi * wj * wk * np.array([v[k + dk, j + dj, i + di] for v in (x, y, z)])
        out.append(p)
    return np.array(out)


@pytest.mark.parametrize("shape", [(40, 33, 26), (8, 19, 12)])
def test_donor_search_matches_oracle(sbp, shape):
    x, y, z = _mesh(*shape)
    pts = _points(x, y, z, 60, 4)
    bo, wo, xo = donors(x, y, z, pts)
    bl, wl, xl = sbp.donor_search_3d(x, y, z, pts)
    assert np.array_equal(bl, bo)
    assert np.abs(xl - xo).max() < 1e-12
    assert np.abs(wl - wo).max() < 1e-12


def test_donor_search_failures_match_oracle(sbp):
    x, y, z = _mesh(20, 17, 13)
    pts = _points(x, y, z, 5, 8)
    out = pts.copy()
    out[3] = [1.5, 0.4, 0.5]    # beyond the i-high face
    with pytest.raises(DonorError) as e:
        donors(x, y, z, out)
    assert e.value.args[0] == 3
    with pytest.raises(sbp.SbpError, match="point 3 "):
        sbp.donor_search_3d(x, y, z, out)
    bo, _, _ = donors(x, y, z, pts)
    ib = np.ones(x.shape, np.int8)
    i0, j0, k0 = bo[2]
    ib[k0 + 1, j0 + 2, i0 + 3] = 0
    with pytest.raises(DonorError) as e:
        donors(x, y, z, pts, iblank=ib)
    with pytest.raises(sbp.SbpError, match="point %d " % e.value.args[0]):
        sbp.donor_search_3d(x, y, z, pts, iblank=ib)


def test_hole_cut_matches_oracle(sbp):
    """sbp3c_hole_cut against oracle.curv3d.hole_cut: the nodes of a background box around a
    warped mesh, margin 2 index units."""
    from oracle.curv3d import hole_cut
    x, y, z = _mesh(20, 17, 14)
    t = [np.linspace(-0.2, 1.3, 16), np.linspace(-0.2, 1.1, 13), np.linspace(-0.2, 1.5, 17)]
    Zb, Yb, Xb = np.meshgrid(t[2], t[1], t[0], indexing="ij")
    pts = np.stack([Xb.ravel(), Yb.ravel(), Zb.ravel()], axis=1)
    want = hole_cut(x, y, z, pts, 2.0)
    got = sbp.hole_cut_3d(x, y, z, pts, 2.0)
    assert want.sum() > 100 and (~want).sum() > 1000
    assert np.array_equal(got, want)


def test_hole_cut_of_a_large_background_is_fast(sbp):
    """The hole cut of a 64^3 background box against a warped 48^3 mesh inside it: most
    background nodes lie outside the mesh and are refused by the padded bounding box without a
    search; the whole cut stays within a few seconds (a scan of every mesh node per outside point
    would take minutes). The result agrees with the oracle's on a sample of the nodes."""
    import time
    from oracle.curv3d import hole_cut
    x, y, z = _mesh(48, 48, 48)
    t = [np.linspace(-0.6, 1.7, 64), np.linspace(-0.6, 1.5, 64), np.linspace(-0.6, 1.9, 64)]
    Zb, Yb, Xb = np.meshgrid(t[2], t[1], t[0], indexing="ij")
    pts = np.stack([Xb.ravel(), Yb.ravel(), Zb.ravel()], axis=1)
    t0 = time.perf_counter()
    got = sbp.hole_cut_3d(x, y, z, pts, 2.0)
    el = time.perf_counter() - t0
    assert el < 20.0, el
    assert got.sum() > 1000 and (~got).sum() > 100000
    sample = np.random.default_rng(3).choice(len(pts), 400, replace=False)
    assert np.array_equal(got[sample], hole_cut(x, y, z, pts[sample], 2.0))
