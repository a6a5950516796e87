"""The 3D curvilinear operator on the GPU (sbp3c_*) against the oracle (oracle.curv3d): metric
terms and flux divergences on warped meshes of uneven sizes, Euler and Navier-Stokes, FP64 to
1e-12 relative (metrics to 1e-13), FP32 to the rounding bound of its fluxes; a uniform state
keeps zero divergence (free-stream preservation); the optional far-field SAT on every face
against the oracle's, and zero at the free stream."""
import numpy as np
import pytest

from conftest import build_library
from oracle.curv3d import Curvilinear3D

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sbp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build_library()
    import paper_1805_06607_gb300 as mod
    return mod


def _mesh(ni, nj, nk, eps=0.04):
    Z, Y, X = np.meshgrid(np.linspace(0, 1.3, nk), np.linspace(0, 0.9, nj), np.linspace(0, 1.1, ni), indexing="ij")
    s = 2 * np.pi
    return (X + eps * np.sin(s * Y) * np.sin(s * Z), Y + eps * np.sin(s * X) * np.sin(s * Z),
            Z + eps * np.sin(s * X) * np.sin(s * Y))


def _state(x, y, z, seed):
    rng = np.random.default_rng(seed)
    rho = 1.0 + 0.1 * np.sin(3 * x) * np.cos(2 * y) * np.sin(z)
    u = 0.3 + 0.1 * np.cos(2 * x + z)
    v = -0.2 + 0.1 * np.sin(3 * y) * np.cos(x)
    w = 0.1 * np.sin(x + y)
    p = 0.9 + 0.05 * np.cos(x) * np.cos(2 * y) * np.cos(3 * z) + 1e-3 * rng.standard_normal(x.shape)
    E = p / 0.4 + 0.5 * rho * (u * u + v * v + w * w)
    return np.array([rho, rho * u, rho * v, rho * w, E])


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


PARAMS = {"euler": {"physics": "euler", "gamma": 1.4, "mu": 0.0, "pr": 0.72},
          "ns": {"physics": "ns", "gamma": 1.4, "mu": 0.02, "pr": 0.72}}


@pytest.mark.parametrize("shape", [(20, 17, 13), (8, 11, 9), (33, 9, 16)])
def test_metrics_match_oracle(sbp, shape):
    x, y, z = _mesh(*shape)
    o = Curvilinear3D(x, y, z)
    g = sbp.Curvilinear3DMesh(x, y, z, PARAMS["euler"])
    met = g.metrics()
    for m in range(3):
        for j in range(3):
            want = o.M[m][j]
            assert np.abs(met[3 * m + j] - want).max() <= 1e-13 * np.abs(want).max() + 1e-15, (m, j)
    assert _rel(met[9], o.J) < 1e-14
    g.close()


@pytest.mark.parametrize("phys", ["euler", "ns"])
@pytest.mark.parametrize("shape", [(20, 17, 13), (8, 11, 9)])
def test_rhs_matches_oracle(sbp, phys, shape):
    x, y, z = _mesh(*shape)
    o = Curvilinear3D(x, y, z)
    q = _state(x, y, z, 7)
    P = PARAMS[phys]
    want = o.rhs(q, P["gamma"], P["mu"], P["pr"])
    g = sbp.Curvilinear3DMesh(x, y, z, P)
    got = g.rhs_eval(torch.from_numpy(q).cuda()).cpu().numpy()
    assert _rel(got, want) < 1e-12, _rel(got, want)
    g.close()
    g32 = sbp.Curvilinear3DMesh(x, y, z, P, dtype="f32")
    got32 = g32.rhs_eval(torch.from_numpy(q.astype(np.float32)).cuda()).cpu().numpy()
    # FP32 fluxes carry ~6e-8 |F|; the derivative divides by the spacing while |dq/dt| here is
    # O(1): a few 1e-6 of |F| / h relative
    assert _rel(got32, want) < 2e-4, _rel(got32, want)
    g32.close()


@pytest.mark.parametrize("phys", ["euler", "ns"])
def test_free_stream_preserved(sbp, phys):
    x, y, z = _mesh(24, 21, 19)
    q = np.array([np.full(x.shape, c) for c in (1.1, 0.33, -0.22, 0.165, 0.9 / 0.4 + 0.5 * 1.1 * 0.1325)])
    g = sbp.Curvilinear3DMesh(x, y, z, PARAMS[phys])
    r = g.rhs_eval(torch.from_numpy(q).cuda()).cpu().numpy()
    assert np.abs(r).max() < 1e-11, np.abs(r).max()
    g.close()


def test_larger_mesh_fp64(sbp):
    """A 64^3 warped mesh (262,144 points, 4,096 CTAs per kernel) against the oracle."""
    x, y, z = _mesh(64, 64, 64, eps=0.02)
    o = Curvilinear3D(x, y, z)
    q = _state(x, y, z, 9)
    P = PARAMS["ns"]
    want = o.rhs(q, P["gamma"], P["mu"], P["pr"])
    g = sbp.Curvilinear3DMesh(x, y, z, P)
    got = g.rhs_eval(torch.from_numpy(q).cuda()).cpu().numpy()
    assert _rel(got, want) < 1e-12, _rel(got, want)
    g.close()


def test_bad_sizes_rejected(sbp):
    x, y, z = _mesh(7, 10, 10)
    with pytest.raises(sbp.SbpError):
        sbp.Curvilinear3DMesh(x, y, z, PARAMS["euler"])


QINF = np.array([1.0, 0.35, -0.1, 0.05, 0.9 / 0.4 + 0.5 * (0.35 ** 2 + 0.1 ** 2 + 0.05 ** 2)])


@pytest.mark.parametrize("phys", ["euler", "ns"])
@pytest.mark.parametrize("shape", [(20, 17, 13), (9, 8, 12)])
def test_farfield_sat_matches_oracle(sbp, phys, shape):
    """Far-field SAT on every face (edges and corners carry two or three terms)."""
    x, y, z = _mesh(*shape)
    o = Curvilinear3D(x, y, z)
    q = _state(x, y, z, 13)
    P = PARAMS[phys]
    sigma = 1.3
    want = o.rhs(q, P["gamma"], P["mu"], P["pr"], qinf=QINF, sigma=sigma)
    plain = o.rhs(q, P["gamma"], P["mu"], P["pr"])
    assert np.linalg.norm(want - plain) > 1e-3 * np.linalg.norm(want)
    g = sbp.Curvilinear3DMesh(x, y, z, P)
    g.set_farfield(QINF, sigma)
    got = g.rhs_eval(torch.from_numpy(q).cuda()).cpu().numpy()
    assert _rel(got, want) < 1e-12, _rel(got, want)
    g.set_farfield(None)
    got0 = g.rhs_eval(torch.from_numpy(q).cuda()).cpu().numpy()
    assert _rel(got0, plain) < 1e-12, _rel(got0, plain)
    g.close()
    g32 = sbp.Curvilinear3DMesh(x, y, z, P, dtype="f32")
    g32.set_farfield(QINF, sigma)
    got32 = g32.rhs_eval(torch.from_numpy(q.astype(np.float32)).cuda()).cpu().numpy()
    assert _rel(got32, want) < 2e-4, _rel(got32, want)
    g32.close()


def test_farfield_free_stream_preserved(sbp):
    x, y, z = _mesh(24, 21, 19)
    q = np.array([np.full(x.shape, c) for c in QINF])
    g = sbp.Curvilinear3DMesh(x, y, z, PARAMS["ns"])
    g.set_farfield(QINF, 1.0)
    r = g.rhs_eval(torch.from_numpy(q).cuda()).cpu().numpy()
    assert np.abs(r).max() < 1e-11, np.abs(r).max()
    g.close()


def test_farfield_bad_arguments_rejected(sbp):
    x, y, z = _mesh(10, 10, 10)
    g = sbp.Curvilinear3DMesh(x, y, z, PARAMS["euler"])
    with pytest.raises(sbp.SbpError):
        g.set_farfield(QINF, -1.0)
    bad = QINF.copy()
    bad[4] = 0.0   # negative pressure
    with pytest.raises(sbp.SbpError):
        g.set_farfield(bad, 1.0)
    g.close()


@pytest.mark.parametrize("shape", [(20, 17, 13), (8, 19, 12)])
def test_overset_gather_matches_oracle(sbp, shape):
    """sbp3c_interp with stencils from the library's donor search against the oracle's gather:
    FP64 to 1e-14 relative, FP32 to its rounding."""
    from oracle.curv3d import interpolate
    x, y, z = _mesh(*shape)
    rng = np.random.default_rng(21)
    nk, nj, ni = x.shape
    cells = np.stack([rng.integers(1, n - 2, 70) for n in (ni, nj, nk)], axis=1)
    frac = rng.uniform(0, 1, (70, 3))
    pts = np.array([[(1 - f[0]) * v[k, j, i] + f[0] * v[k, j, i + 1] for v in (x, y, z)]
                    for (i, j, k), f in zip(cells, frac)])
    base, w, _ = sbp.donor_search_3d(x, y, z, pts)
    q = _state(x, y, z, 5)
    want = interpolate(q, base, w)
    g = sbp.Curvilinear3DMesh(x, y, z, PARAMS["euler"])
    got = g.interp(torch.from_numpy(q).cuda(), base, w).cpu().numpy()
    assert _rel(got, want) < 1e-14, _rel(got, want)
    g.close()
    g32 = sbp.Curvilinear3DMesh(x, y, z, PARAMS["euler"], dtype="f32")
    got32 = g32.interp(torch.from_numpy(q.astype(np.float32)).cuda(), base, w).cpu().numpy()
    assert _rel(got32, want) < 1e-6, _rel(got32, want)
    g32.close()


@pytest.mark.parametrize("phys", ["euler", "ns"])
def test_interface_sat_matches_oracle(sbp, phys):
    """sbp3c_interface_sat after sbp3c_rhs_eval against the oracle's right-hand side with the same
    interface terms: receivers on all six faces, a weighted edge, a corner and a point inside
    the mesh (a hole-boundary receiver), donor states and viscous fluxes given."""
    x, y, z = _mesh(13, 11, 12)
    nk, nj, ni = x.shape
    o = Curvilinear3D(x, y, z)
    q = _state(x, y, z, 31)
    P = PARAMS[phys]
    terms = [(0, 3, 4, 0, 1, 0, 1.0), (ni - 1, 5, 2, 0, -1, 1, 1.0), (4, 0, 6, 1, 1, 2, 1.0),
             (6, nj - 1, 3, 1, -1, 3, 1.0), (5, 4, 0, 2, 1, 4, 1.0), (3, 2, nk - 1, 2, -1, 5, 1.0),
             (0, 0, 5, 0, 1, 6, 0.7), (0, 0, 5, 1, 1, 6, 0.7),
             (ni - 1, nj - 1, nk - 1, 0, -1, 7, 1.0), (ni - 1, nj - 1, nk - 1, 2, -1, 7, 1.0),
             (6, 5, 6, 0, -1, 8, 1.0)]
    nrecv = 9
    rng = np.random.default_rng(3)
    cols = {t[5]: (t[0], t[1], t[2]) for t in terms}
    qhat = np.array([q[:, cols[r][2], cols[r][1], cols[r][0]] for r in range(nrecv)]).T
    qhat = qhat * (1.0 + 0.03 * rng.standard_normal(qhat.shape))
    fvhat = 0.05 * rng.standard_normal((12, nrecv))
    sigma = 0.5
    want = o.rhs(q, P["gamma"], P["mu"], P["pr"], interface=dict(terms=terms, qhat=qhat, fvhat=fvhat, sigma=sigma))
    plain = o.rhs(q, P["gamma"], P["mu"], P["pr"])
    assert np.linalg.norm(want - plain) > 1e-3 * np.linalg.norm(want)
    for dtype, tol in (("f64", 1e-12), ("f32", 2e-4)):
        nd = np.float64 if dtype == "f64" else np.float32
        g = sbp.Curvilinear3DMesh(x, y, z, P, dtype=dtype)
        g.set_interface(terms, nrecv, sigma)
        qd = torch.from_numpy(q.astype(nd)).cuda()
        r = g.rhs_eval(qd)
        g.interface_sat(qd, torch.from_numpy(qhat.astype(nd)).cuda(), r,
                        fvhat=torch.from_numpy(fvhat.astype(nd)).cuda() if phys == "ns" else None)
        got = r.cpu().numpy()
        assert _rel(got, want) < tol, (dtype, _rel(got, want))
        g.close()


def test_interface_terms_rejected(sbp):
    x, y, z = _mesh(10, 10, 10)
    g = sbp.Curvilinear3DMesh(x, y, z, PARAMS["euler"])
    for bad in ([(10, 0, 0, 0, 1, 0, 1.0)], [(0, 0, 0, 3, 1, 0, 1.0)], [(0, 0, 0, 0, 0, 0, 1.0)],
                [(0, 0, 0, 0, 1, 2, 1.0)]):
        with pytest.raises(sbp.SbpError):
            g.set_interface(bad, 2)
    g.close()
