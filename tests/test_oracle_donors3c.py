"""Pins of the curvilinear 3D donor search (oracle.curv3d.donors) by closed forms:

* on a mesh whose coordinates are an affine map of the index coordinates, the computational
  coordinates of a point are that map's inverse;
* on a mesh whose coordinates are cubic in each index coordinate (tensor cubic), the 4 x 4 x 4
  Lagrange map is that polynomial itself, so a point given as the polynomial's image of known
  index coordinates is found at exactly those coordinates; the stencil starts at
  floor(s) - 1 clamped into the mesh;
* the weights reproduce any tensor-cubic field of the index coordinates at the found point;
* points outside the mesh and stencils over inactive points are refused."""
import numpy as np
import pytest

from oracle.curv3d import DonorError, donors, interpolate

NI, NJ, NK = 12, 10, 9


def _index_grid():
    return np.meshgrid(np.arange(NK, dtype=float), np.arange(NJ, dtype=float), np.arange(NI, dtype=float),
                       indexing="ij")


def _tricubic(i, j, k):
    return (0.1 * i + 0.002 * j * j + 0.0003 * i * i * k - 1e-5 * i ** 3,
            0.08 * j + 0.001 * i * k + 2e-5 * j ** 3 + 0.003 * k,
            0.12 * k + 0.002 * i * j - 0.0004 * k * k + 0.0001 * i * j * k)


def _samples(n, seed, margin=0.0):
    rng = np.random.default_rng(seed)
    return rng.uniform([margin] * 3, [NI - 1 - margin, NJ - 1 - margin, NK - 1 - margin], (n, 3))


def test_affine_mesh_inverse_is_closed_form():
    K, J, I = _index_grid()
    A = np.array([[0.1, 0.02, -0.01], [0.015, 0.09, 0.02], [-0.02, 0.01, 0.11]])
    b = np.array([0.3, -0.2, 1.0])
    X = np.einsum("ab,bkji->akji", A, np.stack([I, J, K])) + b[:, None, None, None]
    xs = _samples(25, 1)
    pts = xs @ A.T + b
    base, w, xi = donors(*X, pts)
    assert np.abs(xi - np.linalg.solve(A, (pts - b).T).T).max() < 1e-12


def test_tricubic_mesh_recovers_index_coordinates_and_stencil_start():
    K, J, I = _index_grid()
    X = _tricubic(I, J, K)
    xs = _samples(40, 2)
    xs[:3] = [[0.0, 0.0, 0.0], [NI - 1, NJ - 1, NK - 1], [0.4, NJ - 1.3, 4.5]]   # corners and a face
    pts = np.array([_tricubic(*c) for c in xs])
    base, w, xi = donors(*X, pts)
    assert np.abs(xi - xs).max() < 1e-12
    n = np.array([NI, NJ, NK])
    assert np.array_equal(base, np.clip(np.floor(xs).astype(int) - 1, 0, n - 4))


def test_weights_reproduce_tensor_cubics():
    K, J, I = _index_grid()
    X = _tricubic(I, J, K)
    xs = _samples(30, 3)
    pts = np.array([_tricubic(*c) for c in xs])
    base, w, xi = donors(*X, pts)

    def f(i, j, k):
        return np.stack([1.0 + 0.3 * i ** 3 - 0.2 * j * j * k + 0.05 * i * j * k ** 3, 2.0 - i + k ** 3 * j])

    got = interpolate(f(I, J, K), base, w)
    want = f(xs[:, 0], xs[:, 1], xs[:, 2])
    assert np.abs(got - want).max() < 1e-11 * np.abs(want).max()
    # a quartic is not reproduced: the basis is cubic
    q4 = interpolate((I ** 4)[None], base, w)[0]
    assert np.abs(q4 - xs[:, 0] ** 4).max() > 1e-3


def test_outside_points_and_inactive_stencils_refused():
    K, J, I = _index_grid()
    X = _tricubic(I, J, K)
    inside = np.array([_tricubic(5.5, 4.5, 4.2)])
    outside = np.array([_tricubic(NI - 1 + 0.5, 3.0, 3.0)])
    with pytest.raises(DonorError) as e:
        donors(*X, np.vstack([inside, outside]))
    assert e.value.args[0] == 1
    ib = np.ones((NK, NJ, NI), np.int8)
    ib[4, 4, 5] = 0    # inside the first point's stencil (base (4, 3, 3))
    with pytest.raises(DonorError) as e:
        donors(*X, inside, iblank=ib)
    assert e.value.args[0] == 0
    ib[:] = 1
    ib[0, 0, 0] = 0    # outside its stencil
    donors(*X, inside, iblank=ib)


def test_hole_cut_on_affine_mesh_is_the_index_box():
    """Hole cut against a mesh affine in its index coordinates: a point is a hole exactly when the
    inverse map's closed form puts it more than `margin` index units inside every face."""
    from oracle.curv3d import hole_cut
    K, J, I = _index_grid()
    A = np.array([[0.1, 0.02, -0.01], [0.015, 0.09, 0.02], [-0.02, 0.01, 0.11]])
    b = np.array([0.3, -0.2, 1.0])
    X = np.einsum("ab,bkji->akji", A, np.stack([I, J, K])) + b[:, None, None, None]
    rng = np.random.default_rng(9)
    xs = rng.uniform([-2, -2, -2], [NI + 1, NJ + 1, NK + 1], (300, 3))
    pts = xs @ A.T + b
    margin = 2.5
    want = np.all((xs > margin) & (xs < np.array([NI, NJ, NK]) - 1 - margin), axis=1)
    got = hole_cut(*X, pts, margin)
    assert want.sum() >= 10 and (~want).sum() > 100
    assert np.array_equal(got, want)
