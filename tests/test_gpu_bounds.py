"""Bounds checks on the GPU: the curvilinear gather (sbp3c_interp) takes stencil bases from the
caller; a base whose 4 x 4 x 4 stencil leaves the mesh gives zeros for that receiver and records
SBP_ERR_BOUNDS (read by sbp3c_mesh_check) without reading out of range, while the other
receivers' values are unchanged. The call goes to the C ABI directly (the Python binding refuses
such bases on the host before the call)."""
import ctypes

import numpy as np
import pytest

from conftest import build_library

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sbp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build_library()
    import paper_1805_06607_gb300 as mod
    return mod


def _mesh(ni, nj, nk):
    Z, Y, X = np.meshgrid(np.linspace(0, 1.3, nk), np.linspace(0, 0.9, nj), np.linspace(0, 1.1, ni), indexing="ij")
    return X + 0.02 * np.sin(6 * Y), Y + 0.02 * np.sin(6 * Z), Z + 0.02 * np.sin(6 * X)


def test_out_of_range_stencil_is_recorded_not_read(sbp):
    x, y, z = _mesh(12, 10, 9)
    g = sbp.Curvilinear3DMesh(x, y, z, {"physics": "euler", "gamma": 1.4, "mu": 0.0, "pr": 0.72})
    rng = np.random.default_rng(0)
    q = torch.from_numpy(1.0 + 0.1 * rng.standard_normal((5,) + x.shape)).cuda()
    good = np.array([[1, 2, 3], [8, 6, 5], [0, 0, 0]], np.int32)
    w = np.tile(np.array([0.1, 0.2, 0.3, 0.4]), (3, 3))
    ref = g.interp(q, good, w).cpu().numpy()
    g.check()
    for bad_row in ([9, 2, 3], [-1, 2, 3], [1, 7, 3], [1, 2, 6]):   # i0 > ni - 4, i0 < 0, j0 > nj - 4, k0 > nk - 4
        base = good.copy()
        base[1] = bad_row
        b = torch.from_numpy(base).cuda()
        wt = torch.from_numpy(w).cuda()
        out = torch.full((5, 3), 7.0, dtype=torch.float64, device="cuda")
        st = sbp.lib().sbp3c_interp(g.h, ctypes.c_void_p(q.data_ptr()), 3, ctypes.c_void_p(b.data_ptr()),
                                    ctypes.c_void_p(wt.data_ptr()), ctypes.c_void_p(out.data_ptr()), None)
        assert st == 0
        with pytest.raises(sbp.SbpError) as e:
            g.check()
        assert e.value.status == -8
        got = out.cpu().numpy()
        assert np.all(got[:, 1] == 0.0)
        assert np.array_equal(got[:, [0, 2]], ref[:, [0, 2]])
        g.check()   # cleared
    g.close()
