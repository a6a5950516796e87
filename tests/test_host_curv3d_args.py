"""Host-side argument checks of the curvilinear mesh binding: the kernels index q, rhs, qhat
and fvhat by the mesh's sizes and the receiver count given to set_interface, so a tensor of
another shape, element type or device is refused with ValueError before any device call. The
checks run without a GPU on a mesh object whose sizes are set by hand (no C handle: a call
that got past the checks would fail on the missing handle instead)."""
import numpy as np
import pytest

from conftest import build_library

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sbp():
    build_library()
    import paper_1805_06607_gb300 as mod
    return mod


def _mesh(sbp, viscous=True, dtype=None):
    m = sbp.Curvilinear3DMesh.__new__(sbp.Curvilinear3DMesh)
    m.torch = torch
    m.tdtype = dtype or torch.float64
    m.viscous = viscous
    m.shape = (6, 5, 4)
    m.nrecv = 3
    m.h = None
    return m


def test_refuses_host_tensors(sbp):
    m = _mesh(sbp)
    q = torch.zeros((5, 6, 5, 4), dtype=torch.float64)
    with pytest.raises(ValueError, match="CUDA"):
        m.rhs_eval(q)
    with pytest.raises(ValueError, match="CUDA"):
        m.interp(q, np.zeros((1, 3), np.int32), np.zeros((1, 12)))
    with pytest.raises(ValueError, match="CUDA"):
        m.interface_sat(q, torch.zeros((5, 3), dtype=torch.float64), q, torch.zeros((12, 3), dtype=torch.float64))


def test_interface_sat_needs_set_interface(sbp):
    m = _mesh(sbp)
    m.nrecv = None
    with pytest.raises(ValueError, match="set_interface"):
        m.interface_sat(None, None, None)


def test_field_checks(sbp):
    m = _mesh(sbp)

    class FakeCuda:
        """Stands in for a CUDA tensor in the shape and dtype checks (no device needed)."""
        is_cuda = True

        def __init__(self, shape, dtype=torch.float64):
            self.shape = shape
            self.dtype = dtype

        def contiguous(self):
            return self

    orig = torch.Tensor
    try:
        torch.Tensor = FakeCuda        # isinstance(t, torch.Tensor) accepts the stand-in
        good = FakeCuda((5, 6, 5, 4))
        assert m._field(good, "q", (5,) + m.shape) is good
        with pytest.raises(ValueError, match="shape"):
            m._field(FakeCuda((5, 6, 5, 3)), "q", (5,) + m.shape)
        with pytest.raises(ValueError, match="float64"):
            m._field(FakeCuda((5, 6, 5, 4), torch.float32), "q", (5,) + m.shape)
        with pytest.raises(ValueError, match="qhat"):
            m._field(FakeCuda((5, 2)), "qhat", (5, m.nrecv))
        with pytest.raises(ValueError, match="fvhat"):
            m._field(FakeCuda((6, 3)), "fvhat", (12, m.nrecv))
    finally:
        torch.Tensor = orig
