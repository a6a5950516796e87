"""sbp_f32_to_f64: the integer FP32 -> FP64 widening that the FP32 forms use inside their FP64
accumulations must equal the hardware conversion bit for bit, for every exponent (normal,
subnormal, zero, infinity / NaN) and sign, with random and edge fractions."""
import numpy as np
import pytest

from conftest import build_library

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_widen_matches_hardware_conversion():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build_library()
    import paper_1805_06607_gb300 as sbp

    rng = np.random.default_rng(7)
    frac = np.concatenate([np.array([0, 1, 2, 0x400000, 0x7FFFFE, 0x7FFFFF], dtype=np.uint32),
                           rng.integers(0, 1 << 23, 4096, dtype=np.uint32)])
    exp = np.arange(256, dtype=np.uint32)
    bits = (exp[:, None] << 23) | frac[None, :]
    bits = np.concatenate([bits.ravel(), bits.ravel() | np.uint32(0x80000000)])
    x = torch.from_numpy(bits.view(np.float32)).cuda()
    y = sbp.f32_to_f64(x)
    want = x.double()
    torch.cuda.synchronize()
    yb = y.cpu().numpy().view(np.int64)
    wb = want.cpu().numpy().view(np.int64)
    nan = np.isnan(want.cpu().numpy())
    assert np.isnan(y.cpu().numpy()[nan]).all()
    assert np.array_equal(yb[~nan], wb[~nan])
    # zero-length call is a no-op
    sbp.f32_to_f64(torch.empty(0, dtype=torch.float32, device="cuda"))
