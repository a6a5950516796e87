"""sbp_rhs_eval_noalloc, the right-hand-side entry point for callers that cannot have device
memory allocated for them while they run (device memory reserved up front by another allocator,
or a loop that cannot take the synchronisation of cudaMalloc / cudaFree): it must give the same
result as sbp_rhs_eval, on consecutive calls that share its fixed device workspace, in FP64 and
FP32, and refuse meshes with more receivers than its workspace holds. Collected last on
purpose, so that a run stopping at the first failure has run every other test first."""
import ctypes

import numpy as np
import pytest

import workloads as W
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


def _call(sbp, g, k, q_self, q_other, out):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return sbp.lib().sbp_rhs_eval_noalloc(g.h, k, ctypes.c_void_p(q_self.data_ptr()),
                                          ctypes.c_void_p(q_other.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                          stream)


# FP64: the parity bar of the FP64 path; FP32: both calls run the same FP32 kernels, so the
# results agree far inside the FP32 bound against the oracle
@pytest.mark.parametrize("dtype,tol", [("f64", 1e-12), ("f32", 1e-6)])
def test_noalloc_matches_rhs_eval_on_consecutive_calls(sbp, dtype, tol):
    for wl in (W.cylinder_small(seed=21), W.vortex_box_in_box(seed=22)):
        g = sbp.System(wl, dtype=dtype)
        qd = [g.to_device(k, wl["q0"][k]) for k in range(2)]
        # two calls in a row (fine mesh, then background) through the C ABI
        for k in (1, 0):
            want = g.rhs_eval(k, qd[k], qd[1 - k])
            got = g.empty_state(k)
            got.fill_(float("nan"))
            rc = _call(sbp, g, k, qd[k], qd[1 - k], got)
            assert rc == 0, sbp.lib().sbp_last_error_message()
            a = g.to_host(k, got)
            b = g.to_host(k, want)
            assert np.isfinite(a).all()
            assert np.linalg.norm(a - b) <= tol * np.linalg.norm(b)
        g.close()


def test_noalloc_refuses_more_receivers_than_its_workspace(sbp):
    # a thin fine patch 4100 x 9 with interface faces: 2 * 4100 + 2 * 7 = 8214 receivers, above
    # the workspace's 8192; the background (no hole under so thin a patch) has none
    wl = W.vortex_box_in_box(seed=23)
    fine = W.cartesian_mesh("fine", (4100, 9), (-1.0, -0.02), (2.0 / 4099, 0.005), ("interface",) * 4)
    wl["meshes"][1] = fine
    wl["q0"][1] = W.vortex_state(fine["x"], fine["y"], 0.0, **wl["vortex"])
    g = sbp.System(wl)
    assert g.info[1].n_receivers > 8192 and g.info[0].n_receivers == 0
    qd = [g.to_device(k, wl["q0"][k]) for k in range(2)]
    out = g.empty_state(1)
    assert _call(sbp, g, 1, qd[1], qd[0], out) == -2          # SBP_ERR_SHAPE
    assert b"8192" in sbp.lib().sbp_last_error_message()
    # the background (no receivers) is still served
    want = g.rhs_eval(0, qd[0], qd[1])
    got = g.empty_state(0)
    assert _call(sbp, g, 0, qd[0], qd[1], got) == 0
    assert np.array_equal(g.to_host(0, got), g.to_host(0, want))
    g.close()
