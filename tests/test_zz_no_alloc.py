"""sbp_rhs_eval_noalloc, the right-hand-side entry point for callers that cannot have device
memory allocated for them while they run (inside a global-mode stream capture, or with all
device memory reserved by another allocator): it must give the same result as sbp_rhs_eval,
on consecutive calls that share its fixed device workspace. Collected last on purpose."""
import ctypes

import numpy as np
import pytest

import workloads as W
from conftest import build_library

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_noalloc_matches_rhs_eval_on_consecutive_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build_library()
    import paper_1805_06607_gb300 as sbp

    L = sbp.lib()
    for wl in (W.cylinder_small(seed=21), W.vortex_box_in_box(seed=22)):
        g = sbp.System(wl)
        qd = [g.to_device(k, wl["q0"][k]) for k in range(2)]
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        # two calls in a row (fine mesh, then background) through the C ABI
        for k in (1, 0):
            want = g.rhs_eval(k, qd[k], qd[1 - k])
            got = g.empty_state(k)
            got.fill_(float("nan"))
            rc = L.sbp_rhs_eval_noalloc(g.h, k, ctypes.c_void_p(qd[k].data_ptr()),
                                         ctypes.c_void_p(qd[1 - k].data_ptr()), ctypes.c_void_p(got.data_ptr()),
                                         stream)
            assert rc == 0, L.sbp_last_error_message()
            a = g.to_host(k, got)
            b = g.to_host(k, want)
            assert np.isfinite(a).all()
            assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)
        g.close()
