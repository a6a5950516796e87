"""Failure detection without a GPU fault: the kernels report through the system's device error
word, which sbp_check / sbp_batch_check / sbp3_check read on the host.

* A non-finite value or a non-positive density planted in the initial state on the host reaches
  the MRAB update epilogue, which records SBP_ERR_NONFINITE; the run ends normally and the check
  raises (2D systems, batches, 3D systems). A clean run reports nothing.
* The batch launch's grid barrier waits with a bound: a launch whose CTAs wait for more arrivals
  than the grid has gives up after its poll limit with SBP_ERR_TIMEOUT, every CTA returns, and
  the context stays usable (the same barrier then opens for a reachable count)."""
import numpy as np
import pytest

import workloads as W
from conftest import build_library

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

NONFINITE, TIMEOUT = -5, -7


@pytest.fixture(scope="module")
def sbp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build_library()
    import paper_1805_06607_gb300 as mod
    return mod


def _planted(wl, value, var=0):
    q = [np.array(x) for x in wl["q0"]]
    j, i = q[0].shape[1] // 2, q[0].shape[2] // 3
    q[0][var, j, i] = value
    return q


def _clean_step(sbp, wl, dtype="f64"):
    g = sbp.System(wl, dtype=dtype)
    qd = [g.to_device(k, wl["q0"][k]) for k in range(2)]
    _, H = g.timestep(qd[0], qd[1])
    return g, H


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("value,var", [(float("nan"), 3), (float("inf"), 1), (-1.0, 0)], ids=["nan", "inf", "rho<0"])
def test_planted_bad_state_is_reported(sbp, dtype, value, var):
    wl = W.vortex_box_in_box(seed=61, n_bg=40, n_fine=25)
    g, H = _clean_step(sbp, wl, dtype)
    g.autotune(False)
    g.bind(_planted(wl, value, var))
    g.mrab_init(H)
    g.mrab_step(1)
    with pytest.raises(sbp.SbpError) as e:
        g.check()
    assert e.value.status == NONFINITE
    g.check()      # the word was cleared by the read
    g.close()


def test_clean_run_reports_nothing(sbp):
    wl = W.vortex_box_in_box(seed=62, n_bg=40, n_fine=25)
    g, H = _clean_step(sbp, wl)
    g.bind(wl["q0"])
    g.mrab_init(H)
    g.mrab_step(3)
    g.check()
    g.close()


def test_batch_reports_bad_member(sbp):
    wls = W.batched_vortices(seed=63, n_systems=3, n_range=(96, 128), ratios=(2, 4))
    members = []
    for n, wl in enumerate(wls):
        g, H = _clean_step(sbp, wl)
        g.autotune(False)
        g.bind(_planted(wl, float("nan"), 2) if n == 1 else wl["q0"])
        g.mrab_init(H)
        members.append(g)
    b = sbp.Batch(members, autotune=False)
    b.step(1)
    with pytest.raises(sbp.SbpError) as e:
        b.check()
    assert e.value.status == NONFINITE
    b.close()
    for g in members:
        g.close()


def test_3d_reports_bad_state(sbp):
    wl = W.taylor_green_small(seed=64)
    g = sbp.System3D(wl)
    qd = [g.to_device(k, wl["q0"][k]) for k in range(2)]
    _, H = g.timestep(qd[0], qd[1])
    q = [np.array(x) for x in wl["q0"]]
    q[0][4, 5, 6, 7] = float("nan")
    g.bind(q)
    g.mrab_init(H)
    g.mrab_step(1)
    with pytest.raises(sbp.SbpError) as e:
        g.check()
    assert e.value.status == NONFINITE
    g.close()


def test_grid_barrier_wait_is_bounded(sbp):
    # 2 CTAs wait for 3 arrivals: nobody can pass; each gives up after 4096 polls (~1 ms)
    status, passed = sbp.barrier_selftest(2, 3, 4096)
    assert status == TIMEOUT and passed == 0
    # the context is still usable, and the same barrier opens for a count the grid reaches
    x = torch.arange(8, device="cuda", dtype=torch.float64)
    assert float((x * 2).sum()) == 56.0
    status, passed = sbp.barrier_selftest(4, 4, 4096)
    assert status == 0 and passed == 4


def test_barrier_selftest_refuses_unbounded_arguments(sbp):
    for args in ((0, 1, 10), (9, 1, 10), (2, 0, 10), (2, 3, 0), (2, 3, 1 << 20)):
        with pytest.raises(sbp.SbpError):
            sbp.barrier_selftest(*args)
