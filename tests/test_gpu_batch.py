"""Batched persistent stepping (one cooperative launch per micro step over all member systems)
against the oracle (each member's bootstrap and macro steps against OracleSystem's, on states and
increments), and against stepping each member alone: the same kernels' arithmetic, so the states
must agree bit for bit, over more macro steps than the ring-phase period."""
import numpy as np
import pytest

import workloads as W
from conftest import build_library
from oracle import OracleSystem
from tolerances import U32, U64, fp32_rhs_tol, increment_tol, rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sbp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build_library()
    import paper_1805_06607_gb300 as mod
    return mod


def _members(sbp, wls, dtype):
    out = []
    for wl in wls:
        g = sbp.System(wl, dtype=dtype)
        g.bind(wl["q0"])
        g.mrab_init()
        out.append(g)
    return out


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_batch_matches_oracle(sbp, dtype):
    """Four small members with step ratios 2, 4, 8 and 2 (backgrounds 96..128 points a side with a
    hole under the patch, patch spacing ratio = step ratio), stepped together: each member's states against the oracle's
    bootstrap + macro steps, FP64 to 1e-12 on states and increments; FP32 states to 1e-5 and
    increments within the derived FP32 right-hand-side bound."""
    spec = [(96, 2, 101), (104, 4, 102), (128, 8, 103), (112, 2, 104)]
    wls = [W.vortex_box_in_box(seed=s, n_bg=n, n_fine=int(round(n * r / 8.0)) + 1, bg_half=5.0,
                               fine_half=5.0 / 8.0, step_ratio=r, jitter=0.3) for n, r, s in spec]
    members = _members(sbp, wls, dtype)
    b = sbp.Batch(members, autotune=True)
    start = [[g.to_host(k, g.current_state(k)) for k in range(2)] for g in members]
    nsteps = 3
    b.step(nsteps)
    b.check()
    for wl, g, st in zip(wls, members, start):
        ref = OracleSystem(wl)
        H = ref.macro_step_size(wl["q0"])
        Hg, _ = g.mrab_time()
        # the FP32 form takes its step from its FP32 state; the oracle then runs with that step
        assert abs(Hg - H) <= (1e-14 if dtype == "f64" else 1e-6) * H
        H = Hg
        y, hf, hs = ref.bootstrap(wl["q0"], H)
        want, _, _ = ref.mrab(y, hf, hs, H, nsteps)
        q0, sr = wl["q0"], wl["params"]["step_ratio"]
        if dtype == "f64":
            bar, unit, stol = 1e-12, U64, 1e-12
        else:
            bar = max(fp32_rhs_tol(ref.met[j], q0[j], ref.iblank[j] != 0, ref.coupled_rhs(j, q0[j], q0[1 - j]),
                               ref.mu, ref.pr)
                      for j in range(2))
            unit, stol = U32, 1e-5
        for k in range(2):
            act = ref.iblank[k] != 0
            got = g.to_host(k, g.current_state(k))[:, act]
            assert rel(got, want[k][:, act]) < stol, (sr, k)
            ei = rel(got - st[k][:, act], want[k][:, act] - y[k][:, act])
            tol = increment_tol(bar, y[k][:, act], want[k][:, act], nsteps * sr, unit)
            assert ei < tol, (dtype, sr, k, ei, tol)
    b.close()
    for g in members:
        g.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_batch_matches_single_systems(sbp, dtype):
    wls = W.batched_vortices(seed=5, n_systems=5, n_range=(40, 72), ratios=(1, 2, 3, 4))
    single = _members(sbp, wls, dtype)
    batched = _members(sbp, wls, dtype)
    b = sbp.Batch(batched, autotune=True)
    info = b.info()
    assert info["members"] == 5 and info["rows_per_cta"] in (8, 16, 32, 64) and info["grid"] > 0
    nsteps = 7
    b.step(nsteps)
    b.check()
    for g in single:
        g.mrab_step(nsteps)
        g.check()
    for gs, gb in zip(single, batched):
        for k in range(2):
            a = gs.to_host(k, gs.current_state(k))
            c = gb.to_host(k, gb.current_state(k))
            assert np.array_equal(a, c)
        assert gs.mrab_time() == gb.mrab_time()
    b.close()
    for g in single + batched:
        g.close()


@pytest.mark.parametrize("rows", [8, 16, 32, 64])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_batch_shapes_match_single_systems(sbp, dtype, rows):
    """Every work-item shape (tile pairs of 8 / 16 rows, single-pass strips of 32 / 64 rows)
    reproduces each member stepped alone bit for bit, also after a change of shape between
    steps (the plan is rebuilt from the members' current ring phase)."""
    wls = W.batched_vortices(seed=6, n_systems=4, n_range=(40, 150), ratios=(1, 2, 4))
    single = _members(sbp, wls, dtype)
    batched = _members(sbp, wls, dtype)
    b = sbp.Batch(batched, autotune=False)
    b.step(2)
    b.set_shape(rows)
    assert b.info()["rows_per_cta"] == rows
    b.step(5)
    b.check()
    for g in single:
        g.mrab_step(7)
        g.check()
    for gs, gb in zip(single, batched):
        for k in range(2):
            assert np.array_equal(gs.to_host(k, gs.current_state(k)), gb.to_host(k, gb.current_state(k)))
    b.close()
    for g in single + batched:
        g.close()


@pytest.mark.parametrize("rows", [16, 32])
def test_batch_curvilinear_euler_shapes(sbp, rows):
    """Euler systems with a curvilinear fine mesh (small cylinders at step ratios 2 and 3) in a
    batch: tile pairs and single-pass strips on both mesh kinds reproduce the members."""
    wls = []
    for seed, sr in ((41, 2), (42, 3), (43, 2)):
        wl = W.cylinder_small(seed=seed, step_ratio=sr)
        wls.append(dict(wl, params=dict(wl["params"], physics="euler", mu=0.0)))
    single = _members(sbp, wls, "f32")
    batched = _members(sbp, wls, "f32")
    b = sbp.Batch(batched, autotune=False)
    b.set_shape(rows)
    b.step(4)
    b.check()
    for g in single:
        g.mrab_step(4)
        g.check()
    for gs, gb in zip(single, batched):
        for k in range(2):
            assert np.array_equal(gs.to_host(k, gs.current_state(k)), gb.to_host(k, gb.current_state(k)))
    b.close()
    for g in single + batched:
        g.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_batch_viscous_matches_single_systems(sbp, dtype):
    """Navier-Stokes members (small cylinders at step ratios 2 and 3; donor values with viscous
    fluxes, the primitives handed from micro step to micro step) in tile pairs of 16 rows: the
    batch reproduces each member stepped alone bit for bit."""
    wls = [W.cylinder_small(seed=s, step_ratio=sr) for s, sr in ((4, 2), (5, 3))]
    single = _members(sbp, wls, dtype)
    batched = _members(sbp, wls, dtype)
    b = sbp.Batch(batched, autotune=False)
    b.set_shape(16)
    b.step(4)
    b.check()
    for g in single:
        g.mrab_step(4)
        g.check()
    for gs, gb in zip(single, batched):
        for k in range(2):
            assert np.array_equal(gs.to_host(k, gs.current_state(k)), gb.to_host(k, gb.current_state(k)))
    b.close()
    for g in single + batched:
        g.close()


def test_batch_shape_viscous_rejects_strips(sbp):
    gs = _members(sbp, [W.cylinder_small(seed=3)], "f64")
    b = sbp.Batch(gs, autotune=False)
    with pytest.raises(sbp.SbpError):
        b.set_shape(32)
    b.close()
    for g in gs:
        g.close()


def test_batch_member_kinds_must_match(sbp):
    wl_e = W.vortex_box_in_box(seed=1, n_bg=40, n_fine=25)
    wl_n = W.cylinder_small(seed=2)
    gs = _members(sbp, [wl_e, wl_n], "f64")
    with pytest.raises(sbp.SbpError):
        sbp.Batch(gs)
    for g in gs:
        g.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_full_size_batch_matches_single_systems(sbp, dtype):
    """The benchmark's batch at full size (64 systems, backgrounds 128^2..512^2, step ratios 2, 4
    and 8) with the autotuner's work-item shape: one macro step of the batch equals each member's
    own macro step bit for bit."""
    wls = W.batched_vortices(seed=0)
    single = _members(sbp, wls, dtype)
    batched = _members(sbp, wls, dtype)
    b = sbp.Batch(batched, autotune=True)
    b.step(1)
    b.check()
    for g in single:
        g.mrab_step(1)
        g.check()
    for gs, gb in zip(single, batched):
        for k in range(2):
            assert np.array_equal(gs.to_host(k, gs.current_state(k)), gb.to_host(k, gb.current_state(k)))
    b.close()
    for g in single + batched:
        g.close()
