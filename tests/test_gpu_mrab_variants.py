"""The slowest-first MRAB variants of Sec. 3.3's design choices on the GPU path, against the
oracle's macro steps (oracle.mrab_macro_step_slowest_first), on the increments over the tested
steps: 1e-12 relative in FP64; in FP32 the states within 1e-5 and the increments within the
derived FP32 right-hand-side bound; CUDA-graph replay (slow right-hand side and fast micro steps on parallel branches) equal
to kernel-by-kernel launches; at step ratio 1 every ordering is single-rate AB, bit for bit."""
import numpy as np
import pytest

import workloads as W
from conftest import build_library
from oracle import OracleSystem
from tolerances import U32, U64, fp32_rhs_tol, increment_tol, rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SCHEMES = ["slowest_first", "slowest_first_reextrapolate"]


@pytest.fixture(scope="module")
def sbp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build_library()
    import paper_1805_06607_gb300 as mod
    return mod


def with_scheme(wl, scheme):
    return dict(wl, params=dict(wl["params"], scheme=scheme))


CASES = {
    "vortex": lambda: W.vortex_box_in_box(seed=31),
    "vortex_sr3_ab34": lambda: W.vortex_box_in_box(seed=32, n_bg=48, n_fine=33, step_ratio=3, hist_len=4),
    "cylinder": lambda: W.cylinder_small(seed=33),
}


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("case", sorted(CASES))
def test_variant_matches_oracle_fp64(sbp, case, scheme):
    wl = with_scheme(CASES[case](), scheme)
    ref = OracleSystem(wl)
    H = ref.macro_step_size(wl["q0"])
    y, hf, hs = ref.bootstrap(wl["q0"], H)
    n = 4
    want, _, _ = ref.mrab(y, hf, hs, H, n, scheme=scheme)
    g = sbp.System(wl)
    g.bind(wl["q0"])
    g.mrab_init(H)
    start = [g.to_host(k, g.current_state(k)) for k in range(2)]
    g.mrab_step(n)
    g.check()
    sr = wl["params"]["step_ratio"]
    for k in range(2):
        got = g.to_host(k, g.current_state(k))
        e = rel(got, want[k])
        assert e < 1e-12, (k, e)
        ei = rel(got - start[k], want[k] - y[k])
        tol = increment_tol(1e-12, y[k], want[k], n * sr, U64)
        assert ei < tol, (k, ei, tol)
    g.close()


@pytest.mark.parametrize("scheme", SCHEMES)
def test_variant_fp32(sbp, scheme):
    wl = with_scheme(CASES["cylinder"](), scheme)
    ref = OracleSystem(wl)
    H = ref.macro_step_size(wl["q0"])
    y, hf, hs = ref.bootstrap(wl["q0"], H)
    want, _, _ = ref.mrab(y, hf, hs, H, 3, scheme=scheme)
    g = sbp.System(wl, dtype="f32")
    g.bind(wl["q0"])
    g.mrab_init(H)
    start = [g.to_host(k, g.current_state(k)) for k in range(2)]
    g.mrab_step(3)
    g.check()
    q0 = wl["q0"]
    bar = max(fp32_rhs_tol(ref.met[j], q0[j], ref.iblank[j] != 0, ref.coupled_rhs(j, q0[j], q0[1 - j]),
                               ref.mu, ref.pr)
              for j in range(2))
    sr = wl["params"]["step_ratio"]
    for k in range(2):
        act = ref.iblank[k] != 0
        got = g.to_host(k, g.current_state(k))[:, act]
        assert rel(got, want[k][:, act]) < 1e-5
        ei = rel(got - start[k][:, act], want[k][:, act] - y[k][:, act])
        tol = increment_tol(bar, y[k][:, act], want[k][:, act], 3 * sr, U32)
        assert ei < tol, (k, ei, tol)
    g.close()


@pytest.mark.parametrize("scheme", SCHEMES)
def test_variant_graph_matches_eager(sbp, scheme):
    wl = with_scheme(CASES["vortex_sr3_ab34"](), scheme)
    out = []
    for graphs in (False, True):
        g = sbp.System(wl)
        g.use_graphs(graphs)
        g.bind(wl["q0"])
        g.mrab_init()
        g.mrab_step(9)
        g.check()
        out.append([g.to_host(k, g.current_state(k)) for k in range(2)])
        g.close()
    for k in range(2):
        assert np.array_equal(out[0][k], out[1][k])


def test_step_ratio_one_orderings_agree(sbp):
    base = W.vortex_box_in_box(seed=34, n_bg=40, n_fine=25, step_ratio=1)
    out = {}
    for scheme in ["fastest_first"] + SCHEMES:
        g = sbp.System(with_scheme(base, scheme))
        g.bind(base["q0"])
        g.mrab_init()
        g.mrab_step(5)
        g.check()
        out[scheme] = [g.to_host(k, g.current_state(k)) for k in range(2)]
        g.close()
    for scheme in SCHEMES:
        for k in range(2):
            assert np.array_equal(out[scheme][k], out["fastest_first"][k]), scheme


def test_variant_state_record_refused(sbp):
    wl = with_scheme(CASES["vortex"](), "slowest_first")
    g = sbp.System(wl)
    g.bind(wl["q0"])
    g.mrab_init()
    with pytest.raises(RuntimeError):
        g.get_state()
    g.close()


@pytest.mark.parametrize("case", ["vortex", "vortex_sr3_ab34", "cylinder"])
def test_variable_macro_step_matches_oracle(sbp, case):
    """The macro step changes between macro steps (Sec. 3.3 Step 1): weights solved on the
    history's node times while it is not uniform, then the plan's weights again."""
    wl = CASES[case]()
    ref = OracleSystem(wl)
    H0 = ref.macro_step_size(wl["q0"])
    y, hf, hs = ref.bootstrap(wl["q0"], H0)
    steps = [H0, 0.7 * H0, 0.7 * H0, 1.1 * H0, 1.1 * H0, 1.1 * H0, 1.1 * H0, 1.1 * H0]
    want = ref.mrab_var(y, hf, hs, H0, steps)
    fixed, _, _ = ref.mrab(y, hf, hs, H0, len(steps))
    g = sbp.System(wl)
    g.bind(wl["q0"])
    g.mrab_init(H0)
    start = [g.to_host(k, g.current_state(k)) for k in range(2)]
    for Hi in steps:
        g.mrab_set_step(Hi)
        g.mrab_step(1)
    g.check()
    Hg, t = g.mrab_time()
    assert Hg == steps[-1] and t == pytest.approx(sum(steps))
    for k in range(2):
        got = g.to_host(k, g.current_state(k))
        assert rel(got, want[k]) < 1e-12, (k, rel(got, want[k]))
        ei = rel(got - start[k], want[k] - y[k])
        tol = increment_tol(1e-12, y[k], want[k], len(steps) * wl["params"]["step_ratio"], U64)
        assert ei < tol, (k, ei, tol)
        # and the run is not the fixed-step one: the increments differ
        assert rel(want[k] - y[k], fixed[k] - y[k]) > 1e-3
    g.close()
