"""The single-pass marching right-hand-side kernel (rows staged by per-thread cp.async, or by
TMA tensor copies) against the kernel pair and the oracle.

Both designs perform the same floating-point operations per point in the same order, so the
right-hand side and whole MRAB runs must agree bit for bit, for every chunk height (chunks that are
not a multiple of the rows per tick, chunks taller than the mesh,
periodic wrap in i and j, holes, ragged edges), in FP64 and FP32; FP64 also matches the oracle
to the 1e-12 parity bar."""
import numpy as np
import pytest

import workloads as W
from conftest import build_library
from oracle import OracleSystem

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sbp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build_library()
    import paper_1805_06607_gb300 as mod
    return mod


CASES = {
    "vortex": lambda: W.vortex_box_in_box(seed=31),
    "cylinder": lambda: W.cylinder_small(seed=32),
    "mms_viscous": lambda: W.mms_box_in_box(52, "viscous"),
    "cylinder_ragged": lambda: W.cylinder_small(seed=33, n_theta=72, n_r=20, bg_n=(90, 50), hist_len=4),
    "cylinder_sponge": lambda: W.cylinder_small(seed=36, sponge_cells=6, sponge_strength=2.0),
    "cylinder_euler": lambda: _euler(W.cylinder_small(seed=37)),
}


def _euler(wl):
    """The same meshes and state with the Euler equations (no viscous terms)."""
    return dict(wl, params=dict(wl["params"], physics="euler", mu=0.0))
TMA = 0x10000   # chunk flag: rows staged by TMA tensor copies (k_march_tma)
SHAPES = [(58, 7), (58, 32), (58, 1), (58, 24), (58, 128), (58, 1000),
          (58, 7 | TMA), (58, 32 | TMA), (58, 1 | TMA), (58, 128 | TMA), (58, 1000 | TMA)]


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_march_rhs_bit_identical(sbp, case, dtype):
    wl = CASES[case]()
    g = sbp.System(wl, dtype=dtype)
    q = [g.to_device(k, wl["q0"][k]) for k in range(2)]
    for k in range(2):
        g.set_rhs_shape(k, 0, 16)
        ref = g.rhs_eval(k, q[k], q[1 - k]).clone()
        for strip, rows in SHAPES:
            g.set_rhs_shape(k, strip, rows)
            info = g.mesh_info(k)
            assert info.single_pass == 1 and info.strip_width == strip and info.rows_per_cta == rows
            got = g.rhs_eval(k, q[k], q[1 - k])
            assert torch.equal(got, ref), (k, strip, rows)
    if dtype == "f64":
        o = OracleSystem(wl)
        for k in range(2):
            g.set_rhs_shape(k, 58, 24)
            got = g.to_host(k, g.rhs_eval(k, q[k], q[1 - k]))
            want = o.coupled_rhs(k, wl["q0"][k], wl["q0"][1 - k])
            act = o.iblank[k] != 0
            assert _rel(got[:, act], want[:, act]) < 1e-12


@pytest.mark.parametrize("case", ["vortex", "cylinder_ragged"])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_pair_row_splits_bit_identical(sbp, case, dtype):
    """Flux and derivative kernels with different rows per CTA (the derivative kernel's 4-row
    blocks search their 8-row group's SAT range) give the same bits, in rhs_eval and in MRAB
    steps (which hand the fast mesh's primitives from micro step to micro step)."""
    wl = CASES[case]()
    g = sbp.System(wl, dtype=dtype)
    q = [g.to_device(k, wl["q0"][k]) for k in range(2)]
    splits = [(8, 4), (16, 4), (16, 8), (32, 16), (32, 4), (4, 4), (4, 8)]
    for k in range(2):
        g.set_rhs_shape(k, 0, 16)
        ref = g.rhs_eval(k, q[k], q[1 - k]).clone()
        for rf, ru in splits:
            g.set_rhs_shape(k, 0, rf, ru)
            assert g.mesh_info(k).rows_update == ru
            assert torch.equal(g.rhs_eval(k, q[k], q[1 - k]), ref), (k, rf, ru)
    g.close()
    runs = []
    for rf, ru in [(16, 0)] + splits:
        g = sbp.System(wl, dtype=dtype)
        g.autotune(False)
        for k in range(2):
            g.set_rhs_shape(k, 0, rf, ru)
        g.bind(wl["q0"])
        g.mrab_init()
        g.mrab_step(5)
        g.check()
        runs.append([g.current_state(k).clone() for k in range(2)])
        g.close()
    for r in runs[1:]:
        for k in range(2):
            assert torch.equal(r[k], runs[0][k])


@pytest.mark.parametrize("case", ["vortex", "cylinder_ragged"])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_march_mrab_bit_identical(sbp, case, dtype):
    wl = CASES[case]()
    runs = []
    for shape in [(0, 8), (58, 40), (58, 16), (58, 16 | TMA), (58, 40 | TMA)]:
        g = sbp.System(wl, dtype=dtype)
        g.autotune(False)
        for k in range(2):
            g.set_rhs_shape(k, *shape)
        g.bind(wl["q0"])
        g.mrab_init()
        g.mrab_step(5)
        g.check()
        runs.append([g.current_state(k).clone() for k in range(2)])
        g.close()
    for r in runs[1:]:
        for k in range(2):
            assert torch.equal(r[k], runs[0][k])


def test_autotuner_reports_a_candidate(sbp):
    wl = W.cylinder_small(seed=34)
    g = sbp.System(wl, dtype="f32")
    g.bind(wl["q0"])
    g.mrab_init()
    for k in range(2):
        info = g.mesh_info(k)
        for sp, sw, rows in ((info.single_pass, info.strip_width, info.rows_per_cta),
                             (info.eval_single_pass, info.eval_strip_width, info.eval_rows_per_cta)):
            if sp:  # marching (58 columns, chunk | TMA staging flag) or column kernels
                assert (sw == 58 and rows & 0xFFFF in (8, 16, 32, 64, 128) and rows >> 16 in (0, 1)) or \
                    (sw in (116, 244) and rows in (32, 64, 128, 256))
            else:   # the kernel pair
                assert sw == 32 and rows in (4, 8, 16, 32)
    # the autotuner's choices give the same bits as any other shape: rhs_eval and a macro step
    # against a fixed kernel pair
    q = [g.to_device(k, wl["q0"][k]) for k in range(2)]
    got = [g.rhs_eval(k, q[k], q[1 - k]).clone() for k in range(2)]
    g2 = sbp.System(wl, dtype="f32")
    g2.autotune(False)
    for k in range(2):
        g2.set_rhs_shape(k, 0, 16)
        assert torch.equal(g2.rhs_eval(k, q[k], q[1 - k]), got[k])
    g.mrab_step(2)
    g2.bind(wl["q0"])
    g2.mrab_init()
    g2.mrab_step(2)
    for k in range(2):
        assert torch.equal(g.current_state(k), g2.current_state(k))
    g.close()
    g2.close()


def test_bad_shapes_rejected(sbp):
    wl = W.vortex_box_in_box(seed=35, n_bg=40, n_fine=25)
    g = sbp.System(wl)
    for args in [(0, 12), (48, 32), (32, 32), (64, 32), (58, 0), (58, -3), (0, 16 | (12 << 8)), (58, TMA),
                 (58, 16 | (2 << 16))]:
        with pytest.raises(sbp.SbpError):
            g.set_rhs_shape(0, *args)


COL_CASES = {
    "vortex_wide": lambda: W.vortex_box_in_box(seed=38, n_bg=160, n_fine=130),
    "cylinder_wide": lambda: W.cylinder_small(seed=39, n_theta=256, n_r=40, bg_n=(270, 150), s_bg=0.04),
    "cylinder_wide_euler": lambda: _euler(W.cylinder_small(seed=40, n_theta=256, n_r=40, bg_n=(270, 150), s_bg=0.04)),
    "mms_viscous_wide": lambda: W.mms_box_in_box(260, "viscous"),
}


@pytest.mark.parametrize("case", sorted(COL_CASES))
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_column_kernel_bit_identical(sbp, case, dtype):
    """The column-marching kernel (128- and 256-thread CTAs, chunks that are and are not
    multiples of 8 rows, chunks taller than the mesh) against the kernel pair, bit for bit, on
    right-hand sides and on MRAB runs; FP64 also against the oracle."""
    wl = COL_CASES[case]()
    g = sbp.System(wl, dtype=dtype)
    g.autotune(False)
    q = [g.to_device(k, wl["q0"][k]) for k in range(2)]
    shapes = [(116, 32), (116, 45), (244, 64), (244, 1000)]
    tried = 0
    for k in range(2):
        g.set_rhs_shape(k, 0, 16)
        ref = g.rhs_eval(k, q[k], q[1 - k]).clone()
        for strip, rows in shapes:
            if g.info[k].ni < strip + 12:
                with pytest.raises(sbp.SbpError):
                    g.set_rhs_shape(k, strip, rows)
                continue
            g.set_rhs_shape(k, strip, rows)
            info = g.mesh_info(k)
            assert info.single_pass == 1 and info.strip_width == strip
            assert torch.equal(g.rhs_eval(k, q[k], q[1 - k]), ref), (k, strip, rows)
            tried += 1
    assert tried >= 2
    if dtype == "f64":
        o = OracleSystem(wl)
        for k in range(2):
            if g.info[k].ni >= 128:
                g.set_rhs_shape(k, 116, 40)
            got = g.to_host(k, g.rhs_eval(k, q[k], q[1 - k]))
            want = o.coupled_rhs(k, wl["q0"][k], wl["q0"][1 - k])
            act = o.iblank[k] != 0
            assert _rel(got[:, act], want[:, act]) < 1e-12
    g.close()
    runs = []
    for shape in [(0, 16), (116, 40), (244, 64)]:
        g = sbp.System(wl, dtype=dtype)
        g.autotune(False)
        for k in range(2):
            if shape[0] == 0 or g.info[k].ni >= shape[0] + 12:
                g.set_rhs_shape(k, *shape)
        g.bind(wl["q0"])
        g.mrab_init()
        g.mrab_step(5)
        g.check()
        runs.append([g.current_state(k).clone() for k in range(2)])
        g.close()
    for r in runs[1:]:
        for k in range(2):
            assert torch.equal(r[k], runs[0][k])
