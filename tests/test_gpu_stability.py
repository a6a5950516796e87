"""Step-matrix stability analysis (Sec. 4.3) on the GPU path.

- The integrator state round-trips through sbp_integrator_state, and a step from a state that
  was set equals a step from the state it was read from (checkpoint / resume).
- The matrix-free G_eps v on the GPU equals the oracle's finite difference of its own MRAB
  step along the same direction around the same state (the oracle's histories carry the newest
  right-hand side explicitly; the GPU computes it at the start of the step).
- The spectral-radius estimate (largest Ritz modulus of a Krylov space) agrees between the GPU
  and the oracle operators from the same start vector; it is below 1 at a small macro step and
  above 1 at a large one.
"""
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


def _small():
    return W.vortex_box_in_box(seed=51, n_bg=32, n_fine=21)


def test_state_roundtrip_and_resume(sbp):
    wl = _small()
    g = sbp.System(wl)
    g.bind(wl["q0"])
    g.mrab_init()
    g.mrab_step(2)
    st = g.get_state()
    g.mrab_step(3)
    a = [g.current_state(k).clone() for k in range(2)]
    g.set_state(st)
    g.mrab_step(3)
    b = [g.current_state(k).clone() for k in range(2)]
    for k in range(2):
        assert torch.equal(a[k], b[k])


def test_step_matrix_matches_oracle(sbp):
    from paper_1805_06607_gb300.stability import StepMatrix
    wl = _small()
    g = sbp.System(wl)
    g.bind(wl["q0"])
    q0 = [g.current_state(k) for k in range(2)]
    _, H = g.timestep(q0[0], q0[1])
    S = StepMatrix(g, H)
    o = OracleSystem(wl)
    m = wl["params"]["hist_len"]
    F, Sl = o.fast, o.slow
    act = [o.iblank[k] != 0 for k in range(2)]

    def to_host(state):
        return [(g.to_host(k, q), np.stack([g.to_host(k, hh) for hh in h])) for k, (q, h) in enumerate(state)]

    def pack(hs):
        parts = []
        for k, (q, h) in enumerate(hs):
            parts.append(q[:, act[k]].reshape(-1))
            parts.append(h[:, :, act[k]].reshape(-1))
        return np.concatenate(parts)

    def unpack(vec, like):
        out, o_ = [], 0
        for k, (q, h) in enumerate(like):
            q, h = q.copy(), h.copy()
            n = int(act[k].sum()) * 4
            q[:, act[k]] = vec[o_:o_ + n].reshape(4, -1)
            o_ += n
            nh = n * (m - 1)
            h[:, :, act[k]] = vec[o_:o_ + nh].reshape(m - 1, 4, -1)
            o_ += nh
            out.append((q, h))
        return out

    def oracle_step(hs):
        qs = [hs[0][0], hs[1][0]]
        hist_f = list(hs[F][1]) + [o.coupled_rhs(F, qs[F], qs[Sl])]
        hist_s = list(hs[Sl][1]) + [o.coupled_rhs(Sl, qs[Sl], qs[F])]
        qn, hf, hsl = o.mrab(qs, hist_f, hist_s, H, 1)
        out = [None, None]
        out[F] = (qn[F], np.stack(hf[:-1]))
        out[Sl] = (qn[Sl], np.stack(hsl[:-1]))
        return out

    base_h = to_host(S.phi0)
    assert np.allclose(pack(base_h), S.base, rtol=0, atol=0)
    y0 = pack(oracle_step(base_h))

    def ov_of(v):
        nv = np.linalg.norm(v)
        return (pack(oracle_step(unpack(S.base + S.eps * v / nv, base_h))) - y0) * (nv / S.eps)

    rng = np.random.default_rng(3)
    for _ in range(2):
        v = rng.standard_normal(S.n)
        gv, ov = S.matvec(v), ov_of(v)
        assert np.linalg.norm(gv - ov) <= 1e-5 * np.linalg.norm(ov)
    # the spectral-radius estimate from the same Krylov start agrees
    from paper_1805_06607_gb300.stability import arnoldi_radius
    rg = S.spectral_radius(kdim=20)
    ro = arnoldi_radius(ov_of, S.n, kdim=20)
    assert abs(rg - ro) <= 1e-5 * ro


@pytest.mark.timeout(900)
def test_spectral_radius_brackets_stability(sbp):
    from paper_1805_06607_gb300.stability import StepMatrix
    wl = _small()
    qinf = np.asarray(wl["params"]["qinf"], dtype=np.float64)
    uni = [np.broadcast_to(qinf[:, None, None], (4, m["n"][1], m["n"][0])).copy() for m in wl["meshes"]]
    rho = {}
    for f in (0.3, 1.0):
        g = sbp.System(wl)
        g.bind(uni)
        dts, _ = g.timestep(g.current_state(0), g.current_state(1))
        H = f * wl["params"]["step_ratio"] * dts[1]
        rho[f] = StepMatrix(g, H).spectral_radius()
        g.close()
    assert rho[0.3] <= 1.0 + 1e-3, rho
    assert rho[1.0] > 1.05, rho


def test_checkpoint_blob_resume_is_bit_identical(sbp):
    """sbp_checkpoint_save / _load: steps after a load give the bits of the steps after the
    save, in the same system and in a fresh one (whose right-hand-side shapes were never tuned:
    the kernel designs give the same bits); a checkpoint of another system, a truncated blob
    and a foreign blob are refused."""
    wl = _small()
    g = sbp.System(wl)
    g.bind(wl["q0"])
    g.mrab_init()
    g.mrab_step(3)
    g.mrab_set_step(g.mrab_time()[0] * 0.9)   # a variable-step transition in flight
    g.mrab_step(1)
    blob = g.checkpoint_save()
    t0 = g.mrab_time()
    g.mrab_step(4)
    a = [g.current_state(k).clone() for k in range(2)]
    ta = g.mrab_time()
    g.checkpoint_load(blob)
    assert g.mrab_time() == t0
    g.mrab_step(4)
    b = [g.current_state(k).clone() for k in range(2)]
    assert g.mrab_time() == ta
    for k in range(2):
        assert torch.equal(a[k], b[k])
    fresh = sbp.System(wl)
    fresh.bind(wl["q0"])
    fresh.checkpoint_load(blob)
    fresh.mrab_step(4)
    for k in range(2):
        assert torch.equal(a[k], fresh.current_state(k))
    h32 = sbp.System(wl, dtype="f32")
    h32.bind(wl["q0"])
    with pytest.raises(sbp.SbpError):
        h32.checkpoint_load(blob)
    with pytest.raises(sbp.SbpError):
        fresh.checkpoint_load(blob[:-8])
    with pytest.raises(sbp.SbpError):
        fresh.checkpoint_load(b"x" * len(blob))
    for s in (g, fresh, h32):
        s.close()
