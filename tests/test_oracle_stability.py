"""Step-matrix stability (Sec. 4.3) of the oracle's MRAB step, pinned to theory.

On a uniform flow the linearised semi-discretisation is the periodic SBP operator (spectral
radius 1.3722 / dx on the imaginary axis, Sec. 4.4) times the wave speeds, so single-rate AB3
at the fast mesh's micro step is stable up to (AB3 imaginary-axis bound) / 1.3722 of the
Sec. 4.1 step estimate. The AB3 bound is computed here from the AB3 weights by the boundary
locus. MRAB with step ratio 2 on the vortex geometry, where the fine patch sets the limit,
must reach that bound (the paper's ~100 % efficiency below the spacing ratio).
"""
import numpy as np

import workloads as W
from conftest import golden
from oracle import OracleSystem, ab_coefficients


def _arnoldi_radius(matvec, n, kdim=60, seed=0):
    V = np.zeros((kdim + 1, n))
    Hm = np.zeros((kdim + 1, kdim))
    v = np.random.default_rng(seed).standard_normal(n)
    V[0] = v / np.linalg.norm(v)
    for j in range(kdim):
        w = matvec(V[j])
        for _ in range(2):
            for i in range(j + 1):
                c = V[i] @ w
                Hm[i, j] += c
                w -= c * V[i]
        Hm[j + 1, j] = np.linalg.norm(w)
        V[j + 1] = w / Hm[j + 1, j]
    return float(np.abs(np.linalg.eigvals(Hm[:kdim, :kdim])).max())


def _ab3_imaginary_bound():
    """Largest y with AB3 stable at lambda dt = i y: boundary locus z = e^{i theta},
    lambda dt = (z^3 - z^2) / sum_k alpha_k z^k, first crossing of the imaginary axis."""
    a = ab_coefficients(np.array([-2.0, -1.0, 0.0]), 0.0, 1.0, 3)  # oldest first
    th = np.linspace(0.05, np.pi, 200001)  # away from the tangency at the origin
    z = np.exp(1j * th)
    mu = (z ** 3 - z ** 2) / (a[0] + a[1] * z + a[2] * z ** 2)
    s = np.sign(mu.real)
    idx = np.nonzero(s[1:] != s[:-1])[0]
    return float(np.min(np.abs(mu.imag[idx])))


def test_arnoldi_radius_finds_outlier():
    rng = np.random.default_rng(1)
    n = 300
    Q = np.linalg.qr(rng.standard_normal((n, n)))[0]
    ev = np.concatenate([[1.3], 0.9 * np.exp(2j * np.pi * rng.uniform(size=n - 1)).real])
    A = Q @ np.diag(ev) @ Q.T
    assert abs(_arnoldi_radius(lambda v: A @ v, n) - 1.3) < 1e-8


def test_ab3_imaginary_axis_bound():
    assert abs(_ab3_imaginary_bound() - 0.7236) < 1e-3


def test_mrab_uniform_flow_stability_limit_matches_theory():
    wl = W.vortex_box_in_box(seed=51, n_bg=32, n_fine=21)
    o = OracleSystem(wl)
    qinf = np.asarray(wl["params"]["qinf"])
    uni = [np.broadcast_to(qinf[:, None, None], (4, m["n"][1], m["n"][0])).copy() for m in wl["meshes"]]
    m = wl["params"]["hist_len"]
    sr = wl["params"]["step_ratio"]
    F, Sl = o.fast, o.slow
    act = [o.iblank[k] != 0 for k in range(2)]
    spectral = float(golden("periodic_spectrum.txt")[0][0])
    f_star = _ab3_imaginary_bound() / spectral
    dt_fast = o.dt_mesh(F, uni[F])

    def pack(hs):
        return np.concatenate([x for k, (q, h) in enumerate(hs)
                               for x in (q[:, act[k]].reshape(-1), h[:, :, act[k]].reshape(-1))])

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

    def rho(H):
        qs, hf, hs = o.bootstrap(uni, H)
        base = [None, None]
        base[F] = (qs[F], np.stack(hf[:-1]))
        base[Sl] = (qs[Sl], np.stack(hs[:-1]))

        def step(state):
            q = [state[0][0], state[1][0]]
            hist_f = list(state[F][1]) + [o.coupled_rhs(F, q[F], q[Sl])]
            hist_s = list(state[Sl][1]) + [o.coupled_rhs(Sl, q[Sl], q[F])]
            qn, a, b = o.mrab(q, hist_f, hist_s, H, 1)
            out = [None, None]
            out[F] = (qn[F], np.stack(a[:-1]))
            out[Sl] = (qn[Sl], np.stack(b[:-1]))
            return pack(out)

        b0 = pack(base)
        y0 = step(base)

        def mv(v):
            nv = np.linalg.norm(v)
            return (step(unpack(b0 + 1e-7 * v / nv, base)) - y0) * (nv / 1e-7)

        return _arnoldi_radius(mv, b0.size)

    assert rho(0.95 * f_star * sr * dt_fast) <= 1.0 + 1e-3
    assert rho(1.05 * f_star * sr * dt_fast) > 1.0 + 1e-3
