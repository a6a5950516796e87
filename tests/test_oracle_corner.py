"""The corner-penalty weight of Sec. 4.2 eq. (penalty_interp) in the oracle, pinned by what the
equation and the paper's study fix.

* Omega multiplies the interpolation penalty at fringe points with more than one interface term
  and nothing else: on the paper's box-in-box case (31^2 + 41^2, rho u = 1.25 - 0.01|x|) the
  derivative of the coupled right-hand side along any direction is affine in Omega, and its
  Omega-dependent part lives on the inner box's corner points alone (the two inflow corners carry
  it; at the supersonic outflow corners the characteristic penalty is zero).
* The case is mirror-symmetric in y, so its linearised operator commutes with the reflection
  (y -> -y, rho v -> -rho v); a sign or index slip in either direction's metric, flux or penalty
  breaks that.
* The study's finding: with the penalty sigma^I = 1 a corner-localised eigenvalue on the negative
  real axis moves outward as Omega goes from 1/2 to 1 (on a coarser copy of the case, 16^2 + 21^2
  on the same boxes, where the dense spectrum takes seconds).
Planted mistake: Omega applied to every interface term (on the CPU, in the oracle) puts the
Omega-dependent part on the faces.
"""
import numpy as np
import pytest

import workloads as W
from oracle import OracleSystem
from oracle.adjoint import coupled_rhs_jvp


def _jvp_all(o, q, d):
    return [coupled_rhs_jvp(o, k, q[k], q[1 - k], d[k], d[1 - k])[1] for k in range(2)]


def _unknowns(o):
    act = [o.iblank[k] != 0 for k in range(2)]
    return act, [(k, v, p) for k in range(2) for v in range(4) for p in np.flatnonzero(act[k].ravel())]


def _jacobian(o, q):
    act, idx = _unknowns(o)
    n = len(idx)
    J = np.zeros((n, n))
    for c, (k, v, p) in enumerate(idx):
        d = [np.zeros_like(q[0]), np.zeros_like(q[1])]
        d[k].reshape(4, -1)[v, p] = 1.0
        r = _jvp_all(o, q, d)
        J[:, c] = np.concatenate([r[kk].reshape(4, -1)[:, act[kk].ravel()].ravel() for kk in range(2)])
    return J, idx


def _corner_rows(o):
    """Points (mesh, flat index) with more than one interface term."""
    out = set()
    for k in range(2):
        t = o.terms[k]
        pts, cnt = np.unique(t["pt"][t["kind"] == 1], return_counts=True)
        out |= {(k, int(p)) for p in pts[cnt > 1]}
    return out


def _omega_part(make):
    wl0 = W.corner_box_in_box(0.0)
    q = wl0["q0"]
    o = {om: make(W.corner_box_in_box(om)) for om in (0.0, 0.5, 1.0)}
    rng = np.random.default_rng(7)
    parts = []
    for _ in range(3):
        d = [rng.standard_normal(x.shape) for x in q]
        r = {om: _jvp_all(o[om], q, d) for om in o}
        parts.append([(r[1.0][k] - r[0.5][k], r[0.5][k] - r[0.0][k], r[1.0][k]) for k in range(2)])
    return o[1.0], parts


def test_corner_weight_enters_only_at_corner_fringe_points():
    o, parts = _omega_part(OracleSystem)
    corners = _corner_rows(o)
    ni, nj = o.meshes[1]["n"]
    assert {p for k, p in corners if k == 1} == {0, ni - 1, (nj - 1) * ni, nj * ni - 1}
    assert not any(k == 0 for k, _ in corners)
    inflow = {(1, 0), (1, (nj - 1) * ni)}
    for part in parts:
        for k in range(2):
            hi, lo, full = part[k]
            scale = np.abs(full).max()
            assert np.abs(hi - lo).max() <= 1e-12 * scale  # affine in Omega
            nz = np.nonzero(np.abs(hi).max(axis=0).ravel() > 1e-13 * scale)[0]
            assert {(k, int(p)) for p in nz} <= corners
            if k == 1:
                assert inflow <= {(1, int(p)) for p in nz}


def test_planted_omega_on_every_interface_term_is_caught():
    class EveryTerm(OracleSystem):
        def _build_terms(self):
            super()._build_terms()
            for k in range(2):
                t = self.terms[k]
                t["scale"] = np.where(t["kind"] == 1, float(self.p["omega_corner"]), 1.0)

    o, parts = _omega_part(EveryTerm)
    corners = _corner_rows(o)
    hi = parts[0][1][0]
    nz = np.nonzero(np.abs(hi).max(axis=0).ravel() > 1e-13 * np.abs(parts[0][1][2]).max())[0]
    assert not ({(1, int(p)) for p in nz} <= corners)


@pytest.fixture(scope="module")
def coarse_spectra():
    out = {}
    for om in (1.0, 0.5):
        wl = W.corner_box_in_box(om, n_bg=16, n_fine=21)
        o = OracleSystem(wl, sig_int=1.0)
        J, idx = _jacobian(o, wl["q0"])
        out[om] = (np.linalg.eigvals(J), J, idx, wl)
    return out


def test_linearised_operator_is_mirror_symmetric(coarse_spectra):
    _, J, idx, wl = coarse_spectra[1.0]
    pos = {t: a for a, t in enumerate(idx)}
    perm = np.empty(len(idx), dtype=np.int64)
    sign = np.ones(len(idx))
    for a, (k, v, p) in enumerate(idx):
        ni, nj = wl["meshes"][k]["n"]
        i, j = p % ni, p // ni
        jr = (nj - j) % nj if k == 0 else nj - 1 - j  # the periodic background wraps at y = -4 = 4
        perm[a] = pos[(k, v, jr * ni + i)]
        sign[a] = -1.0 if v == 2 else 1.0
    RJR = (sign[:, None] * sign[None, :]) * J[np.ix_(perm, perm)]
    assert np.abs(RJR - J).max() <= 1e-12 * np.abs(J).max()


def _eigvec(J, mu):
    """Eigenvector for the eigenvalue nearest mu (inverse iteration beside it)."""
    import scipy.linalg as sl
    lu = sl.lu_factor(J - (mu + 1e-9 * abs(mu)) * np.eye(J.shape[0]))
    v = np.random.default_rng(0).standard_normal(J.shape[0])
    for _ in range(6):
        v = sl.lu_solve(lu, v)
        v /= np.linalg.norm(v)
    return v


def test_corner_eigenvalue_moves_out_along_the_negative_real_axis(coarse_spectra):
    most = {}
    for om, (lam, J, idx, wl) in coarse_spectra.items():
        scale = np.abs(lam).max()
        assert lam.real.max() <= 1e-3 * scale  # no growing mode at either weight with sigma^I = 1
        real = np.nonzero(np.abs(lam.imag) <= 1e-9 * scale)[0]
        a = real[np.argmin(lam[real].real)]
        most[om] = lam[a].real
        ni, nj = wl["meshes"][1]["n"]
        near = np.array([k == 1 and min(p % ni, ni - 1 - p % ni) <= 2 and min(p // ni, nj - 1 - p // ni) <= 2
                         for (k, v, p) in idx])
        w = np.abs(_eigvec(J, lam[a].real)) ** 2
        assert w[near].sum() / w.sum() > 0.5, (om, lam[a], w[near].sum() / w.sum())
    assert most[1.0] < most[0.5] - 0.2 * abs(most[0.5])


def test_derivative_at_a_zero_wave_speed_is_the_central_difference():
    """With v = 0 the penalty of every y-direction SAT term sits on the kink of the characteristic
    splitting (wave speed k.u = 0): the oracle's derivative there is the mean of the one-sided
    slopes, the limit of a central difference of the plain oracle (a one-sided rule would leave
    an O(1) gap, not an O(eps^2) one)."""
    wl = W.corner_box_in_box(1.0, n_bg=16, n_fine=21)
    o = OracleSystem(wl)
    q = wl["q0"]
    rng = np.random.default_rng(11)
    d = [rng.standard_normal(x.shape) for x in q]
    eps = 1e-6
    for k in range(2):
        got = coupled_rhs_jvp(o, k, q[k], q[1 - k], d[k], d[1 - k])[1]
        plus = o.coupled_rhs(k, q[k] + eps * d[k], q[1 - k] + eps * d[1 - k])
        minus = o.coupled_rhs(k, q[k] - eps * d[k], q[1 - k] - eps * d[1 - k])
        fd = (plus - minus) / (2.0 * eps)
        assert np.abs(got - fd).max() <= 1e-6 * np.abs(fd).max()
