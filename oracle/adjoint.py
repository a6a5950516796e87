"""The oracle's own derivative (TEST INFRASTRUCTURE ONLY: the reference for the GPU's discrete
adjoint; the GPU library never uses it).

``dual.cpp`` compiles the oracle's per-point arithmetic (``orc2d.c``) with dual numbers, so one
pass gives the right-hand side and its exact derivative along one direction of the inputs
(forward mode; no differencing step). On top of it:

* ``coupled_rhs_jvp`` - ``OracleSystem.coupled_rhs`` and its derivative along (dq_self, dq_other,
  dqinf): the receivers' interpolation of the donor state (and of its viscous fluxes), the
  mesh's right-hand side with its SAT terms, and the sponge term, in the same operations;
* ``rhs_vjp`` - the vector-Jacobian product lam^T dR/d(q_self, q_other, qinf), column by column
  of the Jacobian (tiny meshes only: one dual pass per input);
* ``probe_objective_jvp`` - ``system.probe_objective`` (Runge-Kutta bootstrap, MRAB macro steps,
  probe pressures) and its exact derivative along a direction of the initial states and of the
  far-field state, operation for operation on (value, derivative) pairs.
The values carried along are the plain oracle's, bit for bit (the tests check it).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from .system import ab_coefficients, probe_stencil

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liborc_dual.so")
_lib = None


class Dual(ctypes.Structure):
    _fields_ = [("v", ctypes.c_double), ("d", ctypes.c_double)]


def _load():
    global _lib
    if _lib is not None:
        return _lib
    deps = [os.path.join(_HERE, f) for f in ("dual.cpp", "orc2d.c", "orc_sbp.h")]
    if not os.path.exists(_SO) or os.path.getmtime(_SO) < max(os.path.getmtime(d) for d in deps):
        os.makedirs(os.path.dirname(_SO), exist_ok=True)
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["g++", "-O1", "-std=c++17", "-fPIC", "-shared", "-w", "-ffp-contract=off",
                               "-I", _HERE, os.path.join(_HERE, "dual.cpp"), "-o", tmp])
        os.replace(tmp, _SO)
    L = ctypes.CDLL(_SO)
    P, I, D = ctypes.c_void_p, ctypes.c_int, Dual
    L.orc_rhs2d.argtypes = [I, I, I, I, P, P, P, P, I, D, D, D,
                            I, P, P, P, P, P, P, I, P, P, P, D, D, D, P]
    L.orc_rhs2d.restype = I
    L.orc_interp2d.argtypes = [I, I, I, P, I, P, P, P]
    L.orc_interp2d.restype = I
    L.orc_viscflux2d.argtypes = [I, I, I, I, P, P, P, P, D, D, D, P]
    L.orc_viscflux2d.restype = I
    _lib = L
    return L


def pairs(v, d=None):
    """(value, derivative) pairs of an array, derivative 0 when d is None."""
    v = np.asarray(v, dtype=np.float64)
    return np.ascontiguousarray(np.stack([v, np.zeros_like(v) if d is None else np.asarray(d, np.float64)], -1))


def _p(a):
    return ctypes.c_void_p(a.ctypes.data)


def _viscflux(osys, k, qd):
    L = _load()
    m = osys.meshes[k]
    ni, nj = m["n"]
    fv = np.zeros((6, nj, ni, 2))
    met = pairs(osys.met[k])
    L.orc_viscflux2d(ni, nj, int(m["periodic"][0]), int(m["periodic"][1]), _p(osys.ci[k]), _p(osys.cj[k]), _p(met),
                     _p(qd), Dual(osys.gamma, 0.0), Dual(osys.mu, 0.0), Dual(osys.pr, 0.0), _p(fv))
    return fv


def _interp(osys, k, fd):
    L = _load()
    dm = osys.meshes[1 - k]
    nf = fd.shape[0]
    n = osys.recv_pts[k].size
    out = np.zeros((nf, n, 2))
    if n:
        w = pairs(osys.w[k])
        L.orc_interp2d(dm["n"][0], dm["n"][1], nf, _p(fd), n, _p(osys.base[k]), _p(w), _p(out))
    return out


def coupled_rhs_jvp(osys, k, q_self, q_other, dq_self=None, dq_other=None, dqinf=None):
    """(dq/dt, its derivative along dq_self, dq_other, dqinf) of mesh k: the operations of
    OracleSystem.coupled_rhs on (value, derivative) pairs."""
    L = _load()
    m = osys.meshes[k]
    ni, nj = m["n"]
    qs = pairs(q_self, dq_self)
    qo = pairs(q_other, dq_other)
    qhat = _interp(osys, k, qo)
    fvhat = _interp(osys, k, _viscflux(osys, 1 - k, qo)) if osys.viscous else None
    t = osys.terms[k]
    out = np.zeros((4, nj, ni, 2))
    qinf = pairs(osys.p["qinf"], dqinf)
    met = pairs(osys.met[k])
    scale = pairs(t["scale"])
    rc = L.orc_rhs2d(ni, nj, int(m["periodic"][0]), int(m["periodic"][1]), _p(osys.ci[k]), _p(osys.cj[k]), _p(met),
                     _p(qs), int(osys.viscous), Dual(osys.gamma, 0.0), Dual(osys.mu, 0.0), Dual(osys.pr, 0.0),
                     t["pt"].size, _p(t["pt"]), _p(t["dir"]), _p(t["side"]), _p(t["kind"]), _p(t["recv"]),
                     _p(scale), qhat.shape[1], _p(qhat), _p(fvhat) if fvhat is not None else None, _p(qinf),
                     Dual(float(osys.p["twall"]), 0.0), Dual(osys.sig_int, 0.0), Dual(osys.sig_phys, 0.0), _p(out))
    if rc != 0:
        raise RuntimeError("dual oracle rhs failed: %d" % rc)
    v, d = out[..., 0], out[..., 1]
    if int(osys.p.get("sponge_cells", 0)) > 0:
        sg = osys.sponge_strength(k)[None]
        v = v - sg * (qs[..., 0] - qinf[:, None, None, 0])
        d = d - sg * (qs[..., 1] - qinf[:, None, None, 1])
    return v, d


def rhs_vjp(osys, k, q_self, q_other, lam):
    """lam^T dR_k/d(q_self, q_other, qinf) by the Jacobian's columns (one dual pass per input;
    tiny meshes only). Returns (gradient w.r.t. q_self, w.r.t. q_other, w.r.t. qinf[4])."""
    lam = np.asarray(lam, dtype=np.float64)
    out = []
    for which, shape in ((0, np.shape(q_self)), (1, np.shape(q_other))):
        g = np.zeros(shape)
        e = np.zeros(shape)
        for idx in np.ndindex(*shape):
            e[idx] = 1.0
            _, d = coupled_rhs_jvp(osys, k, q_self, q_other, e if which == 0 else None, e if which == 1 else None)
            g[idx] = float(np.sum(lam * d))
            e[idx] = 0.0
        out.append(g)
    gi = np.zeros(4)
    for c in range(4):
        dq = np.zeros(4)
        dq[c] = 1.0
        _, d = coupled_rhs_jvp(osys, k, q_self, q_other, None, None, dq)
        gi[c] = float(np.sum(lam * d))
    out.append(gi)
    return tuple(out)


class _Pair:
    """A state with its derivative: (value, derivative) arrays with the + and scalar * the time
    integrators use."""

    __array_ufunc__ = None

    def __init__(self, v, d):
        self.v, self.d = v, d

    def __add__(self, o):
        return _Pair(self.v + o.v, self.d + o.d)

    def __mul__(self, c):
        return _Pair(c * self.v, c * self.d)

    __rmul__ = __mul__


def _combine(y, coeffs, hist):
    out = y
    for c, a in zip(coeffs, hist):
        out = out + c * a
    return out


def probe_objective_jvp(osys, q0, probe_xy, n_steps, H, dq0, dqinf=None):
    """(J, dJ) of system.probe_objective from the initial states q0 along (dq0, dqinf): the
    oracle's bootstrap (Heun's RK3), fastest-first MRAB macro steps and probe pressures on
    (value, derivative) pairs, operation for operation."""
    fast, slow = osys.fast, osys.slow
    sr = int(osys.p["step_ratio"])
    m = int(osys.p["hist_len"])
    order = int(osys.p["order"])

    def rhs(k, qs):
        v, d = coupled_rhs_jvp(osys, k, qs[k].v, qs[1 - k].v, qs[k].d, qs[1 - k].d, dqinf)
        return _Pair(v, d)

    def rhs_all(qs):
        return [rhs(k, qs) for k in range(2)]

    # bootstrap: OracleSystem.bootstrap with rk3_heun_step's operations
    h = H / sr
    y = [_Pair(np.array(q0[k], dtype=np.float64), np.array(dq0[k], dtype=np.float64)) for k in range(2)]
    hist_f, hist_s = [], []
    nsteps = (m - 1) * sr
    for step in range(nsteps):
        k1 = rhs_all(y)
        k2 = rhs_all([yi + (h / 3.0) * ki for yi, ki in zip(y, k1)])
        k3 = rhs_all([yi + (2.0 * h / 3.0) * ki for yi, ki in zip(y, k2)])
        y = [yi + (h / 4.0) * (a + 3.0 * c) for yi, a, c in zip(y, k1, k3)]
        if step >= nsteps - (m - 1):
            hist_f.append(k1[fast])
        if step % sr == 0:
            hist_s.append(k1[slow])
    a = rhs_all(y)
    hist_f.append(a[fast])
    hist_s.append(a[slow])
    # MRAB macro steps: mrab_macro_step's operations
    nodes = np.arange(-(m - 1), 1, dtype=np.float64)
    alpha_f = ab_coefficients(nodes, 0.0, 1.0, order) * h
    alpha_s = ab_coefficients(nodes, 0.0, 1.0, order) * H
    f, s = y[fast], y[slow]
    bg = osys.meshes[0]
    st = [probe_stencil(bg, xy) for xy in np.asarray(probe_xy, dtype=np.float64).reshape(-1, 2)]
    J, dJ = 0.0, 0.0
    for _ in range(n_steps):
        for j in range(sr):
            f = _combine(f, alpha_f, hist_f)
            if j < sr - 1:
                beta = ab_coefficients(nodes, 0.0, (j + 1) / sr, order) * H
                s_hat = _combine(s, beta, hist_s)
                vals = [None, None]
                vals[fast], vals[slow] = f, s_hat
                hist_f = hist_f[1:] + [rhs(fast, vals)]
        s = _combine(s, alpha_s, hist_s)
        vals = [None, None]
        vals[fast], vals[slow] = f, s
        a_f, a_s = rhs(fast, vals), rhs(slow, vals)
        hist_f = hist_f[1:] + [a_f]
        hist_s = hist_s[1:] + [a_s]
        q_bg = s if slow == 0 else f
        # probe pressures (system.probe_pressure's operations) and J = H sum p^2
        ps, dps = [], []
        for (i0, j0), (wi, wj) in st:
            ni, nj = bg["n"]
            acc, dacc = 0.0, 0.0
            for b in range(4):
                for a_ in range(4):
                    i, jj = (i0 + a_) % ni, (j0 + b) % nj
                    rho, mx, my, E = q_bg.v[:, jj, i]
                    drho, dmx, dmy, dE = q_bg.d[:, jj, i]
                    g1 = osys.gamma - 1.0
                    ke = 0.5 * (mx * mx + my * my) / rho
                    dke = 0.5 * ((2 * mx * dmx + 2 * my * dmy) * rho - (mx * mx + my * my) * drho) / (rho * rho)
                    p = g1 * (E - ke)
                    dp = g1 * (dE - dke)
                    acc += wi[a_] * wj[b] * p
                    dacc += wi[a_] * wj[b] * dp
            ps.append(acc)
            dps.append(dacc)
        J += H * float(np.sum(np.array(ps) ** 2))
        dJ += H * float(np.sum(2.0 * np.array(ps) * np.array(dps)))
    return J, dJ
