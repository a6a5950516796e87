"""Step-matrix stability analysis of the MRAB step (Sec. 4.3) on the library's GPU path.

The integrator state phi of a two-mesh system is its current states and the hist_len - 1
right-hand-side history entries of both meshes (``System.get_state``), restricted to active
points (holes and pad columns are not state: a hole keeps its value, which would add the
trivial eigenvalue 1). One macro step maps phi_n to phi_{n+1}; the step matrix G_eps of
eq. (sm) is its linearisation, applied here matrix-free by the finite difference of eq.
(sm_form) along a direction v instead of a unit vector:

    G_eps v = (Step(phi_0 + eps v) - Step(phi_0)) / eps,   |v| = 1, eps = 1e-7,

and the spectral radius is estimated, in place of SLEPc's Krylov-Schur solver, by the largest
Ritz value modulus of a fixed-size Krylov space (Arnoldi with re-orthogonalisation, 60 vectors
by default): unstable eigenvalues are outliers beyond the unit circle and their Ritz values
converge within a few dozen vectors, while a stable spectrum clusters inside the unit circle,
where a full convergence would take thousands of steps but the Ritz values stay below 1. The
method is stable at H when the estimate is <= 1 + slack, slack = 0.02 by default: on the
non-normal step matrices of the overset coupling a stable, clustered spectrum can give Ritz
values up to about 1 % above 1, while past the stability limit the outliers rise quickly
(several percent within a few percent of H). The largest stable macro step is found by
bisection. Every step runs in the library's kernels; only the small
Krylov algebra runs on the host.

The same analysis applies to the single-rate classical Runge-Kutta baseline (Sec. 4.4), whose
integrator state is the two meshes' current states alone (``integrator="rk4"``); the ratio of
the largest stable steps is the r_RK4 of the performance model, eqs. (perf_RK4), (perf_AB).
"""
from __future__ import annotations

import numpy as np


class StepMatrix:
    """G_eps of one step of ``system`` at step H (``system.bind`` must have run): an MRAB
    macro step around the state reached by the bootstrap from the bound initial states, or
    (integrator="rk4") a classical Runge-Kutta step of both meshes around the bound states."""

    def __init__(self, system, H, eps=1e-7, integrator="mrab"):
        import torch
        if integrator not in ("mrab", "rk4"):
            raise ValueError("integrator must be 'mrab' or 'rk4'")
        self.torch = torch
        self.g = system
        self.H = H
        self.eps = eps
        self.integrator = integrator
        system.autotune(False)
        if integrator == "mrab":
            system.mrab_init(H)
            self.phi0 = system.get_state()
        else:
            self.phi0 = [(system.current_state(k).clone(), None) for k in range(2)]
        self.masks = []
        for k in range(2):
            inf = system.info[k]
            ib = torch.from_numpy(system.tables(k)["iblank"] != 0).cuda()
            m = torch.zeros((inf.nj, inf.pitch), dtype=torch.bool, device="cuda")
            m[:, :inf.ni] = ib
            self.masks.append(m)
        self.base = self.pack(self.phi0)
        self.y0 = self._step(self.phi0)
        self.n = self.base.size
        self.matvecs = 0

    def pack(self, state):
        """Active entries of (state, history) of both meshes as one host vector."""
        parts = []
        for k, (q, h) in enumerate(state):
            m = self.masks[k]
            parts.append(q[:, m].reshape(-1))
            if h is not None:
                parts.append(h[:, :, m].reshape(-1))
        return self.torch.cat(parts).double().cpu().numpy()

    def unpack(self, vec):
        """A state with the active entries taken from vec and everything else from phi_0."""
        out, o = [], 0
        t = self.torch.from_numpy(np.ascontiguousarray(vec)).cuda()
        for k, (q0, h0) in enumerate(self.phi0):
            m = self.masks[k]
            q = q0.clone()
            n = int(m.sum()) * q.shape[0]
            q[:, m] = t[o:o + n].reshape(q.shape[0], -1).to(q.dtype)
            o += n
            h = None
            if h0 is not None:
                h = h0.clone()
                nh = int(m.sum()) * h.shape[0] * h.shape[1]
                h[:, :, m] = t[o:o + nh].reshape(h.shape[0], h.shape[1], -1).to(h.dtype)
                o += nh
            out.append((q, h))
        return out

    def _step(self, state):
        if self.integrator == "mrab":
            self.g.set_state(state)
            self.g.mrab_step(1)
            return self.pack(self.g.get_state())
        for k in range(2):
            self.g.current_state(k).copy_(state[k][0])
        self.g.rk4_step(1, self.H)
        return self.pack([(self.g.current_state(k), None) for k in range(2)])

    def matvec(self, v):
        v = np.asarray(v, dtype=np.float64).reshape(-1)
        nv = np.linalg.norm(v)
        if nv == 0.0:
            return np.zeros_like(v)
        self.matvecs += 1
        y = self._step(self.unpack(self.base + self.eps * v / nv))
        return (y - self.y0) * (nv / self.eps)

    def spectral_radius(self, kdim=60, seed=0):
        return arnoldi_radius(self.matvec, self.n, kdim=kdim, seed=seed)


def arnoldi_radius(matvec, n, kdim=60, seed=0):
    """Largest modulus of the Ritz values of a kdim-dimensional Krylov space of the operator
    (Arnoldi, modified Gram-Schmidt applied twice), from a seeded random start vector. A step
    that leaves the finite numbers (a state driven non-physical) counts as unstable: inf."""
    V = np.zeros((kdim + 1, n))
    Hm = np.zeros((kdim + 1, kdim))
    v = np.random.default_rng(seed).standard_normal(n)
    V[0] = v / np.linalg.norm(v)
    k = kdim
    for j in range(kdim):
        w = matvec(V[j])
        if not np.all(np.isfinite(w)):
            return float("inf")
        for _ in range(2):
            for i in range(j + 1):
                c = V[i] @ w
                Hm[i, j] += c
                w -= c * V[i]
        Hm[j + 1, j] = np.linalg.norm(w)
        if Hm[j + 1, j] < 1e-14:
            k = j + 1
            break
        V[j + 1] = w / Hm[j + 1, j]
    return float(np.abs(np.linalg.eigvals(Hm[:k, :k])).max())


def max_stable_step(make_system, H_lo, H_hi, rel_tol=1e-3, slack=0.02, integrator="mrab", **kw):
    """Largest H in [H_lo, H_hi] with rho(G_eps(H)) <= 1 + slack, by bisection; make_system()
    returns a freshly bound system. H_lo must be stable and H_hi unstable. Returns (H, evaluations)."""

    def radius(H):
        g = make_system()
        rho = StepMatrix(g, H, integrator=integrator).spectral_radius(**kw)
        g.close()
        return rho

    return bisect_stable_step(radius, H_lo, H_hi, rel_tol=rel_tol, slack=slack)


def bisect_stable_step(radius, H_lo, H_hi, rel_tol=1e-3, slack=0.02):
    """Largest H in [H_lo, H_hi] with radius(H) <= 1 + slack, by bisection on the step, for any
    spectral-radius estimate radius(H) of a step matrix. Returns (H, [(H, radius), ...])."""
    evals = []

    def stable(H):
        rho = radius(H)
        evals.append((H, rho))
        return rho <= 1.0 + slack

    if not stable(H_lo):
        raise ValueError("H_lo is not stable")
    if stable(H_hi):
        raise ValueError("H_hi is stable")
    lo, hi = H_lo, H_hi
    while (hi - lo) > rel_tol * lo:
        mid = 0.5 * (lo + hi)
        if stable(mid):
            lo = mid
        else:
            hi = mid
    return lo, evals
