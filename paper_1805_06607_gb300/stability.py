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


# -- the linearised coupled operator (Sec. 4.2, eq. (penalty_interp)) -----------------------------

def active_index(system):
    """Unknowns of the coupled operator: per mesh, per variable, the active points (row-major
    j * ni + i), meshes first, then variables. Returns [(flat device index into the mesh's
    pitched (4, nj, pitch) state, count)] per mesh and the host list of (mesh, var, i, j)."""
    import torch
    out, host = [], []
    for k in range(2):
        inf = system.info[k]
        ib = system.tables(k)["iblank"] != 0
        jj, ii = np.nonzero(ib)
        flat = []
        for v in range(4):
            flat.append(v * inf.nj * inf.pitch + jj * inf.pitch + ii)
            host.extend((k, v, int(i), int(j)) for j, i in zip(jj, ii))
        out.append((torch.from_numpy(np.concatenate(flat)).cuda(), 4 * ii.size))
    return out, host


def coupled_jacobian(system, q=None):
    """The Jacobian of both meshes' right-hand sides with respect to both meshes' states at
    q = (q0, q1) (device states; default the bound states), restricted to active points, as a dense
    FP64 device tensor with the unknowns of ``active_index``. Column c is the library's
    forward-mode derivative (sbp_rhs_eval_jvp) along the unit direction of unknown c: the own
    mesh's right-hand side and the other mesh's receivers, whose interpolated donor values depend
    on it. Exact to rounding (no differencing step). FP64 systems only."""
    import torch
    if q is None:
        q = [system.current_state(k) for k in range(2)]
    idx, host = active_index(system)
    n = sum(c for _, c in idx)
    Jm = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    dq = [system.empty_state(k) for k in range(2)]
    offs = [0, idx[0][1]]
    col = 0
    for k in range(2):
        flat_k = idx[k][0].tolist()
        dflat = dq[k].view(-1)
        for e in flat_k:
            dflat[e] = 1.0
            r_own = system.rhs_eval_jvp(k, q[k], q[1 - k], dq[k], dq[1 - k])
            r_oth = system.rhs_eval_jvp(1 - k, q[1 - k], q[k], dq[1 - k], dq[k])
            dflat[e] = 0.0
            Jm[offs[k]:offs[k] + idx[k][1], col] = r_own.view(-1)[idx[k][0]]
            Jm[offs[1 - k]:offs[1 - k] + idx[1 - k][1], col] = r_oth.view(-1)[idx[1 - k][0]]
            col += 1
    return Jm, host


def mirror_permutation(system, host, axis=1, tol=1e-9):
    """The reflection x_axis -> -x_axis of both meshes as a signed permutation of the unknowns
    ``host`` (from ``active_index``): perm[a] is the unknown at the mirrored point (same mesh and
    variable; a periodic mesh's images one period away count as the same point), sign[a] = -1 for
    the momentum component along the axis. None when some active point has no active mirror
    image within tol (relative to the mesh's extent)."""
    from scipy.spatial import cKDTree
    pos = {h: a for a, h in enumerate(host)}
    perm = np.empty(len(host), dtype=np.int64)
    sign = np.ones(len(host))
    for k, m in enumerate(system.meshes):
        ni, nj = m["n"]
        pts = np.c_[m["x"].ravel(), m["y"].ravel()]
        scale = max(np.ptp(pts[:, 0]), np.ptp(pts[:, 1]), 1e-300)
        imgs, ids = [], []
        (s0x, s0y), (s1x, s1y) = m["shift"]
        for di in ((0,) if not m["periodic"][0] else (-1, 0, 1)):
            for dj in ((0,) if not m["periodic"][1] else (-1, 0, 1)):
                imgs.append(pts + [di * s0x + dj * s1x, di * s0y + dj * s1y])
                ids.append(np.arange(ni * nj))
        tree = cKDTree(np.concatenate(imgs))
        ids = np.concatenate(ids)
        mir = pts.copy()
        mir[:, axis] = -mir[:, axis]
        d, nb = tree.query(mir)
        for a, (kk, v, i, j) in enumerate(host):
            if kk != k:
                continue
            p = j * ni + i
            if d[p] > tol * scale:
                return None
            q = ids[nb[p]]
            b = pos.get((k, v, int(q % ni), int(q // ni)))
            if b is None:
                return None
            perm[a] = b
            sign[a] = -1.0 if v == 1 + axis else 1.0
    return perm, sign


def mirror_blocks(Jm, perm, sign, tol=1e-10):
    """The operator split into its mirror-even and mirror-odd parts: for a signed permutation R
    (R e_a = sign_a e_perm[a], an involution) that commutes with Jm, the spectrum of Jm is the union
    of the spectra of U_e^T Jm U_e and U_o^T Jm U_o, U_e and U_o the orthonormal bases of R's +1
    and -1 eigenspaces made of (e_a +- sign_a e_perm[a]) / sqrt(2) over the pairs a < perm[a] and
    of e_a over the fixed points (sign_a = +1 even, -1 odd). Returns the two blocks (host arrays),
    or None when |R Jm R - Jm| > tol max|Jm|."""
    A = Jm if isinstance(Jm, np.ndarray) else Jm.double().cpu().numpy()
    n = A.shape[0]
    if np.any(perm[perm] != np.arange(n)):
        return None
    RAR = (sign[:, None] * sign[None, :]) * A[np.ix_(perm, perm)]
    if np.abs(RAR - A).max() > tol * np.abs(A).max():
        return None
    del RAR
    a = np.arange(n)
    pairs = a[a < perm]
    fixed = a[a == perm]
    r2 = 1.0 / np.sqrt(2.0)
    blocks = []
    for par in (1.0, -1.0):
        fx = fixed[sign[fixed] == par]
        # basis vector p = c1[p] e_{i1[p]} + c2[p] e_{i2[p]}
        i1 = np.concatenate([pairs, fx])
        i2 = np.concatenate([perm[pairs], fx])
        c1 = np.concatenate([np.full(pairs.size, r2), np.ones(fx.size)])
        c2 = np.concatenate([par * sign[pairs] * r2, np.zeros(fx.size)])
        AU = A[:, i1] * c1[None, :] + A[:, i2] * c2[None, :]
        blocks.append(c1[:, None] * AU[i1, :] + c2[:, None] * AU[i2, :])
    return blocks


def operator_spectrum(Jm, mirror=None):
    """All eigenvalues of the linearised operator (dense eigensolver, host LAPACK), through the
    mirror blocks when ``mirror`` = (perm, sign) is a symmetry of Jm (a quarter of the work of
    the full matrix); otherwise of the full matrix."""
    blocks = mirror_blocks(Jm, *mirror) if mirror is not None else None
    if blocks is None:
        A = Jm if isinstance(Jm, np.ndarray) else Jm.double().cpu().numpy()
        return np.linalg.eigvals(A)
    return np.concatenate([np.linalg.eigvals(B) for B in blocks])


# -- stability regions of the scalar test equation (Sec. 3.2, App. approx_stab) -------------------

GROWTH_100 = 2.0 ** (1.0 / 100.0)
"""Largest per-step amplification the approximate stability regions accept: the marching test of
the appendix on plotting stability regions deems a step unstable when |y| passes 2 within 100
steps from y = 1, i.e. (after the transient) an amplification above 2^(1/100)."""


def ab_amplification(ab, z):
    """Largest modulus of the amplification factors of an Adams-Bashforth step applied to
    y' = lambda y at z = lambda dt: the spectral radius of the step matrix G of Sec. 3.2 (first row
    1 + z a_newest, z a_..., z a_oldest; ones on the subdiagonal) for the weights ``ab`` of one
    step on unit-spaced history nodes, oldest first (``HostTables.plan``). Vectorised over z."""
    ab = np.asarray(ab, dtype=np.float64)
    z = np.atleast_1d(np.asarray(z, dtype=np.complex128))
    m = ab.size
    G = np.zeros((z.size, m, m), dtype=np.complex128)
    G[:, 0, 0] = 1.0 + z * ab[m - 1]
    for c in range(1, m):
        G[:, 0, c] = z * ab[m - 1 - c]
        G[:, c, c - 1] = 1.0
    return np.abs(np.linalg.eigvals(G)).max(axis=-1)


def rk4_amplification(z):
    """|R(z)| of the classical fourth-order Runge-Kutta method, R(z) = sum_{k<=4} z^k / k!."""
    z = np.atleast_1d(np.asarray(z, dtype=np.complex128))
    return np.abs(1.0 + z * (1.0 + z * (0.5 + z * (1.0 / 6.0 + z / 24.0))))


def largest_stable_step(amplification, lam, dt_hi, growth=GROWTH_100, n_scan=512, rel_tol=1e-7):
    """Largest step dt in (0, dt_hi] with amplification(dt lambda) <= growth for every eigenvalue
    lambda in ``lam``: a uniform scan for the first step that fails, then bisection between it and
    the last step that passed (a region need not be star-shaped, so the scan comes first). Returns
    (dt, the eigenvalue that limits it, or None when dt_hi passes)."""
    lam = np.asarray(lam, dtype=np.complex128).ravel()

    def worst(dt):
        a = amplification(dt * lam)
        i = int(np.argmax(a))
        return a[i], i

    lo = 0.0
    for s in range(1, n_scan + 1):
        dt = dt_hi * s / n_scan
        a, i = worst(dt)
        if a > growth:
            hi = dt
            break
        lo = dt
    else:
        return dt_hi, None
    while hi - lo > rel_tol * hi:
        mid = 0.5 * (lo + hi)
        if worst(mid)[0] > growth:
            hi = mid
        else:
            lo = mid
    return lo, lam[worst(hi)[1]]
