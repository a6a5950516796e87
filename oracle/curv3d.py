"""Plain FP64 CPU oracle: the flux divergence of the 3D compressible Navier-Stokes equations on
one curvilinear structured mesh.

TEST INFRASTRUCTURE ONLY. The GPU library never imports it; only tests may use it. It is the
definition the GPU's curvilinear operator (sbp3c_*) is checked against, pinned by
tests/test_oracle_curv3d.py.

What it computes (App. C.1's equations in curvilinear coordinates, Sec. 2.1's SBP operator):
  * coordinate derivatives X_a = D_a X by the SBP 4-2 first derivative along each index
    direction a (xi = i, eta = j, zeta = k), closures at both ends of every line (Sec. 2.1);
  * metric terms xi_m,x_j / J in the symmetric conservative form of Thomas and Lombard (the
    reading; the paper defers the metrics to other work): for (m, a, b) and (j, c, e) cyclic,
        M[m][j] = D_b((X_c)_a X_e) - D_a((X_c)_b X_e),
    which satisfies the discrete metric identity sum_m D_m M[m][j] = 0 because D_a and D_b act
    on different index directions and commute;
  * J^-1 = det(X_a) from the same coordinate derivatives;
  * gradients d f / d x_j = J sum_m M[m][j] D_m f of (u, v, w, T) (the viscous term's first
    application of D), stresses with Stokes' hypothesis, Fourier heat flux (App. C.1);
  * dq/dt = -J sum_m D_m (sum_j M[m][j] (F_j - F^V_j)).
Optionally (qinf given) the far-field SAT of Sec. 5.1 on all six faces (reading: the
characteristic penalty of eq. (int) towards qinf with sigma, no viscous term, as for the 2D
far field): at a point on the low (side +1) or high (side -1) face of index direction m,
    dq/dt += -(sigma / p0) K^side_k (q - qinf),   k = grad xi_m = J M[m][:],
summed over the directions whose face the point lies on (edges and corners), with K^side_k the
characteristic splitting of the flux Jacobian along k (the Cartesian oracle's
orc_penalty_matrix3d) and p0 = 17/48.

Optionally interface SAT terms (Sec. 2.2 eq. (int)) at receiver points with given donor values,
the Cartesian oracle's interface term with the normal k = J M[m][:] (see _interface).

Donor search (Sec. 2.2's donor-receiver pairing and Lagrange interpolation, in 3D as the 2D
oracle's orc_donors2d does it): for a point p, computational coordinates (s, r, t) on the mesh
with X(s, r, t) = p, X the mesh map interpolated by the 4 x 4 x 4 Lagrange basis on the stencil
starting at (floor(s) - 1, ...) clamped into the mesh; Newton from the nearest node until three
consecutive steps are below 1e-10; the weights are that basis at the solution.

Arrays are (nk, nj, ni) per variable, i fastest; q = (rho, rho u, rho v, rho w, rho E).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import lib


def d_matrix(n):
    """The SBP 4-2 first derivative on a line of n points with closures at both ends, as an
    n x n matrix: columns are the oracle's pinned 1D operator (orc_apply_d1) applied to unit
    vectors."""
    if n < 8:
        raise ValueError("a line needs at least 8 points")
    cls = np.zeros(n, np.int8)
    for r in range(4):
        cls[r] = 1 + r          # closure row r at the low end
        cls[n - 1 - r] = 5 + r  # closure row r counted from the high end
    L = lib()
    D = np.zeros((n, n))
    out = np.zeros(n)
    for c in range(n):
        e = np.zeros(n)
        e[c] = 1.0
        L.orc_apply_d1(n, ctypes.c_void_p(cls.ctypes.data), ctypes.c_void_p(e.ctypes.data),
                       ctypes.c_void_p(out.ctypes.data))
        D[:, c] = out
    return D


class Curvilinear3D:
    """One structured mesh with node coordinates x, y, z (each (nk, nj, ni)), non-periodic in
    every direction.

    With an iblank (nonzero: active), the flux divergence and the viscous gradients take every
    maximal active run along a line as one SBP segment with closures at both of its ends (Sec.
    2.2 hole cutting; the Cartesian oracle's stencil classes, orc_classes3d, which also makes
    runs shorter than 8 points inactive, so the mask in ``self.iblank`` may have grown), and
    the right-hand side is 0 at inactive points. The metric terms always take whole lines: the
    mesh map is defined at every node, holes included (reading)."""

    def __init__(self, x, y, z, iblank=None):
        X = [np.asarray(v, dtype=np.float64) for v in (x, y, z)]
        nk, nj, ni = X[0].shape
        self.shape = (nk, nj, ni)
        self.D = [d_matrix(ni), d_matrix(nj), d_matrix(nk)]
        self.cls = None
        self.iblank = None
        # derivative along index direction a (0: i, 1: j, 2: k) acts on array axis 2 - a
        dX = [[self.deriv(X[c], a) for a in range(3)] for c in range(3)]   # dX[c][a] = D_a X_c
        self.Jinv = (dX[0][0] * (dX[1][1] * dX[2][2] - dX[1][2] * dX[2][1])
                     - dX[0][1] * (dX[1][0] * dX[2][2] - dX[1][2] * dX[2][0])
                     + dX[0][2] * (dX[1][0] * dX[2][1] - dX[1][1] * dX[2][0]))
        self.J = 1.0 / self.Jinv
        cyc = [(0, 1, 2), (1, 2, 0), (2, 0, 1)]
        self.M = [[None] * 3 for _ in range(3)]
        for m, a, b in cyc:
            for j, c, e in cyc:
                self.M[m][j] = (self.deriv(dX[c][a] * X[e], b) - self.deriv(dX[c][b] * X[e], a))
        if iblank is not None:
            ib = np.ascontiguousarray(np.asarray(iblank) != 0, dtype=np.int8).copy()
            cls = [np.zeros(self.shape, np.int8) for _ in range(3)]
            rc = lib().orc_classes3d(ni, nj, nk, 0, 0, 0, ctypes.c_void_p(ib.ctypes.data),
                                     *[ctypes.c_void_p(c.ctypes.data) for c in cls])
            if rc < 0:
                raise RuntimeError("hole growing did not converge")
            self.iblank = ib
            self.cls = cls
            self._lines = {}

    def deriv(self, f, a):
        """D_a f: the SBP derivative along index direction a (unit index spacing); on a mesh with
        holes, per active segment (0 at inactive points)."""
        ax = 2 - a
        if self.cls is None:
            g = np.tensordot(self.D[a], np.moveaxis(f, ax, 0), axes=(1, 0))
            return np.moveaxis(g, 0, ax)
        cl = np.moveaxis(self.cls[a], ax, -1)
        fl = np.moveaxis(np.asarray(f, dtype=np.float64), ax, -1)
        n = cl.shape[-1]
        lines, vals = cl.reshape(-1, n), fl.reshape(-1, n)
        out = np.zeros_like(vals)
        pats, which = np.unique(lines, axis=0, return_inverse=True)
        for u, pat in enumerate(pats):
            sel = which.reshape(-1) == u
            out[sel] = vals[sel] @ self._line_matrix(pat).T
        return np.moveaxis(out.reshape(fl.shape), -1, ax)

    def _line_matrix(self, pat):
        """The derivative on one line with stencil classes pat, as a matrix: the pinned 1D
        operator (orc_apply_d1) applied to unit vectors."""
        key = pat.tobytes()
        if key not in self._lines:
            n = pat.size
            cls = np.ascontiguousarray(pat, dtype=np.int8)
            D = np.zeros((n, n))
            out = np.zeros(n)
            for c in range(n):
                e = np.zeros(n)
                e[c] = 1.0
                lib().orc_apply_d1(n, ctypes.c_void_p(cls.ctypes.data), ctypes.c_void_p(e.ctypes.data),
                                   ctypes.c_void_p(out.ctypes.data))
                D[:, c] = out
            self._lines[key] = D
        return self._lines[key]

    def gradient(self, f):
        """(d f/dx, d f/dy, d f/dz) by the chain rule with the metric terms."""
        Df = [self.deriv(f, m) for m in range(3)]
        return [self.J * (self.M[0][j] * Df[0] + self.M[1][j] * Df[1] + self.M[2][j] * Df[2]) for j in range(3)]

    def rhs(self, q, gamma, mu=0.0, pr=0.72, qinf=None, sigma=1.0, interface=None):
        """dq/dt = -J sum_m D_m F^_m (5 arrays), F^_m = sum_j M[m][j] (F_j - F^V_j), plus the
        far-field SAT on every face when qinf (5 values) is given, plus interface SAT terms when
        `interface` is given (see _interface)."""
        rho = q[0]
        vel = [q[1] / rho, q[2] / rho, q[3] / rho]
        E = q[4]
        p = (gamma - 1.0) * (E - 0.5 * rho * (vel[0] ** 2 + vel[1] ** 2 + vel[2] ** 2))
        F = [[rho * vel[d]] + [rho * vel[d] * vel[c] + (p if c == d else 0.0) for c in range(3)]
             + [(E + p) * vel[d]] for d in range(3)]
        Fv = None
        if mu > 0.0:
            Fv = self._viscous(q, gamma, mu, pr)
            for d in range(3):
                for c in range(3):
                    F[d][1 + c] = F[d][1 + c] - Fv[d][c]
                F[d][4] = F[d][4] - Fv[d][3]
        out = []
        for v in range(5):
            s = 0.0
            for m in range(3):
                Fh = self.M[m][0] * F[0][v] + self.M[m][1] * F[1][v] + self.M[m][2] * F[2][v]
                s = s + self.deriv(Fh, m)
            out.append(-self.J * s)
        out = np.array(out)
        if self.iblank is not None:
            out[:, self.iblank == 0] = 0.0
        if qinf is not None:
            self._farfield(out, q, gamma, np.asarray(qinf, dtype=np.float64), sigma)
        if interface is not None:
            self._interface(out, q, gamma, mu, Fv, **interface)
        return out

    def _viscous(self, q, gamma, mu, pr):
        """Cartesian viscous fluxes Fv[d] = (tau_d0, tau_d1, tau_d2, u . tau_d + kappa T_d) for
        d = x, y, z (App. C.1: Stokes' hypothesis, Fourier heat flux, T = gamma p / rho), with
        the gradients of (u, v, w, T) by the chain rule."""
        rho = q[0]
        vel = [q[1] / rho, q[2] / rho, q[3] / rho]
        p = (gamma - 1.0) * (q[4] - 0.5 * rho * (vel[0] ** 2 + vel[1] ** 2 + vel[2] ** 2))
        T = gamma * p / rho
        g = [self.gradient(f) for f in vel + [T]]   # g[f][d]
        div = g[0][0] + g[1][1] + g[2][2]
        lam, kap = -2.0 / 3.0 * mu, mu / (pr * (gamma - 1.0))
        Fv = []
        for d in range(3):
            tau = [mu * (g[d][c] + g[c][d]) + (lam * div if c == d else 0.0) for c in range(3)]
            Fv.append(tau + [vel[0] * tau[0] + vel[1] * tau[1] + vel[2] * tau[2] + kap * g[3][d]])
        return Fv

    def viscous_fluxes(self, q, gamma, mu, pr):
        """The 12 planes (F^V_x, F^V_y, F^V_z; each momentum x, y, z and energy) of the Cartesian
        viscous fluxes, 0 at inactive points: the donor values of Navier-Stokes receivers."""
        Fv = self._viscous(np.asarray(q, dtype=np.float64), gamma, mu, pr)
        out = np.array([Fv[d][c] for d in range(3) for c in range(4)])
        if self.iblank is not None:
            out[:, self.iblank == 0] = 0.0
        return out

    def _interface(self, out, q, gamma, mu, Fv, terms, qhat, fvhat=None, sigma=0.5):
        """Interface SAT of Sec. 2.2 eq. (int) at receiver points, with the metric normal in place
        of the Cartesian one: for each term (i, j, k, m, side, r, scale) -- receiver point
        (i, j, k), normal index direction m, side +1 (low face) or -1 (high face), donor values
        column r of qhat (5, nrecv) and of fvhat (12, nrecv: F^V_d's 4 components (momentum x,
        y, z, energy) for d = x, y, z, Cartesian, interpolated from the donor mesh; Navier-Stokes
        only) --
            dq/dt += scale * (-(1/p0) [(sigma K^side_k + sigma1 I)(q - qhat)
                                      - side/2 (F^V_k - F^V_k hat)]),
        k = grad xi_m = J M[m][:], sigma1 = mu |k|^2 / 2 (0 for Euler), F^V_k = sum_d k_d F^V_d
        (momentum and energy rows)."""
        L = lib()
        p0 = 17.0 / 48.0
        K = np.zeros((5, 5))
        for (i, j, k, m, side, r, scale) in terms:
            kv = [self.J[k, j, i] * self.M[m][jj][k, j, i] for jj in range(3)]
            qp = np.ascontiguousarray(q[:, k, j, i], dtype=np.float64)
            L.orc_penalty_matrix3d(ctypes.c_void_p(qp.ctypes.data), gamma, kv[0], kv[1], kv[2], side,
                                   ctypes.c_void_p(K.ctypes.data))
            dq = qp - qhat[:, r]
            sig1 = 0.5 * mu * (kv[0] ** 2 + kv[1] ** 2 + kv[2] ** 2) if mu > 0.0 else 0.0
            sat = -(sigma * (K @ dq) + sig1 * dq) / p0
            if mu > 0.0:
                for c in range(4):
                    own = sum(kv[d] * Fv[d][c][k, j, i] for d in range(3))
                    hat = sum(kv[d] * fvhat[4 * d + c, r] for d in range(3))
                    sat[1 + c] += 0.5 * side * (own - hat) / p0
            out[:, k, j, i] += scale * sat

    def _farfield(self, out, q, gamma, qinf, sigma):
        L = lib()
        p0 = 17.0 / 48.0
        nk, nj, ni = self.shape
        n = (ni, nj, nk)
        K = np.zeros((5, 5))
        for k in range(nk):
            for j in range(nj):
                for i in range(ni):
                    c = (i, j, k)
                    for m in range(3):
                        if c[m] == 0:
                            side = 1
                        elif c[m] == n[m] - 1:
                            side = -1
                        else:
                            continue
                        kv = [self.J[k, j, i] * self.M[m][jj][k, j, i] for jj in range(3)]
                        qp = np.ascontiguousarray(q[:, k, j, i], dtype=np.float64)
                        L.orc_penalty_matrix3d(ctypes.c_void_p(qp.ctypes.data), gamma, kv[0], kv[1], kv[2], side,
                                               ctypes.c_void_p(K.ctypes.data))
                        out[:, k, j, i] -= (sigma / p0) * (K @ (qp - qinf))


def lagrange4(s):
    """Cubic Lagrange basis on nodes 0, 1, 2, 3 at s, and its derivative."""
    d = [s - 0.0, s - 1.0, s - 2.0, s - 3.0]
    den = [-6.0, 2.0, -2.0, 6.0]
    l, dl = [], []
    for a in range(4):
        o = [d[b] for b in range(4) if b != a]
        l.append(o[0] * o[1] * o[2] / den[a])
        dl.append((o[1] * o[2] + o[0] * o[2] + o[0] * o[1]) / den[a])
    return np.array(l), np.array(dl)


def _start(s, n):
    return int(min(max(np.floor(s) - 1, 0), n - 4))


class DonorError(ValueError):
    pass


def _invert(X, p):
    """Index coordinates c with the Lagrange-interpolated map X(c) = p (Newton from the nearest
    node, three consecutive steps below 1e-10), or None (no convergence, or outside the mesh)."""
    nk, nj, ni = X.shape[1:]
    n = (ni, nj, nk)
    d2 = ((X - p[:, None, None, None]) ** 2).sum(axis=0)
    k, j, i = np.unravel_index(np.argmin(d2), d2.shape)
    c = np.array([i, j, k], dtype=np.float64)
    small = 0
    for _ in range(100):
        b0 = [_start(c[a], n[a]) for a in range(3)]
        L = [lagrange4(c[a] - b0[a]) for a in range(3)]
        cube = X[:, b0[2]:b0[2] + 4, b0[1]:b0[1] + 4, b0[0]:b0[0] + 4]   # (3, 4k, 4j, 4i)
        val = np.einsum("xkji,i,j,k->x", cube, L[0][0], L[1][0], L[2][0])
        jac = np.stack([np.einsum("xkji,i,j,k->x", cube, L[0][0 if a != 0 else 1], L[1][0 if a != 1 else 1],
                                  L[2][0 if a != 2 else 1]) for a in range(3)], axis=1)
        try:
            step = np.linalg.solve(jac, val - p)
        except np.linalg.LinAlgError:
            return None
        c = c - step
        if not np.all(np.abs(c) < 1e7):
            return None
        small = small + 1 if np.all(np.abs(step) < 1e-10) else 0
        if small == 3:
            break
    if small < 3 or any(c[a] < -1e-9 or c[a] > n[a] - 1 + 1e-9 for a in range(3)):
        return None
    return c


def hole_cut(x, y, z, points, margin):
    """Hole cut against a curvilinear mesh (Sec. 2.2; reading, as for the Cartesian 3D hole cut
    with the overlapping mesh's index units): a point is a hole when it lies inside the mesh at
    index coordinates more than `margin` from each of the mesh's faces. Returns a bool array."""
    X = np.stack([np.asarray(v, dtype=np.float64) for v in (x, y, z)])
    nk, nj, ni = X.shape[1:]
    n = (ni, nj, nk)
    # points outside the nodes' bounding box padded by the longest edge between neighbouring
    # nodes are outside the mesh (the interpolated map of a mesh whose cells are not folded
    # does not reach there): no search
    edge = max(float(np.sqrt((np.diff(X, axis=ax) ** 2).sum(axis=0)).max()) for ax in (1, 2, 3))
    lo = X.reshape(3, -1).min(axis=1) - edge
    hi = X.reshape(3, -1).max(axis=1) + edge
    out = []
    for p in np.asarray(points, dtype=np.float64).reshape(-1, 3):
        if np.any(p < lo) or np.any(p > hi):
            out.append(False)
            continue
        c = _invert(X, p)
        out.append(c is not None and all(margin < c[a] < n[a] - 1 - margin for a in range(3)))
    return np.array(out, bool)


def donors(x, y, z, points, iblank=None):
    """Donor stencils on a curvilinear mesh (coordinates (nk, nj, ni)) for points (npts, 3):
    base (npts, 3) ints (i0, j0, k0), weights (npts, 12) (4 along i, 4 along j, 4 along k) and
    computational coordinates (npts, 3). Raises DonorError(index) for the first point with no
    valid stencil (outside the mesh, no convergence, or an inactive point in the stencil)."""
    X = np.stack([np.asarray(v, dtype=np.float64) for v in (x, y, z)])
    nk, nj, ni = X.shape[1:]
    n = (ni, nj, nk)
    act = np.ones((nk, nj, ni), bool) if iblank is None else np.asarray(iblank) != 0
    P = np.asarray(points, dtype=np.float64).reshape(-1, 3)
    base = np.zeros((len(P), 3), np.int64)
    w = np.zeros((len(P), 12))
    xi = np.zeros((len(P), 3))
    for t, p in enumerate(P):
        c = _invert(X, p)
        if c is None:
            raise DonorError(t)
        b0 = [_start(c[a], n[a]) for a in range(3)]
        if not act[b0[2]:b0[2] + 4, b0[1]:b0[1] + 4, b0[0]:b0[0] + 4].all():
            raise DonorError(t)
        base[t] = b0
        for a in range(3):
            w[t, 4 * a:4 * a + 4] = lagrange4(c[a] - b0[a])[0]
        xi[t] = c
    return base, w, xi


def interpolate(f, base, w):
    """sum over the 4 x 4 x 4 stencil of wi wj wk f, for fields f (nf, nk, nj, ni)."""
    out = np.zeros((f.shape[0], len(base)))
    for t in range(len(base)):
        i0, j0, k0 = base[t]
        cube = f[:, k0:k0 + 4, j0:j0 + 4, i0:i0 + 4]
        out[:, t] = np.einsum("fkji,i,j,k->f", cube, w[t, 0:4], w[t, 4:8], w[t, 8:12])
    return out
