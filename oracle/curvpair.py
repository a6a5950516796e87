"""Oracle assembly for a 3D curvilinear overset pair (TEST INFRASTRUCTURE ONLY: the GPU library
never imports it; only tests, the smoke check and the benchmark's CPU baseline may use it).

Two curvilinear meshes (``workloads.curvilinear_pair`` layout): mesh 0, the background, with the
far-field SAT on all six faces; mesh 1, the overset mesh, with interface SAT terms on all six
faces. The readings are the Cartesian 3D systems' (``system3d``), with the curvilinear operator
of ``curv3d``:
  * hole cut (Sec. 2.2): a background node whose computational coordinates on mesh 1 lie more
    than ``params["hole_cells"]`` index units of mesh 1 inside each of its faces is a hole
    (``curv3d.hole_cut``); every maximal active run along a line is an SBP segment of at least
    8 points (shorter runs become holes, ``orc_classes3d``);
  * receivers: the points of mesh 1's faces, and the background's active points next to a
    hole; one interface SAT term (Sec. 2.2 eq. (int), the normal k = grad xi_m) per face
    direction and side, the face terms first (direction, then low before high), then the hole
    neighbours (same order); a point with more than one interface term weights them by
    Omega (Sec. 4.2 eq. (penalty_interp));
  * donors: the receiver's node located on the other mesh by ``curv3d.donors`` (4 x 4 x 4
    Lagrange stencils, no hole in the stencil); donor values are the other mesh's state and,
    for Navier-Stokes, its Cartesian viscous fluxes, gathered with the same weights;
  * time step (reading: the 2D curvilinear form, orc_dt2d, over three directions): per active
    point 1 / (sum_m |u . k_m| + c |K| + 2 nu |K|^2), k_m = grad xi_m = J M[m][:],
    |K|^2 = sum_m |k_m|^2, nu = max(mu, gamma mu / Pr) / rho; the mesh's time step is the
    minimum. On a Cartesian mesh this is orc_dt3d's.
  * sponge layer (Sec. 5.1; the 2D systems' reading carried to three directions): with
    ``params["sponge_cells"]`` = D > 0, the background's right-hand side gains -sigma (q - qinf)
    after its SAT terms, sigma = A ((D - d) / D)^2 for the index distance d < D to the nearest of
    its six far-field faces (A = ``params["sponge_strength"]``), 0 elsewhere and at holes; the
    overset mesh has no far-field face and no sponge.
Time integration (bootstrap, fastest-first MRAB) is inherited from the 2D class: it needs only
the coupled right-hand side and the time step.
"""
from __future__ import annotations

import numpy as np

from .curv3d import Curvilinear3D, donors, hole_cut, interpolate
from .system import OracleSystem


class OracleCurvPair(OracleSystem):
    """Background (mesh 0) + one overset mesh (mesh 1), both 3D curvilinear."""

    def __init__(self, wl, sig_int=0.5, sig_phys=1.0):
        self.meshes = wl["meshes"]
        self.p = dict(wl["params"])
        self.viscous = self.p["physics"] == "ns"
        self.gamma = float(self.p["gamma"])
        self.mu = float(self.p["mu"]) if self.viscous else 0.0
        self.pr = float(self.p["pr"])
        self.sig_int = sig_int
        self.sig_phys = sig_phys
        self.fast = int(self.p["fast_mesh"])
        self.slow = 1 - self.fast
        bg, ov = self.meshes
        pts = np.stack([bg["x"].ravel(), bg["y"].ravel(), bg["z"].ravel()], axis=1)
        holes = hole_cut(ov["x"], ov["y"], ov["z"], pts, float(self.p["hole_cells"]))
        self.ops = [Curvilinear3D(bg["x"], bg["y"], bg["z"], iblank=~holes.reshape(bg["x"].shape)),
                    Curvilinear3D(ov["x"], ov["y"], ov["z"])]
        self.iblank = [self.ops[0].iblank, np.ones(ov["x"].shape, np.int8)]
        self._build_terms()
        self._build_donors()

    # -- SAT terms and receivers ------------------------------------------------------------
    def _build_terms(self):
        """Per mesh: terms (i, j, k, m, side, r, scale) for curv3d's interface SAT, and the
        receivers' linear point indices (k nj + j) ni + i, sorted."""
        self.terms, self.recv_pts = [], []
        for k, m in enumerate(self.meshes):
            ni, nj, nk = m["n"]
            n = (ni, nj, nk)
            ib = self.iblank[k]
            per_point = {}
            for kq, j, i in np.argwhere(ib != 0):
                idx = (int(i), int(j), int(kq))
                ts = []
                if k == 1:
                    for a in range(3):
                        for side, end in ((1, 0), (-1, n[a] - 1)):
                            if idx[a] == end:
                                ts.append((a, side))
                for a in range(3):
                    for side, off in ((1, -1), (-1, 1)):
                        nb = list(idx)
                        nb[a] += off
                        if 0 <= nb[a] < n[a] and not ib[nb[2], nb[1], nb[0]]:
                            ts.append((a, side))
                if ts:
                    per_point[(idx[2] * nj + idx[1]) * ni + idx[0]] = (idx, ts)
            recv = sorted(per_point)
            terms = []
            for r, p in enumerate(recv):
                idx, ts = per_point[p]
                scale = float(self.p["omega_corner"]) if len(ts) > 1 else 1.0
                for a, side in ts:
                    terms.append((idx[0], idx[1], idx[2], a, side, r, scale))
            self.terms.append(terms)
            self.recv_pts.append(np.array(recv, np.int64))

    def _build_donors(self):
        self.base, self.w = [], []
        for k, m in enumerate(self.meshes):
            dm = self.meshes[1 - k]
            pts = np.stack([m["x"].ravel()[self.recv_pts[k]], m["y"].ravel()[self.recv_pts[k]],
                            m["z"].ravel()[self.recv_pts[k]]], axis=1)
            base, w, _ = donors(dm["x"], dm["y"], dm["z"], pts, iblank=self.iblank[1 - k])
            self.base.append(base)
            self.w.append(w)

    # -- operators ----------------------------------------------------------------------------
    def viscflux(self, k, q):
        return self.ops[k].viscous_fluxes(q, self.gamma, self.mu, self.pr)

    def interp(self, k, field):
        return interpolate(np.asarray(field, dtype=np.float64), self.base[k], self.w[k])

    def sponge_strength(self, k):
        """sigma per point of mesh k (nk, nj, ni): A ((D - d) / D)^2 for the index distance d < D
        to the nearest far-field face (the background's six faces), 0 elsewhere, at holes and on
        the overset mesh."""
        shape = self.meshes[k]["x"].shape
        D = int(self.p.get("sponge_cells", 0))
        if k != 0 or D <= 0:
            return np.zeros(shape)
        A = float(self.p.get("sponge_strength", 1.0))
        nk, nj, ni = shape
        kk, jj, ii = np.meshgrid(np.arange(nk), np.arange(nj), np.arange(ni), indexing="ij")
        d = np.minimum.reduce([ii, ni - 1 - ii, jj, nj - 1 - jj, kk, nk - 1 - kk])
        sig = np.where(d < D, A * ((D - d) / D) ** 2, 0.0)
        return np.where(self.iblank[k] != 0, sig, 0.0)

    def rhs(self, k, q, qhat, fvhat=None):
        """dq/dt on mesh k given the interpolated donor values at its receivers."""
        q = np.asarray(q, dtype=np.float64)
        qinf = np.asarray(self.p["qinf"], dtype=np.float64) if k == 0 else None
        iface = dict(terms=self.terms[k], qhat=np.asarray(qhat), fvhat=fvhat, sigma=self.sig_int)
        out = self.ops[k].rhs(q, self.gamma, self.mu, self.pr, qinf=qinf, sigma=self.sig_phys, interface=iface)
        if k == 0 and int(self.p.get("sponge_cells", 0)) > 0:
            # relaxation toward the far-field state in the sponge layer, after the SAT terms
            out = out - self.sponge_strength(k)[None] * (q - qinf[:, None, None, None])
        return out

    def dt_mesh(self, k, q):
        op = self.ops[k]
        q = np.asarray(q, dtype=np.float64)
        rho = q[0]
        u = [q[1] / rho, q[2] / rho, q[3] / rho]
        pres = (self.gamma - 1.0) * (q[4] - 0.5 * rho * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]))
        c = np.sqrt(self.gamma * pres / rho)
        conv, g2 = 0.0, 0.0
        for m in range(3):
            kv = [op.J * op.M[m][j] for j in range(3)]
            conv = conv + np.abs(u[0] * kv[0] + u[1] * kv[1] + u[2] * kv[2])
            g2 = g2 + kv[0] * kv[0] + kv[1] * kv[1] + kv[2] * kv[2]
        nu = max(self.mu, self.gamma * self.mu / self.pr) / rho
        dt = 1.0 / (conv + c * np.sqrt(g2) + 2.0 * nu * g2)
        return float(dt[self.iblank[k] != 0].min())

    def cell_sizes(self):
        """Cell volume J^-1 per point (eq. (l2error)), holes 0."""
        return [np.where(self.iblank[k] != 0, 1.0 / self.ops[k].J, 0.0) for k in range(2)]
