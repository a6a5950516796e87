"""Oracle assembly for two overset 3D Cartesian meshes (TEST INFRASTRUCTURE ONLY).

The 3D counterpart of ``system.OracleSystem`` for uniform Cartesian meshes (the paper's 3D
workloads): a background box and one overset fine box. The readings are the 2D ones, per
direction:
  * background points inside the fine box and more than ``hole_cells`` background spacings
    from each of its non-periodic faces are holes (Sec. 2.2 hole cutting);
  * every maximal active run along a line is an SBP segment of at least 8 points;
  * receivers are the points of interface faces and the segment ends next to a hole, one SAT
    term per normal direction and side, scaled by Omega where a point has several
    (Sec. 4.2 eq. (penalty_interp));
  * donors: 4 x 4 x 4 Lagrange cells starting at floor(xi) - 1, shifted inward at
    non-periodic ends (Sec. 2.2).
Time integration (bootstrap, MRAB) is inherited from the 2D class: it only needs the coupled
right-hand side.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import lib
from .system import OracleSystem

CL_HOLE = 15
KIND = {"interface": 1, "farfield": 2}


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def lagrange_weights(t):
    """Lagrange basis of the nodes 0, 1, 2, 3 at t."""
    w = np.ones(4)
    for a in range(4):
        for b in range(4):
            if b != a:
                w[a] *= (t - b) / (a - b)
    return w


class OracleSystem3D(OracleSystem):
    """Background (mesh 0) + one overset fine box (mesh 1), 3D Cartesian."""

    def __init__(self, wl, hole_cells=4, sig_int=0.5, sig_phys=1.0):
        L = lib()
        self.meshes = wl["meshes"]
        self.p = dict(wl["params"])
        self.viscous = self.p["physics"] == "ns"
        self.gamma = float(self.p["gamma"])
        self.mu = float(self.p["mu"])
        self.pr = float(self.p["pr"])
        self.sig_int = sig_int
        self.sig_phys = sig_phys
        self.fast = int(self.p["fast_mesh"])
        self.slow = 1 - self.fast
        bg, fine = self.meshes
        self.iblank = [np.ones(self._shape(m), np.int8) for m in self.meshes]
        # hole cut: inside the fine box, more than the margin from its non-periodic faces
        margin = hole_cells * max(bg["h"])
        inside = np.ones(self._shape(bg), bool)
        axes = self._axes(bg)
        for d in range(3):
            if fine["periodic"][d]:
                continue
            lo = fine["lo"][d]
            hi = fine["lo"][d] + (fine["n"][d] - 1) * fine["h"][d]
            x = axes[d]
            ok = (x > lo + margin) & (x < hi - margin)
            shape = [1, 1, 1]
            shape[2 - d] = -1
            inside &= ok.reshape(shape)
        self.iblank[0][inside] = 0
        self.cls = []
        for k, m in enumerate(self.meshes):
            ni, nj, nk = m["n"]
            c = [np.zeros((nk, nj, ni), np.int8) for _ in range(3)]
            rc = L.orc_classes3d(ni, nj, nk, int(m["periodic"][0]), int(m["periodic"][1]), int(m["periodic"][2]),
                                 _p(self.iblank[k]), _p(c[0]), _p(c[1]), _p(c[2]))
            if rc < 0:
                raise RuntimeError("hole growing did not converge")
            self.cls.append(c)
        self._build_terms3d()
        self._build_donors3d()

    @staticmethod
    def _shape(m):
        return (m["n"][2], m["n"][1], m["n"][0])

    @staticmethod
    def _axes(m):
        return [m["lo"][d] + m["h"][d] * np.arange(m["n"][d]) for d in range(3)]

    # -- SAT terms and receivers ------------------------------------------------------------
    def _build_terms3d(self):
        self.terms, self.recv_pts = [], []
        for k, m in enumerate(self.meshes):
            ni, nj, nk = m["n"]
            n = (ni, nj, nk)
            ib = self.iblank[k]
            terms = {}

            def add(p, d, side, kind):
                terms.setdefault(p, []).append((d, side, kind))

            act = np.argwhere(ib != 0)
            for face in range(6):
                d, side = face // 2, (1 if face % 2 == 0 else -1)
                kind = m["bc"][face]
                if kind == "periodic":
                    continue
                idx = 0 if side == 1 else n[d] - 1
                for kq, j, i in act:
                    if (i, j, kq)[d] == idx:
                        add((kq * nj + j) * ni + i, d, side, KIND[kind])
            # segment ends next to holes
            for kq, j, i in act:
                idx3 = (i, j, kq)
                for d in range(3):
                    for side, off in ((1, -1), (-1, 1)):
                        nb = list(idx3)
                        nb[d] += off
                        if m["periodic"][d]:
                            nb[d] %= n[d]
                        elif nb[d] < 0 or nb[d] >= n[d]:
                            continue
                        if not ib[nb[2], nb[1], nb[0]]:
                            add((kq * nj + j) * ni + i, d, side, KIND["interface"])
            recv = sorted(p for p, ts in terms.items() if any(t[2] == 1 for t in ts))
            rid = {p: r for r, p in enumerate(recv)}
            rows = []
            for p in sorted(terms):
                ts = terms[p]
                n_int = sum(1 for t in ts if t[2] == 1)
                for d, side, kind in ts:
                    scale = self.p["omega_corner"] if (kind == 1 and n_int > 1) else 1.0
                    rows.append((p, d, side, kind, rid.get(p, -1) if kind == 1 else -1, scale))
            self.terms.append({
                "pt": np.array([r[0] for r in rows], np.int64),
                "dir": np.array([r[1] for r in rows], np.int32),
                "side": np.array([r[2] for r in rows], np.int32),
                "kind": np.array([r[3] for r in rows], np.int32),
                "recv": np.array([r[4] for r in rows], np.int32),
                "scale": np.array([r[5] for r in rows], np.float64),
            })
            self.recv_pts.append(np.array(recv, np.int64))

    def _build_donors3d(self):
        self.base, self.w = [], []
        for k, m in enumerate(self.meshes):
            dm = self.meshes[1 - k]
            ni, nj, nk = m["n"]
            pts = self.recv_pts[k]
            i = pts % ni
            j = (pts // ni) % nj
            kq = pts // (ni * nj)
            xs = [m["lo"][0] + m["h"][0] * i, m["lo"][1] + m["h"][1] * j, m["lo"][2] + m["h"][2] * kq]
            base = np.zeros((pts.size, 3), np.int32)
            w = np.zeros((pts.size, 12))
            for d in range(3):
                nd = dm["n"][d]
                xi = (xs[d] - dm["lo"][d]) / dm["h"][d]
                if dm["periodic"][d]:
                    xi = np.mod(xi, nd)
                b = np.floor(xi).astype(np.int64) - 1
                if not dm["periodic"][d]:
                    if np.any(xi < 0) or np.any(xi > nd - 1):
                        raise RuntimeError("receiver outside donor mesh %d" % (1 - k))
                    b = np.clip(b, 0, nd - 4)
                t = xi - b
                base[:, d] = b
                for r in range(pts.size):
                    w[r, 4 * d:4 * d + 4] = lagrange_weights(t[r])
            # every donor point active
            dib = self.iblank[1 - k]
            for r in range(pts.size):
                ii = (base[r, 0] + np.arange(4)) % dm["n"][0]
                jj = (base[r, 1] + np.arange(4)) % dm["n"][1]
                kk = (base[r, 2] + np.arange(4)) % dm["n"][2]
                if not np.all(dib[np.ix_(kk, jj, ii)]):
                    raise RuntimeError("donor cell of receiver %d of mesh %d touches a hole" % (r, k))
            self.base.append(base)
            self.w.append(w)

    # -- operators ----------------------------------------------------------------------------
    def viscflux(self, k, q):
        L = lib()
        m = self.meshes[k]
        ni, nj, nk = m["n"]
        q = np.ascontiguousarray(q, dtype=np.float64)
        fv = np.zeros((12, nk, nj, ni))
        c = self.cls[k]
        L.orc_viscflux3d(ni, nj, nk, _p(c[0]), _p(c[1]), _p(c[2]), *m["h"], _p(q), self.gamma, self.mu, self.pr,
                         _p(fv))
        return fv

    def interp(self, k, field):
        L = lib()
        dm = self.meshes[1 - k]
        field = np.ascontiguousarray(field, dtype=np.float64)
        nf = field.shape[0]
        n = self.recv_pts[k].size
        out = np.zeros((nf, n))
        if n:
            base = np.ascontiguousarray(self.base[k])
            w = np.ascontiguousarray(self.w[k])
            L.orc_interp3d(dm["n"][0], dm["n"][1], dm["n"][2], nf, _p(field), n, _p(base), _p(w), _p(out))
        return out

    def rhs(self, k, q, qhat, fvhat=None):
        L = lib()
        m = self.meshes[k]
        ni, nj, nk = m["n"]
        q = np.ascontiguousarray(q, dtype=np.float64)
        qhat = np.ascontiguousarray(qhat, dtype=np.float64)
        if fvhat is not None:
            fvhat = np.ascontiguousarray(fvhat, dtype=np.float64)
        t = self.terms[k]
        out = np.zeros((5, nk, nj, ni))
        qinf = np.ascontiguousarray(self.p["qinf"], dtype=np.float64)
        c = self.cls[k]
        rc = L.orc_rhs3d(ni, nj, nk, _p(c[0]), _p(c[1]), _p(c[2]), *m["h"], _p(q), int(self.viscous), self.gamma,
                         self.mu, self.pr, t["pt"].size, _p(t["pt"]), _p(t["dir"]), _p(t["side"]), _p(t["kind"]),
                         _p(t["recv"]), _p(t["scale"]), qhat.shape[1], _p(qhat), _p(fvhat), _p(qinf),
                         self.sig_int, self.sig_phys, _p(out))
        if rc != 0:
            raise RuntimeError("oracle rhs failed: %d" % rc)
        if int(self.p.get("sponge_cells", 0)) > 0:
            # relaxation toward the far-field state in the sponge layer, after the SAT terms
            out -= self.sponge_strength(k)[None] * (q - qinf[:, None, None, None])
        return out

    def sponge_strength(self, k):
        """The sponge layer of Sec. 5.1 in three directions (the 2D reading): sigma = A ((D - d) /
        D)^2 for the index distance d < D to the nearest far-field face, the largest over the
        faces, A = `sponge_strength`, D = `sponge_cells`; 0 elsewhere and at holes."""
        m = self.meshes[k]
        ni, nj, nk = m["n"]
        D = int(self.p.get("sponge_cells", 0))
        sig = np.zeros((nk, nj, ni))
        if D <= 0:
            return sig
        A = float(self.p.get("sponge_strength", 1.0))
        kk, jj, ii = np.meshgrid(np.arange(nk), np.arange(nj), np.arange(ni), indexing="ij")
        for face, d in zip(m["bc"], (ii, ni - 1 - ii, jj, nj - 1 - jj, kk, nk - 1 - kk)):
            if face == "farfield":
                sig = np.maximum(sig, np.where(d < D, A * ((D - d) / D) ** 2, 0.0))
        return np.where(self.iblank[k] != 0, sig, 0.0)

    def dt_mesh(self, k, q):
        L = lib()
        m = self.meshes[k]
        q = np.ascontiguousarray(q, dtype=np.float64)
        return L.orc_dt3d(m["n"][0], m["n"][1], m["n"][2], _p(self.cls[k][0]), *m["h"], _p(q), self.gamma, self.mu,
                          self.pr)

    def cell_sizes(self):
        """Cell size hx hy hz per point, holes 0 (eq. (l2error))."""
        return [np.where(self.iblank[k] != 0, float(np.prod(m["h"])), 0.0) for k, m in enumerate(self.meshes)]
