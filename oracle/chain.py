"""Oracle for a chain of nested overset meshes stepped at one rate per mesh (TEST INFRASTRUCTURE
ONLY).

Sec. 3.3 notes that the multi-rate scheme extends to any number of rates; Sec. 2.2's overset
coupling extends the same way. The reading here: meshes 0..R-1, mesh r overset on mesh r-1.
Mesh r's outer boundary cuts a hole into mesh r-1 (the hole rule of the two-mesh system,
Sec. 2.2: points inside the outer boundary and more than ``hole_cells`` spacings of mesh r-1
from it); the receivers of mesh r are its interface faces, fed by mesh r-1, and the segment ends
next to the hole cut by mesh r+1, fed by mesh r+1. Every receiver takes its values from a 4 x 4
Lagrange stencil on its donor mesh and gets the interface SAT of eq. (int). Time stepping is
``mrab_macro_step_multirate`` (the two-rate recursion nested level by level), mesh 0 slowest;
the bootstrap is Heun's RK3 at the finest step, recording each mesh's right-hand side at its
own step. With two meshes every piece is ``OracleSystem``'s, operation for operation.
"""
from __future__ import annotations

import numpy as np

from . import lib
from .system import (CL_HOLE, KIND, _outer_polygon, _p, mrab_macro_step_multirate, rk3_heun_step)


class OracleChain:
    """meshes[0] is the outermost (Cartesian) mesh; meshes[r] (r >= 1) lies inside meshes[r-1].
    All but the innermost mesh must be Cartesian (the hole margin is in their spacing).
    ratios[r-1] = step of mesh r-1 / step of mesh r."""

    def __init__(self, wl, hole_cells=4, sig_int=0.5, sig_phys=1.0):
        L = lib()
        self.meshes = wl["meshes"]
        R = self.R = len(self.meshes)
        self.p = dict(wl["params"])
        self.ratios = [int(r) for r in wl["ratios"]]
        if len(self.ratios) != R - 1 or R < 2:
            raise ValueError("R >= 2 meshes and R - 1 step ratios")
        self.viscous = self.p["physics"] == "ns"
        self.gamma, self.mu, self.pr = float(self.p["gamma"]), float(self.p["mu"]), float(self.p["pr"])
        self.sig_int, self.sig_phys = sig_int, sig_phys
        self.iblank = [np.ones((m["n"][1], m["n"][0]), np.int8) for m in self.meshes]
        for r in range(1, R):
            outer = self.meshes[r - 1]
            if not outer["cartesian"]:
                raise ValueError("every mesh but the innermost must be Cartesian")
            bx, by = _outer_polygon(self.meshes[r])
            margin = hole_cells * max(outer["h"])
            L.orc_holecut2d(outer["x"].size, _p(outer["x"]), _p(outer["y"]), bx.size, _p(bx), _p(by), margin,
                            _p(self.iblank[r - 1]))
        self.ci, self.cj, self.met, self.shift = [], [], [], []
        for k, m in enumerate(self.meshes):
            ni, nj = m["n"]
            ci = np.zeros((nj, ni), np.int8)
            cj = np.zeros((nj, ni), np.int8)
            if L.orc_classes2d(ni, nj, int(m["periodic"][0]), int(m["periodic"][1]), _p(self.iblank[k]), _p(ci),
                               _p(cj)) < 0:
                raise RuntimeError("hole growing did not converge")
            shift = np.array([m["shift"][0][0], m["shift"][0][1], m["shift"][1][0], m["shift"][1][1]])
            met = np.zeros((5, nj, ni))
            if m["cartesian"]:
                # exact constants on a uniform Cartesian map (D reproduces linear functions exactly)
                hx, hy = m["h"]
                act = ci != CL_HOLE
                for c, val in enumerate((hy, 0.0, 0.0, hx, 1.0 / (hx * hy))):
                    met[c] = np.where(act, val, 1.0 if c in (0, 3, 4) else 0.0)
            elif L.orc_metrics2d(ni, nj, _p(shift), _p(m["x"]), _p(m["y"]), _p(ci), _p(cj), _p(met)) != 0:
                raise RuntimeError("non-positive cell volume")
            self.ci.append(ci)
            self.cj.append(cj)
            self.met.append(met)
            self.shift.append(shift)
        self._build_terms()
        self._build_donors()

    # -- SAT terms, receivers and their donor meshes -------------------------------------------
    def _build_terms(self):
        """As OracleSystem._build_terms, with each receiver's donor mesh: k - 1 for a point on an
        interface face of mesh k, k + 1 for a segment end next to the hole mesh k + 1 cut."""
        self.terms, self.recv_pts, self.recv_src = [], [], []
        for k, m in enumerate(self.meshes):
            ni, nj = m["n"]
            ib = self.iblank[k]
            terms, src = {}, {}

            def add(p, d, side, kind, donor=None):
                terms.setdefault(p, []).append((d, side, kind))
                if donor is not None:
                    if src.get(p, donor) != donor:
                        raise ValueError("a receiver next to both its outer face and a hole")
                    src[p] = donor

            for face, (d, side) in enumerate(((0, 1), (0, -1), (1, 1), (1, -1))):
                kind = m["bc"][face]
                if kind == "periodic":
                    continue
                if d == 0:
                    pts = [j * ni + (0 if side == 1 else ni - 1) for j in range(nj)]
                else:
                    pts = [(0 if side == 1 else nj - 1) * ni + i for i in range(ni)]
                for p in pts:
                    if ib.flat[p]:
                        add(p, d, side, KIND[kind], k - 1 if kind == "interface" else None)
            for j in range(nj):
                for i in range(ni):
                    if not ib[j, i]:
                        continue
                    p = j * ni + i
                    for d, (n, idx, per) in enumerate(((ni, i, m["periodic"][0]), (nj, j, m["periodic"][1]))):
                        for side, nb in ((1, idx - 1), (-1, idx + 1)):
                            if per:
                                nb %= n
                            elif nb < 0 or nb >= n:
                                continue
                            nbp = (j * ni + nb) if d == 0 else (nb * ni + i)
                            if not ib.flat[nbp]:
                                add(p, d, side, KIND["interface"], k + 1)
            recv = sorted(p for p, ts in terms.items() if any(t[2] == 1 for t in ts))
            if any(not 0 <= src[p] < self.R for p in recv):
                raise ValueError("an interface face of the outermost mesh or a hole with no overset mesh")
            rid = {p: r for r, p in enumerate(recv)}
            rows = []
            for p in sorted(terms):
                ts = terms[p]
                n_int = sum(1 for t in ts if t[2] == 1)
                for d, side, kind in ts:
                    scale = self.p["omega_corner"] if (kind == 1 and n_int > 1) else 1.0
                    rows.append((p, d, side, kind, rid.get(p, -1) if kind == 1 else -1, scale))
            self.terms.append({
                "pt": np.array([r[0] for r in rows], np.int32), "dir": np.array([r[1] for r in rows], np.int32),
                "side": np.array([r[2] for r in rows], np.int32), "kind": np.array([r[3] for r in rows], np.int32),
                "recv": np.array([r[4] for r in rows], np.int32), "scale": np.array([r[5] for r in rows], np.float64)})
            self.recv_pts.append(np.array(recv, np.int64))
            self.recv_src.append(np.array([src[p] for p in recv], np.int64))

    def _build_donors(self):
        """4 x 4 Lagrange stencils of every receiver on its donor mesh (orc_donors2d)."""
        L = lib()
        self.base, self.w = [], []
        for k, m in enumerate(self.meshes):
            pts = self.recv_pts[k]
            base = np.zeros((pts.size, 2), np.int32)
            w = np.zeros((pts.size, 8))
            for dk in (k - 1, k + 1):
                sel = np.nonzero(self.recv_src[k] == dk)[0]
                if sel.size == 0:
                    continue
                dm = self.meshes[dk]
                px = np.ascontiguousarray(m["x"].ravel()[pts[sel]])
                py = np.ascontiguousarray(m["y"].ravel()[pts[sel]])
                b = np.zeros((sel.size, 2), np.int32)
                ww = np.zeros((sel.size, 8))
                xe = np.zeros((sel.size, 2))
                rc = L.orc_donors2d(dm["n"][0], dm["n"][1], int(dm["periodic"][0]), int(dm["periodic"][1]),
                                    _p(self.shift[dk]), _p(dm["x"]), _p(dm["y"]), _p(self.iblank[dk]),
                                    sel.size, _p(px), _p(py), _p(b), _p(ww), _p(xe))
                if rc != 0:
                    raise RuntimeError("no donor for receiver %d of mesh %d" % (sel[rc - 1], k))
                base[sel] = b
                w[sel] = ww
            self.base.append(base)
            self.w.append(w)

    # -- right-hand sides ----------------------------------------------------------------------
    def viscflux(self, k, q):
        L = lib()
        m = self.meshes[k]
        ni, nj = m["n"]
        fv = np.zeros((6, nj, ni))
        qc = np.ascontiguousarray(q, dtype=np.float64)
        L.orc_viscflux2d(ni, nj, int(m["periodic"][0]), int(m["periodic"][1]), _p(self.ci[k]), _p(self.cj[k]),
                         _p(self.met[k]), _p(qc), self.gamma, self.mu, self.pr, _p(fv))
        return fv

    def interp(self, k, fields):
        """Values at mesh k's receivers: fields[dk] is a full field (nf, nj, ni) on donor mesh dk
        for each donor mesh of mesh k; each receiver reads its own donor mesh's field."""
        L = lib()
        nr = self.recv_pts[k].size
        nf = next(iter(fields.values())).shape[0]
        out = np.zeros((nf, nr))
        for dk, field in fields.items():
            sel = np.nonzero(self.recv_src[k] == dk)[0]
            if sel.size == 0:
                continue
            dm = self.meshes[dk]
            part = np.zeros((nf, sel.size))
            # the arrays stay referenced here for the duration of the call
            fld = np.ascontiguousarray(field, dtype=np.float64)
            base = np.ascontiguousarray(self.base[k][sel])
            w = np.ascontiguousarray(self.w[k][sel])
            L.orc_interp2d(dm["n"][0], dm["n"][1], nf, _p(fld), sel.size, _p(base), _p(w), _p(part))
            out[:, sel] = part
        return out

    def rhs(self, k, vals):
        """dq/dt of mesh k with its receivers fed from vals[k - 1] and vals[k + 1]."""
        L = lib()
        m = self.meshes[k]
        ni, nj = m["n"]
        donors = [dk for dk in (k - 1, k + 1) if np.any(self.recv_src[k] == dk)]
        qhat = self.interp(k, {dk: vals[dk] for dk in donors}) if donors else np.zeros((4, 0))
        fvhat = None
        if self.viscous and donors:
            fvhat = np.ascontiguousarray(self.interp(k, {dk: self.viscflux(dk, vals[dk]) for dk in donors}))
        q = np.ascontiguousarray(vals[k], dtype=np.float64)
        qhat = np.ascontiguousarray(qhat)
        t = self.terms[k]
        out = np.zeros((4, nj, ni))
        qinf = np.ascontiguousarray(self.p["qinf"], dtype=np.float64)
        rc = L.orc_rhs2d(ni, nj, int(m["periodic"][0]), int(m["periodic"][1]), _p(self.ci[k]), _p(self.cj[k]),
                         _p(self.met[k]), _p(q), int(self.viscous), self.gamma, self.mu, self.pr,
                         t["pt"].size, _p(t["pt"]), _p(t["dir"]), _p(t["side"]), _p(t["kind"]), _p(t["recv"]),
                         _p(t["scale"]), qhat.shape[1], _p(qhat), _p(fvhat), _p(qinf),
                         float(self.p["twall"]), self.sig_int, self.sig_phys, _p(out))
        if rc != 0:
            raise RuntimeError("oracle rhs failed: %d" % rc)
        return out

    def rhs_all(self, qs):
        return [self.rhs(k, qs) for k in range(self.R)]

    # -- time step, bootstrap, MRAB ------------------------------------------------------------
    def ticks(self):
        """Steps of the innermost mesh per step of mesh r."""
        t = [1] * self.R
        for r in range(self.R - 2, -1, -1):
            t[r] = t[r + 1] * self.ratios[r]
        return t

    def dt_mesh(self, k, q):
        L = lib()
        m = self.meshes[k]
        qc = np.ascontiguousarray(q, dtype=np.float64)
        return L.orc_dt2d(m["n"][0], m["n"][1], _p(self.ci[k]), _p(self.met[k]), _p(qc), self.gamma, self.mu,
                          self.pr)

    def macro_step_size(self, qs):
        """H = min over meshes of CFL dt_r times the steps mesh r takes per step of mesh 0, so that
        every mesh's own step h_r = H / (ratios[0] ... ratios[r-1]) respects the CFL limit (the
        two-mesh rule min(CFL dt_slow, SR CFL dt_fast) for R = 2)."""
        cfl = float(self.p["cfl"])
        t = self.ticks()
        return min(cfl * self.dt_mesh(k, qs[k]) * (t[0] // t[k]) for k in range(self.R))

    def bootstrap(self, qs, H):
        """Heun's RK3 at the innermost step h = H / ticks[0] for (m - 1) ticks[0] steps, recording
        mesh r's right-hand side every ticks[r] steps over the last m - 1 steps of mesh r, then all
        right-hand sides at the end: m values per mesh, ending at the bootstrap end time."""
        m = int(self.p["hist_len"])
        t = self.ticks()
        h = H / t[0]
        hists = [[] for _ in range(self.R)]
        y = [np.array(q, dtype=np.float64) for q in qs]
        nsteps = (m - 1) * t[0]
        for step in range(nsteps):
            y, k1 = rk3_heun_step(y, h, self.rhs_all)
            for r in range(self.R):
                if step % t[r] == 0 and step >= nsteps - (m - 1) * t[r]:
                    hists[r].append(k1[r])
        a = self.rhs_all(y)
        for r in range(self.R):
            hists[r].append(a[r])
        return y, hists

    def mrab(self, qs, hists, H, n_steps):
        """n_steps macro steps of mesh 0 with every mesh at its own step (fastest first)."""
        order = int(self.p["order"])
        ys = [np.array(q, dtype=np.float64) for q in qs]
        for _ in range(n_steps):
            ys, hists = mrab_macro_step_multirate(ys, hists, H, self.ratios, order,
                                                  lambda r, vals: self.rhs(r, vals))
        return ys, hists

    def cell_sizes(self):
        return [np.where(self.iblank[k] != 0, 1.0 / self.met[k][4], 0.0) for k in range(self.R)]
