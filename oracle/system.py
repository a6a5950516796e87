"""Oracle assembly and time integration (TEST INFRASTRUCTURE ONLY).

- ``ab_coefficients``: Adams-Bashforth weights from the Vandermonde moment
  system of Sec. 3.1 eq. (vandermonde), minimum-norm for extended histories
  (Sec. 3.2 eq. (ext_ab)).
- ``mrab_macro_step``: the fastest-first, no-re-extrapolation multi-rate
  scheme of Sec. 3.3 (Steps 1-7), generalised from step ratio 2 to any
  integer step ratio.
- ``rk3_heun_step``: the third-order Runge-Kutta bootstrap of Sec. 3.1.
- ``OracleSystem``: a two-mesh overset system (background + one fine mesh):
  hole cut, stencil classes, metrics, SAT terms, donors (Sec. 2.2), the
  coupled right-hand side, the time step of Sec. 4.1 and the error norm of
  App. C eq. (l2error).

Parity unpinned: the shape of the sponge profile inside the layer
(``OracleSystem.sponge_strength``, a reading; its depth, its relaxation toward
the free stream and its decay away from the face are pinned).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import lib

CL_HOLE = 15
KIND = {"interface": 1, "farfield": 2, "wall": 3}


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


# ---------------------------------------------------------------------------------------------
# Time integration
# ---------------------------------------------------------------------------------------------

def ab_coefficients(nodes, a, b, order):
    """Weights alpha with sum_k alpha_k t_k^i = int_a^b tau^i dtau for i = 0..order-1.

    Sec. 3.1 eq. (vandermonde) with the moment index read as i = 0..n-1 and the
    right-hand side (b^(i+1) - a^(i+1))/(i+1); for more nodes than the order the
    minimum-2-norm solution of Sec. 3.2 eq. (ext_ab). ``nodes`` are the history
    times, oldest first, in any unit; the interval uses the same unit.
    """
    t = np.asarray(nodes, dtype=np.float64)
    V = np.vander(t, order, increasing=True)            # m x n, row k = (1, t_k, ..., t_k^(n-1))
    rhs = np.array([(b ** (i + 1) - a ** (i + 1)) / (i + 1) for i in range(order)])
    alpha, *_ = np.linalg.lstsq(V.T, rhs, rcond=None)   # minimum-norm solution when m > n
    return alpha


def rk3_heun_step(y, h, f):
    """Heun's third-order Runge-Kutta step (the AB3 bootstrap of Sec. 3.1):
    c = (0, 1/3, 2/3), a21 = 1/3, a32 = 2/3, b = (1/4, 0, 3/4). Returns (y_new, k1)."""
    k1 = f(y)
    k2 = f([yi + (h / 3.0) * ki for yi, ki in zip(y, k1)])
    k3 = f([yi + (2.0 * h / 3.0) * ki for yi, ki in zip(y, k2)])
    return [yi + (h / 4.0) * (a + 3.0 * c) for yi, a, c in zip(y, k1, k3)], k1


def rk4_step(y, h, f):
    """The classical fourth-order Runge-Kutta step, the single-rate baseline integrator of
    Sec. 4.4 and 6.1: k1 = f(y), k2 = f(y + h/2 k1), k3 = f(y + h/2 k2), k4 = f(y + h k3),
    y_new = y + h/6 (k1 + 2 k2 + 2 k3 + k4). y is a list of per-component arrays."""
    k1 = f(y)
    k2 = f([yi + (h / 2.0) * ki for yi, ki in zip(y, k1)])
    k3 = f([yi + (h / 2.0) * ki for yi, ki in zip(y, k2)])
    k4 = f([yi + h * ki for yi, ki in zip(y, k3)])
    return [yi + (h / 6.0) * (a + 2.0 * b + 2.0 * c + d) for yi, a, b, c, d in zip(y, k1, k2, k3, k4)]


def _combine(y, coeffs, hist):
    out = y
    for c, a in zip(coeffs, hist):
        out = out + c * a
    return out


def mrab_macro_step(f, s, hist_f, hist_s, H, sr, order, rhs_fast, rhs_slow):
    """One macro step of the fastest-first MRAB scheme without re-extrapolation (Sec. 3.3).

    On entry the histories hold m right-hand-side values each, oldest first, ending
    with the values at the current time t: fast at t-(m-1)h, ..., t and slow at
    t-(m-1)H, ..., t, with h = H/sr.
      Step 1: the extrapolants are the polynomials through these histories.
      Steps 2, 6: f advances by the integral of the fast extrapolant over each micro step.
      Steps 2-4: at each intermediate micro time the slow state is the slow extrapolant
               integrated from t (s itself is not advanced yet), and the fast RHS is
               evaluated there and appended to the fast history.
      Step 5: s advances over [t, t+H] by the integral of the slow extrapolant.
      Step 7: both right-hand sides are evaluated at t+H and appended.
    rhs_fast(f, s_hat) and rhs_slow(s, f) evaluate the coupled right-hand sides.
    """
    m = len(hist_f)
    h = H / sr
    nodes = np.arange(-(m - 1), 1, dtype=np.float64)         # in units of the own step
    alpha_f = ab_coefficients(nodes, 0.0, 1.0, order) * h
    alpha_s = ab_coefficients(nodes, 0.0, 1.0, order) * H
    hist_f = list(hist_f)
    hist_s = list(hist_s)
    for j in range(sr):
        f = _combine(f, alpha_f, hist_f)
        if j < sr - 1:
            beta = ab_coefficients(nodes, 0.0, (j + 1) / sr, order) * H
            s_hat = _combine(s, beta, hist_s)
            hist_f = hist_f[1:] + [rhs_fast(f, s_hat)]
    s = _combine(s, alpha_s, hist_s)
    a_f = rhs_fast(f, s)
    a_s = rhs_slow(s, f)
    hist_f = hist_f[1:] + [a_f]
    hist_s = hist_s[1:] + [a_s]
    return f, s, hist_f, hist_s


def mrab_macro_step_multirate(ys, hists, H, ratios, order, rhs):
    """One macro step [t, t+H] of fastest-first MRAB without re-extrapolation for any number
    of rates. Sec. 3.3 notes that the two-rate scheme extends to any number of rates without
    spelling the extension out; this is the reading: the two-rate recursion nested level by
    level.

    Components 0..R-1 run from slowest to fastest; component r steps with
    h_r = H / (ratios[0] * ... * ratios[r-1]) (ratios: R-1 integers). hists[r] holds m
    right-hand-side values of component r, oldest first, ending at t (nodes t-(m-1)h_r .. t).
    To advance component r over [tau, tau + h_r], component r+1 first takes its ratios[r] steps
    over the same interval; then y_r advances by the integral of its extrapolant (the polynomial
    through hist_r), and its right-hand side at tau + h_r is evaluated with the faster components'
    states (already at tau + h_r) and the slower ones extrapolated: the slower component's state
    at the start of its current step plus the integral of its polynomial up to tau + h_r.
    rhs(r, vals) evaluates component r's right-hand side from the values of all components.
    Times are counted in steps of the fastest component, so that the extrapolation intervals are
    exact ratios. For two rates this is mrab_macro_step operation for operation; with every
    ratio 1 it is single-rate Adams-Bashforth (srab_step) on the whole system."""
    R = len(ys)
    if len(ratios) != R - 1 or len(hists) != R:
        raise ValueError("one history per component and R - 1 step ratios")
    m = len(hists[0])
    nodes = np.arange(-(m - 1), 1, dtype=np.float64)
    ticks = [1] * R                      # steps of the fastest component per step of component r
    for r in range(R - 2, -1, -1):
        ticks[r] = ticks[r + 1] * int(ratios[r])
    h = [H]
    for r in range(1, R):
        h.append(h[-1] / ratios[r - 1])
    alpha = [ab_coefficients(nodes, 0.0, 1.0, order) * h[r] for r in range(R)]
    ys = list(ys)
    hists = [list(x) for x in hists]
    start = [0] * R                      # tick at which each component's current step began

    def extrapolated(c, tick):
        frac = (tick - start[c]) / ticks[c]
        return _combine(ys[c], ab_coefficients(nodes, 0.0, frac, order) * h[c], hists[c])

    def advance(r, tick0):
        if r + 1 < R:
            for j in range(int(ratios[r])):
                advance(r + 1, tick0 + j * ticks[r + 1])
        ys[r] = _combine(ys[r], alpha[r], hists[r])
        tick1 = tick0 + ticks[r]
        vals = [extrapolated(c, tick1) if c < r else ys[c] for c in range(R)]
        hists[r] = hists[r][1:] + [rhs(r, vals)]
        start[r] = tick1

    advance(0, 0)
    return ys, hists


def mrab_macro_step_var(f, s, hist_f, times_f, hist_s, times_s, t, H, sr, order, rhs_fast, rhs_slow):
    """Fastest-first MRAB macro step [t, t+H] for histories at arbitrary past times (the macro
    step may change from one macro step to the next, Sec. 3.3 Step 1): every weight solves the
    moment conditions on the actual node times, shifted to the start of the interval it
    integrates and scaled by its step, so that uniform histories give mrab_macro_step's
    weights. times_f, times_s: the node times of hist_f, hist_s (oldest first, ending at t).
    Returns the states and histories (with their times) at t+H."""
    h = H / sr
    tf = np.asarray(times_f, dtype=np.float64)
    ts = np.asarray(times_s, dtype=np.float64)
    hist_f = list(hist_f)
    for j in range(sr):
        tj = t + j * h
        f = _combine(f, ab_coefficients((tf - tj) / h, 0.0, 1.0, order) * h, hist_f)
        if j < sr - 1:
            beta = ab_coefficients((ts - t) / H, 0.0, (j + 1) / sr, order) * H
            s_hat = _combine(s, beta, hist_s)
            hist_f = hist_f[1:] + [rhs_fast(f, s_hat)]
            tf = np.append(tf[1:], t + (j + 1) * h)
    s = _combine(s, ab_coefficients((ts - t) / H, 0.0, 1.0, order) * H, hist_s)
    hist_f = hist_f[1:] + [rhs_fast(f, s)]
    hist_s = list(hist_s[1:]) + [rhs_slow(s, f)]
    return f, s, hist_f, np.append(tf[1:], t + H), hist_s, np.append(ts[1:], t + H)


def mrab_macro_step_slowest_first(f, s, hist_f, hist_s, H, sr, order, rhs_fast, rhs_slow, reextrapolate=False):
    """One macro step of the slowest-first MRAB variants, the other ordering of Sec. 3.3's
    design choices (the paper's runs use fastest-first; the variants follow its description of
    the alternatives). Entry: histories of m values each, oldest first, ending at t.
      1. s advances over [t, t+H] by the integral of the slow extrapolant (history ending at t).
      2. The fast state at t+H is extrapolated: f^ = f(t) + integral of the fast extrapolant
         over [t, t+H].
      3. The slow right-hand side at t+H is evaluated with it, a_s(s(t+H), f^), and appended.
      4. The fast micro steps as in fastest-first; the slow state at the intermediate micro
         times is s(t) + the integral from t of the slow polynomial through the slow history:
         without re-extrapolation the one of step 1 (history ending at t), with
         re-extrapolation the one through the updated history (ending at t+H).
      5. The fast right-hand side at t+H, a_f(f(t+H), s(t+H)), is appended.
    """
    m = len(hist_f)
    h = H / sr
    nodes = np.arange(-(m - 1), 1, dtype=np.float64)
    alpha_f = ab_coefficients(nodes, 0.0, 1.0, order) * h
    alpha_s = ab_coefficients(nodes, 0.0, 1.0, order) * H
    s_new = _combine(s, alpha_s, hist_s)
    f_hat = _combine(f, ab_coefficients(nodes, 0.0, float(sr), order) * h, hist_f)
    hist_s_new = list(hist_s[1:]) + [rhs_slow(s_new, f_hat)]
    nodes_new = nodes + 1.0  # the updated slow history, relative to t in units of H
    hist_f = list(hist_f)
    for j in range(sr):
        f = _combine(f, alpha_f, hist_f)
        if j < sr - 1:
            if reextrapolate:
                beta = ab_coefficients(nodes_new, 0.0, (j + 1) / sr, order) * H
                s_hat = _combine(s, beta, hist_s_new)
            else:
                beta = ab_coefficients(nodes, 0.0, (j + 1) / sr, order) * H
                s_hat = _combine(s, beta, hist_s)
            hist_f = hist_f[1:] + [rhs_fast(f, s_hat)]
    hist_f = hist_f[1:] + [rhs_fast(f, s_new)]
    return f, s_new, hist_f, hist_s_new


def srab_step(y, hist, dt, order, rhs):
    """Single-rate Adams-Bashforth step of Sec. 3.1 eq. (ab_general) on the whole system:
    y(t+dt) = y(t) + sum_k alpha_k F_k; then F at t+dt is appended to the history.
    y and each history entry are lists of per-component arrays."""
    m = len(hist)
    nodes = np.arange(-(m - 1), 1, dtype=np.float64)
    alpha = ab_coefficients(nodes, 0.0, 1.0, order) * dt
    y = [_combine(yc, alpha, [hk[c] for hk in hist]) for c, yc in enumerate(y)]
    return y, list(hist[1:]) + [rhs(y)]


def l2_norm(errs, vols):
    """App. C eq. (l2error): sqrt(sum over meshes and points of eps^2 * cell size)."""
    return float(np.sqrt(sum(float(np.sum(e * e * v)) for e, v in zip(errs, vols))))


# ---------------------------------------------------------------------------------------------
# Two-mesh overset system
# ---------------------------------------------------------------------------------------------

def _outer_polygon(mesh):
    """Closed outer boundary of a mesh as a polygon (counter-clockwise for the layouts used)."""
    x, y = mesh["x"], mesh["y"]
    ni, nj = mesh["n"]
    if mesh["periodic"][0]:                       # O-grid: outermost ring
        return x[nj - 1].copy(), y[nj - 1].copy()
    px = np.concatenate([x[0, :], x[1:, ni - 1], x[nj - 1, ni - 2::-1], x[nj - 2:0:-1, 0]])
    py = np.concatenate([y[0, :], y[1:, ni - 1], y[nj - 1, ni - 2::-1], y[nj - 2:0:-1, 0]])
    return px.copy(), py.copy()


class OracleSystem:
    """Background (mesh 0) + one overset fine mesh (mesh 1), 2D.

    Setup follows the readings of Sec. 2.2 for what the paper defers:
      * background points inside the fine mesh's outer boundary and more than
        ``hole_cells`` background spacings from it are holes;
      * every maximal active run along a line is an SBP segment (>= 8 points);
      * receivers are the points of interface faces and the segment ends next
        to a hole; each gets one SAT term per normal direction and side, scaled
        by Omega (Sec. 4.2 eq. (penalty_interp)) where a point has several;
      * donors: 4x4 Lagrange stencils on the other mesh.
    """

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
        # hole cut of the background by the fine mesh
        self.iblank = [np.ones((m["n"][1], m["n"][0]), np.int8) for m in self.meshes]
        bx, by = _outer_polygon(fine)
        margin = hole_cells * max(bg["h"])
        L.orc_holecut2d(bg["x"].size, _p(bg["x"]), _p(bg["y"]), bx.size, _p(bx), _p(by), margin,
                        _p(self.iblank[0]))
        self.ci, self.cj, self.met, self.shift = [], [], [], []
        for k, m in enumerate(self.meshes):
            ni, nj = m["n"]
            ci = np.zeros((nj, ni), np.int8)
            cj = np.zeros((nj, ni), np.int8)
            rc = L.orc_classes2d(ni, nj, int(m["periodic"][0]), int(m["periodic"][1]),
                                 _p(self.iblank[k]), _p(ci), _p(cj))
            if rc < 0:
                raise RuntimeError("hole growing did not converge")
            shift = np.array([m["shift"][0][0], m["shift"][0][1], m["shift"][1][0], m["shift"][1][1]])
            met = np.zeros((5, nj, ni))
            if m["cartesian"]:
                # a uniform Cartesian map is linear and D reproduces linear functions exactly, so
                # the metrics are the exact constants (y_eta, -x_eta, -y_xi, x_xi, 1/(hx hy))
                hx, hy = m["h"]
                act = ci != CL_HOLE
                for c, val in enumerate((hy, 0.0, 0.0, hx, 1.0 / (hx * hy))):
                    met[c] = np.where(act, val, 1.0 if c in (0, 3, 4) else 0.0)
            else:
                rc = L.orc_metrics2d(ni, nj, _p(shift), _p(m["x"]), _p(m["y"]), _p(ci), _p(cj), _p(met))
                if rc != 0:
                    raise RuntimeError("non-positive cell volume at point %d" % (-1 - rc))
            self.ci.append(ci)
            self.cj.append(cj)
            self.met.append(met)
            self.shift.append(shift)
        self._build_terms()
        self._build_donors()

    # -- SAT terms and receivers ------------------------------------------------------------
    def _build_terms(self):
        self.terms = []
        self.recv_pts = []
        for k, m in enumerate(self.meshes):
            ni, nj = m["n"]
            ib = self.iblank[k]
            terms = {}   # point -> list of (dir, side, kind)

            def add(p, d, side, kind):
                terms.setdefault(p, []).append((d, side, kind))

            bc = m["bc"]
            for face, (d, side) in enumerate(((0, 1), (0, -1), (1, 1), (1, -1))):
                kind = bc[face]
                if kind == "periodic":
                    continue
                if d == 0:
                    i = 0 if side == 1 else ni - 1
                    pts = [j * ni + i for j in range(nj)]
                else:
                    j = 0 if side == 1 else nj - 1
                    pts = [j * ni + i for i in range(ni)]
                for p in pts:
                    if ib.flat[p]:
                        add(p, d, side, KIND[kind])
            # segment ends next to holes
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
                                add(p, d, side, KIND["interface"])
            recv = sorted(p for p, ts in terms.items() if any(t[2] == 1 for t in ts))
            rid = {p: r for r, p in enumerate(recv)}
            rows = []
            for p in sorted(terms):
                ts = terms[p]
                n_int = sum(1 for t in ts if t[2] == 1)
                for d, side, kind in ts:
                    scale = self.p["omega_corner"] if (kind == 1 and n_int > 1) else 1.0
                    rows.append((p, d, side, kind, rid.get(p, -1) if kind == 1 else -1, scale))
            arr = {
                "pt": np.array([r[0] for r in rows], np.int32),
                "dir": np.array([r[1] for r in rows], np.int32),
                "side": np.array([r[2] for r in rows], np.int32),
                "kind": np.array([r[3] for r in rows], np.int32),
                "recv": np.array([r[4] for r in rows], np.int32),
                "scale": np.array([r[5] for r in rows], np.float64),
            }
            self.terms.append(arr)
            self.recv_pts.append(np.array(recv, np.int64))

    def _build_donors(self):
        L = lib()
        self.base, self.w, self.xe = [], [], []
        for k, m in enumerate(self.meshes):
            dm = self.meshes[1 - k]
            pts = self.recv_pts[k]
            px = np.ascontiguousarray(m["x"].ravel()[pts])
            py = np.ascontiguousarray(m["y"].ravel()[pts])
            n = pts.size
            base = np.zeros((n, 2), np.int32)
            w = np.zeros((n, 8))
            xe = np.zeros((n, 2))
            if n:
                rc = L.orc_donors2d(dm["n"][0], dm["n"][1], int(dm["periodic"][0]), int(dm["periodic"][1]),
                                    _p(self.shift[1 - k]), _p(dm["x"]), _p(dm["y"]), _p(self.iblank[1 - k]),
                                    n, _p(px), _p(py), _p(base), _p(w), _p(xe))
                if rc != 0:
                    raise RuntimeError("no donor for receiver %d of mesh %d" % (rc - 1, k))
            self.base.append(base)
            self.w.append(w)
            self.xe.append(xe)

    # -- pointwise operators ------------------------------------------------------------------
    def viscflux(self, k, q):
        L = lib()
        m = self.meshes[k]
        ni, nj = m["n"]
        q = np.ascontiguousarray(q, dtype=np.float64)
        fv = np.zeros((6, nj, ni))
        L.orc_viscflux2d(ni, nj, int(m["periodic"][0]), int(m["periodic"][1]), _p(self.ci[k]),
                         _p(self.cj[k]), _p(self.met[k]), _p(q), self.gamma, self.mu, self.pr, _p(fv))
        return fv

    def interp(self, k, field):
        """Values at mesh k's receivers interpolated from a full field on the other mesh."""
        L = lib()
        dm = self.meshes[1 - k]
        field = np.ascontiguousarray(field, dtype=np.float64)
        nf = field.shape[0]
        n = self.recv_pts[k].size
        out = np.zeros((nf, n))
        if n:
            L.orc_interp2d(dm["n"][0], dm["n"][1], nf, _p(field), n, _p(self.base[k]), _p(self.w[k]),
                           _p(out))
        return out

    def sponge_strength(self, k):
        """Sponge layer of Sec. 5.1 (far-field boundaries with a sponge `sponge_cells` points deep,
        the form cited to Bodony's sponge analysis, not printed): per point the strength
        sigma = A ((D - d) / D)^2 for the index distance d < D from a far-field face, the largest
        over the faces, A = `sponge_strength`; 0 elsewhere, at holes, or with D = 0."""
        m = self.meshes[k]
        ni, nj = m["n"]
        D = int(self.p.get("sponge_cells", 0))
        sig = np.zeros((nj, ni))
        if D <= 0:
            return sig
        A = float(self.p.get("sponge_strength", 1.0))
        i = np.arange(ni)[None, :] + 0 * np.arange(nj)[:, None]
        j = np.arange(nj)[:, None] + 0 * np.arange(ni)[None, :]
        for face, d in zip(m["bc"], (i, ni - 1 - i, j, nj - 1 - j)):
            if face == "farfield":
                sig = np.maximum(sig, np.where(d < D, A * ((D - d) / D) ** 2, 0.0))
        return np.where(self.iblank[k] != 0, sig, 0.0)

    def rhs(self, k, q, qhat, fvhat=None):
        """dq/dt on mesh k given the interpolated donor values at its receivers."""
        L = lib()
        m = self.meshes[k]
        ni, nj = m["n"]
        q = np.ascontiguousarray(q, dtype=np.float64)
        qhat = np.ascontiguousarray(qhat, dtype=np.float64)
        if fvhat is not None:
            fvhat = np.ascontiguousarray(fvhat, dtype=np.float64)
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
        if int(self.p.get("sponge_cells", 0)) > 0:
            # relaxation toward the far-field state in the sponge layer
            out -= self.sponge_strength(k)[None] * (q - qinf[:, None, None])
        return out

    def coupled_rhs(self, k, q_self, q_other):
        """Right-hand side of mesh k with receivers fed from the other mesh's state."""
        qhat = self.interp(k, q_other)
        fvhat = self.interp(k, self.viscflux(1 - k, q_other)) if self.viscous else None
        return self.rhs(k, q_self, qhat, fvhat)

    def rhs_all(self, qs):
        return [self.coupled_rhs(k, qs[k], qs[1 - k]) for k in range(2)]

    # -- time step, bootstrap, MRAB ------------------------------------------------------------
    def dt_mesh(self, k, q):
        L = lib()
        m = self.meshes[k]
        q = np.ascontiguousarray(q, dtype=np.float64)
        return L.orc_dt2d(m["n"][0], m["n"][1], _p(self.ci[k]), _p(self.met[k]), _p(q), self.gamma, self.mu,
                          self.pr)

    def macro_step_size(self, qs):
        """H = min(CFL dt_slow, SR CFL dt_fast) so that both meshes respect the CFL limit."""
        cfl = float(self.p["cfl"])
        sr = int(self.p["step_ratio"])
        return min(cfl * self.dt_mesh(self.slow, qs[self.slow]), sr * cfl * self.dt_mesh(self.fast, qs[self.fast]))

    def bootstrap(self, qs, H):
        """RK3 at the micro step h for (m-1)*SR steps; returns states and full histories
        (m values each, ending at the bootstrap end time)."""
        sr = int(self.p["step_ratio"])
        m = int(self.p["hist_len"])
        h = H / sr
        hist_f, hist_s = [], []
        y = [np.array(q, dtype=np.float64) for q in qs]
        nsteps = (m - 1) * sr
        for step in range(nsteps):
            y, k1 = rk3_heun_step(y, h, self.rhs_all)
            if step >= nsteps - (m - 1):
                hist_f.append(k1[self.fast])
            if step % sr == 0:
                hist_s.append(k1[self.slow])
        a = self.rhs_all(y)
        hist_f.append(a[self.fast])
        hist_s.append(a[self.slow])
        return y, hist_f, hist_s

    def mrab(self, qs, hist_f, hist_s, H, n_steps, scheme="fastest_first"):
        """n_steps MRAB macro steps; scheme "fastest_first" (the paper's), "slowest_first" or
        "slowest_first_reextrapolate" (Sec. 3.3's alternatives)."""
        f, s = qs[self.fast], qs[self.slow]
        sr = int(self.p["step_ratio"])
        order = int(self.p["order"])
        for _ in range(n_steps):
            kw = dict(rhs_fast=lambda ff, ss: self.coupled_rhs(self.fast, ff, ss),
                      rhs_slow=lambda ss, ff: self.coupled_rhs(self.slow, ss, ff))
            if scheme == "fastest_first":
                f, s, hist_f, hist_s = mrab_macro_step(f, s, hist_f, hist_s, H, sr, order, **kw)
            elif scheme in ("slowest_first", "slowest_first_reextrapolate"):
                f, s, hist_f, hist_s = mrab_macro_step_slowest_first(
                    f, s, hist_f, hist_s, H, sr, order, reextrapolate=scheme.endswith("reextrapolate"), **kw)
            else:
                raise ValueError("unknown MRAB scheme " + scheme)
        out = [None, None]
        out[self.fast], out[self.slow] = f, s
        return out, hist_f, hist_s

    def rk4(self, qs, h, n_steps):
        """n_steps classical Runge-Kutta steps of size h on both meshes at one rate, every stage
        with the overset coupling (the baseline integrator of Sec. 4.4 and 6.1)."""
        y = [np.array(q, dtype=np.float64) for q in qs]
        for _ in range(n_steps):
            y = rk4_step(y, h, self.rhs_all)
        return y

    def mrab_var(self, qs, hist_f, hist_s, H0, steps):
        """Fastest-first MRAB with a macro step that changes between macro steps: the
        histories come from bootstrap(qs, H0) (node times -(m-1)..0 in units of its micro and
        macro step), then one macro step per entry of `steps`."""
        sr = int(self.p["step_ratio"])
        order = int(self.p["order"])
        m = len(hist_f)
        h0 = H0 / sr
        tf = np.array([(k - (m - 1)) * h0 for k in range(m)])
        ts = np.array([(k - (m - 1)) * H0 for k in range(m)])
        f, s, t = qs[self.fast], qs[self.slow], 0.0
        for H in steps:
            f, s, hist_f, tf, hist_s, ts = mrab_macro_step_var(
                f, s, hist_f, tf, hist_s, ts, t, H, sr, order,
                rhs_fast=lambda ff, ss: self.coupled_rhs(self.fast, ff, ss),
                rhs_slow=lambda ss, ff: self.coupled_rhs(self.slow, ss, ff))
            t = t + H
        out = [None, None]
        out[self.fast], out[self.slow] = f, s
        return out

    def cell_sizes(self):
        """Cell size per point for eq. (l2error): J^-1 (= dx dy on Cartesian meshes), holes 0."""
        return [np.where(self.iblank[k] != 0, 1.0 / self.met[k][4], 0.0) for k in range(2)]


# ---------------------------------------------------------------------------------------------
# Probe-pressure objective (the objective of the discrete adjoint; the paper has none)
# ---------------------------------------------------------------------------------------------
def probe_stencil(mesh, xy):
    """4 x 4 Lagrange stencil of point xy on a Cartesian mesh, the stencil kind of Sec. 2.2's
    interpolation: nodes i0..i0+3 along each direction with i0 = floor(xi) - 1 (the point in
    the middle cell), shifted inward at non-periodic edges; weights are the Lagrange basis
    polynomials of those nodes at the point. Returns ((i0, j0), (w_i[4], w_j[4]))."""
    base, ws = [], []
    for d in range(2):
        xi = (xy[d] - mesh["lo"][d]) / mesh["h"][d]
        n = mesh["n"][d]
        i0 = int(np.floor(xi)) - 1
        if not mesh["periodic"][d]:
            if xi < 0.0 or xi > n - 1:
                raise ValueError("probe outside the mesh")
            i0 = max(0, min(n - 4, i0))
        t = xi - i0
        w = []
        for a in range(4):
            others = [b for b in range(4) if b != a]
            w.append(np.prod([(t - b) / (a - b) for b in others]))
        base.append(i0)
        ws.append(np.array(w))
    return tuple(base), tuple(ws)


def probe_pressure(mesh, q, stencil, gamma):
    """Pressure interpolated at a probe: sum over the 4 x 4 nodes of w_a w_b p(q)."""
    (i0, j0), (wi, wj) = stencil
    ni, nj = mesh["n"]
    acc = 0.0
    for b in range(4):
        for a in range(4):
            i, j = (i0 + a) % ni, (j0 + b) % nj
            rho, mx, my, E = q[:, j, i]
            p = (gamma - 1.0) * (E - 0.5 * (mx * mx + my * my) / rho)
            acc += wi[a] * wj[b] * p
    return acc


def probe_objective(osys, q0, probe_xy, n_steps, H):
    """J = H sum_{n=1..n_steps} sum_p p_p(t_n)^2 over the bootstrap + n_steps MRAB macro steps
    (Sec. 3.1, Sec. 3.3) from the initial states q0, probes on the background (mesh 0).
    Returns (J, pressures[n_steps, n_probes])."""
    bg = osys.meshes[0]
    st = [probe_stencil(bg, xy) for xy in np.asarray(probe_xy, dtype=np.float64).reshape(-1, 2)]
    qs, hf, hs = osys.bootstrap([np.array(q, dtype=np.float64) for q in q0], H)
    pr = np.zeros((n_steps, len(st)))
    J = 0.0
    for n in range(n_steps):
        qs, hf, hs = osys.mrab(qs, hf, hs, H, 1)
        for p, s in enumerate(st):
            pr[n, p] = probe_pressure(bg, qs[0], s, osys.gamma)
        J += H * float(np.sum(pr[n] ** 2))
    return J, pr
