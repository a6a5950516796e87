"""Comparison helpers and the tolerances the parity tests derive from the arithmetic.

* Increments, not states: a time step is checked on y_end - y_start, where y_start is the state
  at the start of the tested steps on both sides, so that a state that did not advance fails
  (its increment error is 100 %). The bar applies to the increment, except where the rounding of
  the stored state itself (one half unit in the last place per stored update, growing like the
  square root of the number of updates) is a larger fraction of the increment; that floor is
  added to the bar.
* FP32 right-hand sides against the FP64 oracle: every flux value carries the rounding of the
  ~12 FP32 operations that form it and the derivative stencil adds its own four, so the
  absolute error of dq/dt is at most (12 + 4) u32 sum_k |c_k| J (|F_xi| + |F_eta|) with
  u32 = 2^-24 and sum_k |c_k| = 3/2 for the interior row; relative to |dq/dt| this is large
  where the flux differences cancel (a nearly uniform flow), which the bound measures case by
  case from the oracle's state and metrics. Navier-Stokes adds the rounding of the primitives
  taken through two derivatives (the gradient, then the divergence of the viscous flux), which
  grows like |grad xi|^2: large on the finely stretched cells of a wall-resolving mesh.
"""
import math

import numpy as np

U32 = 2.0 ** -24
U64 = 2.0 ** -53
GAMMA = 1.4


def rel(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def rel_increment(got, want, start):
    """Relative L2 error of the increment got - start against want - start."""
    return rel(np.asarray(got) - start, np.asarray(want) - start)


def increment_tol(bar, start, want, n_updates, unit):
    """bar plus the rounding floor of the stored state: 2 sqrt(n_updates) unit |q| / |dq|.
    Asserts that the comparison is not vacuous (the floor well below the increment)."""
    dq = np.linalg.norm(np.asarray(want) - start)
    floor = 2.0 * math.sqrt(max(n_updates, 1)) * unit * np.linalg.norm(start) / max(dq, 1e-300)
    assert floor < 0.1, "the increment is below the state's own rounding: run more steps"
    return bar + floor


def fp32_rhs_bound(met, q, act, mu=0.0, pr=0.72):
    """Numerator of the derived FP32 bound (module docstring), from the state q (4, nj, ni) and
    the metric planes met (xi_x/J, xi_y/J, eta_x/J, eta_y/J, J), over the active points:
    the flux term 16 u32 (3/2) J (|F_xi| + |F_eta|), plus, for Navier-Stokes (mu > 0), the
    rounding of the primitives carried through two derivatives: 16 u32 (3/2)^2
    (|grad xi| + |grad eta|)^2 mu (4/3 (|u| + |v|)(1 + |u| + |v|) + |T| / (Pr (gamma - 1))), the
    largest of the momentum and energy viscous terms."""
    rho, mx, my, E = q
    u, v = mx / rho, my / rho
    p = (GAMMA - 1.0) * (E - 0.5 * rho * (u * u + v * v))
    F = np.stack([mx, mx * u + p, mx * v, (E + p) * u])
    G = np.stack([my, my * u, my * v + p, (E + p) * v])
    fx = np.abs(met[0] * F + met[1] * G)
    fe = np.abs(met[2] * F + met[3] * G)
    b = 16.0 * U32 * 1.5 * met[4] * (fx + fe)
    if mu > 0.0:
        gk = met[4] * (np.hypot(met[0], met[1]) + np.hypot(met[2], met[3]))
        T = GAMMA * p / rho
        au, av = np.abs(u), np.abs(v)
        visc = mu * (4.0 / 3.0 * (au + av) * (1.0 + au + av) + np.abs(T) / (pr * (GAMMA - 1.0)))
        b = b + 16.0 * U32 * 2.25 * gk * gk * visc
    return float(np.linalg.norm(b[:, act]))


def fp32_rhs_tol(met, q, act, rhs_ref, mu=0.0, pr=0.72):
    """The derived FP32 bound relative to the oracle's right-hand side rhs_ref."""
    return fp32_rhs_bound(met, q, act, mu, pr) / float(np.linalg.norm(rhs_ref[:, act]))


def fp32_rhs_tol_3d(q, h, act, rhs_ref):
    """The same bound on a 3D Cartesian mesh of spacings h = (hx, hy, hz): 16 u32 (3/2)
    |(|F|/hx + |G|/hy + |H|/hz)| / |dq/dt| over the active points, q = (rho, rho u, rho v,
    rho w, rho E)."""
    rho, mx, my, mz, E = q
    u, v, w = mx / rho, my / rho, mz / rho
    p = (GAMMA - 1.0) * (E - 0.5 * rho * (u * u + v * v + w * w))
    F = np.stack([mx, mx * u + p, mx * v, mx * w, (E + p) * u])
    G = np.stack([my, my * u, my * v + p, my * w, (E + p) * v])
    H = np.stack([mz, mz * u, mz * v, mz * w + p, (E + p) * w])
    s = np.abs(F) / h[0] + np.abs(G) / h[1] + np.abs(H) / h[2]
    return 16.0 * U32 * 1.5 * float(np.linalg.norm(s[:, act])) / float(np.linalg.norm(rhs_ref[:, act]))


def fp32_rhs_tol_curv(q, op, act, rhs_ref, mu=0.0, pr=0.72, unit=U32):
    """The same bound on a 3D curvilinear mesh (op: an oracle.curv3d.Curvilinear3D): the flux term
    16 u (3/2) J sum_m |F^_m| with the contravariant fluxes F^_m = sum_j M[m][j] F_j, plus,
    for Navier-Stokes, 16 u (3/2)^2 (sum_m |grad xi_m|)^2 mu (4/3 |u|_1 (1 + |u|_1) + |T| /
    (Pr (gamma - 1))) with |u|_1 = |u| + |v| + |w|; relative to the oracle's right-hand side
    over the active points. u = u32 by default; with unit = U64 it is the FP64 rounding bound,
    which exceeds 1e-12 where a nearly uniform stream makes the flux differences cancel."""
    rho, mx, my, mz, E = q
    u, v, w = mx / rho, my / rho, mz / rho
    p = (GAMMA - 1.0) * (E - 0.5 * rho * (u * u + v * v + w * w))
    F = [np.stack([mx, mx * u + p, mx * v, mx * w, (E + p) * u]),
         np.stack([my, my * u, my * v + p, my * w, (E + p) * v]),
         np.stack([mz, mz * u, mz * v, mz * w + p, (E + p) * w])]
    s = 0.0
    for m in range(3):
        s = s + np.abs(op.M[m][0] * F[0] + op.M[m][1] * F[1] + op.M[m][2] * F[2])
    b = 16.0 * unit * 1.5 * op.J * s
    if mu > 0.0:
        gk = sum(op.J * np.sqrt(op.M[m][0] ** 2 + op.M[m][1] ** 2 + op.M[m][2] ** 2) for m in range(3))
        T = GAMMA * p / rho
        a1 = np.abs(u) + np.abs(v) + np.abs(w)
        visc = mu * (4.0 / 3.0 * a1 * (1.0 + a1) + np.abs(T) / (pr * (GAMMA - 1.0)))
        b = b + 16.0 * unit * 2.25 * gk * gk * visc
    return float(np.linalg.norm(b[:, act])) / float(np.linalg.norm(rhs_ref[:, act]))


def viscous_flux_rounding_curv(q, op, act, mu, pr=0.72, unit=U64):
    """Largest absolute rounding of the Cartesian viscous fluxes on a 3D curvilinear mesh over its
    active points: the primitives' rounding carried through the gradient (the derivative's row,
    sum |c| = 3/2, times |grad xi| summed over the three directions) into the stress and the heat
    flux, 16 u (3/2) (sum_m |grad xi_m|) mu (4/3 |u|_1 (1 + |u|_1) + |T| / (Pr (gamma - 1)))."""
    rho, mx, my, mz, E = q
    u, v, w = mx / rho, my / rho, mz / rho
    p = (GAMMA - 1.0) * (E - 0.5 * rho * (u * u + v * v + w * w))
    gk = sum(op.J * np.sqrt(op.M[m][0] ** 2 + op.M[m][1] ** 2 + op.M[m][2] ** 2) for m in range(3))
    a1 = np.abs(u) + np.abs(v) + np.abs(w)
    T = GAMMA * p / rho
    b = 16.0 * unit * 1.5 * gk * mu * (4.0 / 3.0 * a1 * (1.0 + a1) + np.abs(T) / (pr * (GAMMA - 1.0)))
    return float(b[act].max())
