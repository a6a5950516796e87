"""Seeded synthetic inputs: mesh coordinates and initial conditions.

This module is shared by the CPU oracle, the tests and the benchmark. It
holds none of the method's arithmetic (no derivative operators, metrics,
fluxes, penalties, interpolation weights or time-integration coefficients):
it only lays out grid coordinates and fills initial states, so that both
implementations receive identical inputs.

Meshes are plain dicts::

    {"name": str, "dim": 2, "n": (ni, nj), "periodic": (bool, bool),
     "cartesian": bool, "lo": (x0, y0), "h": (hx, hy),
     "x": (nj, ni) float64, "y": (nj, ni) float64,
     "shift": ((sx_i, sy_i), (sx_j, sy_j)),   # coordinate jump across a periodic wrap
     "bc": (i_lo, i_hi, j_lo, j_hi)}          # "periodic" | "interface" | "farfield" | "wall"

The index i (the xi direction) runs fastest in every array. States are
(nvar, nj, ni) float64 arrays of conserved variables (rho, rho u, rho v, rho E).

The workloads follow the paper's test problems: the convecting isentropic
vortex of App. C.2 on a box-in-box pair, and a cylinder in cross-flow on an
O-grid inside a Cartesian background (Sec. 5.1), with the sizes listed in
the DESIGN notes.
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = 1.4


def cartesian_mesh(name, n, lo, h, bc, periodic=(False, False)):
    """Uniform Cartesian mesh with n points per direction starting at lo."""
    ni, nj = n
    xi = lo[0] + h[0] * np.arange(ni, dtype=np.float64)
    yj = lo[1] + h[1] * np.arange(nj, dtype=np.float64)
    x, y = np.meshgrid(xi, yj, indexing="xy")
    return {
        "name": name, "dim": 2, "n": (ni, nj), "periodic": tuple(bool(p) for p in periodic),
        "cartesian": True, "lo": tuple(map(float, lo)), "h": tuple(map(float, h)),
        "x": np.ascontiguousarray(x), "y": np.ascontiguousarray(y),
        "shift": ((ni * h[0] if periodic[0] else 0.0, 0.0), (0.0, nj * h[1] if periodic[1] else 0.0)),
        "bc": tuple(bc),
    }


def ogrid_mesh(name, n_theta, n_r, r_in, dr0, stretch, center=(0.0, 0.0), bc_inner="wall",
               bc_outer="interface"):
    """O-grid around a circle: i runs over the angle (periodic), j outward.

    Radial spacing grows geometrically: r_j = r_in + dr0 (stretch^j - 1)/(stretch - 1).
    """
    # clockwise angle so that (i, j) = (angle, radius) is a right-handed frame (J^-1 > 0)
    th = -2.0 * math.pi * np.arange(n_theta, dtype=np.float64) / n_theta
    j = np.arange(n_r, dtype=np.float64)
    if stretch == 1.0:
        r = r_in + dr0 * j
    else:
        r = r_in + dr0 * (stretch ** j - 1.0) / (stretch - 1.0)
    x = center[0] + r[:, None] * np.cos(th)[None, :]
    y = center[1] + r[:, None] * np.sin(th)[None, :]
    return {
        "name": name, "dim": 2, "n": (n_theta, n_r), "periodic": (True, False),
        "cartesian": False, "lo": (0.0, 0.0), "h": (0.0, 0.0),
        "x": np.ascontiguousarray(x), "y": np.ascontiguousarray(y),
        "shift": ((0.0, 0.0), (0.0, 0.0)),
        "bc": ("periodic", "periodic", bc_inner, bc_outer),
        "r": r,
    }


def freestream(mach, gamma=GAMMA, angle=0.0):
    """Free stream with rho = 1, c = 1 (p = 1/gamma), speed = mach."""
    rho = 1.0
    p = 1.0 / gamma
    u = mach * math.cos(angle)
    v = mach * math.sin(angle)
    return np.array([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)])


def vortex_state(x, y, t, x0, y0, u0, v0, omega, phi, gamma=GAMMA):
    """Convecting isentropic vortex of App. C.2 with p_inf = rho_inf = 1, c0^2 = gamma."""
    c0sq = gamma
    dx = x - x0 - u0 * t
    dy = y - y0 - v0 * t
    r2 = dx * dx + dy * dy
    ex = np.exp(1.0 - phi * phi * r2)
    rho = (1.0 - omega * omega * (gamma - 1.0) / (8.0 * math.pi ** 2 * c0sq) * ex) ** (1.0 / (gamma - 1.0))
    amp = omega / (2.0 * math.pi) * phi * np.sqrt(ex)
    u = u0 - amp * dy
    v = v0 + amp * dx
    p = rho ** gamma
    return np.stack([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)])


def noisy_uniform(shape, qinf, amp, rng):
    """Uniform state qinf plus amp * N(0,1) per point and variable, scaled by (1, 1, 1, rhoE_inf)."""
    scale = np.array([1.0, 1.0, 1.0, qinf[3]])
    q = np.empty((4,) + tuple(shape))
    for v in range(4):
        q[v] = qinf[v] + amp * scale[v] * rng.standard_normal(shape)
    return q


# --------------------------------------------------------------------------------------------
# Workloads
# --------------------------------------------------------------------------------------------

def vortex_box_in_box(seed=0, n_bg=64, n_fine=41, bg_half=5.0, fine_half=1.0, omega=5.0, phi=1.0,
                      mach=0.5, order=3, hist_len=None, step_ratio=2, cfl=0.5, jitter=0.5):
    """2D Euler vortex on a periodic background with a fine box patch (all faces interface)."""
    rng = np.random.default_rng(seed)
    hb = 2.0 * bg_half / n_bg
    bg = cartesian_mesh("background", (n_bg, n_bg), (-bg_half, -bg_half), (hb, hb),
                        ("periodic",) * 4, periodic=(True, True))
    hf = 2.0 * fine_half / (n_fine - 1)
    fine = cartesian_mesh("fine", (n_fine, n_fine), (-fine_half, -fine_half), (hf, hf),
                          ("interface",) * 4)
    c0 = math.sqrt(GAMMA)
    x0, y0 = (rng.uniform(-jitter, jitter, 2) if jitter > 0 else (0.0, 0.0))
    vort = dict(x0=float(x0), y0=float(y0), u0=mach * c0, v0=0.0, omega=omega, phi=phi)
    q = [vortex_state(m["x"], m["y"], 0.0, gamma=GAMMA, **vort) for m in (bg, fine)]
    params = dict(physics="euler", gamma=GAMMA, mu=0.0, pr=0.72, order=order,
                  hist_len=hist_len or order, step_ratio=step_ratio, fast_mesh=1, cfl=cfl,
                  qinf=np.array([1.0, vort["u0"], 0.0, 1.0 / (GAMMA - 1.0) + 0.5 * vort["u0"] ** 2]),
                  twall=1.0, omega_corner=1.0)
    return {"meshes": [bg, fine], "q0": q, "params": params, "vortex": vort, "seed": seed}


def cylinder_overset(seed=0, n_theta=512, n_r=128, r_in=0.5, stretch=1.05, s_bg=0.05,
                     bg_n=(1024, 512), bg_lo=(-12.8, -12.8), mach=0.2, re=200.0, pr=0.72,
                     order=3, hist_len=None, step_ratio=4, cfl=0.5, amp=1e-3, twall=1.0):
    """2D Navier-Stokes cylinder in cross-flow: O-grid (wall inside, interface outside) on a
    Cartesian background with far-field faces. The first radial spacing is chosen so that the
    outermost O-grid spacing equals the background spacing."""
    rng = np.random.default_rng(seed)
    dr0 = s_bg / stretch ** (n_r - 2)
    og = ogrid_mesh("ogrid", n_theta, n_r, r_in, dr0, stretch)
    bg = cartesian_mesh("background", bg_n, bg_lo, (s_bg, s_bg), ("farfield",) * 4)
    qinf = freestream(mach)
    q_og = noisy_uniform((n_r, n_theta), qinf, amp, rng)
    q_bg = noisy_uniform((bg_n[1], bg_n[0]), qinf, amp, rng)
    params = dict(physics="ns", gamma=GAMMA, mu=mach / re, pr=pr, order=order,
                  hist_len=hist_len or order, step_ratio=step_ratio, fast_mesh=1, cfl=cfl,
                  qinf=qinf, twall=twall, omega_corner=1.0)
    return {"meshes": [bg, og], "q0": [q_bg, q_og], "params": params, "seed": seed}


def cylinder_small(seed=0, **kw):
    """A scaled-down cylinder case for parity tests (several tiles, ragged edges)."""
    args = dict(n_theta=96, n_r=24, s_bg=0.1, bg_n=(100, 60), bg_lo=(-3.0, -3.0), stretch=1.08)
    args.update(kw)
    return cylinder_overset(seed=seed, **args)


def mms_box_in_box(n, kind="inviscid", gamma=GAMMA, mu=1.0):
    """Box-in-box pair of App. C.1: periodic outer [-1,1]^2 with n x n points, inner
    [-0.5,0.5]^2 with n/2 x n/2 points (all faces interface). The prescribed states are
    rho = 1, rho v = 0, constant pressure 1/gamma, and rho u = sin(2 pi (x - 0.5)) ("inviscid")
    or sin(2 pi (y - 0.5)) ("viscous")."""
    h_out = 2.0 / n
    bg = cartesian_mesh("background", (n, n), (-1.0, -1.0), (h_out, h_out), ("periodic",) * 4,
                        periodic=(True, True))
    ni = n // 2
    h_in = 1.0 / (ni - 1)
    fine = cartesian_mesh("fine", (ni, ni), (-0.5, -0.5), (h_in, h_in), ("interface",) * 4)
    qs = []
    for m in (bg, fine):
        c = m["x"] if kind == "inviscid" else m["y"]
        rho = np.ones_like(c)
        mom = np.sin(2.0 * math.pi * (c - 0.5))
        p = np.full_like(c, 1.0 / gamma)
        qs.append(np.stack([rho, mom, np.zeros_like(c), p / (gamma - 1.0) + 0.5 * mom * mom / rho]))
    params = dict(physics="euler" if kind == "inviscid" else "ns", gamma=gamma,
                  mu=0.0 if kind == "inviscid" else mu, pr=0.72, order=3, hist_len=3, step_ratio=1,
                  fast_mesh=1, cfl=0.5, qinf=np.array([1.0, 0.0, 0.0, 1.0 / (gamma * (gamma - 1.0))]),
                  twall=1.0, omega_corner=1.0)
    return {"meshes": [bg, fine], "q0": qs, "params": params}


def batched_vortices(seed=0, n_systems=64, n_range=(128, 512), ratios=(2, 4, 8), bg_half=5.0, omega=5.0,
                     mach=0.5, order=3, cfl=0.5):
    """Many independent 2D Euler vortex systems: background N x N periodic on [-bg_half, bg_half]^2
    with N ~ U{n_range}, one fine patch of 1/8 of the background side whose spacing is the
    background spacing / r, r drawn from `ratios` and used as the MRAB step ratio; vortex centres
    seeded near the patch."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(n_systems):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        r = int(rng.choice(ratios))
        fine_half = bg_half / 8.0
        n_fine = int(round(n * r / 8.0)) + 1
        wl = vortex_box_in_box(seed=int(rng.integers(1 << 30)), n_bg=n, n_fine=n_fine, bg_half=bg_half,
                               fine_half=fine_half, omega=omega, phi=1.0, mach=mach, order=order,
                               step_ratio=r, cfl=cfl, jitter=0.5 * fine_half)
        out.append(wl)
    return out


def wake_probes(seed=0, n=8, x_range=(1.8, 3.5), y_range=(-0.6, 0.6)):
    """n probe points (x, y) drawn uniformly in a box behind the cylinder (the wake region)."""
    rng = np.random.default_rng(seed)
    return np.stack([rng.uniform(x_range[0], x_range[1], n), rng.uniform(y_range[0], y_range[1], n)], axis=1)


def cylinder_adjoint(seed=0, **kw):
    """The adjoint workload: the cylinder geometry at half resolution (O-grid 256 x 64 on a
    512 x 256 background of spacing 0.1), step ratio 4, with 8 wake probes."""
    args = dict(n_theta=256, n_r=64, s_bg=0.1, bg_n=(512, 256), bg_lo=(-12.8, -12.8), step_ratio=4)
    args.update(kw)
    wl = cylinder_overset(seed=seed, **args)
    wl["probes"] = wake_probes(seed + 1, 8, x_range=(3.0, 6.0), y_range=(-1.0, 1.0))
    return wl
