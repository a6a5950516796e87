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
O-grid inside a Cartesian background (Sec. 5.1); each function states its
sizes.
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


def vortex_chain(seed=0, n_bg=48, ratios=(2, 2), halves=(5.0, 2.2, 0.9), omega=5.0, phi=1.0, mach=0.5, order=3,
                 hist_len=None, cfl=0.5, jitter=0.3):
    """2D Euler vortex on a chain of nested overset meshes, one step ratio per level: a periodic
    n_bg^2 background on [-halves[0], halves[0]]^2 and boxes [-halves[r], halves[r]]^2 (interface
    faces) whose spacing is the enclosing mesh's divided by ratios[r-1]; mesh r steps ratios[r-1]
    times per step of mesh r-1."""
    rng = np.random.default_rng(seed)
    hb = 2.0 * halves[0] / n_bg
    meshes = [cartesian_mesh("background", (n_bg, n_bg), (-halves[0], -halves[0]), (hb, hb), ("periodic",) * 4,
                             periodic=(True, True))]
    h = hb
    for r, ratio in enumerate(ratios, start=1):
        h = h / ratio
        n = int(round(2.0 * halves[r] / h)) + 1
        hr = 2.0 * halves[r] / (n - 1)
        meshes.append(cartesian_mesh("level%d" % r, (n, n), (-halves[r], -halves[r]), (hr, hr), ("interface",) * 4))
    c0 = math.sqrt(GAMMA)
    x0, y0 = rng.uniform(-jitter, jitter, 2)
    vort = dict(x0=float(x0), y0=float(y0), u0=mach * c0, v0=0.0, omega=omega, phi=phi)
    q = [vortex_state(m["x"], m["y"], 0.0, gamma=GAMMA, **vort) for m in meshes]
    params = dict(physics="euler", gamma=GAMMA, mu=0.0, pr=0.72, order=order, hist_len=hist_len or order,
                  step_ratio=int(ratios[0]), fast_mesh=1, cfl=cfl,
                  qinf=np.array([1.0, vort["u0"], 0.0, 1.0 / (GAMMA - 1.0) + 0.5 * vort["u0"] ** 2]),
                  twall=1.0, omega_corner=1.0)
    return {"meshes": meshes, "q0": q, "params": params, "ratios": [int(r) for r in ratios], "vortex": vort,
            "seed": seed}


def cylinder_overset(seed=0, n_theta=512, n_r=128, r_in=0.5, stretch=1.05, s_bg=0.05,
                     bg_n=(1024, 512), bg_lo=(-12.8, -12.8), mach=0.2, re=200.0, pr=0.72,
                     order=3, hist_len=None, step_ratio=4, cfl=0.5, amp=1e-3, twall=1.0,
                     sponge_cells=0, sponge_strength=1.0, pulse_amp=0.0, pulse_at=(-1.2, 0.3), pulse_width=0.4):
    """2D Navier-Stokes cylinder in cross-flow: O-grid (wall inside, interface outside) on a
    Cartesian background with far-field faces. The first radial spacing is chosen so that the
    outermost O-grid spacing equals the background spacing. The state is the free stream plus
    amp N(0,1) noise per point, plus (pulse_amp > 0) a smooth pressure pulse
    p (1 + pulse_amp exp(-|x - pulse_at|^2 / pulse_width^2)) at fixed density."""
    rng = np.random.default_rng(seed)
    dr0 = s_bg / stretch ** (n_r - 2)
    og = ogrid_mesh("ogrid", n_theta, n_r, r_in, dr0, stretch)
    bg = cartesian_mesh("background", bg_n, bg_lo, (s_bg, s_bg), ("farfield",) * 4)
    qinf = freestream(mach)
    q_og = noisy_uniform((n_r, n_theta), qinf, amp, rng)
    q_bg = noisy_uniform((bg_n[1], bg_n[0]), qinf, amp, rng)
    if pulse_amp > 0.0:
        p_inf = (GAMMA - 1.0) * (qinf[3] - 0.5 * (qinf[1] ** 2 + qinf[2] ** 2) / qinf[0])
        for m, q in ((og, q_og), (bg, q_bg)):
            r2 = (m["x"] - pulse_at[0]) ** 2 + (m["y"] - pulse_at[1]) ** 2
            q[3] += p_inf * pulse_amp * np.exp(-r2 / pulse_width ** 2) / (GAMMA - 1.0)
    params = dict(physics="ns", gamma=GAMMA, mu=mach / re, pr=pr, order=order,
                  hist_len=hist_len or order, step_ratio=step_ratio, fast_mesh=1, cfl=cfl,
                  qinf=qinf, twall=twall, omega_corner=1.0, sponge_cells=sponge_cells,
                  sponge_strength=sponge_strength)
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


def corner_box_in_box(omega_corner=1.0, n_bg=31, n_fine=41, bg_half=4.0, fine_half=2.0, gamma=GAMMA,
                      order=3, hist_len=4):
    """Box-in-box pair of the corner-penalty study (Sec. 4.2): periodic background [-4,4]^2 with
    31 x 31 points, inner box [-2,2]^2 with 41 x 41 points (all faces interface), inviscid. The
    state is effectively one-dimensional: rho = 1, rho u = 1.25 - 0.01 |x|, rho v = 0 and
    constant pressure 1/gamma (the paper gives the momentum alone; density and pressure follow
    the unit-density, unit-sound-speed convention of the other cases). omega_corner weights the
    interface penalty at fringe points with more than one interface term (eq. (penalty_interp))."""
    hb = 2.0 * bg_half / n_bg
    bg = cartesian_mesh("background", (n_bg, n_bg), (-bg_half, -bg_half), (hb, hb), ("periodic",) * 4,
                        periodic=(True, True))
    hf = 2.0 * fine_half / (n_fine - 1)
    fine = cartesian_mesh("fine", (n_fine, n_fine), (-fine_half, -fine_half), (hf, hf), ("interface",) * 4)
    qs = []
    for m in (bg, fine):
        rho = np.ones_like(m["x"])
        mom = 1.25 - 0.01 * np.abs(m["x"])
        p = np.full_like(m["x"], 1.0 / gamma)
        qs.append(np.stack([rho, mom, np.zeros_like(mom), p / (gamma - 1.0) + 0.5 * mom * mom / rho]))
    params = dict(physics="euler", gamma=gamma, mu=0.0, pr=0.72, order=order, hist_len=hist_len, step_ratio=1,
                  fast_mesh=1, cfl=1.0, qinf=np.array([1.0, 1.25, 0.0, 1.0 / (gamma * (gamma - 1.0)) + 0.5 * 1.25 ** 2]),
                  twall=1.0, omega_corner=float(omega_corner))
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


# --------------------------------------------------------------------------------------------
# 3D Cartesian workloads
# --------------------------------------------------------------------------------------------

def cartesian_mesh3d(name, n, lo, h, bc, periodic=(False, False, False)):
    """Uniform 3D Cartesian mesh with n points per direction starting at lo. Faces are ordered
    i-low, i-high, j-low, j-high, k-low, k-high."""
    return {"name": name, "dim": 3, "n": tuple(int(v) for v in n), "periodic": tuple(bool(v) for v in periodic),
            "cartesian": True, "lo": tuple(map(float, lo)), "h": tuple(map(float, h)), "bc": tuple(bc)}


def axes3d(m):
    """Coordinates of a 3D Cartesian mesh as three 1D arrays (x along i, y along j, z along k)."""
    return [m["lo"][d] + m["h"][d] * np.arange(m["n"][d], dtype=np.float64) for d in range(3)]


def freestream3d(mach, gamma=GAMMA):
    return np.array([1.0, mach, 0.0, 0.0, 1.0 / (gamma * (gamma - 1.0)) + 0.5 * mach * mach])


def taylor_green_box(seed=0, n_bg=256, n_fine=192, ratio=4, mach=0.1, re=1600.0, pr=0.72, pulse_amp=1e-3,
                     pulse_width=4.0, order=3, hist_len=None, step_ratio=4, cfl=0.5, physics="ns"):
    """3D Taylor-Green vortex on a periodic n_bg^3 background over [0, 2 pi)^3 with an overset
    n_fine^3 box at 1/ratio of the background spacing centred at (pi, pi, pi) (interface on all
    six faces), plus a Gaussian pressure pulse of relative amplitude pulse_amp and width
    pulse_width fine spacings at the box centre jittered by the seed. Velocity
    u = M sin x cos y cos z, v = -M cos x sin y cos z, w = 0; pressure
    p = 1/gamma + M^2/16 (cos 2x + cos 2y)(cos 2z + 2); temperature T = gamma p / rho = 1."""
    rng = np.random.default_rng(seed)
    h = 2.0 * math.pi / n_bg
    hf = h / ratio
    bg = cartesian_mesh3d("background", (n_bg,) * 3, (0.0,) * 3, (h,) * 3, ("periodic",) * 6, (True,) * 3)
    lo_f = math.pi - 0.5 * (n_fine - 1) * hf
    fine = cartesian_mesh3d("fine", (n_fine,) * 3, (lo_f,) * 3, (hf,) * 3, ("interface",) * 6)
    centre = np.full(3, math.pi) + rng.uniform(-1.0, 1.0, 3) * hf
    qs = []
    for m in (bg, fine):
        x, y, z = axes3d(m)
        Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
        u = mach * np.sin(X) * np.cos(Y) * np.cos(Z)
        v = -mach * np.cos(X) * np.sin(Y) * np.cos(Z)
        p = 1.0 / GAMMA + mach * mach / 16.0 * (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2.0)
        r2 = (X - centre[0]) ** 2 + (Y - centre[1]) ** 2 + (Z - centre[2]) ** 2
        p = p * (1.0 + pulse_amp * np.exp(-r2 / (pulse_width * hf) ** 2))
        rho = GAMMA * p
        E = p / (GAMMA - 1.0) + 0.5 * rho * (u * u + v * v)
        qs.append(np.stack([rho, rho * u, rho * v, np.zeros_like(rho), E]))
        del X, Y, Z
    params = dict(physics=physics, gamma=GAMMA, mu=(mach / re if physics == "ns" else 0.0), pr=pr, order=order,
                  hist_len=hist_len or order, step_ratio=step_ratio, fast_mesh=1, cfl=cfl,
                  qinf=freestream3d(0.0), twall=1.0, omega_corner=1.0)
    return {"meshes": [bg, fine], "q0": qs, "params": params, "seed": seed}


def taylor_green_small(seed=0, **kw):
    """A scaled-down Taylor-Green box for parity tests: 24^3 background, 21^3 box at ratio 2."""
    args = dict(n_bg=24, n_fine=21, ratio=2, step_ratio=2, pulse_width=2.0, mach=0.3, re=100.0)
    args.update(kw)
    return taylor_green_box(seed=seed, **args)


def extrude_to_3d(wl, nk, lz, axis=2):
    """A 2D Cartesian two-mesh workload extruded along a new periodic direction of nk points
    over length lz: axis = 2 puts the 2D plane in (x, y) and extrudes along z; axis = 1 puts it
    in (x, z) and extrudes along y. The velocity component along the new direction is 0."""
    meshes, qs = [], []
    for m, q in zip(wl["meshes"], wl["q0"]):
        bc = list(m["bc"])
        per = list(m["periodic"])
        if axis == 2:
            n = (m["n"][0], m["n"][1], nk)
            lo = (m["lo"][0], m["lo"][1], 0.0)
            h = (m["h"][0], m["h"][1], lz / nk)
            bc3 = bc + ["periodic", "periodic"]
            per3 = (per[0], per[1], True)
            q3 = np.stack([q[0], q[1], q[2], np.zeros_like(q[0]), q[3]])
            q3 = np.broadcast_to(q3[:, None], (5, nk) + q.shape[1:]).copy()
        else:
            n = (m["n"][0], nk, m["n"][1])
            lo = (m["lo"][0], 0.0, m["lo"][1])
            h = (m["h"][0], lz / nk, m["h"][1])
            bc3 = bc[:2] + ["periodic", "periodic"] + bc[2:]
            per3 = (per[0], True, per[1])
            q3 = np.stack([q[0], q[1], np.zeros_like(q[0]), q[2], q[3]])
            q3 = np.broadcast_to(q3[:, :, None, :], (5, q.shape[1], nk, q.shape[2])).copy()
        meshes.append(cartesian_mesh3d(m["name"], n, lo, h, bc3, per3))
        qs.append(q3)
    p = dict(wl["params"])
    qi = np.asarray(p["qinf"], dtype=np.float64)
    p["qinf"] = (np.array([qi[0], qi[1], qi[2], 0.0, qi[3]]) if axis == 2
                 else np.array([qi[0], qi[1], 0.0, qi[2], qi[3]]))
    return {"meshes": meshes, "q0": qs, "params": p}


# --------------------------------------------------------------------------------------------
# 3D curvilinear overset pair
# --------------------------------------------------------------------------------------------

def curvilinear_mesh3d(name, x, y, z):
    """A 3D curvilinear mesh (non-periodic in every direction) from node coordinates, each
    (nk, nj, ni) with i fastest."""
    x, y, z = (np.ascontiguousarray(v, dtype=np.float64) for v in (x, y, z))
    nk, nj, ni = x.shape
    return {"name": name, "dim": 3, "n": (ni, nj, nk), "curvilinear": True, "x": x, "y": y, "z": z}


def rotation3d(angles):
    """The rotation Rz(c) Ry(b) Rx(a) for angles (a, b, c) in radians, as a 3 x 3 array."""
    a, b, c = angles
    rx = np.array([[1, 0, 0], [0, math.cos(a), -math.sin(a)], [0, math.sin(a), math.cos(a)]])
    ry = np.array([[math.cos(b), 0, math.sin(b)], [0, 1, 0], [-math.sin(b), 0, math.cos(b)]])
    rz = np.array([[math.cos(c), -math.sin(c), 0], [math.sin(c), math.cos(c), 0], [0, 0, 1]])
    return rz @ ry @ rx


def curvilinear_pair(seed=0, n_bg=24, n_fine=25, ratio=2, eps_bg=0.03, eps_fine=0.02, angles=(0.25, -0.15, 0.35),
                     hole_cells=7, physics="euler", mach=0.3, re=200.0, pr=0.72, pulse_amp=0.05, order=3,
                     hist_len=None, step_ratio=2, cfl=0.5, omega_corner=1.0, sponge_cells=0, sponge_strength=1.0):
    """A 3D curvilinear overset pair. Mesh 0: n_bg^3 points over [-1, 1]^3, each coordinate
    displaced by eps_bg sin(2 pi s) sin(2 pi t) of the other two index fractions s, t (far
    field on all six faces). Mesh 1: an n_fine^3 box at 1/ratio of the background spacing,
    displaced the same way by eps_fine times its width, turned by rotation3d(angles) and
    centred near the origin (jittered by the seed; interface on all six faces). Background
    points more than hole_cells index units of mesh 1 inside it are holes. Initial state: a
    uniform stream of Mach `mach` (rho = 1, p = 1 / gamma) along a seeded direction, plus a
    Gaussian bump of relative amplitude pulse_amp and width 4 spacings of mesh 1 at its centre
    in pressure and density, and a swirl about the z axis through the centre of the same
    width. Navier-Stokes: mu = mach / re. The defaults (13,824 + 15,625 points, 125 holes) are
    the parity-test size; the overset box must stay inside the background, and a hole wider
    than n_bg - 16 background points along a line grows (segments shorter than 8 points become
    holes) until the setup finds no donors."""
    rng = np.random.default_rng(seed)
    t = np.linspace(0.0, 1.0, n_bg)
    T3, T2, T1 = np.meshgrid(t, t, t, indexing="ij")
    s2 = 2.0 * math.pi
    xb = -1.0 + 2.0 * T1 + eps_bg * np.sin(s2 * T2) * np.sin(s2 * T3)
    yb = -1.0 + 2.0 * T2 + eps_bg * np.sin(s2 * T1) * np.sin(s2 * T3)
    zb = -1.0 + 2.0 * T3 + eps_bg * np.sin(s2 * T1) * np.sin(s2 * T2)
    hf = 2.0 / (n_bg - 1) / ratio
    width = (n_fine - 1) * hf
    t = np.linspace(0.0, 1.0, n_fine)
    T3, T2, T1 = np.meshgrid(t, t, t, indexing="ij")
    loc = np.stack([(T1 - 0.5) * width + eps_fine * width * np.sin(s2 * T2) * np.sin(s2 * T3),
                    (T2 - 0.5) * width + eps_fine * width * np.sin(s2 * T1) * np.sin(s2 * T3),
                    (T3 - 0.5) * width + eps_fine * width * np.sin(s2 * T1) * np.sin(s2 * T2)])
    R = rotation3d(angles)
    centre = rng.uniform(-0.5, 0.5, 3) * hf
    xf, yf, zf = (centre[a] + sum(R[a, b] * loc[b] for b in range(3)) for a in range(3))
    meshes = [curvilinear_mesh3d("background", xb, yb, zb), curvilinear_mesh3d("overset", xf, yf, zf)]
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    w = 4.0 * hf
    qs = []
    for m in meshes:
        x, y, z = m["x"], m["y"], m["z"]
        G = np.exp(-((x - centre[0]) ** 2 + (y - centre[1]) ** 2 + (z - centre[2]) ** 2) / (w * w))
        rho = 1.0 + 0.5 * pulse_amp * G
        p = (1.0 + pulse_amp * G) / GAMMA
        u = mach * d[0] - pulse_amp * (y - centre[1]) / w * G
        v = mach * d[1] + pulse_amp * (x - centre[0]) / w * G
        wz = np.full_like(G, mach * d[2])
        E = p / (GAMMA - 1.0) + 0.5 * rho * (u * u + v * v + wz * wz)
        qs.append(np.stack([rho, rho * u, rho * v, rho * wz, E]))
    qinf = np.array([1.0, mach * d[0], mach * d[1], mach * d[2], 1.0 / (GAMMA * (GAMMA - 1.0)) + 0.5 * mach * mach])
    params = dict(physics=physics, gamma=GAMMA, mu=(mach / re if physics == "ns" else 0.0), pr=pr, order=order,
                  hist_len=hist_len or order, step_ratio=step_ratio, fast_mesh=1, cfl=cfl, qinf=qinf, twall=1.0,
                  omega_corner=omega_corner, hole_cells=hole_cells, sponge_cells=sponge_cells,
                  sponge_strength=sponge_strength)
    return {"meshes": meshes, "q0": qs, "params": params, "seed": seed}
