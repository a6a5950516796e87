"""Energy stability of the oracle's interface SAT (Sec. 2.2 eq. (int)), pinned by the spectrum of
the linearised two-mesh operator.

Two overlapping uniform meshes, A on [0, 1] and B on [0.73, 1.73] (non-coinciding nodes, spacings
1/20 and 1/25), each periodic along y with the same period and far-field faces at their outer
ends, are coupled at their inner ends by the interface SAT with 4 x 4 Lagrange donors. A state
that does not vary along y stays so, so the right-hand side restricted to such states is a
one-dimensional two-mesh SBP-SAT operator (4 x 47 = 188 unknowns). Its Jacobian at a uniform flow
(central differences of the oracle's right-hand side) must have no eigenvalue with a positive
real part: the semi-discretisation is stable, as the SAT's energy estimate makes it for
sigma^I = 1/2 with the p0^-1 factor. Planted mistakes (on the CPU, in the oracle): a flipped
penalty sign, and the p0^-1 factor dropped (equivalent to sigma^I = 17/96), give growing modes;
so does the viscous flux-jump term with a flipped sign (a copy of the oracle compiled with the
mistake)."""
import numpy as np
import pytest

import workloads as W
from conftest import planted_oracle, run_with_oracle
from oracle import OracleSystem

P0 = 17.0 / 48.0


def _pair(mach=0.5, angle=0.0, physics="euler", mu=0.0, nA=21, nB=26, ny=(8, 10), Ly=0.4):
    hA, hB = 1.0 / (nA - 1), 1.0 / (nB - 1)
    A = W.cartesian_mesh("A", (nA, ny[0]), (0.0, 0.0), (hA, Ly / ny[0]),
                         ("farfield", "interface", "periodic", "periodic"), periodic=(False, True))
    B = W.cartesian_mesh("B", (nB, ny[1]), (0.73, 0.0), (hB, Ly / ny[1]),
                         ("interface", "farfield", "periodic", "periodic"), periodic=(False, True))
    qinf = W.freestream(mach, angle=angle)
    params = dict(physics=physics, gamma=W.GAMMA, mu=mu, pr=0.72, order=3, hist_len=3, step_ratio=1,
                  fast_mesh=1, cfl=0.5, qinf=qinf, twall=1.0, omega_corner=1.0)
    q = [np.broadcast_to(qinf[:, None, None], (4, m["n"][1], m["n"][0])).copy() for m in (A, B)]
    return {"meshes": [A, B], "q0": q, "params": params}


def _jacobian_1d(wl, osys, eps=1e-6):
    """Jacobian of the coupled right-hand side with respect to y-uniform perturbations, read
    on the first row of each mesh (every row is the same); central differences."""
    n = [m["n"][0] for m in wl["meshes"]]
    N = 4 * sum(n)
    Jm = np.zeros((N, N))
    col = 0
    for k in range(2):
        for v in range(4):
            for i in range(n[k]):
                outs = []
                for s in (1.0, -1.0):
                    q = [x.copy() for x in wl["q0"]]
                    q[k][v, :, i] += s * eps
                    r = osys.rhs_all(q)
                    # the response is uniform along y
                    assert all(np.allclose(r[kk], r[kk][:, :1, :], rtol=0, atol=1e-9) for kk in range(2))
                    outs.append(np.concatenate([r[kk][:, 0, :].ravel() for kk in range(2)]))
                Jm[:, col] = (outs[0] - outs[1]) / (2.0 * eps)
                col += 1
    return Jm


def _max_real(wl, **kw):
    osys = OracleSystem(wl, hole_cells=1000, **kw)   # no hole: the meshes overlap only at their ends
    assert all(int((ib == 0).sum()) == 0 for ib in osys.iblank)
    lam = np.linalg.eigvals(_jacobian_1d(wl, osys))
    return float(lam.real.max()), float(np.abs(lam).max())


# Rounding of the central differences (~1e-9 in the Jacobian's entries) moves eigenvalues of
# this non-normal matrix by far less than this; the planted mistakes move them by O(1).
def _tol(rho):
    return 1e-7 * rho


EULER_FLOWS = [dict(mach=0.5), dict(mach=-0.5), dict(mach=0.5, angle=0.6), dict(mach=1.3), dict(mach=0.0)]


@pytest.mark.parametrize("flow", EULER_FLOWS, ids=["M0.5", "M-0.5", "oblique", "supersonic", "at_rest"])
def test_interface_sat_spectrum_is_stable_euler(flow):
    re_max, rho = _max_real(_pair(**flow))
    assert re_max <= _tol(rho), (flow, re_max, rho)


@pytest.mark.parametrize("flow", [dict(mach=0.5, mu=0.01), dict(mach=0.2, mu=0.05), dict(mach=0.5, mu=0.002)])
def test_interface_sat_spectrum_is_stable_navier_stokes(flow):
    re_max, rho = _max_real(_pair(physics="ns", **flow))
    assert re_max <= _tol(rho), (flow, re_max, rho)


@pytest.mark.parametrize("flow", EULER_FLOWS[:4], ids=["M0.5", "M-0.5", "oblique", "supersonic"])
def test_planted_penalty_mistakes_grow(flow):
    wl = _pair(**flow)
    flipped, rho = _max_real(wl, sig_int=-0.5)
    assert flipped > 0.1 * rho, flipped
    dropped_p0, _ = _max_real(wl, sig_int=0.5 * P0)
    assert dropped_p0 > 1.0, dropped_p0


def test_planted_viscous_jump_sign_grows(tmp_path):
    root = planted_oracle(tmp_path, "orc2d.c", "sat[v] += 0.5 * side * (own[v] - hat[v])",
                          "sat[v] -= 0.5 * side * (own[v] - hat[v])")
    out = run_with_oracle(root, "import test_oracle_interface_spectrum as T\n"
                                "print(T._max_real(T._pair(physics='ns', mach=0.2, mu=0.05))[0])\n")
    assert float(out) > 1.0
