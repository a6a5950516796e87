"""Pins of the oracle's operation counter (oracle.flops: orc2d.c compiled with a counting double,
the FLOP numerator of the benchmark's FP64 roofline):

* the counting build computes the plain oracle's right-hand sides bit for bit (so it runs the
  same operations), Euler and Navier-Stokes, with receivers, SAT terms and holes;
* on a periodic Cartesian mesh without SAT terms every point runs the same operations: the count
  is a + b N on meshes of N points of different sizes and for different states (the viscous
  branches count alike), a the few operations per call."""
import ctypes

import numpy as np
import pytest

import workloads as W
from oracle import OracleSystem
from oracle.flops import _load, count_rhs_flops


@pytest.mark.parametrize("make", [lambda: W.vortex_box_in_box(seed=2, n_bg=32, n_fine=21),
                                  lambda: W.cylinder_small(seed=2)], ids=["euler", "navier_stokes"])
def test_counting_build_computes_the_oracle(make):
    wl = make()
    o = OracleSystem(wl)
    for k in range(2):
        c = count_rhs_flops(o, k, wl["q0"][k], wl["q0"][1 - k])
        assert np.array_equal(c["rhs_out"], o.coupled_rhs(k, wl["q0"][k], wl["q0"][1 - k]))
        assert c["rhs"] > 50 * c["points"]


def _periodic_count(ni, nj, viscous, seed):
    L = _load()
    rng = np.random.default_rng(seed)
    ci = np.zeros((nj, ni), np.int8)
    cj = np.zeros((nj, ni), np.int8)
    h = 0.1
    met = np.zeros((5, nj, ni))
    met[0] = h     # xi_x / J = y_eta
    met[3] = h     # eta_y / J = x_xi
    met[4] = 1.0 / (h * h)
    rho = 1.0 + 0.1 * rng.random((nj, ni))
    u, v = 0.3 * rng.standard_normal((2, nj, ni))
    p = 1.0 / 1.4 + 0.05 * rng.random((nj, ni))
    q = np.ascontiguousarray(np.stack([rho, rho * u, rho * v, p / 0.4 + 0.5 * rho * (u * u + v * v)]))
    out = np.zeros((4, nj, ni))
    qinf = np.array([1.0, 0.2, 0.0, 1.0 / (1.4 * 0.4) + 0.02])
    P = lambda a: ctypes.c_void_p(a.ctypes.data)
    e = np.zeros(1, np.int64)
    ei = np.zeros(1, np.int32)
    ed = np.zeros(1)
    L.orc_flops_read(1)
    rc = L.orc_rhs2d(ni, nj, 1, 1, P(ci), P(cj), P(met), P(q), int(viscous), 1.4, 0.01 if viscous else 0.0, 0.72,
                     0, P(e), P(ei), P(ei), P(ei), P(ei), P(ed), 0, P(ed), None, P(qinf), 1.0, 0.5, 1.0, P(out))
    assert rc == 0
    return L.orc_flops_read(1)


@pytest.mark.parametrize("viscous", [False, True])
def test_count_is_the_same_at_every_point(viscous):
    """count = a + b N: b operations per point and a few per call (the viscous coefficients)."""
    n1 = _periodic_count(16, 12, viscous, 1)
    n2 = _periodic_count(24, 20, viscous, 2)
    assert (n2 - n1) % (24 * 20 - 16 * 12) == 0
    b = (n2 - n1) // (24 * 20 - 16 * 12)
    a = n1 - b * 16 * 12
    assert b > 100 and 0 <= a < 16, (a, b)
    assert _periodic_count(16, 12, viscous, 3) == n1
    assert _periodic_count(30, 8, viscous, 4) == a + b * 240
