"""Algorithmic floating-point operation counts of the oracle's right-hand side (TEST
INFRASTRUCTURE ONLY: the FLOP numerator of the benchmark's FP64 roofline; the GPU library never
uses it).

``flopcount.cpp`` compiles ``orc2d.c`` with a counting double (one count per +, -, *, / and
square root). ``count_rhs_flops`` runs one coupled right-hand side of an ``OracleSystem`` mesh
through that build with the arguments ``OracleSystem.coupled_rhs`` passes to the plain one: the
receivers' interpolation of the donor state (and, for Navier-Stokes, of the donor viscous
fluxes, counted at the distinct donor points only: the GPU path evaluates them there, the oracle
on the whole donor mesh) and the mesh's own right-hand side (fluxes, viscous gradients,
derivatives, SAT terms).

Run as a script, it prints the counts per active point for the benchmark's cylinder workload.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liborc_count.so")
_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    deps = [os.path.join(_HERE, f) for f in ("flopcount.cpp", "orc2d.c", "orc_sbp.h")]
    if not os.path.exists(_SO) or os.path.getmtime(_SO) < max(os.path.getmtime(d) for d in deps):
        os.makedirs(os.path.dirname(_SO), exist_ok=True)
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["g++", "-O1", "-std=c++17", "-fPIC", "-shared", "-w", "-ffp-contract=off",
                               "-I", _HERE, os.path.join(_HERE, "flopcount.cpp"), "-o", tmp])
        os.replace(tmp, _SO)
    L = ctypes.CDLL(_SO)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    L.orc_rhs2d.argtypes = [I, I, I, I, P, P, P, P, I, D, D, D,
                            I, P, P, P, P, P, P, I, P, P, P, D, D, D, P]
    L.orc_rhs2d.restype = I
    L.orc_interp2d.argtypes = [I, I, I, P, I, P, P, P]
    L.orc_interp2d.restype = I
    L.orc_viscflux2d.argtypes = [I, I, I, I, P, P, P, P, D, D, D, P]
    L.orc_viscflux2d.restype = I
    L.orc_flops_read.argtypes = [I]
    L.orc_flops_read.restype = ctypes.c_ulonglong
    _lib = L
    return L


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def count_rhs_flops(osys, k, q_self, q_other):
    """FLOPs of one coupled right-hand side of mesh k: {'rhs', 'interp', 'donor_viscous',
    'total', 'points'} with points = the mesh's active points."""
    L = _load()
    m, dm = osys.meshes[k], osys.meshes[1 - k]
    ni, nj = m["n"]
    dni, dnj = dm["n"]
    q_self = np.ascontiguousarray(q_self, dtype=np.float64)
    q_other = np.ascontiguousarray(q_other, dtype=np.float64)
    nr = osys.recv_pts[k].size
    qhat = np.zeros((4, max(nr, 1)))
    fvhat = None
    L.orc_flops_read(1)
    if nr:
        L.orc_interp2d(dni, dnj, 4, _p(q_other), nr, _p(osys.base[k]), _p(osys.w[k]), _p(qhat))
    interp = L.orc_flops_read(1)
    donor_visc = 0.0
    if osys.viscous:
        fv = np.zeros((6, dnj, dni))
        L.orc_viscflux2d(dni, dnj, int(dm["periodic"][0]), int(dm["periodic"][1]), _p(osys.ci[1 - k]),
                         _p(osys.cj[1 - k]), _p(osys.met[1 - k]), _p(q_other), osys.gamma, osys.mu, osys.pr, _p(fv))
        whole = L.orc_flops_read(1)
        # the whole donor mesh's count scaled to its distinct donor points
        dpts = {((i0 + a) % dni, (j0 + b) % dnj) for i0, j0 in osys.base[k] for a in range(4) for b in range(4)}
        donor_visc = whole * len(dpts) / int((osys.iblank[1 - k] != 0).sum())
        fvhat = np.zeros((6, max(nr, 1)))
        if nr:
            L.orc_interp2d(dni, dnj, 6, _p(fv), nr, _p(osys.base[k]), _p(osys.w[k]), _p(fvhat))
        interp += L.orc_flops_read(1)
    t = osys.terms[k]
    out = np.zeros((4, nj, ni))
    qinf = np.ascontiguousarray(osys.p["qinf"], dtype=np.float64)
    rc = L.orc_rhs2d(ni, nj, int(m["periodic"][0]), int(m["periodic"][1]), _p(osys.ci[k]), _p(osys.cj[k]),
                     _p(osys.met[k]), _p(q_self), int(osys.viscous), osys.gamma, osys.mu, osys.pr,
                     t["pt"].size, _p(t["pt"]), _p(t["dir"]), _p(t["side"]), _p(t["kind"]), _p(t["recv"]),
                     _p(t["scale"]), nr, _p(qhat), _p(fvhat), _p(qinf), float(osys.p["twall"]), osys.sig_int, osys.sig_phys, _p(out))
    if rc != 0:
        raise RuntimeError("counting rhs failed: %d" % rc)
    rhs = L.orc_flops_read(1)
    pts = int((osys.iblank[k] != 0).sum())
    return {"rhs": int(rhs), "interp": int(interp), "donor_viscous": float(donor_visc),
            "total": rhs + interp + donor_visc, "points": pts, "rhs_out": out}


if __name__ == "__main__":
    import sys
    sys.path.insert(0, os.path.dirname(_HERE))
    import workloads as W
    from oracle import OracleSystem

    wl = W.cylinder_overset(seed=0)
    osys = OracleSystem(wl)
    m = int(wl["params"]["hist_len"])
    for k, name in enumerate(("background", "ogrid")):
        c = count_rhs_flops(osys, k, wl["q0"][k], wl["q0"][1 - k])
        ref = osys.coupled_rhs(k, wl["q0"][k], wl["q0"][1 - k])
        assert np.array_equal(c["rhs_out"], ref), "the counting build must compute the same values"
        per = c["total"] / c["points"]
        print("%s: points %d, rhs %.1f, interp %.2f, donor viscous %.2f FLOP/pt; right-hand side %.1f, "
              "+ MRAB update (2 m nvar = %d) %.1f FLOP/pt"
              % (name, c["points"], c["rhs"] / c["points"], c["interp"] / c["points"],
                 c["donor_viscous"] / c["points"], per, 8 * m, per + 8 * m))
