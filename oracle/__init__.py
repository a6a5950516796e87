"""Plain, slow FP64 CPU oracle for the SBP-SAT overset RHS with MRAB time stepping.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / ``--impl reference`` legs use it to check and
time the GPU library. The GPU library never imports it and shares no code
with it; the two meet only through the seeded inputs of ``workloads``.

The C part (``orc2d.c``, ``orc3d.c``, ``orc_sbp.h``) holds the per-point
arithmetic; ``system.py`` (2D) and ``system3d.py`` (3D Cartesian) hold the
assembly (hole cut, receivers, donors), the Adams-Bashforth coefficient solve
and the time integrators, each citing the passage it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, "orc2d.c"), os.path.join(_HERE, "orc3d.c")]
_DEPS = _SRC + [os.path.join(_HERE, "orc_sbp.h")]
_SO = os.path.join(_HERE, "_build", "liborc.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle's C part with gcc (no FMA contraction, so x86 and Arm agree)."""
    newest = max(os.path.getmtime(s) for s in _DEPS)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= newest:
        return _SO
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    tmp = _SO + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
                           *_SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _SO)
    return _SO


def lib():
    """Load (building first if needed) the oracle's C library."""
    global _lib
    if _lib is not None:
        return _lib
    build()
    L = ctypes.CDLL(_SO)
    P = ctypes.c_void_p
    I = ctypes.c_int
    D = ctypes.c_double
    Lg = ctypes.c_long
    L.orc_set_threads.argtypes = [I]
    L.orc_set_threads.restype = I
    L.orc_classes2d.argtypes = [I, I, I, I, P, P, P]
    L.orc_classes2d.restype = I
    L.orc_metrics2d.argtypes = [I, I, P, P, P, P, P, P]
    L.orc_metrics2d.restype = I
    L.orc_viscflux2d.argtypes = [I, I, I, I, P, P, P, P, D, D, D, P]
    L.orc_viscflux2d.restype = I
    L.orc_penalty_matrix2d.argtypes = [P, D, D, D, I, P]
    L.orc_penalty_matrix2d.restype = None
    L.orc_rhs2d.argtypes = [I, I, I, I, P, P, P, P, I, D, D, D,
                            I, P, P, P, P, P, P, I, P, P, P, D, D, D, P]
    L.orc_rhs2d.restype = I
    L.orc_interp2d.argtypes = [I, I, I, P, I, P, P, P]
    L.orc_interp2d.restype = I
    L.orc_donors2d.argtypes = [I, I, I, I, P, P, P, P, I, P, P, P, P, P]
    L.orc_donors2d.restype = I
    L.orc_holecut2d.argtypes = [Lg, P, P, I, P, P, D, P]
    L.orc_holecut2d.restype = I
    L.orc_dt2d.argtypes = [I, I, P, P, P, D, D, D]
    L.orc_dt2d.restype = D
    L.orc_apply_d1.argtypes = [I, P, P, P]
    L.orc_apply_d1.restype = I
    L.orc_classes3d.argtypes = [I, I, I, I, I, I, P, P, P, P]
    L.orc_classes3d.restype = I
    L.orc_viscflux3d.argtypes = [I, I, I, P, P, P, D, D, D, P, D, D, D, P]
    L.orc_viscflux3d.restype = I
    L.orc_penalty_matrix3d.argtypes = [P, D, D, D, D, I, P]
    L.orc_penalty_matrix3d.restype = None
    L.orc_rhs3d.argtypes = [I, I, I, P, P, P, D, D, D, P, I, D, D, D,
                            I, P, P, P, P, P, P, I, P, P, P, D, D, P]
    L.orc_rhs3d.restype = I
    L.orc_interp3d.argtypes = [I, I, I, I, P, I, P, P, P]
    L.orc_interp3d.restype = I
    L.orc_dt3d.argtypes = [I, I, I, P, D, D, D, P, D, D, D]
    L.orc_dt3d.restype = D
    _lib = L
    return L


from .system import (OracleSystem, ab_coefficients, mrab_macro_step, mrab_macro_step_multirate,  # noqa: E402
                     mrab_macro_step_slowest_first,
                     mrab_macro_step_var, rk3_heun_step, rk4_step, srab_step, l2_norm)
from .system3d import OracleSystem3D  # noqa: E402

__all__ = ["build", "lib", "OracleSystem", "OracleSystem3D", "ab_coefficients", "mrab_macro_step",
           "mrab_macro_step_multirate",
           "mrab_macro_step_slowest_first", "mrab_macro_step_var", "rk3_heun_step", "rk4_step", "srab_step",
           "l2_norm"]
