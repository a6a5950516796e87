"""GB300 (sm_103a) library for multi-rate Adams-Bashforth integration of the SBP-SAT
compressible Euler / Navier-Stokes equations on overset meshes (arXiv 1805.06607).

This module is a thin ctypes binding of the C ABI declared in ``include/sbp_mrab.h``:
it marshals arguments and owns device buffers through PyTorch; every step of the
method runs in the library's CUDA kernels. There is no CPU fallback: importing the
module fails when the compiled library is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# SBP_MRAB_LIBRARY may name another build of the library (e.g. the bounds-checked one of
# build.build(bounds_check=True)); the default is the in-tree build
LIB_PATH = os.environ.get("SBP_MRAB_LIBRARY") or os.path.join(_HERE, "_build", "libsbpmrab.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libsbpmrab.so is not built: run paper_1805_06607_gb300.build.build() "
                      "(or __graft_entry__.build()) first")

_lib = ctypes.CDLL(LIB_PATH)

BC = {"periodic": 0, "interface": 1, "farfield": 2, "wall": 3}
PHYSICS = {"euler": 0, "ns": 1}
DTYPE = {"f64": 0, "f32": 1}


class MeshDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 2), ("periodic", ctypes.c_int * 2), ("bc", ctypes.c_int * 4),
                ("cartesian", ctypes.c_int), ("lo", ctypes.c_double * 2), ("h", ctypes.c_double * 2),
                ("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("shift", ctypes.c_double * 4)]


class Params(ctypes.Structure):
    _fields_ = [("physics", ctypes.c_int), ("dtype", ctypes.c_int), ("gamma", ctypes.c_double),
                ("mu", ctypes.c_double), ("pr", ctypes.c_double), ("twall", ctypes.c_double),
                ("omega_corner", ctypes.c_double), ("sigma_interface", ctypes.c_double),
                ("sigma_physical", ctypes.c_double), ("cfl", ctypes.c_double), ("qinf", ctypes.c_double * 4),
                ("order", ctypes.c_int), ("hist_len", ctypes.c_int), ("step_ratio", ctypes.c_int),
                ("fast_mesh", ctypes.c_int), ("hole_cells", ctypes.c_double), ("scheme", ctypes.c_int),
                ("sponge_cells", ctypes.c_int), ("sponge_strength", ctypes.c_double)]

# MRAB orderings of Sec. 3.3 (sbp_mrab_scheme)
SCHEMES = {"fastest_first": 0, "slowest_first": 1, "slowest_first_reextrapolate": 2}


class MeshInfo(ctypes.Structure):
    _fields_ = [("ni", ctypes.c_int), ("nj", ctypes.c_int), ("pitch", ctypes.c_int),
                ("field_elems", ctypes.c_size_t), ("state_bytes", ctypes.c_size_t),
                ("hist_bytes", ctypes.c_size_t), ("nvar", ctypes.c_int), ("n_holes", ctypes.c_int),
                ("n_receivers", ctypes.c_int), ("n_sat_points", ctypes.c_int), ("elem_size", ctypes.c_int),
                ("strip_width", ctypes.c_int), ("rows_per_cta", ctypes.c_int), ("single_pass", ctypes.c_int),
                ("rows_update", ctypes.c_int), ("eval_strip_width", ctypes.c_int),
                ("eval_rows_per_cta", ctypes.c_int), ("eval_single_pass", ctypes.c_int),
                ("eval_rows_update", ctypes.c_int)]


class Mesh3Desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("periodic", ctypes.c_int * 3), ("bc", ctypes.c_int * 6),
                ("lo", ctypes.c_double * 3), ("h", ctypes.c_double * 3)]


class Mesh3Info(ctypes.Structure):
    _fields_ = [("ni", ctypes.c_int), ("nj", ctypes.c_int), ("nk", ctypes.c_int), ("pitch", ctypes.c_int),
                ("field_elems", ctypes.c_size_t), ("state_bytes", ctypes.c_size_t), ("nvar", ctypes.c_int),
                ("n_holes", ctypes.c_int), ("n_receivers", ctypes.c_int), ("n_sat_points", ctypes.c_int),
                ("elem_size", ctypes.c_int)]


class Mesh3cDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("z", ctypes.c_void_p)]


class AdjointDesc(ctypes.Structure):
    _fields_ = [("n_steps", ctypes.c_int), ("n_snapshots", ctypes.c_int), ("n_probes", ctypes.c_int),
                ("probe_xy", ctypes.c_void_p), ("H", ctypes.c_double)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_SIGS = {
    "sbp_system_create": [ctypes.POINTER(MeshDesc), _I, ctypes.POINTER(Params), ctypes.POINTER(_P)],
    "sbp_system_destroy": [_P],
    "sbp_mesh_info_get": [_P, _I, ctypes.POINTER(MeshInfo)],
    "sbp_get_tables": [_P, _I, _P, _P, _P, _P, _P],
    "sbp_overset_interp": [_P, _I, _P, _P, _P, _P],
    "sbp_rhs_eval": [_P, _I, _P, _P, _P, _P],
    "sbp_rhs_eval_noalloc": [_P, _I, _P, _P, _P, _P],
    "sbp_timestep": [_P, _P, _P, _P, _P, _P],
    "sbp_bind": [_P, _I, _P, _P, _P],
    "sbp_current_state": [_P, _I, ctypes.POINTER(_P)],
    "sbp_mrab_init": [_P, _D, _P],
    "sbp_mrab_step": [_P, _I, _P],
    "sbp_mrab_time": [_P, ctypes.POINTER(_D), ctypes.POINTER(_D)],
    "sbp_rk4_step": [_P, _I, _D, _P],
    "sbp_mrab_set_step": [_P, _D],
    "sbp_check": [_P, _P],
    "sbp_profile_enable": [_P, _I],
    "sbp_use_graphs": [_P, _I],
    "sbp_graph_launches": [_P, _P],
    "sbp_autotune": [_P, _I, _P],
    "sbp_profile_read": [_P, _P, _P, _I],
    "sbp_set_rhs_shape": [_P, _I, _I, _I],
    "sbp_integrator_state": [_P, _I, _P, _P, _I, _P],
    "sbp_checkpoint_save": [_P, _P, ctypes.POINTER(ctypes.c_size_t), _P],
    "sbp_checkpoint_load": [_P, _P, ctypes.c_size_t, _P],
}
_SIGS.update({
    "sbp_batch_create": [ctypes.POINTER(_P), _I, _I, _P, ctypes.POINTER(_P)],
    "sbp_batch_destroy": [_P],
    "sbp_batch_step": [_P, _I, _P],
    "sbp_batch_info": [_P, _P, _P, _P, _P],
    "sbp_batch_set_shape": [_P, _I],
    "sbp_batch_check": [_P, _P],
})
_SIGS.update({
    "sbp_set_freestream": [_P, _P],
    "sbp_rhs_eval_vjp": [_P, _I, _P, _P, _P, _P, _P, _P, _P],
    "sbp_rhs_eval_jvp": [_P, _I, _P, _P, _P, _P, _P, _P, _P],
    "sbp_overset_interp_vjp": [_P, _I, _P, _P, _P, _P, _P],
    "sbp_adjoint_probe": [_P, ctypes.POINTER(AdjointDesc), _P, _P, _P, _P, _P, _P, _P, _P, _P],
})
_SIGS.update({
    "sbp3_system_create": [ctypes.POINTER(Mesh3Desc), _I, ctypes.POINTER(Params), ctypes.POINTER(_P)],
    "sbp3_system_destroy": [_P],
    "sbp3_mesh_info_get": [_P, _I, ctypes.POINTER(Mesh3Info)],
    "sbp3_set_freestream": [_P, _P],
    "sbp3_get_tables": [_P, _I, _P, _P, _P, _P],
    "sbp3_overset_interp": [_P, _I, _P, _P, _P, _P],
    "sbp3_rhs_eval": [_P, _I, _P, _P, _P, _P],
    "sbp3_timestep": [_P, _P, _P, _P, _P, _P],
    "sbp3_bind": [_P, _I, _P, _P, _P],
    "sbp3_current_state": [_P, _I, ctypes.POINTER(_P)],
    "sbp3_mrab_init": [_P, _D, _P],
    "sbp3_mrab_step": [_P, _I, _P],
    "sbp3_check": [_P, _P],
    "sbp3_set_rhs_kernel": [_P, _I, _I],
    "sbp_f32_to_f64": [_P, _P, ctypes.c_size_t, _P],
    "sbp_fp64_rate_probe": [_P, _I, _I, ctypes.c_long, ctypes.POINTER(_D), _P],
    "sbp_barrier_selftest": [_I, _I, ctypes.c_uint, ctypes.POINTER(_I), ctypes.POINTER(_I), _P],
    "sbp_chain_create": [ctypes.POINTER(MeshDesc), _I, _P, ctypes.POINTER(Params), ctypes.POINTER(_P)],
    "sbp_chain_destroy": [_P],
    "sbp_chain_mesh_info": [_P, _I, ctypes.POINTER(MeshInfo)],
    "sbp_chain_tables": [_P, _I, _P, _P, _P, _P, _P],
    "sbp_chain_rhs_eval": [_P, _I, _P, _P, _P],
    "sbp_chain_timestep": [_P, _P, _P, _P, _P],
    "sbp_chain_bind": [_P, _I, _P, _P, _P],
    "sbp_chain_current_state": [_P, _I, ctypes.POINTER(_P)],
    "sbp_chain_mrab_init": [_P, _D, _P],
    "sbp_chain_mrab_step": [_P, _I, _P],
    "sbp_chain_mrab_time": [_P, ctypes.POINTER(_D), ctypes.POINTER(_D)],
    "sbp_chain_check": [_P, _P],
    "sbp_host_tables_create": [ctypes.POINTER(MeshDesc), _I, ctypes.POINTER(Params), ctypes.POINTER(_P)],
    "sbp_host_tables_destroy": [_P],
    "sbp_host_tables_get": [_P, _I, _P, _P, _P, _P, _P],
    "sbp_host_tables_plan": [_P, _P, _P, _P, _P],
    "sbp3_host_tables_create": [ctypes.POINTER(Mesh3Desc), _I, ctypes.POINTER(Params), ctypes.POINTER(_P)],
    "sbp3_host_tables_destroy": [_P],
    "sbp3_host_tables_get": [_P, _I, _P, _P, _P, _P, _P],
    "sbp3c_mesh_create": [_P, _P, _P, _P, ctypes.POINTER(Params), ctypes.POINTER(_P)],
    "sbp3c_mesh_destroy": [_P],
    "sbp3c_get_metrics": [_P, _P],
    "sbp3c_rhs_eval": [_P, _P, _P, _P],
    "sbp3c_set_farfield": [_P, _P, ctypes.c_double],
    "sbp3c_donor_search": [_P, _P, _P, _P, _P, _I, _P, _P, _P, _P, _P],
    "sbp3c_interp": [_P, _P, _I, _P, _P, _P, _P],
    "sbp3c_hole_cut": [_P, _P, _P, _P, _I, _P, ctypes.c_double, _P],
    "sbp3c_set_interface": [_P, _I, _P, _P, _I, ctypes.c_double],
    "sbp3c_interface_sat": [_P, _P, _P, _P, _P, _P],
    "sbp3c_mesh_check": [_P, _P],
    "sbp3c_system_create": [ctypes.POINTER(Mesh3cDesc), _I, ctypes.POINTER(Params), ctypes.POINTER(_P)],
    "sbp3c_system_destroy": [_P],
    "sbp3c_system_info": [_P, _I, ctypes.POINTER(Mesh3Info)],
    "sbp3c_system_set_freestream": [_P, _P],
    "sbp3c_system_tables": [_P, _I, _P, _P, _P, _P],
    "sbp3c_host_tables_create": [ctypes.POINTER(Mesh3cDesc), _I, ctypes.POINTER(Params), ctypes.POINTER(_P)],
    "sbp3c_host_tables_destroy": [_P],
    "sbp3c_host_tables_get": [_P, _I, _P, _P, _P, _P, _P],
    "sbp3c_system_interp": [_P, _I, _P, _P, _P, _P],
    "sbp3c_system_rhs_eval": [_P, _I, _P, _P, _P, _P],
    "sbp3c_system_timestep": [_P, _P, _P, _P, _P, _P],
    "sbp3c_system_bind": [_P, _I, _P, _P, _P],
    "sbp3c_system_current_state": [_P, _I, ctypes.POINTER(_P)],
    "sbp3c_system_mrab_init": [_P, _D, _P],
    "sbp3c_system_mrab_step": [_P, _I, _P],
    "sbp3c_system_mrab_time": [_P, ctypes.POINTER(_D), ctypes.POINTER(_D)],
    "sbp3c_system_check": [_P, _P],
})
for _name, _args in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = ctypes.c_int
_lib.sbp_status_string.argtypes = [ctypes.c_int]
_lib.sbp_status_string.restype = ctypes.c_char_p
_lib.sbp_last_error_message.argtypes = []
_lib.sbp_last_error_message.restype = ctypes.c_char_p


# Flag in the marching kernel's chunk rows (set_rhs_shape): TMA tensor-copy staging.
STAGE_TMA = 0x10000


class SbpError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = _lib.sbp_status_string(status).decode()
        detail = _lib.sbp_last_error_message().decode()
        super().__init__("%s: %s (%d) %s" % (where, msg, status, detail))


def _check(status, where):
    if status != 0:
        raise SbpError(status, where)


def lib():
    return _lib


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _descriptors(wl, dtype, sigma_interface, sigma_physical, hole_cells):
    """C descriptors (sbp_mesh_desc[n], sbp_params) of a workload dict, and the arrays they point
    into (to be kept alive by the caller)."""
    p = wl["params"]
    descs = (MeshDesc * len(wl["meshes"]))()
    keep = []
    for k, m in enumerate(wl["meshes"]):
        d = descs[k]
        d.n[0], d.n[1] = m["n"]
        d.periodic[0], d.periodic[1] = int(m["periodic"][0]), int(m["periodic"][1])
        for f in range(4):
            d.bc[f] = BC[m["bc"][f]]
        d.cartesian = int(m["cartesian"])
        d.lo[0], d.lo[1] = m["lo"]
        d.h[0], d.h[1] = m["h"]
        x = np.ascontiguousarray(m["x"], dtype=np.float64)
        y = np.ascontiguousarray(m["y"], dtype=np.float64)
        keep += [x, y]
        d.x = x.ctypes.data
        d.y = y.ctypes.data
        sh = m["shift"]
        d.shift[0], d.shift[1], d.shift[2], d.shift[3] = sh[0][0], sh[0][1], sh[1][0], sh[1][1]
    pr = Params()
    pr.physics = PHYSICS[p["physics"]]
    pr.dtype = DTYPE[dtype]
    pr.gamma = p["gamma"]
    pr.mu = p["mu"]
    pr.pr = p["pr"]
    pr.twall = p["twall"]
    pr.omega_corner = p["omega_corner"]
    pr.sigma_interface = sigma_interface
    pr.sigma_physical = sigma_physical
    pr.cfl = p["cfl"]
    for v in range(4):
        pr.qinf[v] = float(p["qinf"][v])
    pr.order = p["order"]
    pr.hist_len = p["hist_len"]
    pr.step_ratio = p["step_ratio"]
    pr.fast_mesh = p["fast_mesh"]
    pr.hole_cells = hole_cells
    pr.scheme = SCHEMES[p.get("scheme", "fastest_first")]
    pr.sponge_cells = int(p.get("sponge_cells", 0))
    pr.sponge_strength = float(p.get("sponge_strength", 1.0))
    return descs, pr, keep


class HostTables:
    """The host part of system creation alone (sbp_host_tables_*): setup tables and the MRAB
    coefficient plan, without touching a GPU."""

    def __init__(self, wl, hole_cells=4):
        descs, pr, self._keep = _descriptors(wl, "f64", 0.5, 1.0, hole_cells)
        h = ctypes.c_void_p()
        _check(_lib.sbp_host_tables_create(descs, 2, ctypes.byref(pr), ctypes.byref(h)), "sbp_host_tables_create")
        self.h = h
        self.meshes = wl["meshes"]

    def tables(self, k):
        ni, nj = self.meshes[k]["n"]
        nr = ctypes.c_int()
        _check(_lib.sbp_host_tables_get(self.h, k, None, None, None, None, ctypes.byref(nr)), "sbp_host_tables_get")
        nr = nr.value
        ib = np.zeros(ni * nj, np.int8)
        rec = np.zeros(max(nr, 1), np.int32)
        base = np.zeros(max(2 * nr, 1), np.int32)
        w = np.zeros(max(8 * nr, 1))
        _check(_lib.sbp_host_tables_get(self.h, k, ib.ctypes.data, rec.ctypes.data, base.ctypes.data, w.ctypes.data,
                                        None), "sbp_host_tables_get")
        return {"iblank": ib.reshape(nj, ni), "receivers": rec[:nr], "base": base[:2 * nr].reshape(nr, 2),
                "w": w[:8 * nr].reshape(nr, 8)}

    def plan(self):
        m, sr = ctypes.c_int(), ctypes.c_int()
        _check(_lib.sbp_host_tables_plan(self.h, None, None, ctypes.byref(m), ctypes.byref(sr)), "sbp_host_tables_plan")
        ab = np.zeros(m.value)
        ext = np.zeros((sr.value, m.value))
        _check(_lib.sbp_host_tables_plan(self.h, ab.ctypes.data, ext.ctypes.data, None, None), "sbp_host_tables_plan")
        return ab, ext

    def close(self):
        if getattr(self, "h", None):
            _lib.sbp_host_tables_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class System:
    """A two-mesh overset system on the current CUDA device.

    ``wl`` is a workload dict (``workloads`` layout: meshes, params). States are exchanged
    as numpy arrays (nvar, nj, ni) or as device tensors in the library's pitched layout.
    """

    def __init__(self, wl, dtype="f64", sigma_interface=0.5, sigma_physical=1.0, hole_cells=4):
        import torch
        self.torch = torch
        self.dtype = dtype
        self.tdtype = torch.float64 if dtype == "f64" else torch.float32
        self.meshes = wl["meshes"]
        p = wl["params"]
        descs, pr, self._keep = _descriptors(wl, dtype, sigma_interface, sigma_physical, hole_cells)
        self.params = p
        h = ctypes.c_void_p()
        torch.cuda.init()
        _check(_lib.sbp_system_create(descs, 2, ctypes.byref(pr), ctypes.byref(h)), "sbp_system_create")
        self.h = h
        self.info = []
        for k in range(2):
            inf = MeshInfo()
            _check(_lib.sbp_mesh_info_get(self.h, k, ctypes.byref(inf)), "sbp_mesh_info_get")
            self.info.append(inf)
        self.bound = None


    def close(self):
        if getattr(self, "h", None):
            _lib.sbp_system_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- layout helpers ------------------------------------------------------------------------
    def empty_state(self, k, n=1):
        inf = self.info[k]
        t = self.torch.zeros((n, 4, inf.nj, inf.pitch), dtype=self.tdtype, device="cuda")
        return t if n > 1 else t[0]

    def to_device(self, k, q):
        inf = self.info[k]
        t = self.empty_state(k)
        t[:, :, :inf.ni] = self.torch.from_numpy(np.ascontiguousarray(q)).to(self.tdtype).cuda()
        return t

    def to_host(self, k, t):
        inf = self.info[k]
        return t[..., :inf.ni].double().cpu().numpy()

    # -- calls ---------------------------------------------------------------------------------
    def tables(self, k):
        inf = self.info[k]
        n = inf.ni * inf.nj
        nr = inf.n_receivers
        ib = np.zeros(n, np.int8)
        met = np.zeros(5 * n)
        rec = np.zeros(max(nr, 1), np.int32)
        base = np.zeros(max(2 * nr, 1), np.int32)
        w = np.zeros(max(8 * nr, 1))
        _check(_lib.sbp_get_tables(self.h, k, ib.ctypes.data, met.ctypes.data, rec.ctypes.data, base.ctypes.data,
                                   w.ctypes.data), "sbp_get_tables")
        return {"iblank": ib.reshape(inf.nj, inf.ni), "metrics": met.reshape(5, inf.nj, inf.ni),
                "receivers": rec[:nr], "base": base[:2 * nr].reshape(nr, 2), "w": w[:8 * nr].reshape(nr, 8)}

    def overset_interp(self, recv, q_donor, viscous_fluxes=True, stream=None):
        nr = self.info[recv].n_receivers
        qhat = self.torch.zeros((4, max(nr, 1)), dtype=self.tdtype, device="cuda")
        fvhat = self.torch.zeros((6, max(nr, 1)), dtype=self.tdtype, device="cuda") if viscous_fluxes else None
        _check(_lib.sbp_overset_interp(self.h, recv, _ptr(q_donor), _ptr(qhat), _ptr(fvhat), _stream(stream)),
               "sbp_overset_interp")
        return qhat[:, :nr], (fvhat[:, :nr] if fvhat is not None else None)

    def rhs_eval(self, k, q_self, q_other, out=None, stream=None):
        if out is None:
            out = self.empty_state(k)
        _check(_lib.sbp_rhs_eval(self.h, k, _ptr(q_self), _ptr(q_other), _ptr(out), _stream(stream)), "sbp_rhs_eval")
        return out

    def timestep(self, q0, q1, stream=None):
        dt = (ctypes.c_double * 2)()
        H = ctypes.c_double()
        _check(_lib.sbp_timestep(self.h, _ptr(q0), _ptr(q1), ctypes.cast(dt, ctypes.c_void_p),
                                 ctypes.cast(ctypes.pointer(H), ctypes.c_void_p), _stream(stream)), "sbp_timestep")
        return [dt[0], dt[1]], H.value

    def bind(self, q_host):
        """Allocate and bind integrator buffers; load the initial states (numpy, per mesh)."""
        self.bound = []
        for k in range(2):
            qa = self.to_device(k, q_host[k])
            qb = self.empty_state(k)
            hist = self.empty_state(k, n=self.params["hist_len"]) if self.params["hist_len"] > 1 else \
                self.empty_state(k)[None]
            _check(_lib.sbp_bind(self.h, k, _ptr(qa), _ptr(qb), _ptr(hist)), "sbp_bind")
            self.bound.append((qa, qb, hist))

    def current_state(self, k):
        p = ctypes.c_void_p()
        _check(_lib.sbp_current_state(self.h, k, ctypes.byref(p)), "sbp_current_state")
        qa, qb, _ = self.bound[k]
        return qa if p.value == qa.data_ptr() else qb

    def mrab_init(self, H=0.0, stream=None):
        _check(_lib.sbp_mrab_init(self.h, float(H), _stream(stream)), "sbp_mrab_init")

    def mrab_step(self, n=1, stream=None):
        _check(_lib.sbp_mrab_step(self.h, int(n), _stream(stream)), "sbp_mrab_step")

    def mrab_set_step(self, H):
        """Macro step H for the following macro steps (weights solved on the history's node
        times until the histories are uniform in H again)."""
        _check(_lib.sbp_mrab_set_step(self.h, float(H)), "sbp_mrab_set_step")

    def rk4_step(self, n, h, stream=None):
        """n classical Runge-Kutta steps of size h on both meshes (single rate), in place on the
        bound states; the MRAB history must be rebuilt (mrab_init) before the next mrab_step."""
        _check(_lib.sbp_rk4_step(self.h, int(n), float(h), _stream(stream)), "sbp_rk4_step")

    def get_state(self, stream=None):
        """Integrator state per mesh: (state, history entries oldest first) device tensors."""
        out = []
        m = self.params["hist_len"]
        for k in range(2):
            q = self.empty_state(k)
            h = self.empty_state(k, n=max(m - 1, 1)) if m > 2 else self.empty_state(k)[None]
            _check(_lib.sbp_integrator_state(self.h, k, _ptr(q), _ptr(h), 0, _stream(stream)), "sbp_integrator_state")
            out.append((q, h[:m - 1]))
        return out

    def set_state(self, state, stream=None):
        for k in range(2):
            q, h = state[k]
            _check(_lib.sbp_integrator_state(self.h, k, _ptr(q.contiguous()), _ptr(h.contiguous()), 1,
                                             _stream(stream)), "sbp_integrator_state")

    def checkpoint_save(self, stream=None):
        """The whole integrator (states, history rings, node times, H, t) as bytes."""
        n = ctypes.c_size_t(0)
        _check(_lib.sbp_checkpoint_save(self.h, None, ctypes.byref(n), _stream(stream)), "sbp_checkpoint_save")
        buf = (ctypes.c_char * n.value)()
        _check(_lib.sbp_checkpoint_save(self.h, ctypes.addressof(buf), ctypes.byref(n), _stream(stream)),
               "sbp_checkpoint_save")
        return bytes(buf)

    def checkpoint_load(self, blob, stream=None):
        """Restore the integrator from checkpoint_save's bytes (buffers must be bound)."""
        buf = ctypes.create_string_buffer(bytes(blob), len(blob))
        _check(_lib.sbp_checkpoint_load(self.h, ctypes.addressof(buf), len(blob), _stream(stream)),
               "sbp_checkpoint_load")

    def mrab_time(self):
        H = ctypes.c_double()
        t = ctypes.c_double()
        _check(_lib.sbp_mrab_time(self.h, ctypes.byref(H), ctypes.byref(t)), "sbp_mrab_time")
        return H.value, t.value

    PHASES = ("interp_slow", "rhs_slow", "interp_fast", "rhs_fast")

    def mesh_info(self, k):
        inf = MeshInfo()
        _check(_lib.sbp_mesh_info_get(self.h, k, ctypes.byref(inf)), "sbp_mesh_info_get")
        return inf

    def autotune(self, on=True, stream=None):
        _check(_lib.sbp_autotune(self.h, int(bool(on)), _stream(stream)), "sbp_autotune")

    def set_rhs_shape(self, k, strip, rows, rows_update=0):
        """strip 0: kernel pair with `rows` rows per CTA of the flux kernel and `rows_update`
        (0: the same) of the derivative kernel; 58: marching kernel, chunks of `rows` (| STAGE_TMA:
        rows staged by TMA tensor copies); 116 / 244: column-marching kernel, chunks of `rows`."""
        code = int(rows) | (int(rows_update) << 8) if int(strip) == 0 else int(rows)
        _check(_lib.sbp_set_rhs_shape(self.h, k, int(strip), code), "sbp_set_rhs_shape")
        self.info[k] = self.mesh_info(k)

    def use_graphs(self, on=True):
        _check(_lib.sbp_use_graphs(self.h, int(bool(on))), "sbp_use_graphs")

    def graph_launches(self):
        """Kernel launches in the macro-step graph replayed last (0 before the first replay)."""
        n = ctypes.c_int(0)
        _check(_lib.sbp_graph_launches(self.h, ctypes.byref(n)), "sbp_graph_launches")
        return n.value

    def profile_enable(self, on=True):
        _check(_lib.sbp_profile_enable(self.h, int(bool(on))), "sbp_profile_enable")

    def profile_read(self, reset=True):
        """Per-phase device milliseconds and launch counts recorded by sbp_mrab_step."""
        ms = (ctypes.c_double * 4)()
        n = (ctypes.c_int * 4)()
        _check(_lib.sbp_profile_read(self.h, ctypes.cast(ms, ctypes.c_void_p), ctypes.cast(n, ctypes.c_void_p),
                                     int(reset)), "sbp_profile_read")
        return {p: (ms[i], n[i]) for i, p in enumerate(self.PHASES)}

    def check(self, stream=None):
        _check(_lib.sbp_check(self.h, _stream(stream)), "sbp_check")

    # -- discrete adjoint (FP64 systems) -------------------------------------------------------
    def set_freestream(self, qinf):
        arr = (ctypes.c_double * 4)(*[float(v) for v in qinf])
        _check(_lib.sbp_set_freestream(self.h, ctypes.cast(arr, ctypes.c_void_p)), "sbp_set_freestream")

    def rhs_eval_vjp(self, k, q_self, q_other, lam, stream=None):
        """((dR_k/dq_self)^T lam, (dR_k/dq_other)^T lam, (dR_k/dqinf)^T lam as numpy[4])."""
        lq_s = self.empty_state(k)
        lq_o = self.empty_state(1 - k)
        lqinf = (ctypes.c_double * 4)()
        _check(_lib.sbp_rhs_eval_vjp(self.h, k, _ptr(q_self), _ptr(q_other), _ptr(lam), _ptr(lq_s), _ptr(lq_o),
                                     ctypes.cast(lqinf, ctypes.c_void_p), _stream(stream)), "sbp_rhs_eval_vjp")
        return lq_s, lq_o, np.array(lqinf[:])

    def rhs_eval_jvp(self, k, q_self, q_other, dq_self, dq_other, dqinf=None, stream=None):
        out = self.empty_state(k)
        arr = (ctypes.c_double * 4)(*[float(v) for v in dqinf]) if dqinf is not None else None
        _check(_lib.sbp_rhs_eval_jvp(self.h, k, _ptr(q_self), _ptr(q_other), _ptr(dq_self), _ptr(dq_other),
                                     ctypes.cast(arr, ctypes.c_void_p) if arr is not None else None, _ptr(out),
                                     _stream(stream)), "sbp_rhs_eval_jvp")
        return out

    def overset_interp_vjp(self, recv, q_donor, lqhat, lfvhat=None, stream=None):
        nr = self.info[recv].n_receivers
        lq = self.empty_state(1 - recv)
        lqh = self.torch.zeros((4, max(nr, 1)), dtype=self.torch.float64, device="cuda")
        lqh[:, :nr] = lqhat
        lfv = None
        if lfvhat is not None:
            lfv = self.torch.zeros((6, max(nr, 1)), dtype=self.torch.float64, device="cuda")
            lfv[:, :nr] = lfvhat
        if nr:
            lqh = lqh[:, :nr].contiguous()
            lfv = lfv[:, :nr].contiguous() if lfv is not None else None
        _check(_lib.sbp_overset_interp_vjp(self.h, recv, _ptr(q_donor), _ptr(lqh), _ptr(lfv), _ptr(lq),
                                           _stream(stream)), "sbp_overset_interp_vjp")
        return lq

    def adjoint_probe(self, q0, probe_xy, n_steps, H, n_snapshots=None, grad=True, stream=None):
        """Probe objective J of a run from device states q0 = (mesh 0, mesh 1) and, with grad,
        its gradients w.r.t. q0 (device tensors) and the far-field state (numpy[4])."""
        xy = np.ascontiguousarray(probe_xy, dtype=np.float64).reshape(-1, 2)
        d = AdjointDesc()
        d.n_steps = int(n_steps)
        d.n_snapshots = int(n_steps if n_snapshots is None else n_snapshots)
        d.n_probes = xy.shape[0]
        d.probe_xy = xy.ctypes.data
        d.H = float(H)
        J = ctypes.c_double()
        pp = np.zeros(max(int(n_steps) * xy.shape[0], 1))
        fwd = ctypes.c_long()
        g = [self.empty_state(0), self.empty_state(1)] if grad else [None, None]
        gq = (ctypes.c_double * 4)()
        _check(_lib.sbp_adjoint_probe(self.h, ctypes.byref(d), _ptr(q0[0]), _ptr(q0[1]),
                                      ctypes.cast(ctypes.pointer(J), ctypes.c_void_p), pp.ctypes.data,
                                      _ptr(g[0]), _ptr(g[1]), ctypes.cast(gq, ctypes.c_void_p) if grad else None,
                                      ctypes.cast(ctypes.pointer(fwd), ctypes.c_void_p), _stream(stream)),
               "sbp_adjoint_probe")
        out = {"J": J.value, "p": pp[:int(n_steps) * xy.shape[0]].reshape(int(n_steps), xy.shape[0]),
               "forward_steps": fwd.value}
        if grad:
            out.update({"dq0": g, "dqinf": np.array(gq[:])})
        return out


def _descriptors3(wl, dtype, sigma_interface, sigma_physical, hole_cells):
    """C descriptors (sbp3_mesh_desc[2], sbp_params) of a 3D workload dict (qinf's first four
    entries: rho, rho u, rho v, rho E; the full 5-component state goes through
    sbp3_set_freestream)."""
    p = wl["params"]
    descs = (Mesh3Desc * 2)()
    for k, m in enumerate(wl["meshes"]):
        d = descs[k]
        for a in range(3):
            d.n[a] = m["n"][a]
            d.periodic[a] = int(m["periodic"][a])
            d.lo[a] = m["lo"][a]
            d.h[a] = m["h"][a]
        for f in range(6):
            d.bc[f] = BC[m["bc"][f]]
    pr = Params()
    pr.physics = PHYSICS[p["physics"]]
    pr.dtype = DTYPE[dtype]
    pr.gamma = p["gamma"]
    pr.mu = p["mu"]
    pr.pr = p["pr"]
    pr.twall = p["twall"]
    pr.omega_corner = p["omega_corner"]
    pr.sigma_interface = sigma_interface
    pr.sigma_physical = sigma_physical
    pr.cfl = p["cfl"]
    qi = np.asarray(p["qinf"], dtype=np.float64)
    for v, c in enumerate((0, 1, 2, 4)):
        pr.qinf[v] = float(qi[c])
    pr.order = p["order"]
    pr.hist_len = p["hist_len"]
    pr.step_ratio = p["step_ratio"]
    pr.fast_mesh = p["fast_mesh"]
    pr.hole_cells = hole_cells
    pr.sponge_cells = int(p.get("sponge_cells", 0))
    pr.sponge_strength = float(p.get("sponge_strength", 1.0))
    return descs, pr


class HostTables3D:
    """The host part of 3D system creation alone (sbp3_host_tables_*), without a GPU."""

    def __init__(self, wl, hole_cells=4):
        descs, pr = _descriptors3(wl, "f64", 0.5, 1.0, hole_cells)
        h = ctypes.c_void_p()
        _check(_lib.sbp3_host_tables_create(descs, 2, ctypes.byref(pr), ctypes.byref(h)), "sbp3_host_tables_create")
        self.h = h
        self.meshes = wl["meshes"]

    def tables(self, k):
        ni, nj, nk = self.meshes[k]["n"]
        nr = ctypes.c_int()
        _check(_lib.sbp3_host_tables_get(self.h, k, None, None, None, None, ctypes.byref(nr)), "sbp3_host_tables_get")
        nr = nr.value
        ib = np.zeros(ni * nj * nk, np.int8)
        rec = np.zeros(max(nr, 1), np.int64)
        base = np.zeros(max(3 * nr, 1), np.int32)
        w = np.zeros(max(12 * nr, 1))
        _check(_lib.sbp3_host_tables_get(self.h, k, ib.ctypes.data, rec.ctypes.data, base.ctypes.data,
                                         w.ctypes.data, None), "sbp3_host_tables_get")
        return {"iblank": ib.reshape(nk, nj, ni), "receivers": rec[:nr], "base": base[:3 * nr].reshape(nr, 3),
                "w": w[:12 * nr].reshape(nr, 12)}

    def close(self):
        if getattr(self, "h", None):
            _lib.sbp3_host_tables_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class System3D:
    """A two-mesh 3D Cartesian overset system (C ABI sbp3_*). ``wl`` is a 3D workload dict
    (``workloads.taylor_green_box`` layout). States are numpy arrays (5, nk, nj, ni) or device
    tensors (5, nk, nj, pitch)."""

    def __init__(self, wl, dtype="f64", sigma_interface=0.5, sigma_physical=1.0, hole_cells=4):
        import torch
        self.torch = torch
        self.dtype = dtype
        self.tdtype = torch.float64 if dtype == "f64" else torch.float32
        self.meshes = wl["meshes"]
        p = wl["params"]
        descs, pr = _descriptors3(wl, dtype, sigma_interface, sigma_physical, hole_cells)
        qi = np.asarray(p["qinf"], dtype=np.float64)
        self.params = p
        h = ctypes.c_void_p()
        torch.cuda.init()
        _check(_lib.sbp3_system_create(descs, 2, ctypes.byref(pr), ctypes.byref(h)), "sbp3_system_create")
        self.h = h
        arr = (ctypes.c_double * 5)(*[float(v) for v in qi])
        _check(_lib.sbp3_set_freestream(self.h, ctypes.cast(arr, ctypes.c_void_p)), "sbp3_set_freestream")
        self.info = []
        for k in range(2):
            inf = Mesh3Info()
            _check(_lib.sbp3_mesh_info_get(self.h, k, ctypes.byref(inf)), "sbp3_mesh_info_get")
            self.info.append(inf)
        self.bound = None

    def close(self):
        if getattr(self, "h", None):
            _lib.sbp3_system_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def empty_state(self, k, n=1):
        inf = self.info[k]
        t = self.torch.zeros((n, 5, inf.nk, inf.nj, inf.pitch), dtype=self.tdtype, device="cuda")
        return t if n > 1 else t[0]

    def to_device(self, k, q):
        inf = self.info[k]
        t = self.empty_state(k)
        t[..., :inf.ni] = self.torch.from_numpy(np.ascontiguousarray(q)).to(self.tdtype).cuda()
        return t

    def to_host(self, k, t):
        return t[..., :self.info[k].ni].double().cpu().numpy()

    def tables(self, k):
        inf = self.info[k]
        n = inf.ni * inf.nj * inf.nk
        nr = inf.n_receivers
        ib = np.zeros(n, np.int8)
        rec = np.zeros(max(nr, 1), np.int64)
        base = np.zeros(max(3 * nr, 1), np.int32)
        w = np.zeros(max(12 * nr, 1))
        _check(_lib.sbp3_get_tables(self.h, k, ib.ctypes.data, rec.ctypes.data, base.ctypes.data, w.ctypes.data),
               "sbp3_get_tables")
        return {"iblank": ib.reshape(inf.nk, inf.nj, inf.ni), "receivers": rec[:nr],
                "base": base[:3 * nr].reshape(nr, 3), "w": w[:12 * nr].reshape(nr, 12)}

    def overset_interp(self, recv, q_donor, stream=None):
        nr = self.info[recv].n_receivers
        qhat = self.torch.zeros((5, max(nr, 1)), dtype=self.tdtype, device="cuda")
        fvhat = self.torch.zeros((12, max(nr, 1)), dtype=self.tdtype, device="cuda")
        if nr:
            qhat, fvhat = qhat[:, :nr].contiguous(), fvhat[:, :nr].contiguous()
        _check(_lib.sbp3_overset_interp(self.h, recv, _ptr(q_donor), _ptr(qhat), _ptr(fvhat), _stream(stream)),
               "sbp3_overset_interp")
        return qhat[:, :nr], fvhat[:, :nr]

    def rhs_eval(self, k, q_self, q_other, out=None, stream=None):
        if out is None:
            out = self.empty_state(k)
        _check(_lib.sbp3_rhs_eval(self.h, k, _ptr(q_self), _ptr(q_other), _ptr(out), _stream(stream)),
               "sbp3_rhs_eval")
        return out

    def timestep(self, q0, q1, stream=None):
        dt = (ctypes.c_double * 2)()
        H = ctypes.c_double()
        _check(_lib.sbp3_timestep(self.h, _ptr(q0), _ptr(q1), ctypes.cast(dt, ctypes.c_void_p),
                                  ctypes.cast(ctypes.pointer(H), ctypes.c_void_p), _stream(stream)), "sbp3_timestep")
        return [dt[0], dt[1]], H.value

    def bind(self, q_host):
        self.bound = []
        for k in range(2):
            qa = self.to_device(k, q_host[k])
            qb = self.empty_state(k)
            hist = self.empty_state(k, n=self.params["hist_len"]) if self.params["hist_len"] > 1 else \
                self.empty_state(k)[None]
            _check(_lib.sbp3_bind(self.h, k, _ptr(qa), _ptr(qb), _ptr(hist)), "sbp3_bind")
            self.bound.append((qa, qb, hist))

    def current_state(self, k):
        p = ctypes.c_void_p()
        _check(_lib.sbp3_current_state(self.h, k, ctypes.byref(p)), "sbp3_current_state")
        qa, qb, _ = self.bound[k]
        return qa if p.value == qa.data_ptr() else qb

    def mrab_init(self, H=0.0, stream=None):
        _check(_lib.sbp3_mrab_init(self.h, float(H), _stream(stream)), "sbp3_mrab_init")

    def mrab_step(self, n=1, stream=None):
        _check(_lib.sbp3_mrab_step(self.h, int(n), _stream(stream)), "sbp3_mrab_step")

    def check(self, stream=None):
        _check(_lib.sbp3_check(self.h, _stream(stream)), "sbp3_check")

    def set_rhs_kernel(self, mesh, kchunk):
        """kchunk > 0: the k-marching right-hand side with kchunk planes per CTA; 0: per point."""
        _check(_lib.sbp3_set_rhs_kernel(self.h, int(mesh), int(kchunk)), "sbp3_set_rhs_kernel")


class Batch:
    """Member systems (already bound and initialised) advanced together, one cooperative
    persistent launch per micro step (C ABI: sbp_batch_*)."""

    def __init__(self, systems, autotune=True, stream=None):
        self.systems = list(systems)
        arr = (ctypes.c_void_p * len(self.systems))(*[g.h.value for g in self.systems])
        h = ctypes.c_void_p()
        _check(_lib.sbp_batch_create(arr, len(self.systems), int(bool(autotune)), _stream(stream), ctypes.byref(h)),
               "sbp_batch_create")
        self.h = h

    def step(self, n=1, stream=None):
        _check(_lib.sbp_batch_step(self.h, int(n), _stream(stream)), "sbp_batch_step")

    def info(self):
        v = [ctypes.c_int() for _ in range(4)]
        _check(_lib.sbp_batch_info(self.h, *[ctypes.cast(ctypes.pointer(x), ctypes.c_void_p) for x in v]),
               "sbp_batch_info")
        return {"members": v[0].value, "rows_per_cta": v[1].value, "grid": v[2].value, "period": v[3].value}

    def set_shape(self, rows):
        """Work items of `rows` rows: 8, 16 (tile pairs) or, for Euler, 32, 64, 128 (strips)."""
        _check(_lib.sbp_batch_set_shape(self.h, int(rows)), "sbp_batch_set_shape")

    def check(self, stream=None):
        _check(_lib.sbp_batch_check(self.h, _stream(stream)), "sbp_batch_check")

    def close(self):
        if getattr(self, "h", None):
            _lib.sbp_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def f32_to_f64(x, stream=None):
    """Widen a contiguous FP32 CUDA tensor to FP64 with the library's integer re-encoding (the
    conversion inside the FP32 forms' FP64 accumulations)."""
    import torch
    if x.dtype != torch.float32 or not x.is_cuda or not x.is_contiguous():
        raise ValueError("a contiguous float32 CUDA tensor is required")
    y = torch.empty(x.shape, dtype=torch.float64, device=x.device)
    _check(_lib.sbp_f32_to_f64(_ptr(x), _ptr(y), x.numel(), _stream(stream)), "sbp_f32_to_f64")
    return y


class Chain:
    """A chain of nested overset meshes, each at its own rate (C ABI sbp_chain_*). ``wl`` is a
    workload dict with meshes (outermost first), params and ratios (``workloads.vortex_chain``
    layout). States are numpy arrays (4, nj, ni) or device tensors in the pitched layout."""

    def __init__(self, wl, dtype="f64", sigma_interface=0.5, sigma_physical=1.0, hole_cells=4):
        import torch
        self.torch = torch
        self.tdtype = torch.float64 if dtype == "f64" else torch.float32
        self.params = wl["params"]
        self.R = len(wl["meshes"])
        descs, pr, self._keep = _descriptors(wl, dtype, sigma_interface, sigma_physical, hole_cells)
        ratios = (ctypes.c_int * max(self.R - 1, 1))(*[int(r) for r in wl["ratios"]])
        h = ctypes.c_void_p()
        torch.cuda.init()
        _check(_lib.sbp_chain_create(descs, self.R, ctypes.cast(ratios, ctypes.c_void_p), ctypes.byref(pr),
                                     ctypes.byref(h)), "sbp_chain_create")
        self.h = h
        self.info = []
        for k in range(self.R):
            inf = MeshInfo()
            _check(_lib.sbp_chain_mesh_info(self.h, k, ctypes.byref(inf)), "sbp_chain_mesh_info")
            self.info.append(inf)
        self.bound = None

    def close(self):
        if getattr(self, "h", None):
            _lib.sbp_chain_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    empty_state = System.empty_state
    to_device = System.to_device
    to_host = System.to_host

    def tables(self, k):
        inf = self.info[k]
        n, nr = inf.ni * inf.nj, inf.n_receivers
        ib = np.zeros(n, np.int8)
        rec = np.zeros(max(nr, 1), np.int32)
        src = np.zeros(max(nr, 1), np.int32)
        base = np.zeros(max(2 * nr, 1), np.int32)
        w = np.zeros(max(8 * nr, 1))
        _check(_lib.sbp_chain_tables(self.h, k, ib.ctypes.data, rec.ctypes.data, src.ctypes.data, base.ctypes.data,
                                     w.ctypes.data), "sbp_chain_tables")
        return {"iblank": ib.reshape(inf.nj, inf.ni), "receivers": rec[:nr], "donor_mesh": src[:nr],
                "base": base[:2 * nr].reshape(nr, 2), "w": w[:8 * nr].reshape(nr, 8)}

    def _ptrs(self, qs):
        return (ctypes.c_void_p * self.R)(*[t.data_ptr() for t in qs])

    def rhs_eval(self, k, qs, out=None, stream=None):
        if out is None:
            out = self.empty_state(k)
        _check(_lib.sbp_chain_rhs_eval(self.h, k, ctypes.cast(self._ptrs(qs), ctypes.c_void_p), _ptr(out),
                                       _stream(stream)), "sbp_chain_rhs_eval")
        return out

    def timestep(self, qs, stream=None):
        dt = (ctypes.c_double * self.R)()
        H = ctypes.c_double()
        _check(_lib.sbp_chain_timestep(self.h, ctypes.cast(self._ptrs(qs), ctypes.c_void_p),
                                       ctypes.cast(dt, ctypes.c_void_p), ctypes.cast(ctypes.pointer(H), ctypes.c_void_p),
                                       _stream(stream)), "sbp_chain_timestep")
        return list(dt), H.value

    def bind(self, q_host):
        self.bound = []
        for k in range(self.R):
            qa = self.to_device(k, q_host[k])
            qb = self.empty_state(k)
            hist = self.empty_state(k, n=self.params["hist_len"]) if self.params["hist_len"] > 1 else \
                self.empty_state(k)[None]
            _check(_lib.sbp_chain_bind(self.h, k, _ptr(qa), _ptr(qb), _ptr(hist)), "sbp_chain_bind")
            self.bound.append((qa, qb, hist))

    def current_state(self, k):
        p = ctypes.c_void_p()
        _check(_lib.sbp_chain_current_state(self.h, k, ctypes.byref(p)), "sbp_chain_current_state")
        qa, qb, _ = self.bound[k]
        return qa if p.value == qa.data_ptr() else qb

    def mrab_init(self, H=0.0, stream=None):
        _check(_lib.sbp_chain_mrab_init(self.h, float(H), _stream(stream)), "sbp_chain_mrab_init")

    def mrab_step(self, n=1, stream=None):
        _check(_lib.sbp_chain_mrab_step(self.h, int(n), _stream(stream)), "sbp_chain_mrab_step")

    def mrab_time(self):
        H, t = ctypes.c_double(), ctypes.c_double()
        _check(_lib.sbp_chain_mrab_time(self.h, ctypes.byref(H), ctypes.byref(t)), "sbp_chain_mrab_time")
        return H.value, t.value

    def check(self, stream=None):
        _check(_lib.sbp_chain_check(self.h, _stream(stream)), "sbp_chain_check")


def barrier_selftest(grid, arrivals, max_spins, stream=None):
    """The batch launch's bounded grid barrier on `grid` CTAs waiting for `arrivals` arrivals
    (C ABI sbp_barrier_selftest): returns (error word, CTAs that passed)."""
    st, npass = ctypes.c_int(0), ctypes.c_int(0)
    _check(_lib.sbp_barrier_selftest(int(grid), int(arrivals), int(max_spins), ctypes.byref(st),
                                     ctypes.byref(npass), _stream(stream)), "sbp_barrier_selftest")
    return st.value, npass.value


def fp64_rate_probe(out, grid, block, iters, stream=None):
    """Launch the FP64 fused multiply-add probe (grid x block threads, 8 chains of iters FMAs
    each) on stream; out is a float64 CUDA tensor of at least grid * block elements. Returns the
    FP64 operations the launch performs."""
    import torch
    if out.dtype != torch.float64 or not out.is_cuda or out.numel() < grid * block:
        raise ValueError("a float64 CUDA tensor of grid * block elements is required")
    flops = ctypes.c_double(0.0)
    _check(_lib.sbp_fp64_rate_probe(_ptr(out), int(grid), int(block), int(iters), ctypes.byref(flops),
                                    _stream(stream)), "sbp_fp64_rate_probe")
    return flops.value


class Curvilinear3DMesh:
    """One 3D curvilinear structured mesh on the current CUDA device (C ABI sbp3c_*): device
    metric terms and the flux divergence of a state. x, y, z: (nk, nj, ni) coordinate arrays;
    params: a workload's params dict (physics, gamma, mu, pr)."""

    def __init__(self, x, y, z, params, dtype="f64"):
        import torch
        self.torch = torch
        self.tdtype = torch.float64 if dtype == "f64" else torch.float32
        self.viscous = params["physics"] == "ns"
        self.nrecv = None
        X = [np.ascontiguousarray(v, dtype=np.float64) for v in (x, y, z)]
        self.shape = X[0].shape
        nk, nj, ni = self.shape
        n = (ctypes.c_int * 3)(ni, nj, nk)
        pr = Params()
        pr.physics = PHYSICS[params["physics"]]
        pr.dtype = DTYPE[dtype]
        pr.gamma = params["gamma"]
        pr.mu = params.get("mu", 0.0)
        pr.pr = params.get("pr", 0.72)
        h = ctypes.c_void_p()
        torch.cuda.init()
        _check(_lib.sbp3c_mesh_create(ctypes.cast(n, ctypes.c_void_p), X[0].ctypes.data, X[1].ctypes.data,
                                      X[2].ctypes.data, ctypes.byref(pr), ctypes.byref(h)), "sbp3c_mesh_create")
        self.h = h

    def _field(self, t, name, shape):
        """t as a contiguous device tensor of the mesh's element type and the given shape; the
        kernels index it by the mesh's sizes, so anything else is refused before the call."""
        torch = self.torch
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise ValueError("%s must be a CUDA tensor" % name)
        if t.dtype != self.tdtype:
            raise ValueError("%s must be %s, got %s" % (name, self.tdtype, t.dtype))
        if tuple(t.shape) != tuple(shape):
            raise ValueError("%s must have shape %s, got %s" % (name, tuple(shape), tuple(t.shape)))
        return t.contiguous()

    def metrics(self):
        out = np.zeros((10,) + self.shape)
        _check(_lib.sbp3c_get_metrics(self.h, out.ctypes.data), "sbp3c_get_metrics")
        return out

    def set_farfield(self, qinf, sigma=1.0):
        """Far-field SAT towards qinf (5 conserved values) on every face; None turns it off."""
        if qinf is None:
            _check(_lib.sbp3c_set_farfield(self.h, None, 0.0), "sbp3c_set_farfield")
            return
        qi = np.ascontiguousarray(qinf, dtype=np.float64)
        if qi.shape != (5,):
            raise ValueError("qinf needs 5 values")
        _check(_lib.sbp3c_set_farfield(self.h, qi.ctypes.data, float(sigma)), "sbp3c_set_farfield")

    def set_interface(self, terms, nrecv, sigma=0.5):
        """Interface SAT terms: a list of (i, j, k, m, side, r, scale)."""
        t = np.ascontiguousarray([x[:6] for x in terms], dtype=np.int32).reshape(-1, 6)
        sc = np.ascontiguousarray([x[6] for x in terms], dtype=np.float64)
        _check(_lib.sbp3c_set_interface(self.h, len(t), t.ctypes.data if len(t) else None,
                                        sc.ctypes.data if len(t) else None, int(nrecv), float(sigma)),
               "sbp3c_set_interface")
        self.nrecv = int(nrecv)

    def interface_sat(self, q, qhat, rhs, fvhat=None, stream=None):
        """rhs += the interface SAT terms at state q (device tensors of the mesh's element type:
        q and rhs (5, nk, nj, ni), qhat (5, nrecv), fvhat (12, nrecv) for Navier-Stokes, with
        nrecv as given to set_interface)."""
        if self.nrecv is None:
            raise ValueError("set_interface first")
        q = self._field(q, "q", (5,) + self.shape)
        if not rhs.is_contiguous():
            raise ValueError("rhs must be contiguous")
        self._field(rhs, "rhs", (5,) + self.shape)
        qhat = self._field(qhat, "qhat", (5, self.nrecv))
        fv = None
        if self.viscous:
            if fvhat is None:
                raise ValueError("fvhat (12, nrecv) is required for Navier-Stokes")
            fv = self._field(fvhat, "fvhat", (12, self.nrecv))
        _check(_lib.sbp3c_interface_sat(self.h, _ptr(q), _ptr(qhat), None if fv is None else _ptr(fv), _ptr(rhs),
                                        _stream(stream)), "sbp3c_interface_sat")
        return rhs

    def interp(self, q, base, w, stream=None):
        """Overset gather of q (5, nk, nj, ni) at stencils (base (n, 3) ints, w (n, 12)), as
        donor_search_3d returns them: a (5, n) device tensor."""
        torch = self.torch
        q = self._field(q, "q", (5,) + self.shape)
        bh = np.ascontiguousarray(base, dtype=np.int32).reshape(-1, 3)
        nk, nj, ni = self.shape
        if len(bh) and ((bh.min(axis=0) < 0).any() or (bh.max(axis=0) > np.array([ni, nj, nk]) - 4).any()):
            raise ValueError("donor stencil outside the mesh")
        b = torch.as_tensor(bh).cuda()
        wt = torch.as_tensor(np.ascontiguousarray(w, dtype=np.float64)).cuda()
        n = int(b.shape[0])
        if b.shape != (n, 3) or wt.shape != (n, 12):
            raise ValueError("base (n, 3) and w (n, 12) expected")
        out = torch.empty((5, n), dtype=self.tdtype, device="cuda")
        _check(_lib.sbp3c_interp(self.h, _ptr(q), n, _ptr(b), _ptr(wt), _ptr(out), _stream(stream)), "sbp3c_interp")
        return out

    def check(self, stream=None):
        """Synchronise and report the mesh's device error word (SBP_ERR_BOUNDS from interp)."""
        _check(_lib.sbp3c_mesh_check(self.h, _stream(stream)), "sbp3c_mesh_check")

    def rhs_eval(self, q, out=None, stream=None):
        """q: (5, nk, nj, ni) device tensor of the mesh's element type."""
        q = self._field(q, "q", (5,) + self.shape)
        if out is None:
            out = self.torch.empty_like(q)
        elif not out.is_contiguous():
            raise ValueError("out must be contiguous")
        else:
            self._field(out, "out", (5,) + self.shape)
        _check(_lib.sbp3c_rhs_eval(self.h, _ptr(q), _ptr(out), _stream(stream)), "sbp3c_rhs_eval")
        return out

    def close(self):
        if getattr(self, "h", None):
            _lib.sbp3c_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _descriptors_curv(wl, dtype, sigma_interface, sigma_physical):
    """C descriptors (sbp3c_mesh_desc[2], sbp_params) of a curvilinear pair workload
    (``workloads.curvilinear_pair`` layout) and the coordinate arrays they point to (keep them
    alive for the call)."""
    p = wl["params"]
    descs = (Mesh3cDesc * 2)()
    keep = []
    for k, m in enumerate(wl["meshes"]):
        X = [np.ascontiguousarray(m[c], dtype=np.float64) for c in ("x", "y", "z")]
        nk, nj, ni = X[0].shape
        if tuple(m["n"]) != (ni, nj, nk) or any(v.shape != X[0].shape for v in X):
            raise ValueError("mesh %d: coordinates must be (nk, nj, ni) arrays matching n" % k)
        keep.extend(X)
        d = descs[k]
        for a, v in enumerate((ni, nj, nk)):
            d.n[a] = v
        d.x, d.y, d.z = (v.ctypes.data for v in X)
    pr = Params()
    pr.physics = PHYSICS[p["physics"]]
    pr.dtype = DTYPE[dtype]
    pr.gamma = p["gamma"]
    pr.mu = p["mu"]
    pr.pr = p["pr"]
    pr.twall = p.get("twall", 1.0)
    pr.omega_corner = p["omega_corner"]
    pr.sigma_interface = sigma_interface
    pr.sigma_physical = sigma_physical
    pr.cfl = p["cfl"]
    qi = np.asarray(p["qinf"], dtype=np.float64)
    for v, c in enumerate((0, 1, 2, 4)):
        pr.qinf[v] = float(qi[c])
    pr.order = p["order"]
    pr.hist_len = p["hist_len"]
    pr.step_ratio = p["step_ratio"]
    pr.fast_mesh = p["fast_mesh"]
    pr.hole_cells = float(p["hole_cells"])
    pr.sponge_cells = int(p.get("sponge_cells", 0))
    pr.sponge_strength = float(p.get("sponge_strength", 1.0))
    return descs, pr, keep


def _tables3(getter, where, handle, k, shape, nr):
    """iblank, receivers, donor bases and weights of mesh k by a table getter of the C ABI."""
    nk, nj, ni = shape
    ib = np.zeros(ni * nj * nk, np.int8)
    rec = np.zeros(max(nr, 1), np.int64)
    base = np.zeros(max(3 * nr, 1), np.int32)
    w = np.zeros(max(12 * nr, 1))
    _check(getter(handle, k, ib.ctypes.data, rec.ctypes.data, base.ctypes.data, w.ctypes.data), where)
    return {"iblank": ib.reshape(nk, nj, ni), "receivers": rec[:nr], "base": base[:3 * nr].reshape(nr, 3),
            "w": w[:12 * nr].reshape(nr, 12)}


class HostTablesCurvilinearPair:
    """The host part of curvilinear pair creation alone (sbp3c_host_tables_*), without a GPU."""

    def __init__(self, wl, sigma_interface=0.5, sigma_physical=1.0):
        descs, pr, keep = _descriptors_curv(wl, "f64", sigma_interface, sigma_physical)
        h = ctypes.c_void_p()
        _check(_lib.sbp3c_host_tables_create(descs, 2, ctypes.byref(pr), ctypes.byref(h)), "sbp3c_host_tables_create")
        del keep
        self.h = h
        self.shapes = [m["x"].shape for m in wl["meshes"]]

    def tables(self, k):
        nr = ctypes.c_int()
        _check(_lib.sbp3c_host_tables_get(self.h, k, None, None, None, None, ctypes.byref(nr)), "sbp3c_host_tables_get")
        return _tables3(lambda h, kk, a, b, c, d: _lib.sbp3c_host_tables_get(h, kk, a, b, c, d, None),
                        "sbp3c_host_tables_get", self.h, k, self.shapes[k], nr.value)

    def close(self):
        if getattr(self, "h", None):
            _lib.sbp3c_host_tables_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class CurvilinearPair:
    """A 3D curvilinear overset pair on the current CUDA device (C ABI sbp3c_system_*): mesh 0 the
    background (far field on its faces), mesh 1 the overset mesh (interface on its faces).
    ``wl`` is a ``workloads.curvilinear_pair`` dict. States are numpy arrays or device tensors
    (5, nk, nj, ni) of the pair's element type."""

    def __init__(self, wl, dtype="f64", sigma_interface=0.5, sigma_physical=1.0):
        import torch
        self.torch = torch
        self.dtype = dtype
        self.tdtype = torch.float64 if dtype == "f64" else torch.float32
        self.params = wl["params"]
        self.viscous = self.params["physics"] == "ns"
        self.shapes = [m["x"].shape for m in wl["meshes"]]
        descs, pr, keep = _descriptors_curv(wl, dtype, sigma_interface, sigma_physical)
        h = ctypes.c_void_p()
        torch.cuda.init()
        _check(_lib.sbp3c_system_create(descs, 2, ctypes.byref(pr), ctypes.byref(h)), "sbp3c_system_create")
        del keep
        self.h = h
        qi = np.ascontiguousarray(self.params["qinf"], dtype=np.float64)
        _check(_lib.sbp3c_system_set_freestream(self.h, qi.ctypes.data), "sbp3c_system_set_freestream")
        self.info = []
        for k in range(2):
            inf = Mesh3Info()
            _check(_lib.sbp3c_system_info(self.h, k, ctypes.byref(inf)), "sbp3c_system_info")
            self.info.append(inf)
        self.bound = None

    def close(self):
        if getattr(self, "h", None):
            _lib.sbp3c_system_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _state(self, k, t, name):
        torch = self.torch
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != self.tdtype or not t.is_contiguous():
            raise ValueError("%s must be a contiguous CUDA tensor of %s" % (name, self.tdtype))
        if tuple(t.shape) != (5,) + tuple(self.shapes[k]):
            raise ValueError("%s must have shape %s" % (name, (5,) + tuple(self.shapes[k])))
        return t

    def empty_state(self, k, n=1):
        t = self.torch.zeros((n, 5) + tuple(self.shapes[k]), dtype=self.tdtype, device="cuda")
        return t if n > 1 else t[0]

    def to_device(self, k, q):
        return self.torch.from_numpy(np.ascontiguousarray(q)).to(self.tdtype).cuda().contiguous()

    def to_host(self, k, t):
        return t.double().cpu().numpy()

    def tables(self, k):
        return _tables3(_lib.sbp3c_system_tables, "sbp3c_system_tables", self.h, k, self.shapes[k],
                        self.info[k].n_receivers)

    def overset_interp(self, recv, q_donor, stream=None):
        """(qhat (5, n_receivers), fvhat (12, n_receivers)) at mesh recv's receivers."""
        nr = self.info[recv].n_receivers
        q_donor = self._state(1 - recv, q_donor, "q_donor")
        qhat = self.torch.zeros((5, max(nr, 1)), dtype=self.tdtype, device="cuda")
        fvhat = self.torch.zeros((12, max(nr, 1)), dtype=self.tdtype, device="cuda")
        _check(_lib.sbp3c_system_interp(self.h, recv, _ptr(q_donor), _ptr(qhat), _ptr(fvhat), _stream(stream)),
               "sbp3c_system_interp")
        return qhat[:, :nr], fvhat[:, :nr]

    def rhs_eval(self, k, q_self, q_other, out=None, stream=None):
        q_self = self._state(k, q_self, "q_self")
        q_other = self._state(1 - k, q_other, "q_other")
        out = self.empty_state(k) if out is None else self._state(k, out, "out")
        _check(_lib.sbp3c_system_rhs_eval(self.h, k, _ptr(q_self), _ptr(q_other), _ptr(out), _stream(stream)),
               "sbp3c_system_rhs_eval")
        return out

    def timestep(self, q0, q1, stream=None):
        q0, q1 = self._state(0, q0, "q0"), self._state(1, q1, "q1")
        dt = (ctypes.c_double * 2)()
        H = ctypes.c_double()
        _check(_lib.sbp3c_system_timestep(self.h, _ptr(q0), _ptr(q1), ctypes.cast(dt, ctypes.c_void_p),
                                          ctypes.cast(ctypes.pointer(H), ctypes.c_void_p), _stream(stream)),
               "sbp3c_system_timestep")
        return [dt[0], dt[1]], H.value

    def bind(self, q_host):
        self.bound = []
        m = int(self.params["hist_len"])
        for k in range(2):
            qa = self.to_device(k, q_host[k])
            qb = self.empty_state(k)
            hist = self.empty_state(k, n=m) if m > 1 else self.empty_state(k)[None]
            _check(_lib.sbp3c_system_bind(self.h, k, _ptr(qa), _ptr(qb), _ptr(hist)), "sbp3c_system_bind")
            self.bound.append((qa, qb, hist))

    def current_state(self, k):
        p = ctypes.c_void_p()
        _check(_lib.sbp3c_system_current_state(self.h, k, ctypes.byref(p)), "sbp3c_system_current_state")
        qa, qb, _ = self.bound[k]
        return qa if p.value == qa.data_ptr() else qb

    def mrab_init(self, H=0.0, stream=None):
        _check(_lib.sbp3c_system_mrab_init(self.h, float(H), _stream(stream)), "sbp3c_system_mrab_init")

    def mrab_step(self, n=1, stream=None):
        _check(_lib.sbp3c_system_mrab_step(self.h, int(n), _stream(stream)), "sbp3c_system_mrab_step")

    def mrab_time(self):
        H, t = ctypes.c_double(), ctypes.c_double()
        _check(_lib.sbp3c_system_mrab_time(self.h, ctypes.byref(H), ctypes.byref(t)), "sbp3c_system_mrab_time")
        return H.value, t.value

    def check(self, stream=None):
        _check(_lib.sbp3c_system_check(self.h, _stream(stream)), "sbp3c_system_check")


def donor_search_3d(x, y, z, points, iblank=None):
    """Donor stencils on a curvilinear mesh (host, no device calls; C ABI sbp3c_donor_search).
    x, y, z: (nk, nj, ni) coordinates; points (npts, 3). Returns base (npts, 3) int32,
    weights (npts, 12), computational coordinates (npts, 3); raises SbpError (status
    SBP_ERR_DONOR) naming the first point without a valid stencil."""
    X = [np.ascontiguousarray(v, dtype=np.float64) for v in (x, y, z)]
    nk, nj, ni = X[0].shape
    n = (ctypes.c_int * 3)(ni, nj, nk)
    P = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
    npts = len(P)
    base = np.zeros((npts, 3), np.int32)
    w = np.zeros((npts, 12))
    xi = np.zeros((npts, 3))
    ib = None if iblank is None else np.ascontiguousarray(iblank, dtype=np.int8)
    failed = ctypes.c_int(-1)
    _check(_lib.sbp3c_donor_search(ctypes.cast(n, ctypes.c_void_p), X[0].ctypes.data, X[1].ctypes.data,
                                   X[2].ctypes.data, None if ib is None else ib.ctypes.data, npts,
                                   P.ctypes.data, base.ctypes.data, w.ctypes.data, xi.ctypes.data,
                                   ctypes.byref(failed)), "sbp3c_donor_search")
    return base, w, xi


def hole_cut_3d(x, y, z, points, margin):
    """Points (npts, 3) that are holes of the curvilinear mesh x, y, z (host, no device calls;
    C ABI sbp3c_hole_cut): a bool array."""
    X = [np.ascontiguousarray(v, dtype=np.float64) for v in (x, y, z)]
    nk, nj, ni = X[0].shape
    n = (ctypes.c_int * 3)(ni, nj, nk)
    P = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
    ib = np.ones(len(P), np.int8)
    _check(_lib.sbp3c_hole_cut(ctypes.cast(n, ctypes.c_void_p), X[0].ctypes.data, X[1].ctypes.data, X[2].ctypes.data,
                               len(P), P.ctypes.data, float(margin), ib.ctypes.data), "sbp3c_hole_cut")
    return ib == 0


def exported_symbols():
    """Names declared in include/sbp_mrab.h that the library must export."""
    return sorted(list(_SIGS) + ["sbp_status_string", "sbp_last_error_message"])
