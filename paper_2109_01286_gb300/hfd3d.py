"""Python binding of the three-dimensional extension's C ABI (include/hfd3d.h): argument
marshalling only; every step of the residual and the time stepping runs in the library's
kernels (libhfd.so, loaded by `hfd`, which fails loudly when the library is missing).

States are 20 x V float64 CUDA tensors in the input vertex order: rows 0-4 w = (rho, rho u,
rho v, rho w, E), rows 5-9 w_x, rows 10-14 w_y, rows 15-19 w_z."""
import ctypes

import numpy as np

from .hfd import HfdError, _lib, _stream, _dptr

_P = ctypes.c_void_p

__all__ = ["Mesh3", "Options3", "options3", "HfdError"]

EXPORTED = ["hfd3_default_options", "hfd3_mesh_create", "hfd3_mesh_destroy", "hfd3_mesh_info",
            "hfd3_prep_size", "hfd3_prep_get", "hfd3_prep_set", "hfd3_residual", "hfd3_steps",
            "hfd3_steps_profiled", "hfd3_check", "hfd3_mesh_set_lanes"]


class Options3(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("weno_eps", ctypes.c_double),
                ("sens_lo", ctypes.c_double), ("sens_hi", ctypes.c_double),
                ("harten", ctypes.c_double), ("sv_rtol", ctypes.c_double),
                ("div_cond_min", ctypes.c_double), ("force_branch", ctypes.c_int32),
                ("threads", ctypes.c_int32), ("host_only", ctypes.c_int32)]


class MeshDesc3(ctypes.Structure):
    _fields_ = [("nv", ctypes.c_int32), ("x", ctypes.POINTER(ctypes.c_double)),
                ("y", ctypes.POINTER(ctypes.c_double)), ("z", ctypes.POINTER(ctypes.c_double)),
                ("ntet", ctypes.c_int32), ("tet", ctypes.POINTER(ctypes.c_int32)),
                ("Lx", ctypes.c_double), ("Ly", ctypes.c_double), ("Lz", ctypes.c_double)]


_lib.hfd3_default_options.argtypes = [ctypes.POINTER(Options3)]
_lib.hfd3_default_options.restype = None
_lib.hfd3_mesh_create.argtypes = [ctypes.POINTER(MeshDesc3), ctypes.POINTER(Options3),
                                  ctypes.POINTER(_P)]
_lib.hfd3_mesh_destroy.argtypes = [_P]
_lib.hfd3_mesh_destroy.restype = None
_lib.hfd3_mesh_info.argtypes = [_P, ctypes.POINTER(ctypes.c_int64)]
_lib.hfd3_prep_size.argtypes = [_P, ctypes.c_char_p]
_lib.hfd3_prep_size.restype = ctypes.c_int64
_lib.hfd3_prep_get.argtypes = [_P, ctypes.c_char_p, _P, ctypes.c_int64]
_lib.hfd3_prep_set.argtypes = [_P, ctypes.c_char_p, _P, ctypes.c_int64]
_lib.hfd3_residual.argtypes = [_P, _P, _P, _P]
_lib.hfd3_steps.argtypes = [_P, _P, ctypes.c_double, ctypes.c_int32, _P]
_lib.hfd3_steps_profiled.argtypes = [_P, _P, ctypes.c_double, ctypes.c_int32,
                                     ctypes.POINTER(ctypes.c_double), _P]
_lib.hfd3_check.argtypes = [_P]
_lib.hfd3_mesh_set_lanes.argtypes = [_P, ctypes.c_int32]

_INT_ARRAYS = {"edges", "sten", "rank", "vptr", "vidx", "eptr", "eidx"}


def _ok(status, where):
    if status != 0:
        raise HfdError(status, where)


def options3(**kw):
    """hfd3_default_options with keyword overrides (force_branch: 0, 1, 2 or "sensor",
    "hermite", "weno")."""
    o = Options3()
    _lib.hfd3_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if k == "force_branch" and isinstance(v, str):
            v = {"sensor": 0, "hermite": 1, "weno": 2}[v]
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


class Mesh3:
    """A periodic tetrahedral mesh on the device (hfd3_mesh_*), built from a mesh dict with x,
    y, z, tet, Lx, Ly, Lz (as made by synth.three_d.periodic_tet_box).  host_only=1 builds the
    host preprocessing alone (no GPU needed; prep_get and info work)."""

    def __init__(self, mesh, **opts):
        x = np.ascontiguousarray(mesh["x"], dtype=np.float64)
        y = np.ascontiguousarray(mesh["y"], dtype=np.float64)
        z = np.ascontiguousarray(mesh["z"], dtype=np.float64)
        tet = np.ascontiguousarray(mesh["tet"], dtype=np.int32)
        dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        d = MeshDesc3(len(x), dp(x), dp(y), dp(z), len(tet),
                      tet.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                      float(mesh["Lx"]), float(mesh["Ly"]), float(mesh["Lz"]))
        o = options3(**opts)
        h = _P()
        _ok(_lib.hfd3_mesh_create(ctypes.byref(d), ctypes.byref(o), ctypes.byref(h)),
            "hfd3_mesh_create")
        self._h = h
        info = self.info()
        self.nv, self.nedges = info["nv"], info["nedges"]

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _lib.hfd3_mesh_destroy(h)
            self._h = None

    def info(self):
        a = (ctypes.c_int64 * 6)()
        _ok(_lib.hfd3_mesh_info(self._h, a), "hfd3_mesh_info")
        keys = ["nv", "nedges", "div_nv_total", "div_ne_total", "rank_deficient_sides",
                "prep_micros"]
        return dict(zip(keys, list(a)))

    def prep_get(self, name):
        n = _lib.hfd3_prep_size(self._h, name.encode())
        if n < 0:
            raise KeyError(name)
        out = np.empty(n, dtype=np.int32 if name in _INT_ARRAYS else np.float64)
        _ok(_lib.hfd3_prep_get(self._h, name.encode(), out.ctypes.data_as(_P), n), "hfd3_prep_get")
        return out

    def prep_set(self, name, values):
        a = np.ascontiguousarray(values, dtype=np.int32 if name in _INT_ARRAYS else np.float64).ravel()
        _ok(_lib.hfd3_prep_set(self._h, name.encode(), a.ctypes.data_as(_P), a.size),
            "hfd3_prep_set")

    def residual(self, U, R=None, stream=None):
        import torch
        if R is None:
            R = torch.empty_like(U)
        _ok(_lib.hfd3_residual(self._h, _dptr(U), _dptr(R), _stream(stream)), "hfd3_residual")
        return R

    def steps(self, U, dt, nsteps=1, stream=None):
        _ok(_lib.hfd3_steps(self._h, _dptr(U), float(dt), int(nsteps), _stream(stream)),
            "hfd3_steps")
        return U

    def steps_profiled(self, U, dt, nsteps=1, stream=None):
        ms = (ctypes.c_double * 3)()
        _ok(_lib.hfd3_steps_profiled(self._h, _dptr(U), float(dt), int(nsteps), ms,
                                     _stream(stream)), "hfd3_steps_profiled")
        return {"vertex": ms[0], "edge": ms[1], "div": ms[2]}

    def set_lanes(self, lanes):
        _ok(_lib.hfd3_mesh_set_lanes(self._h, int(lanes)), "hfd3_mesh_set_lanes")

    def check(self):
        _ok(_lib.hfd3_check(self._h), "hfd3_check")
