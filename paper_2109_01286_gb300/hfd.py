"""Python binding of the C ABI in include/hfd.h (argument marshalling only).

Every step of the computation runs in libhfd.so: host preprocessing in its C++ part, the
residual and time steps in its CUDA kernels.  PyTorch is used for device memory and streams.
If the library has not been built this module raises at import: there is no fallback.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# HFD_CHECKED=1 loads the bounds-checked build (every gathered index tested on the device; an
# index out of range is reported by check() as HFD_ERR_MESH instead of being read)
LIB_PATH = os.path.join(_HERE, "_lib", "libhfd_check.so" if os.environ.get("HFD_CHECKED") == "1"
                        else "libhfd.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with "
                      "`python -c 'import __graft_entry__ as g; g.build()'`")
_lib = ctypes.CDLL(LIB_PATH)

HFD_OK = 0
STATUS = {0: "HFD_OK", 1: "HFD_ERR_ARG", 2: "HFD_ERR_MESH", 3: "HFD_ERR_STENCIL",
          4: "HFD_ERR_SINGULAR", 5: "HFD_ERR_CUDA", 6: "HFD_ERR_NONFINITE",
          7: "HFD_ERR_POSITIVITY", 8: "HFD_ERR_TIMEOUT", 9: "HFD_ERR_UNSUPPORTED"}

EXPORTED = ["hfd_default_options", "hfd_last_error", "hfd_prep_create", "hfd_prep_destroy",
            "hfd_prep_size", "hfd_prep_get", "hfd_prep_set", "hfd_mesh_create", "hfd_mesh_upload",
            "hfd_mesh_destroy", "hfd_mesh_info", "hfd_mesh_perm", "hfd_state_import",
            "hfd_state_export", "hfd_residual", "hfd_step", "hfd_steps", "hfd_steps_host",
            "hfd_last_dt", "hfd_check", "hfd_steps_profiled", "hfd_residual_static",
            "hfd_prep_concat", "hfd_mesh_set_launch", "hfd_mesh_set_lanes", "hfd_mesh_autotune",
            "hfd_mesh_set_barrier_limit", "hfd_adjoint", "hfd_batch_create", "hfd_batch_destroy",
            "hfd_batch_mesh", "hfd_batch_step", "hfd_measure_fma_peaks",
            "hfd_mesh_set_div_staged", "hfd_edge_branches", "hfd_mesh_set_fp64_div",
            "hfd_check_conversions"]


class HfdError(RuntimeError):
    def __init__(self, status, where):
        msg = _lib.hfd_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")
        self.status = status


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


def _torch_alloc(nbytes, ctx):
    import torch
    try:
        return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device())
    except Exception:                 # out of memory: the library reports HFD_ERR_CUDA
        return None


def _torch_free(ptr, ctx):
    import torch
    torch.cuda.caching_allocator_delete(ptr)


# module-level so that the C function pointers outlive every mesh that holds them
TORCH_ALLOC = _ALLOC_FN(_torch_alloc)
TORCH_FREE = _FREE_FN(_torch_free)


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("div_degree", ctypes.c_int32),
                ("visc_degree", ctypes.c_int32), ("viscous", ctypes.c_int32),
                ("renumber", ctypes.c_int32), ("nthreads", ctypes.c_int32),
                ("gamma", ctypes.c_double), ("mu", ctypes.c_double), ("prandtl", ctypes.c_double),
                ("R_gas", ctypes.c_double), ("weno_eps", ctypes.c_double),
                ("sens_lo", ctypes.c_double), ("sens_hi", ctypes.c_double),
                ("sv_rtol", ctypes.c_double), ("div_cond_min", ctypes.c_double),
                ("harten", ctypes.c_double), ("cfl", ctypes.c_double),
                ("visc_coef_max", ctypes.c_double), ("dev_alloc", _ALLOC_FN),
                ("dev_free", _FREE_FN), ("alloc_ctx", ctypes.c_void_p), ("flux", ctypes.c_int32),
                ("conservative", ctypes.c_int32), ("force_branch", ctypes.c_int32)]


class MeshDesc(ctypes.Structure):
    _fields_ = [("nv", ctypes.c_int32), ("ntri", ctypes.c_int32),
                ("x", ctypes.POINTER(ctypes.c_double)), ("y", ctypes.POINTER(ctypes.c_double)),
                ("tri", ctypes.POINTER(ctypes.c_int32)), ("Lx", ctypes.c_double),
                ("Ly", ctypes.c_double), ("periodic_x", ctypes.c_int32),
                ("periodic_y", ctypes.c_int32), ("nghost", ctypes.c_int32),
                ("ghost_ids", ctypes.POINTER(ctypes.c_int32)),
                ("ghost_donor", ctypes.POINTER(ctypes.c_int32)),
                ("ghost_flags", ctypes.POINTER(ctypes.c_int32))]


class MeshStats(ctypes.Structure):
    _fields_ = [("nv", ctypes.c_int64), ("nactive", ctypes.c_int64), ("nedges", ctypes.c_int64),
                ("nflux_edges", ctypes.c_int64), ("div_nnz", ctypes.c_int64),
                ("div_nv_total", ctypes.c_int64), ("div_ne_total", ctypes.c_int64),
                ("div_nv_max", ctypes.c_int32), ("div_ne_max", ctypes.c_int32),
                ("rank_hist", ctypes.c_int64 * 16), ("div_degree_fallbacks", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("prep_seconds", ctypes.c_double),
                ("nmember", ctypes.c_int32), ("visc_degree_fallbacks", ctypes.c_int64)]


_P = ctypes.c_void_p
_lib.hfd_last_error.restype = ctypes.c_char_p
_lib.hfd_default_options.argtypes = [ctypes.POINTER(Options)]
_lib.hfd_prep_create.argtypes = [ctypes.POINTER(MeshDesc), ctypes.POINTER(Options), ctypes.POINTER(_P)]
_lib.hfd_prep_destroy.argtypes = [_P]
_lib.hfd_prep_size.argtypes = [_P, ctypes.c_char_p]
_lib.hfd_prep_size.restype = ctypes.c_int64
_lib.hfd_prep_get.argtypes = [_P, ctypes.c_char_p, _P, ctypes.c_int64]
_lib.hfd_prep_set.argtypes = [_P, ctypes.c_char_p, _P, ctypes.c_int64]
_lib.hfd_mesh_create.argtypes = [ctypes.POINTER(MeshDesc), ctypes.POINTER(Options), ctypes.POINTER(_P)]
_lib.hfd_mesh_upload.argtypes = [_P, ctypes.c_int32, ctypes.POINTER(_P)]
_lib.hfd_steps_profiled.argtypes = [_P, _P, ctypes.c_double, ctypes.c_int32, _P,
                                    ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]
_lib.hfd_mesh_destroy.argtypes = [_P]
_lib.hfd_mesh_info.argtypes = [_P, ctypes.POINTER(MeshStats)]
_lib.hfd_mesh_perm.argtypes = [_P, _P]
_lib.hfd_state_import.argtypes = [_P, _P, _P, _P]
_lib.hfd_state_export.argtypes = [_P, _P, _P, _P]
_lib.hfd_residual.argtypes = [_P, _P, _P, _P]
_lib.hfd_residual_static.argtypes = [_P, _P, _P, _P]
_lib.hfd_prep_concat.argtypes = [ctypes.POINTER(_P), ctypes.c_int32, ctypes.POINTER(_P)]
_lib.hfd_mesh_set_launch.argtypes = [_P, ctypes.c_int32, ctypes.c_int32]
_lib.hfd_mesh_autotune.argtypes = [_P, _P, _P, ctypes.POINTER(ctypes.c_int32)]
_lib.hfd_mesh_set_barrier_limit.argtypes = [_P, ctypes.c_uint32]
_lib.hfd_mesh_set_lanes.argtypes = [_P, ctypes.c_int32]
_lib.hfd_mesh_set_div_staged.argtypes = [_P, ctypes.c_int32]
_lib.hfd_mesh_set_fp64_div.argtypes = [_P, ctypes.c_int32]
_lib.hfd_edge_branches.argtypes = [_P, _P, _P, _P]
_lib.hfd_check_conversions.argtypes = [ctypes.c_int64, _P, _P, _P, _P, _P, _P]
_lib.hfd_adjoint.argtypes = [_P, _P, _P, _P, ctypes.c_double, _P]
_lib.hfd_step.argtypes = [_P, _P, ctypes.c_double, _P]
_lib.hfd_batch_create.argtypes = [ctypes.POINTER(_P), ctypes.c_int32, ctypes.c_int32,
                                  ctypes.POINTER(_P)]
_lib.hfd_batch_destroy.argtypes = [_P]
_lib.hfd_batch_mesh.argtypes = [_P, ctypes.POINTER(_P)]
_lib.hfd_batch_step.argtypes = [_P, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_double), _P]
_lib.hfd_steps.argtypes = [_P, _P, ctypes.c_double, ctypes.c_int32, _P]
_lib.hfd_measure_fma_peaks.argtypes = [ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_int32), _P]
_lib.hfd_steps_host.argtypes = [_P, _P, _P, ctypes.c_double, ctypes.c_int32, _P]
_lib.hfd_last_dt.argtypes = [_P, _P, _P]
_lib.hfd_check.argtypes = [_P, _P]


def _ok(status, where):
    if status != HFD_OK:
        raise HfdError(status, where)


def options(**kw):
    """hfd_options with the library defaults, overridden by keyword (precision may be 'fp64' or
    'fp32', flux 'roe' or 'rusanov', force_branch 'sensor', 'hermite' or 'weno'; booleans are
    accepted for viscous/renumber;
    allocator='torch' takes the mesh's device memory from PyTorch's caching allocator)."""
    o = Options()
    _lib.hfd_default_options(ctypes.byref(o))
    alloc = kw.pop("allocator", None)
    if alloc == "torch":              # device blocks from PyTorch's caching allocator
        o.dev_alloc, o.dev_free = TORCH_ALLOC, TORCH_FREE
    elif alloc not in (None, "cuda"):
        raise ValueError(f"allocator must be None, 'cuda' or 'torch', not {alloc!r}")
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = {"fp64": 0, "fp32": 1, "mixed": 1}[v]
        if k == "flux" and isinstance(v, str):
            v = {"roe": 0, "rusanov": 1}[v]
        if k == "force_branch" and isinstance(v, str):
            v = {"sensor": 0, "hermite": 1, "weno": 2}[v]
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, int(v) if isinstance(v, bool) else v)
    return o


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _desc(mesh):
    keep = {
        "x": np.ascontiguousarray(mesh["x"], dtype=np.float64),
        "y": np.ascontiguousarray(mesh["y"], dtype=np.float64),
        "tri": np.ascontiguousarray(mesh["tri"], dtype=np.int32),
        "gi": np.ascontiguousarray(mesh.get("ghost_ids", np.zeros(0)), dtype=np.int32),
        "gd": np.ascontiguousarray(mesh.get("ghost_donor", np.zeros(0)), dtype=np.int32),
        "gf": np.ascontiguousarray(mesh.get("ghost_flags", np.zeros(0)), dtype=np.int32),
    }
    d = MeshDesc()
    d.nv = len(keep["x"])
    d.ntri = len(keep["tri"])
    d.x, d.y = _ptr(keep["x"], ctypes.c_double), _ptr(keep["y"], ctypes.c_double)
    d.tri = _ptr(keep["tri"], ctypes.c_int32)
    d.Lx, d.Ly = float(mesh.get("Lx", 0.0)), float(mesh.get("Ly", 0.0))
    d.periodic_x, d.periodic_y = int(mesh.get("periodic_x", 0)), int(mesh.get("periodic_y", 0))
    d.nghost = len(keep["gi"])
    d.ghost_ids = _ptr(keep["gi"], ctypes.c_int32)
    d.ghost_donor = _ptr(keep["gd"], ctypes.c_int32)
    d.ghost_flags = _ptr(keep["gf"], ctypes.c_int32)
    return d, keep


_INT_ARRAYS = {"edges", "flux_edges", "stencil", "rank", "active", "div_vptr", "div_vidx",
               "div_eptr", "div_eidx", "div_degree", "visc_degree"}


class Prep:
    """Host-only geometric preprocessing (hfd_prep_*): needs no GPU."""

    def __init__(self, mesh, **opts):
        if mesh is None:                      # filled by concat()
            self._h = None
            return
        self.options = options(**opts)
        d, keep = _desc(mesh)
        h = _P()
        _ok(_lib.hfd_prep_create(ctypes.byref(d), ctypes.byref(self.options), ctypes.byref(h)),
            "hfd_prep_create")
        self._h = h

    @classmethod
    def concat(cls, preps):
        """Batch: the disjoint union of several preps (hfd_prep_concat)."""
        arr = (_P * len(preps))(*[p._h for p in preps])
        h = _P()
        _ok(_lib.hfd_prep_concat(arr, len(preps), ctypes.byref(h)), "hfd_prep_concat")
        out = cls(None)
        out._h = h
        return out

    def get(self, name):
        n = _lib.hfd_prep_size(self._h, name.encode())
        if n < 0:
            raise KeyError(name)
        a = np.empty(n, dtype=np.int32 if name in _INT_ARRAYS else np.float64)
        _ok(_lib.hfd_prep_get(self._h, name.encode(), a.ctypes.data, n), "hfd_prep_get")
        return a

    def set(self, name, arr):
        a = np.ascontiguousarray(arr, dtype=np.float64).ravel()
        _ok(_lib.hfd_prep_set(self._h, name.encode(), a.ctypes.data, len(a)), "hfd_prep_set")

    def upload(self, precision=None):
        """Device mesh from this preprocessing (precision: None = as created, 'fp64', 'fp32')."""
        return Mesh(prep=self, precision=precision)

    def close(self):
        if self._h:
            _lib.hfd_prep_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def measure_fma_peaks(stream=None):
    """hfd_measure_fma_peaks: measured FP64 and FP32 FMA throughput of the current device in
    FLOP/s, and its SM count."""
    f64, f32, sms = ctypes.c_double(), ctypes.c_double(), ctypes.c_int32()
    _ok(_lib.hfd_measure_fma_peaks(ctypes.byref(f64), ctypes.byref(f32), ctypes.byref(sms),
                                   _stream(stream)), "hfd_measure_fma_peaks")
    return {"fp64_flops": f64.value, "fp32_flops": f32.value, "sm_count": sms.value}


def check_conversions(x, stream=None):
    """hfd_check_conversions: for a contiguous float64 CUDA tensor x, the integer-only and the
    hardware FP64-to-FP32 roundings of x, and FP32-to-FP64 widenings of the floats held in the
    low 32 bits of x, as (f_int, f_hw, d_int, d_hw) tensors."""
    import torch
    if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float64
            and x.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    n = x.numel()
    f_int = torch.empty(n, dtype=torch.float32, device=x.device)
    f_hw = torch.empty_like(f_int)
    d_int = torch.empty(n, dtype=torch.float64, device=x.device)
    d_hw = torch.empty_like(d_int)
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    _ok(_lib.hfd_check_conversions(n, ptr(x), ptr(f_int), ptr(f_hw), ptr(d_int), ptr(d_hw),
                                   _stream(stream)), "hfd_check_conversions")
    return f_int, f_hw, d_int, d_hw


def _dptr(t):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64
            and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


class Mesh:
    """Device mesh (hfd_mesh_*).  State tensors are 12 x V float64 CUDA tensors in the mesh's
    internal order; import_state / export_state convert from / to the input vertex order."""

    def __init__(self, mesh=None, prep=None, precision=None, **opts):
        h = _P()
        if prep is not None:
            pr = {None: -1, "fp64": 0, "fp32": 1, "mixed": 1, 0: 0, 1: 1}[precision]
            _ok(_lib.hfd_mesh_upload(prep._h, pr, ctypes.byref(h)), "hfd_mesh_upload")
        else:
            if precision is not None:
                opts["precision"] = precision
            self.options = options(**opts)
            d, keep = _desc(mesh)
            _ok(_lib.hfd_mesh_create(ctypes.byref(d), ctypes.byref(self.options), ctypes.byref(h)),
                "hfd_mesh_create")
        self._h = h
        s = MeshStats()
        _ok(_lib.hfd_mesh_info(self._h, ctypes.byref(s)), "hfd_mesh_info")
        self.stats = s
        self.nv, self.nactive = int(s.nv), int(s.nactive)
        self.perm = np.empty(self.nv, dtype=np.int32)
        _ok(_lib.hfd_mesh_perm(self._h, self.perm.ctypes.data), "hfd_mesh_perm")

    def stats_dict(self):
        s = self.stats
        return {k: (list(getattr(s, k)) if k == "rank_hist" else getattr(s, k))
                for k, _ in MeshStats._fields_}

    def import_state(self, U_input, out=None, stream=None):
        import torch
        out = torch.empty_like(U_input) if out is None else out
        _ok(_lib.hfd_state_import(self._h, _dptr(U_input), _dptr(out), _stream(stream)),
            "hfd_state_import")
        return out

    def export_state(self, U_internal, out=None, stream=None):
        import torch
        out = torch.empty_like(U_internal) if out is None else out
        _ok(_lib.hfd_state_export(self._h, _dptr(U_internal), _dptr(out), _stream(stream)),
            "hfd_state_export")
        return out

    def residual(self, U, R=None, stream=None):
        import torch
        R = torch.empty_like(U) if R is None else R
        _ok(_lib.hfd_residual(self._h, _dptr(U), _dptr(R), _stream(stream)), "hfd_residual")
        return R

    def residual_static(self, U, R, stream=None):
        """hfd_residual_static: the residual with the library's fixed scratch array, for callers
        that cannot allocate device memory at call time (R must be preallocated)."""
        _ok(_lib.hfd_residual_static(self._h, _dptr(U), _dptr(R), _stream(stream)),
            "hfd_residual_static")
        return R

    def step(self, U, dt=0.0, stream=None):
        _ok(_lib.hfd_step(self._h, _dptr(U), float(dt), _stream(stream)), "hfd_step")
        return U

    def steps(self, U, dt, n, stream=None):
        _ok(_lib.hfd_steps(self._h, _dptr(U), float(dt), int(n), _stream(stream)), "hfd_steps")
        return U

    def steps_host(self, U_in, U_out, dt, n, stream=None):
        """End-to-end form on host buffers (numpy arrays or CPU tensors, ideally pinned)."""
        def hp(a):
            return ctypes.c_void_p(a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data)
        _ok(_lib.hfd_steps_host(self._h, hp(U_in), hp(U_out), float(dt), int(n), _stream(stream)),
            "hfd_steps_host")
        return U_out

    def steps_profiled(self, U, dt, n, stream=None):
        """Like steps() but kernel by kernel with CUDA events; returns (ms per kernel kind
        {ghost, vertex, edge, div, dt}, number of launches).  Synchronises."""
        ms = (ctypes.c_double * 6)()
        nl = ctypes.c_int64()
        _ok(_lib.hfd_steps_profiled(self._h, _dptr(U), float(dt), int(n), _stream(stream), ms,
                                    ctypes.byref(nl)), "hfd_steps_profiled")
        return (dict(zip(["ghost", "vertex", "edge", "div", "dt", "stage"], list(ms))),
                int(nl.value))

    def adjoint(self, U_n, lam_np1, lam_n=None, dt=None, stream=None):
        """lam_n = (d step(U_n, dt) / d U_n)^T lam_np1 (hfd_adjoint; fixed dt > 0)."""
        import torch
        lam_n = torch.empty_like(lam_np1) if lam_n is None else lam_n
        _ok(_lib.hfd_adjoint(self._h, _dptr(U_n), _dptr(lam_np1), _dptr(lam_n), float(dt),
                             _stream(stream)), "hfd_adjoint")
        return lam_n

    def set_launch(self, persistent, grid=0):
        _ok(_lib.hfd_mesh_set_launch(self._h, int(bool(persistent)), int(grid)),
            "hfd_mesh_set_launch")

    def set_barrier_limit(self, polls):
        _ok(_lib.hfd_mesh_set_barrier_limit(self._h, int(polls)), "hfd_mesh_set_barrier_limit")

    def set_lanes(self, lanes):
        """Lanes per vertex in the divergence gather (1, 2, 4 or 8)."""
        _ok(_lib.hfd_mesh_set_lanes(self._h, int(lanes)), "hfd_mesh_set_lanes")

    def autotune(self, U, stream=None):
        """Pick the fastest launch shape for one RK stage on state U; returns
        (persistent, grid, lanes, staged)."""
        c = (ctypes.c_int32 * 4)()
        _ok(_lib.hfd_mesh_autotune(self._h, _dptr(U), _stream(stream), c), "hfd_mesh_autotune")
        return int(c[0]), int(c[1]), int(c[2]), int(c[3])

    def edge_branches(self, U, stream=None):
        """hfd_edge_branches: per flux edge (the preprocessing's flux-edge order) the byte of
        Alg. 1 branches taken on state U (bit side*4+q: the 3-node WENO value)."""
        out = np.zeros(int(self.stats.nflux_edges), dtype=np.uint8)
        _ok(_lib.hfd_edge_branches(self._h, _dptr(U), out.ctypes.data_as(ctypes.c_void_p),
                                   _stream(stream)), "hfd_edge_branches")
        return out

    def set_fp64_div(self, folded):
        """hfd_mesh_set_fp64_div: the folded double-float FP64 divergence (1) or the plain FP64
        one (0)."""
        _ok(_lib.hfd_mesh_set_fp64_div(self._h, int(folded)), "hfd_mesh_set_fp64_div")

    def set_div_staged(self, staged):
        """hfd_mesh_set_div_staged: the staged FP32 divergence (1) or the unstaged one (0)."""
        _ok(_lib.hfd_mesh_set_div_staged(self._h, int(staged)), "hfd_mesh_set_div_staged")

    def last_dt(self, stream=None):
        """dt of the last step: a float, or one value per member for a batch."""
        n = max(1, int(self.stats.nmember))
        v = (ctypes.c_double * n)()
        _ok(_lib.hfd_last_dt(self._h, v, _stream(stream)), "hfd_last_dt")
        return v[0] if n == 1 else list(v)

    def check(self, stream=None):
        _ok(_lib.hfd_check(self._h, _stream(stream)), "hfd_check")

    def save_state(self, path, U_internal, **extra):
        """Checkpoint: writes the state (exported to input vertex order) and the mesh's vertex
        count to an .npz file, with any extra arrays given by keyword (time, step count, ...)."""
        U = self.export_state(U_internal).cpu().numpy()
        np.savez(path, U=U, nv=np.int64(self.nv), **extra)

    def load_state(self, path):
        """Reads a checkpoint written by save_state; returns (state in internal order on the
        current CUDA device, dict of the extra arrays)."""
        import torch
        with np.load(path) as z:
            if int(z["nv"]) != self.nv or z["U"].shape != (12, self.nv):
                raise ValueError(f"checkpoint of {int(z['nv'])} vertices for a mesh of {self.nv}")
            U = torch.from_numpy(np.ascontiguousarray(z["U"])).cuda()
            extra = {k: z[k] for k in z.files if k not in ("U", "nv")}
        return self.import_state(U), extra

    def close(self):
        if getattr(self, "_h", None):
            _lib.hfd_mesh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Several meshes with one state array per member (hfd_batch_*): each state is a 12 x nv_k
    float64 CUDA tensor in that member's input vertex order, updated in place by step()."""

    def __init__(self, preps, precision=None):
        arr = (_P * len(preps))(*[p._h for p in preps])
        pr = {None: -1, "fp64": 0, "fp32": 1, "mixed": 1, 0: 0, 1: 1}[precision]
        h = _P()
        _ok(_lib.hfd_batch_create(arr, len(preps), pr, ctypes.byref(h)), "hfd_batch_create")
        self._h = h
        self.n = len(preps)

    def step(self, states, dt=None, stream=None):
        """One SSP-RK3 step of every member: dt = None (each member's CFL step) or n steps."""
        if len(states) != self.n:
            raise ValueError(f"{len(states)} states for {self.n} members")
        ptrs = (ctypes.c_void_p * self.n)(*[t.data_ptr() for t in states])
        dts = None if dt is None else (ctypes.c_double * self.n)(*[float(x) for x in dt])
        _ok(_lib.hfd_batch_step(self._h, ptrs, dts, _stream(stream)), "hfd_batch_step")

    def last_dt(self, stream=None):
        """The members' steps of the last step()."""
        m = _P()
        _ok(_lib.hfd_batch_mesh(self._h, ctypes.byref(m)), "hfd_batch_mesh")
        v = (ctypes.c_double * self.n)()
        _ok(_lib.hfd_last_dt(m, v, _stream(stream)), "hfd_last_dt")
        return list(v)

    def close(self):
        if getattr(self, "_h", None):
            _lib.hfd_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

