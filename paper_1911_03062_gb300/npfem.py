"""Python binding of libnpfem.so (ctypes; argument marshalling only).

Every step of the solver runs in the library's CUDA kernels; this module
only converts arrays and pointers.  If the library is missing the import of
:class:`Solver` fails loudly -- there is no CPU fallback.

Arrays use the library's public layout: cell-major in the order cells were
added, each cell ``[nV, 3]`` float64.  Host arrays are numpy; device arrays
are torch CUDA tensors (float64, contiguous), passed by pointer.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnpfem.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "npfem.h")

FP64, MIXED_TF32, MIXED_BF16 = 0, 1, 2
PRECISION = {"fp64": FP64, "tf32": MIXED_TF32, "bf16": MIXED_BF16}

OK, EINVAL, ENOMEM, ENOTSPD, ECUDA, ENONFINITE, ETIMEOUT, ESTATE = 0, -1, -2, -3, -4, -5, -6, -7
_NAMES = {EINVAL: "EINVAL", ENOMEM: "ENOMEM", ENOTSPD: "ENOTSPD", ECUDA: "ECUDA",
          ENONFINITE: "ENONFINITE", ETIMEOUT: "ETIMEOUT", ESTATE: "ESTATE"}


class NpfemError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class Options(C.Structure):
    _fields_ = [("precision", C.c_int), ("iters", C.c_int), ("history", C.c_int),
                ("armijo_c1", C.c_double), ("max_backtracks", C.c_int), ("refine_tol", C.c_double),
                ("refine_max", C.c_int), ("use_graph", C.c_int), ("device", C.c_int),
                ("cuda_stream", C.c_void_p), ("autotune_cache", C.c_char_p), ("residual_fp64", C.c_int),
                ("refine_split", C.c_int), ("force_median", C.c_int), ("u_max", C.c_double),
                ("pbd_kappa", C.c_double), ("pik_radius", C.c_double), ("collision_k", C.c_double)]


class Lattice(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("dx", C.c_double), ("x0", C.c_double),
                ("y0", C.c_double), ("z0", C.c_double)]


class Material(C.Structure):
    _fields_ = [("k_strain", C.c_double), ("k_area", C.c_double), ("k_bend", C.c_double),
                ("k_vol", C.c_double), ("dt", C.c_double), ("rayleigh_alpha", C.c_double),
                ("rayleigh_beta", C.c_double)]


class StepStats(C.Structure):
    _fields_ = [("cell_iterations", C.c_int64), ("backtracks", C.c_int64),
                ("capped_searches", C.c_int64), ("fallbacks", C.c_int64),
                ("refine_sweeps", C.c_int64), ("max_refine_residual", C.c_double),
                ("energy_sum", C.c_double), ("launches_per_step", C.c_int64), ("contacts", C.c_int64)]


KCLASSES = ["predict", "iterate", "fallback", "gemm", "gemm_refine", "residual", "fallback_apply", "filter",
            "contact"]


class KernelTimes(C.Structure):
    _fields_ = [("ms", C.c_double * 9), ("launches", C.c_int64 * 9)]


_lib = None


def header_functions(path: str = HEADER):
    """Names of the functions declared in include/npfem.h."""
    src = open(path).read()
    return sorted(set(re.findall(r"\b(npfem_[a-z_0-9]+)\s*\(", src)))


def load(path: str = LIB_PATH):
    """Load libnpfem.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                           "(the npFEM solver has no CPU fallback)")
    L = C.CDLL(path)
    vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.c_int
    L.npfem_default_options.argtypes = [C.POINTER(Options)]
    L.npfem_create.argtypes = [C.POINTER(Options), C.POINTER(vp)]
    L.npfem_destroy.argtypes = [vp]
    L.npfem_create_mesh_type.argtypes = [vp, ip, vp, ip, vp, vp, C.POINTER(Material), C.POINTER(C.c_int)]
    L.npfem_add_cells.argtypes = [vp, ip, ip, vp, vp, C.POINTER(C.c_int64)]
    L.npfem_num_dofs.argtypes = [vp]
    L.npfem_num_dofs.restype = C.c_size_t
    L.npfem_step.argtypes = [vp, vp, ip]
    L.npfem_sync.argtypes = [vp]
    L.npfem_get_positions.argtypes = [vp, vp, C.c_size_t, ip]
    L.npfem_get_velocities.argtypes = [vp, vp, C.c_size_t, ip]
    L.npfem_set_state.argtypes = [vp, vp, vp, C.c_size_t]
    L.npfem_stats.argtypes = [vp, C.POINTER(StepStats)]
    L.npfem_apply_pinv.argtypes = [vp, ip, vp, vp, ip]
    L.npfem_apply_pinv_noalloc.argtypes = [vp, ip, vp, vp, ip]
    L.npfem_profile.argtypes = [vp, ip]
    L.npfem_ibm_forces.argtypes = [vp, C.POINTER(Lattice), vp, C.c_double, ip, vp, vp]
    L.npfem_profile_read.argtypes = [vp, C.POINTER(KernelTimes), ip]
    L.npfem_last_error.argtypes = [vp]
    L.npfem_last_error.restype = C.c_char_p
    for name in ("npfem_create", "npfem_create_mesh_type", "npfem_add_cells", "npfem_step", "npfem_sync",
                 "npfem_get_positions", "npfem_get_velocities", "npfem_set_state", "npfem_stats",
                 "npfem_apply_pinv", "npfem_apply_pinv_noalloc", "npfem_profile", "npfem_profile_read",
                 "npfem_ibm_forces"):
        getattr(L, name).restype = C.c_int
    _lib = L
    return L


def default_options() -> Options:
    o = Options()
    load().npfem_default_options(C.byref(o))
    return o


def _host(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(C.c_void_p)


def _is_device(a) -> bool:
    return hasattr(a, "is_cuda") and a.is_cuda


def _dev_ptr(t):
    import torch
    if t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError("device arrays must be contiguous float64 CUDA tensors")
    return C.c_void_p(t.data_ptr())


class Solver:
    """One npFEM context: mesh types, cells, and the time step on one GPU."""

    def __init__(self, precision="fp64", iters=10, history=5, armijo_c1=1e-4, max_backtracks=8,
                 refine_tol=1e-6, refine_max=3, use_graph=True, device=0, stream=None, residual_fp64=False,
                 refine_split=True, force_median=False, u_max=0.0, pbd_kappa=0.0, pik_radius=0.0,
                 collision_k=0.0):
        self._L = load()
        o = default_options()
        o.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
        o.iters, o.history, o.armijo_c1 = iters, history, armijo_c1
        o.max_backtracks, o.refine_tol, o.refine_max = max_backtracks, refine_tol, refine_max
        o.use_graph, o.device = int(bool(use_graph)), device
        o.residual_fp64 = int(bool(residual_fp64))
        o.refine_split = int(bool(refine_split))
        o.force_median = int(bool(force_median))
        o.u_max = float(u_max)
        o.pbd_kappa = float(pbd_kappa)
        o.pik_radius = float(pik_radius)
        o.collision_k = float(collision_k)
        if stream is not None:
            o.cuda_stream = C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        self.precision = o.precision
        self._ctx = C.c_void_p()
        self._check(self._L.npfem_create(C.byref(o), C.byref(self._ctx)), ctx=False)
        self.types = []

    # -- errors ---------------------------------------------------------------
    def _check(self, rc, ctx=True):
        if rc != OK:
            msg = self._L.npfem_last_error(self._ctx if ctx else None).decode()
            raise NpfemError(rc, msg)

    def close(self):
        if getattr(self, "_ctx", None):
            self._L.npfem_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- set-up -----------------------------------------------------------------
    def create_mesh_type(self, rest, tris, k_strain, k_area, k_bend, k_vol, dt, mass=None,
                         rayleigh_alpha=0.0, rayleigh_beta=0.0) -> int:
        rest, rp = _host(np.asarray(rest).reshape(-1, 3))
        tris = np.ascontiguousarray(np.asarray(tris).reshape(-1, 3), dtype=np.int32)
        mp = None
        if mass is not None:
            mass, mp = _host(mass)
        mat = Material(k_strain, k_area, k_bend, k_vol, dt, rayleigh_alpha, rayleigh_beta)
        tid = C.c_int()
        self._check(self._L.npfem_create_mesh_type(self._ctx, rest.shape[0], rp, tris.shape[0],
                                                   tris.ctypes.data_as(C.c_void_p), mp, C.byref(mat),
                                                   C.byref(tid)))
        self.types.append(rest.shape[0])
        return tid.value

    def create_type(self, mtype) -> int:
        """Register an inputs.MeshType."""
        m = mtype.material
        return self.create_mesh_type(mtype.rest, mtype.tris, m.k_strain, m.k_area, m.k_bend, m.k_vol,
                                     m.dt, mtype.mass, getattr(m, "rayleigh_alpha", 0.0),
                                     getattr(m, "rayleigh_beta", 0.0))

    def add_cells(self, type_id, x0, v0=None) -> int:
        x0, xp = _host(x0)
        n = x0.size // (3 * self.types[type_id])
        vp = None
        if v0 is not None:
            v0, vp = _host(v0)
        first = C.c_int64()
        self._check(self._L.npfem_add_cells(self._ctx, type_id, n, xp, vp, C.byref(first)))
        return first.value

    @property
    def num_dofs(self) -> int:
        return int(self._L.npfem_num_dofs(self._ctx))

    # -- stepping ---------------------------------------------------------------
    def step(self, f_ext):
        if _is_device(f_ext):
            self._check(self._L.npfem_step(self._ctx, _dev_ptr(f_ext), 1))
        else:
            f, fp = _host(f_ext)
            if f.size != self.num_dofs:
                raise ValueError(f"f_ext has {f.size} values, expected {self.num_dofs}")
            self._check(self._L.npfem_step(self._ctx, fp, 0))

    def sync(self):
        self._check(self._L.npfem_sync(self._ctx))

    def _get(self, fn, out):
        n = self.num_dofs
        if out is not None and _is_device(out):
            self._check(fn(self._ctx, _dev_ptr(out), n, 1))
            return out
        if out is None:
            out = np.empty(n)
        self._check(fn(self._ctx, out.ctypes.data_as(C.c_void_p), n, 0))
        return out

    def positions(self, out=None):
        return self._get(self._L.npfem_get_positions, out)

    def velocities(self, out=None):
        return self._get(self._L.npfem_get_velocities, out)

    def set_state(self, x, v=None):
        x, xp = _host(x)
        vp = None
        if v is not None:
            v, vp = _host(v)
        self._check(self._L.npfem_set_state(self._ctx, xp, vp, x.size))

    def stats(self) -> dict:
        s = StepStats()
        self._check(self._L.npfem_stats(self._ctx, C.byref(s)))
        return {k: getattr(s, k) for k, _ in StepStats._fields_}

    def apply_pinv_noalloc(self, type_id, q, z):
        """As apply_pinv, with the library's static scratch instead of allocations."""
        n_cols = q.shape[0]
        self._check(self._L.npfem_apply_pinv_noalloc(self._ctx, type_id, _dev_ptr(q), _dev_ptr(z), n_cols))
        return z

    def ibm_forces(self, u, origin, dx, dt, cycles=1, f_lagr=None, f_grid=None):
        """Immersed-boundary forces (multi-direct forcing) of every vertex from the fluid
        velocity u (torch float64 on the device, [3, nz, ny, nx], nodes origin + (i, j, k) dx).
        Returns (f_lagr [num_dofs], f_grid like u), both device tensors, after the
        context's stream has finished them (the call synchronises it)."""
        import torch
        if u.dim() != 4 or u.shape[0] != 3:
            raise ValueError("u must be [3, nz, ny, nx]")
        _, nz, ny, nx = u.shape
        if f_lagr is None:
            f_lagr = torch.empty(self.num_dofs, dtype=torch.float64, device=u.device)
        if f_grid is None:
            f_grid = torch.empty_like(u)
        if f_lagr.numel() != self.num_dofs or tuple(f_grid.shape) != tuple(u.shape):
            raise ValueError("f_lagr must hold num_dofs values and f_grid the shape of u")
        lat = Lattice(nx, ny, nz, float(dx), float(origin[0]), float(origin[1]), float(origin[2]))
        self._check(self._L.npfem_ibm_forces(self._ctx, C.byref(lat), _dev_ptr(u), float(dt), int(cycles),
                                             _dev_ptr(f_lagr), _dev_ptr(f_grid)))
        self._check(self._L.npfem_sync(self._ctx))
        return f_lagr, f_grid

    def profile(self, enable: bool):
        self._check(self._L.npfem_profile(self._ctx, int(bool(enable))))

    def profile_read(self, reset=True) -> dict:
        k = KernelTimes()
        self._check(self._L.npfem_profile_read(self._ctx, C.byref(k), int(bool(reset))))
        return {n: (k.ms[i], k.launches[i]) for i, n in enumerate(KCLASSES) if k.launches[i]}

    def apply_pinv(self, type_id, q, z):
        """z = P^{-1} q on the device (torch float64 tensors, [n_cols, nV])."""
        n_cols = q.shape[0]
        self._check(self._L.npfem_apply_pinv(self._ctx, type_id, _dev_ptr(q), _dev_ptr(z), n_cols))
        return z
