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
                ("pbd_kappa", C.c_double), ("pik_radius", C.c_double), ("collision_k", C.c_double),
                ("curvature_tol", C.c_double)]


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
    L.npfem_check_wait.argtypes = [vp, ip]
    L.npfem_ibm_forces.argtypes = [vp, C.POINTER(Lattice), vp, C.c_double, ip, vp, vp]
    L.npfem_profile_read.argtypes = [vp, C.POINTER(KernelTimes), ip]
    L.npfem_last_error.argtypes = [vp]
    L.npfem_last_error.restype = C.c_char_p
    for name in ("npfem_create", "npfem_create_mesh_type", "npfem_add_cells", "npfem_step", "npfem_sync",
                 "npfem_get_positions", "npfem_get_velocities", "npfem_set_state", "npfem_stats",
                 "npfem_apply_pinv", "npfem_apply_pinv_noalloc", "npfem_profile", "npfem_profile_read",
                 "npfem_ibm_forces", "npfem_check_wait"):
        getattr(L, name).restype = C.c_int
    _lib = L
    return L


def default_options() -> Options:
    o = Options()
    load().npfem_default_options(C.byref(o))
    return o


def _host(a, n=None, what="array"):
    """Contiguous float64 copy (or view) of a host array and its pointer; n: required size."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None and a.size != n:
        raise ValueError(f"{what} has {a.size} values, expected {n}")
    return a, a.ctypes.data_as(C.c_void_p)


def _is_device(a) -> bool:
    return hasattr(a, "is_cuda") and a.is_cuda


def _dev_ptr(t, device, numel=None, shape=None, what="tensor"):
    """Pointer of a device tensor after checking what the library will assume of it:
    a contiguous float64 CUDA tensor on the context's device, of the given size or shape.
    Raises ValueError before any pointer reaches the library."""
    if not _is_device(t):
        raise ValueError(f"{what} must be a CUDA tensor")
    if str(t.dtype) != "torch.float64" or not t.is_contiguous():
        raise ValueError(f"{what} must be a contiguous float64 CUDA tensor")
    if t.device.index != device:
        raise ValueError(f"{what} is on cuda:{t.device.index}, the context on cuda:{device}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{what} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{what} has {t.numel()} values, expected {numel}")
    return C.c_void_p(t.data_ptr())


class Solver:
    """One npFEM context: mesh types, cells, and the time step on one GPU.

    Stream order: the context runs on one CUDA stream (``stream``, or a stream this
    object creates).  Every call that takes caller device tensors first makes that
    stream wait for the caller's current torch stream (so tensors written there are
    complete) and afterwards makes the current torch stream wait for the context's
    stream (so later torch work on those tensors, or their release to the caching
    allocator, comes after the library's reads and writes)."""

    def __init__(self, precision="fp64", iters=10, history=5, armijo_c1=1e-4, max_backtracks=8,
                 refine_tol=1e-6, refine_max=3, use_graph=True, device=0, stream=None, residual_fp64=False,
                 refine_split=True, force_median=False, u_max=0.0, pbd_kappa=0.0, pik_radius=0.0,
                 collision_k=0.0, curvature_tol=1e-12, autotune_cache=None):
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
        o.curvature_tol = float(curvature_tol)
        self._cache_path = None if autotune_cache is None else os.fsencode(autotune_cache)
        o.autotune_cache = self._cache_path
        self.device = int(device)
        self._stream = None
        import torch
        if stream is not None:
            self._stream = stream if hasattr(stream, "cuda_stream") else \
                torch.cuda.ExternalStream(int(stream), device=torch.device("cuda", self.device))
        elif torch.cuda.is_available():
            self._stream = torch.cuda.Stream(device=self.device)
        if self._stream is not None:
            o.cuda_stream = C.c_void_p(self._stream.cuda_stream)
        self.precision = o.precision
        self._ctx = C.c_void_p()
        self._check(self._L.npfem_create(C.byref(o), C.byref(self._ctx)), ctx=False)
        self.types = []

    # -- errors and stream order ------------------------------------------------
    def _check(self, rc, ctx=True):
        if rc != OK:
            msg = self._L.npfem_last_error(self._ctx if ctx else None).decode()
            raise NpfemError(rc, msg)

    def _torch_stream(self):
        import torch
        return torch.cuda.current_stream(self.device)

    def _enter(self):
        """The context stream waits for the caller's work on the current torch stream."""
        self._stream.wait_stream(self._torch_stream())

    def _leave(self):
        """The current torch stream waits for the context stream's work so far."""
        self._torch_stream().wait_stream(self._stream)

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
        rest, rp = _host(np.asarray(rest, dtype=np.float64).reshape(-1, 3))
        tris = np.ascontiguousarray(np.asarray(tris).reshape(-1, 3), dtype=np.int32)
        mp = None
        if mass is not None:
            mass, mp = _host(mass, rest.shape[0], "mass")
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

    def _nV(self, type_id):
        if not 0 <= type_id < len(self.types):
            raise ValueError(f"unknown mesh type {type_id}")
        return self.types[type_id]

    def add_cells(self, type_id, x0, v0=None) -> int:
        per = 3 * self._nV(type_id)
        x0, xp = _host(x0)
        if x0.size % per:
            raise ValueError(f"x0 has {x0.size} values, not a multiple of 3 nV = {per}")
        n = x0.size // per
        vp = None
        if v0 is not None:
            v0, vp = _host(v0, x0.size, "v0")
        first = C.c_int64()
        self._check(self._L.npfem_add_cells(self._ctx, type_id, n, xp, vp, C.byref(first)))
        return first.value

    @property
    def num_dofs(self) -> int:
        return int(self._L.npfem_num_dofs(self._ctx))

    # -- stepping ---------------------------------------------------------------
    def step(self, f_ext):
        """One time step under f_ext (num_dofs values): a host array (copied during the
        call) or a device tensor read on the context's stream after the caller's
        current-stream work; the call returns once the step is enqueued."""
        if _is_device(f_ext):
            p = _dev_ptr(f_ext, self.device, numel=self.num_dofs, what="f_ext")
            self._enter()
            self._check(self._L.npfem_step(self._ctx, p, 1))
            self._leave()
        else:
            f, fp = _host(f_ext, self.num_dofs, "f_ext")
            self._check(self._L.npfem_step(self._ctx, fp, 0))

    def sync(self):
        self._check(self._L.npfem_sync(self._ctx))

    def _get(self, fn, out):
        n = self.num_dofs
        if out is not None and _is_device(out):
            p = _dev_ptr(out, self.device, numel=n, what="out")
            self._enter()
            self._check(fn(self._ctx, p, n, 1))
            self._leave()
            return out
        if out is None:
            out = np.empty(n)
        if not (isinstance(out, np.ndarray) and out.dtype == np.float64 and out.flags.c_contiguous
                and out.size == n):
            raise ValueError(f"out must be a contiguous float64 numpy array or CUDA tensor of {n} values")
        self._check(fn(self._ctx, out.ctypes.data_as(C.c_void_p), out.size, 0))
        return out

    def positions(self, out=None):
        return self._get(self._L.npfem_get_positions, out)

    def velocities(self, out=None):
        return self._get(self._L.npfem_get_velocities, out)

    def set_state(self, x, v=None):
        x, xp = _host(x, self.num_dofs, "x")
        vp = None
        if v is not None:
            v, vp = _host(v, x.size, "v")
        self._check(self._L.npfem_set_state(self._ctx, xp, vp, x.size))

    def stats(self) -> dict:
        s = StepStats()
        self._check(self._L.npfem_stats(self._ctx, C.byref(s)))
        return {k: getattr(s, k) for k, _ in StepStats._fields_}

    def _apply_args(self, type_id, q, z):
        nV = self._nV(type_id)
        if getattr(q, "dim", lambda: 0)() != 2:
            raise ValueError("q must be a 2-D [n_cols, nV] tensor")
        shape = (q.shape[0], nV)
        pq = _dev_ptr(q, self.device, shape=shape, what="q")
        pz = _dev_ptr(z, self.device, shape=shape, what="z")
        return pq, pz, q.shape[0]

    def apply_pinv(self, type_id, q, z):
        """z = P^{-1} q on the device (float64 CUDA tensors [n_cols, nV]); returns z,
        complete on the caller's current stream."""
        pq, pz, n_cols = self._apply_args(type_id, q, z)
        self._enter()
        self._check(self._L.npfem_apply_pinv(self._ctx, type_id, pq, pz, n_cols))
        self._leave()
        return z

    def apply_pinv_noalloc(self, type_id, q, z):
        """As apply_pinv, with the library's static scratch instead of allocations."""
        pq, pz, n_cols = self._apply_args(type_id, q, z)
        self._enter()
        self._check(self._L.npfem_apply_pinv_noalloc(self._ctx, type_id, pq, pz, n_cols))
        self._leave()
        return z

    def ibm_forces(self, u, origin, dx, dt, cycles=1, f_lagr=None, f_grid=None):
        """Immersed-boundary forces (multi-direct forcing) of every vertex from the fluid
        velocity u (torch float64 on the device, [3, nz, ny, nx], nodes origin + (i, j, k) dx).
        Returns (f_lagr [num_dofs], f_grid like u), both device tensors, after the
        context's stream has finished them (the call synchronises it)."""
        import torch
        if not _is_device(u) or u.dim() != 4 or u.shape[0] != 3:
            raise ValueError("u must be a [3, nz, ny, nx] CUDA tensor")
        _, nz, ny, nx = u.shape
        if f_lagr is None:
            f_lagr = torch.empty(self.num_dofs, dtype=torch.float64, device=u.device)
        if f_grid is None:
            f_grid = torch.empty_like(u)
        pu = _dev_ptr(u, self.device, what="u")
        pl = _dev_ptr(f_lagr, self.device, numel=self.num_dofs, what="f_lagr")
        pg = _dev_ptr(f_grid, self.device, shape=tuple(u.shape), what="f_grid")
        lat = Lattice(nx, ny, nz, float(dx), float(origin[0]), float(origin[1]), float(origin[2]))
        self._enter()
        self._check(self._L.npfem_ibm_forces(self._ctx, C.byref(lat), pu, float(dt), int(cycles), pl, pg))
        self._check(self._L.npfem_sync(self._ctx))
        self._leave()
        return f_lagr, f_grid

    def check_wait(self, limit_ms=50):
        """Enqueue the failure-path self-check: a bounded device wait that expires; the
        next synchronising call raises NpfemError(ETIMEOUT)."""
        self._check(self._L.npfem_check_wait(self._ctx, int(limit_ms)))

    def profile(self, enable: bool):
        self._check(self._L.npfem_profile(self._ctx, int(bool(enable))))

    def profile_read(self, reset=True) -> dict:
        k = KernelTimes()
        self._check(self._L.npfem_profile_read(self._ctx, C.byref(k), int(bool(reset))))
        return {n: (k.ms[i], k.launches[i]) for i, n in enumerate(KCLASSES) if k.launches[i]}
