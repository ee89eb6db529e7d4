"""ctypes binding of the FP64 CPU oracle (npfem_oracle.c).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the CPU
baseline of bench.py are the only users.  Nothing in the product package
imports this module.

Layout of every per-cell array: [nV, 3] float64 (vertex major, xyz inner).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "npfem_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

TERM_INERTIA, TERM_STRAIN, TERM_AREA, TERM_BEND, TERM_VOLUME = 1, 2, 4, 8, 16
TERM_ALL = 31

_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, -O2, no vector intrinsics)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c99", "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(LIB)
            dp = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
            ip = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
            vp = C.c_void_p
            L.orc_type_create.argtypes = [C.c_int, dp, C.c_int, ip, vp, C.c_double, C.c_double,
                                          C.c_double, C.c_double, C.c_double, C.POINTER(vp)]
            L.orc_type_create.restype = C.c_int
            L.orc_type_destroy.argtypes = [vp]
            L.orc_type_info.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_double),
                                        C.POINTER(C.c_int), C.POINTER(C.c_long)]
            L.orc_P_dense.argtypes = [vp, dp]
            L.orc_hinges.argtypes = [vp, ip, dp, dp]
            L.orc_solve.argtypes = [vp, dp, dp]
            L.orc_energy.argtypes = [vp, dp, dp, C.c_int, vp, vp]
            L.orc_energy.restype = C.c_double
            L.orc_polar.argtypes = [dp, dp, dp]
            L.orc_area_project.argtypes = [dp, dp, dp]
            L.orc_area_target.argtypes = [C.c_double, C.c_double, dp]
            L.orc_volume_project.argtypes = [vp, dp, dp]
            L.orc_volume_project.restype = C.c_int
            L.orc_volume.argtypes = [vp, dp]
            L.orc_volume.restype = C.c_double
            L.orc_volume_grad.argtypes = [vp, dp, dp]
            L.orc_step.argtypes = [vp, dp, dp, dp, C.c_int, C.c_int, C.c_double, C.c_int,
                                   dp, dp, vp, vp, vp, vp]
            L.orc_step.restype = C.c_int
            L.orc_step_trace.argtypes = [vp, dp, dp, dp, C.c_int, C.c_int, C.c_double, C.c_int, C.c_double,
                                         dp, dp, dp, dp, ip, ip, dp, dp, dp, ip]
            L.orc_step_trace.restype = C.c_int
            L.orc_step_cells.argtypes = [vp, C.c_int, vp, vp, vp, C.c_int, C.c_int, C.c_double,
                                         C.c_int, vp, vp]
            L.orc_step_cells.restype = C.c_int
            L.orc_force_median.argtypes = [vp, dp, dp]
            L.orc_force_median.restype = C.c_int
            L.orc_velocity_cap.argtypes = [C.c_int, dp, C.c_double]
            L.orc_pbd_damping.argtypes = [vp, dp, dp, C.c_double]
            L.orc_pbd_damping.restype = C.c_int
            L.orc_type_set_damping.argtypes = [vp, C.c_double, C.c_double]
            L.orc_type_set_damping.restype = C.c_int
            L.orc_vertex_normals.argtypes = [vp, dp, dp]
            L.orc_pik.argtypes = [C.c_int, ip, vp, vp, C.c_double, ip, ip, dp]
            L.orc_pik.restype = C.c_int
            L.orc_energy_col.argtypes = [vp, dp, dp, C.c_int, vp, vp, C.c_double, ip, dp]
            L.orc_energy_col.restype = C.c_double
            L.orc_step_cells_col.argtypes = [vp, C.c_int, vp, vp, vp, C.c_int, C.c_int, C.c_double,
                                             C.c_int, C.c_double, vp, vp, vp, vp]
            L.orc_step_cells_col.restype = C.c_int
            L.orc_phi4.argtypes = [C.c_double]
            L.orc_phi4.restype = C.c_double
            L.orc_vertex_areas.argtypes = [vp, dp, dp]
            L.orc_ibm.argtypes = [C.c_int, dp, dp, dp, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                  C.c_double, C.c_double, dp, C.c_double, C.c_int, dp, dp]
            L.orc_ibm.restype = C.c_int
            _lib = L
    return _lib


def _c(a, dtype=np.float64):
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class OracleType:
    """One mesh type: rest shape, topology, material, time step; owns P and its factor."""

    def __init__(self, rest, tris, k_strain, k_area, k_bend, k_vol, dt, mass=None):
        L = lib()
        self.rest = _c(rest).reshape(-1, 3)
        self.tris = _c(tris, np.int32).reshape(-1, 3)
        self.nV, self.nT = self.rest.shape[0], self.tris.shape[0]
        self.dt = float(dt)
        self.mass = None if mass is None else _c(mass)
        h = C.c_void_p()
        rc = L.orc_type_create(self.nV, self.rest, self.nT, self.tris, _ptr(self.mass),
                               k_strain, k_area, k_bend, k_vol, dt, C.byref(h))
        if rc != 0:
            raise ValueError(f"oracle type creation failed ({rc})")
        self._h = h
        nH, V0, nnz, nnzL = C.c_int(), C.c_double(), C.c_int(), C.c_long()
        L.orc_type_info(h, C.byref(nH), C.byref(V0), C.byref(nnz), C.byref(nnzL))
        self.nH, self.V0, self.nnzP, self.nnzL = nH.value, V0.value, nnz.value, nnzL.value

    @classmethod
    def from_mesh_type(cls, mt):
        m = mt.material
        T = cls(mt.rest, mt.tris, m.k_strain, m.k_area, m.k_bend, m.k_vol, m.dt, mt.mass)
        a, b = getattr(m, "rayleigh_alpha", 0.0), getattr(m, "rayleigh_beta", 0.0)
        return T.set_damping(a, b) if (a or b) else T

    def __del__(self):
        try:
            if getattr(self, "_h", None) is not None:
                lib().orc_type_destroy(self._h)
        except Exception:
            pass

    def set_damping(self, alpha, beta):
        """Rayleigh damping C = alpha M + beta L (Sec. 2.1): rebuilds P and factors
        Mt = M + h C for the predictor; (0, 0) is the undamped type."""
        rc = lib().orc_type_set_damping(self._h, float(alpha), float(beta))
        if rc != 0:
            raise ValueError(f"oracle damping set-up failed ({rc})")
        self.alpha, self.beta = float(alpha), float(beta)
        return self

    # -- pieces -------------------------------------------------------------
    def P_dense(self):
        P = np.empty((self.nV, self.nV))
        lib().orc_P_dense(self._h, P)
        return P

    def hinges(self):
        hv = np.empty((self.nH, 4), np.int32)
        hc = np.empty((self.nH, 4))
        hr = np.empty(self.nH)
        lib().orc_hinges(self._h, hv, hc, hr)
        return hv, hc, hr

    def solve(self, b):
        b = _c(b).reshape(self.nV, 3)
        x = np.empty_like(b)
        lib().orc_solve(self._h, b, x)
        return x

    def energy(self, x, y, mask=TERM_ALL, grad=True):
        x = _c(x).reshape(self.nV, 3)
        y = _c(y).reshape(self.nV, 3)
        g = np.empty_like(x) if grad else None
        terms = np.empty(5)
        e = lib().orc_energy(self._h, x, y, mask, _ptr(g), _ptr(terms))
        return e, g, terms

    def energy_col(self, x, y, kc, hit, p, mask=TERM_ALL, grad=True):
        """g with the PIK collision term kc/2 |x_v - p_v|^2 over the vertices with hit != 0."""
        x = _c(x).reshape(self.nV, 3)
        y = _c(y).reshape(self.nV, 3)
        g = np.empty_like(x) if grad else None
        terms = np.empty(5)
        e = lib().orc_energy_col(self._h, x, y, mask, _ptr(g), _ptr(terms), kc,
                                 _c(hit, np.int32), _c(p).reshape(self.nV, 3))
        return e, g, terms

    def normals(self, x):
        """Area-weighted outward vertex normals, normalised ([nV, 3])."""
        x = _c(x).reshape(self.nV, 3)
        n = np.empty_like(x)
        lib().orc_vertex_normals(self._h, x, n)
        return n

    def vertex_areas(self, x):
        """A third of the incident triangles' areas per vertex ([nV])."""
        a = np.empty(self.nV)
        lib().orc_vertex_areas(self._h, _c(x).reshape(self.nV, 3), a)
        return a

    def volume(self, p):
        return lib().orc_volume(self._h, _c(p).reshape(self.nV, 3))

    def volume_grad(self, p):
        g = np.empty((self.nV, 3))
        lib().orc_volume_grad(self._h, _c(p).reshape(self.nV, 3), g)
        return g

    def volume_project(self, x):
        x = _c(x).reshape(self.nV, 3)
        p = np.empty_like(x)
        it = lib().orc_volume_project(self._h, x, p)
        return p, it

    # -- time step ----------------------------------------------------------
    def step(self, xn, vn, f, K=10, m=5, c1=1e-4, max_bt=8, trace=False):
        xn, vn, f = (_c(a).reshape(self.nV, 3) for a in (xn, vn, f))
        xo, vo = np.empty_like(xn), np.empty_like(xn)
        if trace:
            gt, at = np.empty(K + 1), np.empty(K)
            bt, fb = np.empty(K, np.int32), np.empty(K, np.int32)
            caps = lib().orc_step(self._h, xn, vn, f, K, m, c1, max_bt, xo, vo,
                                  _ptr(gt), _ptr(at), _ptr(bt), _ptr(fb))
            return xo, vo, dict(g=gt, alpha=at, backtracks=bt, fallback=fb, caps=caps)
        lib().orc_step(self._h, xn, vn, f, K, m, c1, max_bt, xo, vo, None, None, None, None)
        return xo, vo

    def step_trace(self, xn, vn, f, K=10, m=5, c1=1e-4, max_bt=8, curv_tol=1e-12):
        """One step with the full per-iteration record: iterates x [K+1, nV, 3] (x[0] = y),
        gradients g [K+1, nV, 3], directions d [K, nV, 3], kept [K] (the pair of iteration
        k entered the history), energies, alphas, halvings, fallbacks and the cap count.
        ``curv_tol`` is the history's curvature threshold (the method's is 1e-12)."""
        xn, vn, f = (_c(a).reshape(self.nV, 3) for a in (xn, vn, f))
        xo, vo = np.empty_like(xn), np.empty_like(xn)
        gt, at = np.empty(K + 1), np.empty(K)
        bt, fb, kept = np.empty(K, np.int32), np.empty(K, np.int32), np.empty(K, np.int32)
        xs, gs, ds = np.empty((K + 1, self.nV, 3)), np.empty((K + 1, self.nV, 3)), np.empty((K, self.nV, 3))
        caps = lib().orc_step_trace(self._h, xn, vn, f, K, m, c1, max_bt, float(curv_tol), xo, vo,
                                    gt, at, bt, fb, xs, gs, ds, kept)
        return xo, vo, dict(g=gt, alpha=at, backtracks=bt, fallback=fb, caps=caps, x=xs, grad=gs, d=ds,
                            kept=kept)

    def step_cells_col(self, xn, vn, f, kc, hit, p, K=10, m=5, c1=1e-4, max_bt=8):
        """Step n cells with the PIK collision term: hit [n, nV] (nonzero = contaminated
        vertex: fluid force dropped, kc/2 |x - p|^2 added), p [n, nV, 3] targets."""
        xn, vn, f, p = (_c(a).reshape(-1, self.nV, 3) for a in (xn, vn, f, p))
        hit = _c(hit, np.int32).reshape(-1, self.nV)
        xo, vo = np.empty_like(xn), np.empty_like(xn)
        lib().orc_step_cells_col(self._h, xn.shape[0], _ptr(xn), _ptr(vn), _ptr(f), K, m, c1, max_bt, kc,
                                 _ptr(hit), _ptr(p), _ptr(xo), _ptr(vo))
        return xo, vo

    def step_cells(self, xn, vn, f, K=10, m=5, c1=1e-4, max_bt=8, threads=1):
        """Step n cells ([n, nV, 3]); ``threads`` host threads split the cells."""
        xn, vn, f = (_c(a).reshape(-1, self.nV, 3) for a in (xn, vn, f))
        n = xn.shape[0]
        xo, vo = np.empty_like(xn), np.empty_like(xn)
        L = lib()
        threads = max(1, min(threads, n))
        bounds = np.linspace(0, n, threads + 1).astype(int)

        def run(a, b):
            if b > a:
                L.orc_step_cells(self._h, b - a, _ptr(xn[a:b]), _ptr(vn[a:b]), _ptr(f[a:b]),
                                 K, m, c1, max_bt, _ptr(xo[a:b]), _ptr(vo[a:b]))

        if threads == 1:
            run(0, n)
        else:
            ts = [threading.Thread(target=run, args=(bounds[i], bounds[i + 1])) for i in range(threads)]
            for t in ts:
                t.start()
            for t in ts:
                t.join()
        return xo, vo


def force_median(T, f):
    """One-ring median filter of per-vertex forces ([n, nV, 3] or [nV, 3])."""
    f = _c(f)
    flat = f.reshape(-1, T.nV, 3)
    out = np.empty_like(flat)
    for c in range(flat.shape[0]):
        src = np.ascontiguousarray(flat[c])
        dst = np.empty_like(src)
        if lib().orc_force_median(T._h, src, dst) != 0:
            raise MemoryError("orc_force_median")
        out[c] = dst
    return out.reshape(f.shape)


def velocity_cap(v, umax):
    """Copy of per-vertex velocities ([..., 3]) with |v| > umax scaled to umax."""
    out = _c(v).copy()
    flat = out.reshape(-1, 3)
    lib().orc_velocity_cap(flat.shape[0], flat, float(umax))
    return out


def pbd_damping(T, x, v, kappa):
    """Copy of the velocities of cells ([n, nV, 3] or [nV, 3]) after PBD damping."""
    xs = _c(x).reshape(-1, T.nV, 3)
    out = _c(v).copy().reshape(-1, T.nV, 3)
    for c in range(xs.shape[0]):
        vc = np.ascontiguousarray(out[c])
        if lib().orc_pbd_damping(T._h, np.ascontiguousarray(xs[c]), vc, float(kappa)) != 0:
            raise ValueError("singular inertia tensor")
        out[c] = vc
    return out.reshape(np.shape(v))


def polar(F):
    F = _c(F).reshape(3, 2)
    T, s = np.empty((3, 2)), np.empty(2)
    lib().orc_polar(F, T, s)
    return T, s


def area_project(F):
    F = _c(F).reshape(3, 2)
    P, d = np.empty((3, 2)), np.empty(2)
    lib().orc_area_project(F, P, d)
    return P, d


def area_target(s1, s2):
    d = np.empty(2)
    lib().orc_area_target(float(s1), float(s2), d)
    return d


def predictor(xn, vn, f, dt, nV, mass=None):
    """y = x_n + h v_n + h^2 M^{-1} F_ext (Eq. genericOptimizationNewton, C = 0)."""
    m = (1.0 / nV) if mass is None else np.asarray(mass)[:, None]
    return xn + dt * vn + dt * dt / m * f


def pik(cells, rk):
    """Particle-in-kernel search over all cells (list of (OracleType, x [nV, 3])):
    returns per cell (hit_cell [nV], hit_vert [nV], p [nV, 3]) with -1 where no
    foreign vertex lies within rk, and the targets p (x where none)."""
    xs = [_c(x).reshape(T.nV, 3) for T, x in cells]
    ns = [T.normals(x) for (T, _), x in zip(cells, xs)]
    nV = np.array([T.nV for T, _ in cells], np.int32)
    tot = int(nV.sum())
    hc, hv = np.empty(tot, np.int32), np.empty(tot, np.int32)
    p = np.empty((tot, 3))
    xp = (C.c_void_p * len(cells))(*[x.ctypes.data for x in xs])
    npp = (C.c_void_p * len(cells))(*[n.ctypes.data for n in ns])
    rc = lib().orc_pik(len(cells), nV, C.cast(xp, C.c_void_p), C.cast(npp, C.c_void_p), float(rk), hc, hv, p)
    if rc != 0:
        raise ValueError(f"orc_pik failed ({rc})")
    out, o = [], 0
    for T, _ in cells:
        out.append((hc[o:o + T.nV], hv[o:o + T.nV], p[o:o + T.nV]))
        o += T.nV
    return out


def pik_step(cells, f, rk, kc, K=10, m=5):
    """One step of every cell with the PIK collision framework: the search on the
    state at the start of the step, then each cell's step with its targets.
    cells: list of (OracleType, x, v); f: list of forces.  Returns [(x1, v1)]."""
    res = pik([(T, x) for T, x, _ in cells], rk)
    out = []
    for (T, x, v), fc, (hc, _, p) in zip(cells, f, res):
        xo, vo = T.step_cells_col(x[None], v[None], fc[None], kc, (hc >= 0).astype(np.int32)[None], p[None],
                                  K=K, m=m)
        out.append((xo[0], vo[0]))
    return out


def phi4(r):
    """Peskin's four-point kernel function."""
    return lib().orc_phi4(float(r))


def ibm(X, U, A, u, origin, dx, dt, cycles):
    """Multi-direct forcing (supplementary IBM section): Lagrangian points X, U [N, 3],
    areas A [N]; fluid velocity u [3, nz, ny, nx] on nodes origin + (i, j, k) dx.
    Returns (f [N, 3], F_imm [3, nz, ny, nx])."""
    X, U, A = _c(X).reshape(-1, 3), _c(U).reshape(-1, 3), _c(A).ravel()
    u = _c(u)
    _, nz, ny, nx = u.shape
    f = np.empty_like(X)
    F = np.empty_like(u)
    rc = lib().orc_ibm(X.shape[0], X, U, A, nx, ny, nz, float(dx), float(origin[0]), float(origin[1]),
                       float(origin[2]), u.ravel(), float(dt), int(cycles), f, F.ravel())
    if rc != 0:
        raise ValueError(f"orc_ibm failed ({rc})")
    return f, F
