"""Seeded synthetic inputs for the npFEM cell-suspension workloads.

This module is shared by the FP64 CPU oracle (tests) and by the CUDA path
(tests, bench).  It holds no arithmetic of the method itself: it only builds

* closed triangle meshes (icospheres) and the rest shapes mapped onto them
  (Evans-Fung biconcave red blood cell, oblate-ellipsoid platelet);
* cell placements (uniform position in a box, uniform random rotation);
* per-vertex external forces (seeded random Fourier modes plus a uniform
  shear), which stand in for the immersed-boundary forces of the coupled
  flow runs (the paper's F_ext, Supplementary Sec. 2.1), since those come
  from a fluid solver that is not part of this path.

Everything is seeded; numpy's PCG64 generator makes the draws identical on
x86 and Arm.  Arrays use the public layout of the library: per cell, vertex
major, xyz innermost (``[n_cells, nV, 3]`` float64).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# Evans & Fung (1972) biconcave profile constants; radius in the paper's
# non-dimensional units (about 7.8 um diameter).
RBC_R0 = 3.91
RBC_C0 = 0.207161
RBC_C1 = 2.002558
RBC_C2 = -1.122762
# Platelet: oblate ellipsoid, semi-axes (1.8, 1.8, 0.5).
PLT_AXES = (1.8, 1.8, 0.5)


# --------------------------------------------------------------------------
# meshes
# --------------------------------------------------------------------------
def icosahedron():
    """12 unit vertices and 20 outward-CCW faces, in a fixed order."""
    phi = (1.0 + 5.0 ** 0.5) / 2.0
    v = []
    for a in (-1.0, 1.0):
        for b in (-phi, phi):
            v.append((0.0, a, b))
            v.append((a, b, 0.0))
            v.append((b, 0.0, a))
    v = np.array(v, dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    d = np.linalg.norm(v[:, None, :] - v[None, :, :], axis=2)
    edge = np.min(d[d > 1e-9])
    adj = np.abs(d - edge) < 1e-9
    faces = []
    n = len(v)
    for i in range(n):
        for j in range(i + 1, n):
            if not adj[i, j]:
                continue
            for k in range(j + 1, n):
                if adj[i, k] and adj[j, k]:
                    f = [i, j, k]
                    nrm = np.cross(v[j] - v[i], v[k] - v[i])
                    if np.dot(nrm, v[i] + v[j] + v[k]) < 0:
                        f = [i, k, j]
                    faces.append(f)
    assert len(faces) == 20
    return v, np.array(faces, dtype=np.int32)


def icosphere(level: int):
    """Unit icosphere: 4-way split of every face ``level`` times.

    Midpoints are shared by edge key (min, max) and projected to the unit
    sphere; vertices are numbered in creation order; faces stay CCW seen from
    outside.  nV = 10 * 4**level + 2.
    """
    verts, faces = icosahedron()
    verts = [tuple(p) for p in verts]
    faces = [tuple(f) for f in faces]
    for _ in range(level):
        cache = {}

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            if key in cache:
                return cache[key]
            p = np.add(verts[a], verts[b]) * 0.5
            p = p / np.linalg.norm(p)
            verts.append(tuple(p))
            cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    return np.array(verts, dtype=np.float64), np.array(faces, dtype=np.int32)


def rbc_shape(unit: np.ndarray) -> np.ndarray:
    """Evans-Fung biconcave map of unit-sphere points (radius RBC_R0)."""
    ux, uy, uz = unit[:, 0], unit[:, 1], unit[:, 2]
    rho2 = ux * ux + uy * uy
    half = 0.5 * RBC_R0 * np.sqrt(np.maximum(0.0, 1.0 - rho2))
    z = np.sign(uz) * half * (RBC_C0 + RBC_C1 * rho2 + RBC_C2 * rho2 * rho2)
    return np.stack([RBC_R0 * ux, RBC_R0 * uy, z], axis=1)


def ellipsoid_shape(unit: np.ndarray, axes=PLT_AXES) -> np.ndarray:
    return unit * np.asarray(axes, dtype=np.float64)[None, :]


def tetrahedron():
    """4-vertex closed surface (regular tetrahedron, outward CCW faces)."""
    v = np.array([[1.0, 1.0, 1.0], [1.0, -1.0, -1.0],
                  [-1.0, 1.0, -1.0], [-1.0, -1.0, 1.0]])
    f = []
    for tri in ([0, 1, 2], [0, 1, 3], [0, 2, 3], [1, 2, 3]):
        i, j, k = tri
        nrm = np.cross(v[j] - v[i], v[k] - v[i])
        if np.dot(nrm, v[i] + v[j] + v[k]) < 0:
            tri = [i, k, j]
        f.append(tri)
    return v, np.array(f, dtype=np.int32)


# --------------------------------------------------------------------------
# mesh types and workloads
# --------------------------------------------------------------------------
@dataclass
class Material:
    k_strain: float
    k_area: float
    k_bend: float
    k_vol: float
    dt: float
    rayleigh_alpha: float = 0.0     # Rayleigh damping C = alpha M + beta L (0, 0: none)
    rayleigh_beta: float = 0.0


@dataclass
class MeshType:
    name: str
    rest: np.ndarray          # [nV, 3] float64
    tris: np.ndarray          # [nT, 3] int32, outward CCW
    material: Material
    radius: float             # cell radius used by the error metric
    mass: np.ndarray | None = None   # [nV] or None (uniform 1/nV)

    @property
    def nV(self) -> int:
        return int(self.rest.shape[0])


RBC_MATERIAL = Material(1.0, 5.0, 0.05, 10.0, 1e-3)
PLT_MATERIAL = Material(10.0, 5.0, 0.5, 10.0, 1e-3)


def rbc_type(level: int = 3, material: Material = RBC_MATERIAL, name="rbc") -> MeshType:
    unit, tris = icosphere(level)
    return MeshType(name, rbc_shape(unit), tris, material, RBC_R0)


def plt_type(level: int = 2, material: Material = PLT_MATERIAL, name="plt") -> MeshType:
    unit, tris = icosphere(level)
    return MeshType(name, ellipsoid_shape(unit), tris, material, PLT_AXES[0])


@dataclass
class Group:
    """``n_cells`` cells of one mesh type, with their seeded inputs."""
    mtype: MeshType
    n_cells: int
    seed: int
    amp: float = 0.1
    shear: float = 0.02
    box: float = 200.0
    x0: np.ndarray | None = field(default=None, repr=False)
    v0: np.ndarray | None = field(default=None, repr=False)
    f_ext: np.ndarray | None = field(default=None, repr=False)


def random_rotations(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniform rotations from normalised Gaussian quaternions -> [n,3,3]."""
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def fourier_forces(rest: np.ndarray, radius: float, amp: float, shear: float,
                   e: np.ndarray, k: np.ndarray, phase: np.ndarray) -> np.ndarray:
    """Per-vertex force of C cells from their mode draws.

    f_v = sum_j amp * e_j * sin(k_j . (X_v - c) + phase_j) + shear * (X_v - c)_y * x_hat,
    X_v the rest (body-frame) positions, c their centroid.  e: [C,8,3] unit
    vectors, k: [C,8,3] wave vectors, phase: [C,8].  Returns [C, nV, 3].
    """
    rel = rest - rest.mean(axis=0, keepdims=True)              # [nV,3]
    arg = np.einsum("cjd,vd->cjv", k, rel) + phase[:, :, None]   # [C,8,nV]
    f = amp * np.einsum("cjd,cjv->cvd", e, np.sin(arg))          # [C,nV,3]
    f[:, :, 0] += shear * rel[None, :, 1]
    return f


def materialise(group: Group, chunk: int = 2048) -> Group:
    """Fill x0 (placed rest shapes), v0 (zero) and f_ext for a group."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([group.seed, 0x5EED])))
    C, nV = group.n_cells, group.mtype.nV
    R = random_rotations(rng, C)
    t = rng.uniform(0.0, group.box, size=(C, 3))
    e = rng.standard_normal((C, 8, 3))
    e /= np.linalg.norm(e, axis=2, keepdims=True)
    kmax = 2.0 * np.pi / (2.0 * group.mtype.radius)
    k = rng.uniform(-1.0, 1.0, size=(C, 8, 3)) * kmax
    phase = rng.uniform(0.0, 2.0 * np.pi, size=(C, 8))
    rest = group.mtype.rest
    x0 = np.empty((C, nV, 3))
    f = np.empty((C, nV, 3))
    for s in range(0, C, chunk):
        sl = slice(s, min(C, s + chunk))
        x0[sl] = np.einsum("cij,vj->cvi", R[sl], rest) + t[sl, None, :]
        f[sl] = fourier_forces(rest, group.mtype.radius, group.amp, group.shear,
                               e[sl], k[sl], phase[sl])
    group.x0, group.v0, group.f_ext = x0, np.zeros_like(x0), f
    return group


def subset(group: Group, idx) -> Group:
    """The cells ``idx`` of a materialised group (same draws)."""
    idx = np.asarray(idx, dtype=np.int64)
    g = Group(group.mtype, len(idx), group.seed, group.amp, group.shear, group.box)
    g.x0, g.v0, g.f_ext = group.x0[idx].copy(), group.v0[idx].copy(), group.f_ext[idx].copy()
    return g


# --------------------------------------------------------------------------
# the five suspension workloads (sizes, meshes, stiffness, forces, seeds)
# --------------------------------------------------------------------------
WORKLOADS = {
    "rbc1": dict(desc="1 RBC, 642-vertex Evans-Fung mesh, plain FP64, 20 steps x 10 iterations",
                 groups=[("rbc", 1, 0.1)], seed=0, steps=20, precision="fp64"),
    "rbc4096": dict(desc="4096 RBCs (642 v) in a 200^3 box, plain FP64, 100 steps",
                    groups=[("rbc", 4096, 0.1)], seed=1, steps=100, precision="fp64"),
    "rbc10k_plt1500": dict(desc="10000 RBC (642 v) + 1500 PLT (162 v), TF32 global step + FP64-residual refinement, 50 steps",
                           groups=[("rbc", 10000, 0.1), ("plt", 1500, 0.1)], seed=2, steps=50,
                           precision="tf32"),
    "rbc50k_plt5k": dict(desc="50000 RBC (642 v) + 5000 PLT (162 v), BF16 global step, FP32 accumulate, refinement to 1e-6, 50 steps, force amplitude 0.3",
                         groups=[("rbc", 50000, 0.3), ("plt", 5000, 0.3)], seed=3, steps=50,
                         precision="bf16"),
    "hetero20k": dict(desc="20000 cells over 3 meshes (162/642/2562 v) x 4 k_strain {0.5,1,2,10}: 12 matrices, dt {5e-4,1e-3}, BF16 global step, 20 steps",
                      groups="hetero", seed=4, steps=20, precision="bf16"),
}


def hetero_types():
    """12 mesh types: level {2,3,4} sphere->RBC map x k_strain {0.5,1,2,10}."""
    out = []
    gi = 0
    for level in (2, 3, 4):
        unit, tris = icosphere(level)
        rest = rbc_shape(unit)
        for ks in (0.5, 1.0, 2.0, 10.0):
            dt = 5e-4 if gi % 2 == 0 else 1e-3
            mat = Material(ks, 5.0, 0.05, 10.0, dt)
            out.append(MeshType(f"L{level}_ks{ks:g}", rest, tris, mat, RBC_R0))
            gi += 1
    return out


def workload_groups(name: str, scale: float = 1.0):
    """Groups (unmaterialised) of a named workload; ``scale`` shrinks cell counts."""
    w = WORKLOADS[name]
    seed = w["seed"]
    groups = []
    if w["groups"] == "hetero":
        types = hetero_types()
        total = max(len(types), int(round(20000 * scale)))
        base = total // len(types)
        for i, t in enumerate(types):
            n = base + (1 if i < total - base * len(types) else 0)
            groups.append(Group(t, n, seed * 1000 + i, 0.1))
        return groups
    cache = {}
    for gi, (kind, n, amp) in enumerate(w["groups"]):
        if kind not in cache:
            cache[kind] = rbc_type() if kind == "rbc" else plt_type()
        groups.append(Group(cache[kind], max(1, int(round(n * scale))), seed * 1000 + gi, amp))
    return groups
