"""Shared helpers of the GPU parity tests: run the same seeded workload
through the CUDA library and through the FP64 oracle, and compare.

Error metric: max over cells and vertices of |x_gpu - x_oracle|_2 / R_cell
(R = 3.91 for red blood cells, 1.8 for platelets)."""
from __future__ import annotations

import numpy as np

from paper_1911_03062_gb300 import inputs as I


def make_groups(spec, seed=100):
    """spec: list of (MeshType, n_cells, amp)."""
    return [I.materialise(I.Group(mt, n, seed + i, amp=amp)) for i, (mt, n, amp) in enumerate(spec)]


def public(groups, attr):
    return np.concatenate([getattr(g, attr).ravel() for g in groups])


def split(x, groups):
    out, off = [], 0
    for g in groups:
        n = g.n_cells * g.mtype.nV * 3
        out.append(x[off:off + n].reshape(g.n_cells, g.mtype.nV, 3))
        off += n
    return out


def run_gpu(groups, steps, precision="fp64", **opts):
    from paper_1911_03062_gb300.npfem import Solver
    s = Solver(precision=precision, **opts)
    for g in groups:
        tid = s.create_type(g.mtype)
        s.add_cells(tid, g.x0, g.v0)
    f = public(groups, "f_ext")
    for _ in range(steps):
        s.step(f)
    x, v = s.positions(), s.velocities()
    st = s.stats()
    s.close()
    return split(x, groups), split(v, groups), st


def run_oracle(groups, steps, sample=None, K=10, m=5, threads=4):
    """Oracle trajectories of the sampled cells of every group."""
    from oracle import oracle as O
    xs, vs = [], []
    for gi, g in enumerate(groups):
        T = O.OracleType.from_mesh_type(g.mtype)
        idx = np.arange(g.n_cells) if sample is None else np.asarray(sample[gi])
        x, v, f = g.x0[idx].copy(), g.v0[idx].copy(), g.f_ext[idx]
        for _ in range(steps):
            x, v = T.step_cells(x, v, f, K=K, m=m, threads=threads)
        xs.append((idx, x))
        vs.append((idx, v))
    return xs, vs


def rel_pos_err(xg_groups, xo_groups, groups):
    err = 0.0
    for xg, (idx, xo), g in zip(xg_groups, xo_groups, groups):
        d = np.linalg.norm(xg[idx] - xo, axis=2).max() / g.mtype.radius
        err = max(err, float(d))
    return err


def one_step_parity(groups, steps_before, sample, precision="fp64", **opts):
    """Advance all cells `steps_before` steps on the GPU, then one more step on the
    GPU and, from the same GPU state (positions and velocities), one oracle step for
    the sampled cells; returns the relative position error of that step.

    The cell dynamics amplify any difference in rounding order (the oracle against
    itself with a 1e-12 perturbation grows ~1.16x per step on the amplitude-0.3
    workloads), so parity after many steps is measured on the step map from a shared
    state rather than on two independently integrated trajectories."""
    from oracle import oracle as O
    from paper_1911_03062_gb300.npfem import Solver
    s = Solver(precision=precision, **opts)
    for g in groups:
        s.add_cells(s.create_type(g.mtype), g.x0, g.v0)
    f = public(groups, "f_ext")
    for _ in range(steps_before):
        s.step(f)
    xn, vn = split(s.positions(), groups), split(s.velocities(), groups)
    s.step(f)
    x1 = split(s.positions(), groups)
    st = s.stats()
    s.close()
    err = 0.0
    for gi, g in enumerate(groups):
        idx = np.asarray(sample[gi])
        T = O.OracleType.from_mesh_type(g.mtype)
        xo, _ = T.step_cells(xn[gi][idx].copy(), vn[gi][idx].copy(), g.f_ext[idx], K=10, m=5, threads=4)
        err = max(err, float(np.linalg.norm(x1[gi][idx] - xo, axis=2).max() / g.mtype.radius))
    return err, st


def branch_cell(seed=5, dt=0.05, mirror=False):
    """A level-1 RBC (42 vertices) at dt = 0.05, where the inertia term no longer
    dominates and the quasi-Newton iterations stay far from convergence for K > 15,
    in a deformed state with velocities and forces.  mirror: the cell inside out
    (large non-convex projections; seed 23 gives one negative-curvature pair).
    Returns (MeshType, x_n, v_n, f_ext), each array [nV, 3]."""
    unit, tris = I.icosphere(1)
    rest = I.rbc_shape(unit)
    mt = I.MeshType("rbc-l1", rest, tris, I.Material(1.0, 5.0, 0.5, 10.0, dt), I.RBC_R0)
    rng = np.random.default_rng(seed)
    if mirror:
        xn = rest * np.array([1, 1, -1]) + 0.1 * rng.standard_normal(rest.shape)
    else:
        R = I.random_rotations(np.random.default_rng(seed), 1)[0]
        xn = rest @ R.T + 0.3 * rng.standard_normal(rest.shape)
    vn = rng.standard_normal(rest.shape)
    f = rng.standard_normal(rest.shape)
    return mt, xn, vn, f


def group_of(mt, x0, v0, f):
    """A Group holding the given cells ([n, nV, 3] arrays, or one [nV, 3] cell)."""
    x0, v0, f = (np.asarray(a, dtype=np.float64).reshape(-1, mt.nV, 3) for a in (x0, v0, f))
    g = I.Group(mt, x0.shape[0], seed=0)
    g.x0, g.v0, g.f_ext = x0.copy(), v0.copy(), f.copy()
    return g
