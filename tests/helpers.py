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
