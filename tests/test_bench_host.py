"""CPU checks of bench.py's host logic: the sampled oracle step used for parity
with particle-in-kernel collisions searches each sampled cell against the cells
whose bounding spheres come within the kernel radius, which must give the same
step as the brute-force search over all cells."""
import types

import numpy as np

from paper_1911_03062_gb300 import inputs as I


def test_sampled_collision_step_equals_full_search(oracle_lib, monkeypatch):
    import bench as B
    O = oracle_lib
    rk, kc = 0.5, 200.0
    groups = [I.materialise(I.Group(I.rbc_type(), 6, 700, amp=0.3, box=12.0)),
              I.materialise(I.Group(I.plt_type(), 4, 701, amp=0.3, box=12.0))]
    monkeypatch.setattr(B, "PARITY_CELLS", 3)
    args = types.SimpleNamespace(pik_radius=rk, collision_k=kc, force_median=False)
    xn = np.concatenate([g.x0.ravel() for g in groups])
    vn = np.concatenate([g.v0.ravel() for g in groups])
    sampled = B.oracle_step_sampled(groups, xn, vn, args)
    Ts = [O.OracleType.from_mesh_type(g.mtype) for g in groups]
    cells = [(Ts[gi], g.x0[c]) for gi, g in enumerate(groups) for c in range(g.n_cells)]
    res = O.pik(cells, rk)
    base = np.cumsum([0] + [g.n_cells for g in groups])
    contacts = 0
    for gi, (g, (idx, xo)) in enumerate(zip(groups, sampled)):
        for k, c in enumerate(idx):
            hc, _, p = res[base[gi] + c]
            contacts += int((hc >= 0).sum())
            x1, _ = Ts[gi].step_cells_col(g.x0[c][None], g.v0[c][None], g.f_ext[c][None], kc,
                                          (hc >= 0).astype(np.int32)[None], p[None])
            assert np.array_equal(xo[k], x1[0])
    assert contacts > 100
