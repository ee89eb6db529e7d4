"""Immersed-boundary forces by multi-direct forcing (supplementary IBM section)
on the CUDA path vs the FP64 oracle: every vertex of every cell against a
synthetic fluid velocity on a lattice that the cells partly leave (nodes outside
are left out).  Bar: 1e-12 relative (FP64; the spreading's atomic additions
change only the order of the sums).  All calls go through libnpfem.so."""
import numpy as np
import pytest

from paper_1911_03062_gb300 import inputs as I

from helpers import public, split

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as G
    G.build()


def _field(n, dx, origin, seed):
    idx = np.indices((n, n, n))[::-1].astype(float)
    x = origin[:, None, None, None] + dx * idx
    rng = np.random.default_rng(seed)
    u = np.zeros((3, n, n, n))
    for c in range(3):
        for _ in range(3):
            k = rng.uniform(-0.6, 0.6, 3)
            u[c] += rng.uniform(-0.5, 0.5) * np.sin(np.einsum("d,dzyx->zyx", k, x) + rng.uniform(0, 6.3))
    return u


@pytest.mark.parametrize("cycles", [0, 1, 3])
def test_ibm_forces_match_oracle(cycles):
    import torch
    from oracle import oracle as O
    from paper_1911_03062_gb300.npfem import Solver
    groups = [I.materialise(I.Group(I.rbc_type(), 2, 600, amp=0.3, box=6.0)),
              I.materialise(I.Group(I.plt_type(), 2, 601, amp=0.3, box=6.0))]
    s = Solver(precision="bf16")
    for g in groups:
        s.add_cells(s.create_type(g.mtype), g.x0, g.v0)
    s.step(public(groups, "f_ext"))                       # non-zero vertex velocities
    x, v = s.positions(), s.velocities()
    n, dx, origin, dt = 26, 0.5, np.array([-3.0, -2.5, -3.5]), 0.1   # the cells reach past the lattice
    u = _field(n, dx, origin, 602)
    fl, fg = s.ibm_forces(torch.tensor(u, device="cuda"), origin, dx, dt, cycles)
    fl, fg = fl.cpu().numpy(), fg.cpu().numpy()
    s.close()
    xs, vs = split(x, groups), split(v, groups)
    X = np.concatenate([xx.reshape(-1, 3) for xx in xs])
    U = np.concatenate([vv.reshape(-1, 3) for vv in vs])
    A = np.concatenate([O.OracleType.from_mesh_type(g.mtype).vertex_areas(c) for g, xx in zip(groups, xs) for c in xx])
    fo, Fo = O.ibm(X, U, A, u, origin, dx, dt, cycles)
    assert np.abs(fl.reshape(-1, 3) - fo).max() <= 1e-12 * np.abs(fo).max()
    assert np.abs(fg - Fo).max() <= 1e-12 * np.abs(Fo).max()
    assert np.abs(Fo).max() > 0
    q = (X - origin) / dx                                  # stencil nodes floor(q) - 1 .. floor(q) + 2
    assert (np.floor(q) - 1 < 0).any() and (np.floor(q) + 2 > n - 1).any()   # some leave the lattice


def test_ibm_rejects_bad_arguments():
    import torch
    from paper_1911_03062_gb300.npfem import EINVAL, NpfemError, Solver
    g = I.materialise(I.Group(I.plt_type(), 1, 603))
    s = Solver(precision="fp64")
    s.add_cells(s.create_type(g.mtype), g.x0, g.v0)
    u = torch.zeros((3, 4, 4, 4), dtype=torch.float64, device="cuda")
    for kw in ({"dt": 0.0, "cycles": 1}, {"dt": 0.1, "cycles": -1}):
        with pytest.raises(NpfemError) as e:
            s.ibm_forces(u, np.zeros(3), 0.5, **kw)
        assert e.value.code == EINVAL
    with pytest.raises(NpfemError):
        s.ibm_forces(u, np.zeros(3), 0.0, 0.1)
    s.close()
