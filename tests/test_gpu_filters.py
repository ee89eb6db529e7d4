"""The steps either side of the path (paper Sec. 2.2): one-ring median filter of
the external forces before each step, velocity cap after it.  GPU path vs the
oracle composed the same way (median -> step -> cap), FP64 (1e-10) and BF16
(1e-6).  All calls go through libnpfem.so."""
import numpy as np
import pytest

from paper_1911_03062_gb300 import inputs as I

from helpers import make_groups, public, rel_pos_err, split

pytestmark = pytest.mark.gpu

UMAX = 0.4          # caps about half of the vertices of these cells after one step


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as G
    G.build()


def _gpu(groups, steps, precision, **opts):
    from paper_1911_03062_gb300.npfem import Solver
    s = Solver(precision=precision, **opts)
    for g in groups:
        s.add_cells(s.create_type(g.mtype), g.x0, g.v0)
    f = public(groups, "f_ext")
    for _ in range(steps):
        s.step(f)
    x, v = split(s.positions(), groups), split(s.velocities(), groups)
    s.close()
    return x, v


def _oracle(groups, steps, median, umax, kappa=0.0):
    from oracle import oracle as O
    xs, vs = [], []
    for g in groups:
        T = O.OracleType.from_mesh_type(g.mtype)
        f = O.force_median(T, g.f_ext) if median else g.f_ext
        x, v = g.x0.copy(), g.v0.copy()
        for _ in range(steps):
            x, v = T.step_cells(x, v, f, K=10, m=5, threads=4)
            if kappa > 0:
                v = O.pbd_damping(T, x, v, kappa)
            if umax > 0:
                v = O.velocity_cap(v, umax)
        xs.append((np.arange(g.n_cells), x))
        vs.append((np.arange(g.n_cells), v))
    return xs, vs


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("bf16", 1e-6)])
def test_median_and_cap_match_oracle(precision, tol):
    groups = make_groups([(I.rbc_type(), 4, 0.3), (I.plt_type(), 2, 0.3)], seed=300)
    xg, vg = _gpu(groups, 3, precision, force_median=True, u_max=UMAX)
    xo, vo = _oracle(groups, 3, True, UMAX)
    assert rel_pos_err(xg, xo, groups) <= tol
    for a, (_, b) in zip(vg, vo):
        # velocity = position difference / h: the position bar divided by h = 1e-3
        assert np.abs(a - b).max() <= (1e-5 if precision == "fp64" else 3e-2) * UMAX


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("bf16", 1e-6)])
def test_pbd_damping_matches_oracle(precision, tol):
    # kappa_damping = 0.8 (paper range 0.5-0.9), with the median filter and the cap
    groups = make_groups([(I.rbc_type(), 4, 0.3), (I.plt_type(), 2, 0.3)], seed=302)
    xg, vg = _gpu(groups, 3, precision, force_median=True, u_max=UMAX, pbd_kappa=0.8)
    xo, vo = _oracle(groups, 3, True, UMAX, kappa=0.8)
    assert rel_pos_err(xg, xo, groups) <= tol
    for a, (_, b) in zip(vg, vo):
        assert np.abs(a - b).max() <= (1e-5 if precision == "fp64" else 3e-2) * UMAX


def test_pbd_damping_damps_deformation_keeps_momentum():
    groups = make_groups([(I.rbc_type(), 3, 0.3)], seed=303)
    xa, va = _gpu(groups, 2, "fp64")
    xb, vb = _gpu(groups, 2, "fp64", pbd_kappa=0.9)
    # the damped run deforms less: velocity spread about the cell mean is smaller
    spread = lambda v: np.linalg.norm(v - v.mean(axis=1, keepdims=True), axis=2).mean()
    assert spread(vb[0]) < 0.5 * spread(va[0])


def test_filters_are_active():
    # the median changes the trajectory, the cap bounds every velocity
    groups = make_groups([(I.rbc_type(), 3, 0.3)], seed=301)
    xa, va = _gpu(groups, 2, "fp64")
    xb, vb = _gpu(groups, 2, "fp64", force_median=True)
    xc, vc = _gpu(groups, 2, "fp64", u_max=UMAX)
    assert np.abs(xa[0] - xb[0]).max() > 1e-6
    assert np.linalg.norm(va[0], axis=2).max() > 1.5 * UMAX
    assert np.linalg.norm(vc[0], axis=2).max() <= UMAX * (1 + 1e-12)


def test_median_rejects_high_valence():
    # bipyramid over a 33-gon: each apex has 33 neighbours (> 31)
    from paper_1911_03062_gb300.npfem import EINVAL, NpfemError, Solver
    n = 33
    ang = 2 * np.pi * np.arange(n) / n
    rest = np.vstack([np.c_[np.cos(ang), np.sin(ang), np.zeros(n)], [[0, 0, 1.0], [0, 0, -1.0]]])
    top, bot = n, n + 1
    tris = [[i, (i + 1) % n, top] for i in range(n)] + [[(i + 1) % n, i, bot] for i in range(n)]
    mt = I.MeshType("bipyramid", rest, np.array(tris, dtype=np.int32), I.Material(1.0, 5.0, 0.05, 10.0, 1e-3), 1.0)
    s = Solver(precision="fp64")
    s.create_type(mt)                       # fine without the filter
    s.close()
    s = Solver(precision="fp64", force_median=True)
    with pytest.raises(NpfemError) as e:
        s.create_type(mt)
    assert e.value.code == EINVAL and "neighbours" in str(e.value)
    s.close()
