"""FP64 CUDA path vs the FP64 oracle (bar: 1e-10 relative position error),
plus the C-ABI contract on the GPU: errors, edge cases, invariants and
checkpoint/resume.  All calls go through libnpfem.so."""
import numpy as np
import pytest

from paper_1911_03062_gb300 import inputs as I

from helpers import make_groups, one_step_parity, public, rel_pos_err, run_gpu, run_oracle, split

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as G
    G.build()


def test_one_rbc_twenty_steps():
    # the single-RBC workload: 642-vertex Evans-Fung cell, 20 steps x 10 iterations
    groups = [I.materialise(I.Group(I.rbc_type(), 1, seed=0, amp=0.1))]
    xg, vg, st = run_gpu(groups, 20)
    xo, vo = run_oracle(groups, 20)
    assert rel_pos_err(xg, xo, groups) <= TOL64
    assert np.abs(vg[0] - vo[0][1]).max() <= 1e-6
    assert st["cell_iterations"] == 10


def test_two_types_ragged_tiles():
    # 50 RBC (150 RHS rows: two 128-row tiles, ragged) + 7 platelets
    groups = make_groups([(I.rbc_type(), 50, 0.3), (I.plt_type(), 7, 0.3)])
    xg, _, _ = run_gpu(groups, 3)
    xo, _ = run_oracle(groups, 3)
    assert rel_pos_err(xg, xo, groups) <= TOL64


@pytest.mark.parametrize("graph", [True, False])
def test_graph_and_eager_agree_bitwise(graph):
    groups = make_groups([(I.rbc_type(), 5, 0.3), (I.plt_type(), 3, 0.3)])
    xa, _, _ = run_gpu(groups, 2, use_graph=graph)
    xb, _, _ = run_gpu(groups, 2, use_graph=not graph)
    for a, b in zip(xa, xb):
        assert np.array_equal(a, b)


def test_large_mesh_and_tetrahedron():
    u4, t4 = I.icosphere(4)
    big = I.MeshType("L4", I.rbc_shape(u4), t4, I.Material(1.0, 5.0, 0.05, 10.0, 5e-4), I.RBC_R0)
    v, f = I.tetrahedron()
    tet = I.MeshType("tet", v, f, I.Material(1.0, 5.0, 0.05, 10.0, 1e-2), 1.7)
    groups = make_groups([(big, 2, 0.3), (tet, 5, 1.0)])
    xg, _, _ = run_gpu(groups, 2)
    xo, _ = run_oracle(groups, 2)
    assert rel_pos_err(xg, xo, groups) <= TOL64


def test_sampled_cells_at_4096():
    # the 4096-RBC FP64 workload, 2 steps, sampled cells against the oracle
    g = I.materialise(I.Group(I.rbc_type(), 4096, seed=1, amp=0.1))
    xg, _, _ = run_gpu([g], 2)
    sample = [[0, 1, 2047, 4000, 4095]]
    xo, _ = run_oracle([g], 2, sample=sample)
    assert rel_pos_err(xg, xo, [g]) <= TOL64


def test_late_state_step_at_4096():
    # 4096 RBC after 20 steps: one FP64 GPU step from its own state vs the oracle's
    # step from the same state (trajectories themselves drift apart by rounding
    # amplification, ~1.2x per step)
    groups = [I.materialise(g) for g in I.workload_groups("rbc4096")]
    err, _ = one_step_parity(groups, 20, [[0, 1000, 2048, 4095]], precision="fp64")
    assert err <= TOL64, err


def test_rest_state_stays_at_rest():
    g = I.materialise(I.Group(I.plt_type(), 4, seed=3))
    g.f_ext[:] = 0.0
    xg, vg, _ = run_gpu([g], 3)
    assert np.abs(xg[0] - g.x0).max() <= 1e-12 * I.PLT_AXES[0]
    assert np.abs(vg[0]).max() <= 1e-9


def test_momentum_conserved_without_forces():
    g = I.materialise(I.Group(I.rbc_type(), 3, seed=4))
    rng = np.random.default_rng(5)
    g.v0 = rng.standard_normal(g.v0.shape)
    g.f_ext[:] = 0.0
    _, vg, _ = run_gpu([g], 2)
    assert np.allclose(vg[0].mean(axis=1), g.v0.mean(axis=1), atol=1e-9)


def test_checkpoint_resume_bitwise():
    from paper_1911_03062_gb300.npfem import Solver
    groups = make_groups([(I.rbc_type(), 4, 0.3), (I.plt_type(), 2, 0.3)])
    f = public(groups, "f_ext")

    def solver():
        s = Solver(precision="fp64")
        for g in groups:
            s.add_cells(s.create_type(g.mtype), g.x0, g.v0)
        return s

    a = solver()
    for _ in range(2):
        a.step(f)
    x2, v2 = a.positions(), a.velocities()
    for _ in range(2):
        a.step(f)
    xa = a.positions()
    b = solver()
    b.set_state(x2, v2)
    for _ in range(2):
        b.step(f)
    assert np.array_equal(xa, b.positions())


def test_apply_pinv_fp64():
    import torch
    from oracle import oracle as O
    from paper_1911_03062_gb300.npfem import Solver
    mt = I.rbc_type()
    s = Solver(precision="fp64")
    tid = s.create_type(mt)
    P = O.OracleType.from_mesh_type(mt).P_dense()
    q = np.random.default_rng(6).standard_normal((131, mt.nV))
    z = s.apply_pinv(tid, torch.tensor(q, device="cuda"), torch.empty((131, mt.nV), dtype=torch.float64,
                                                                        device="cuda")).cpu().numpy()
    ref = np.linalg.solve(P, q.T).T
    assert np.abs(z - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("level", [1, 2, 4])
def test_blocked_inverse_matches_library_inverse(level):
    # the set-up's blocked Gauss-Jordan inverse (32-pivot blocks; nV = 42, 162, 2562 pad to
    # 64, 192, 2592) read back through the FP64 apply of identity columns, against numpy
    import torch
    from oracle import oracle as O
    from paper_1911_03062_gb300.npfem import Solver
    u, t = I.icosphere(level)
    mt = I.MeshType(f"L{level}", I.rbc_shape(u), t, I.Material(1.0, 5.0, 0.05, 10.0, 5e-4), I.RBC_R0)
    s = Solver(precision="fp64")
    tid = s.create_type(mt)
    inv = np.linalg.inv(O.OracleType.from_mesh_type(mt).P_dense())
    eye = torch.eye(mt.nV, dtype=torch.float64, device="cuda")
    z = s.apply_pinv(tid, eye, torch.empty_like(eye)).cpu().numpy()
    assert np.abs(z - inv).max() <= 1e-12 * np.abs(inv).max()
    s.close()


def test_errors():
    from paper_1911_03062_gb300.npfem import ENONFINITE, EINVAL, ESTATE, NpfemError, Solver
    s = Solver(precision="fp64")
    with pytest.raises(NpfemError) as e:
        s.step(np.zeros(0))
    assert e.value.code == ESTATE
    v, f = I.tetrahedron()
    with pytest.raises(NpfemError) as e:                      # open mesh
        s.create_mesh_type(v, f[:3], 1, 1, 1, 1, 1e-3)
    assert e.value.code == EINVAL
    with pytest.raises(NpfemError) as e:                      # inward orientation
        s.create_mesh_type(v, f[:, ::-1], 1, 1, 1, 1, 1e-3)
    assert e.value.code == EINVAL
    with pytest.raises(NpfemError) as e:                      # repeated vertex
        s.create_mesh_type(v, np.array([[0, 0, 1], [0, 1, 2], [0, 2, 3], [1, 2, 3]]), 1, 1, 1, 1, 1e-3)
    assert e.value.code == EINVAL
    tid = s.create_mesh_type(v, f, 1, 1, 1, 1, 1e-3)
    assert s.add_cells(tid, np.zeros((0, 4, 3))) == 0
    s.add_cells(tid, v[None] + 1.0)
    bad = np.zeros(s.num_dofs)
    bad[5] = np.nan
    s.step(bad)
    with pytest.raises(NpfemError) as e:
        s.sync()
    assert e.value.code == ENONFINITE
    with pytest.raises(NpfemError) as e:
        s.add_cells(tid, np.full((1, 4, 3), np.inf))
    assert e.value.code == ENONFINITE


@pytest.mark.parametrize("precision", ["fp64", "bf16"])
def test_vertex_numbering_is_internal(precision):
    # the library renumbers vertices internally; a caller's relabelling of the
    # same cells (vertices shuffled, triangles rotated and reordered) gives the
    # same public result up to rounding
    rng = np.random.default_rng(7)
    base = I.rbc_type()
    g = I.materialise(I.Group(base, 5, seed=11, amp=0.3))
    perm = rng.permutation(base.nV)                        # new label k <- old vertex perm[k]
    new_of_old = np.empty_like(perm)
    new_of_old[perm] = np.arange(base.nV)
    tris = new_of_old[base.tris]
    tris = np.roll(tris, 1, axis=1)[rng.permutation(len(tris))].astype(np.int32)
    relabelled = I.MeshType("rbc_relabelled", base.rest[perm], tris, base.material, base.radius)
    g2 = I.Group(relabelled, 5, seed=11, amp=0.3)
    g2.x0, g2.v0, g2.f_ext = g.x0[:, perm], g.v0[:, perm], g.f_ext[:, perm]
    xa, _, _ = run_gpu([g], 3, precision=precision)
    xb, _, _ = run_gpu([g2], 3, precision=precision)
    err = np.abs(xa[0] - xb[0][:, new_of_old]).max() / base.radius
    assert err <= (1e-12 if precision == "fp64" else 1e-6)
