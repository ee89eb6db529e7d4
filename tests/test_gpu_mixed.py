"""Mixed-precision CUDA path (FP32 local step, tcgen05 TF32 / BF16 global
step with FP64-residual refinement) vs the FP64 oracle: bar 1e-6 relative
position error.  All calls go through libnpfem.so."""
import numpy as np
import pytest

from paper_1911_03062_gb300 import inputs as I

from helpers import make_groups, one_step_parity, public, rel_pos_err, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-6


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as G
    G.build()


def _solver(prec, **kw):
    # "bf16-plain": BF16 form with plain (unsplit) refinement corrections
    from paper_1911_03062_gb300.npfem import Solver
    if prec == "bf16-plain":
        return Solver(precision="bf16", refine_split=False, **kw)
    return Solver(precision=prec, **kw)


@pytest.mark.parametrize("prec", ["bf16", "bf16-plain", "tf32"])
def test_apply_pinv_tensor_cores(prec):
    # z = P^{-1} q on tcgen05 + refinement vs the exact FP64 solve; 131 columns
    # (two 128-row tiles, ragged), both mesh sizes (three 224-wide N tiles / one)
    import torch
    from oracle import oracle as O
    for mt in (I.rbc_type(), I.plt_type()):
        s = _solver(prec)
        tid = s.create_type(mt)
        P = O.OracleType.from_mesh_type(mt).P_dense()
        q = np.random.default_rng(7).standard_normal((131, mt.nV))
        z = s.apply_pinv(tid, torch.tensor(q, device="cuda"),
                         torch.empty((131, mt.nV), dtype=torch.float64, device="cuda")).cpu().numpy()
        ref = np.linalg.solve(P, q.T).T
        resid = np.linalg.norm(q - z @ P, axis=1) / np.linalg.norm(q, axis=1)
        assert resid.max() <= 1e-6, (prec, mt.name, resid.max())
        assert np.abs(z - ref).max() <= 2e-6 * np.abs(ref).max()
        st = s.stats()
        assert st["max_refine_residual"] <= 1e-6
        s.close()


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_unrefined_apply_is_low_precision(prec):
    # with no refinement sweep the apply carries the operand rounding (proves
    # the tensor-core path, not an FP64 shortcut, produced the refined result)
    import torch
    from oracle import oracle as O
    from paper_1911_03062_gb300.npfem import Solver
    mt = I.rbc_type()
    s = Solver(precision=prec, refine_max=0)
    tid = s.create_type(mt)
    P = O.OracleType.from_mesh_type(mt).P_dense()
    q = np.random.default_rng(8).standard_normal((60, mt.nV))
    z = s.apply_pinv(tid, torch.tensor(q, device="cuda"),
                     torch.empty((60, mt.nV), dtype=torch.float64, device="cuda")).cpu().numpy()
    resid = (np.linalg.norm(q - z @ P, axis=1) / np.linalg.norm(q, axis=1)).max()
    assert 1e-6 < resid < (2e-2 if prec == "bf16" else 5e-3), resid


def test_split_correction_gains_two_orders():
    # one refinement sweep: the split BF16 correction (hi/lo parts of r and
    # P^{-1}, three products) leaves a residual far below the plain one's
    import torch
    from oracle import oracle as O
    mt = I.rbc_type()
    P = O.OracleType.from_mesh_type(mt).P_dense()
    q = np.random.default_rng(9).standard_normal((96, mt.nV))
    res = {}
    for prec in ("bf16", "bf16-plain"):
        s = _solver(prec, refine_max=1)
        tid = s.create_type(mt)
        z = s.apply_pinv(tid, torch.tensor(q, device="cuda"),
                         torch.empty((96, mt.nV), dtype=torch.float64, device="cuda")).cpu().numpy()
        res[prec] = (np.linalg.norm(q - z @ P, axis=1) / np.linalg.norm(q, axis=1)).max()
        s.close()
    assert res["bf16"] <= 1e-5 and res["bf16"] * 20 <= res["bf16-plain"], res


@pytest.mark.parametrize("prec", ["bf16", "bf16-plain", "tf32"])
def test_two_types_ragged_tiles(prec):
    groups = make_groups([(I.rbc_type(), 50, 0.3), (I.plt_type(), 7, 0.3)])
    if prec == "bf16-plain":
        xg, _, st = run_gpu(groups, 3, precision="bf16", refine_split=False)
    else:
        xg, _, st = run_gpu(groups, 3, precision=prec)
    xo, _ = run_oracle(groups, 3)
    assert rel_pos_err(xg, xo, groups) <= TOL_MIXED
    assert st["max_refine_residual"] <= 1e-6


def test_one_rbc_twenty_steps_bf16():
    groups = [I.materialise(I.Group(I.rbc_type(), 1, seed=0, amp=0.1))]
    xg, _, _ = run_gpu(groups, 20, precision="bf16")
    xo, _ = run_oracle(groups, 20)
    assert rel_pos_err(xg, xo, groups) <= TOL_MIXED


def test_rest_state_and_momentum_bf16():
    g = I.materialise(I.Group(I.rbc_type(), 3, seed=9))
    g.f_ext[:] = 0.0
    xg, vg, _ = run_gpu([g], 2, precision="bf16")
    # Within a step the mixed forms hold positions as FP32 offsets from the cell
    # centroid (half-ulp 1.2e-7 at R = 3.91), so the local step sees the rest
    # shape perturbed by that much and relaxes it by about
    # ulp x (elastic stiffness / (m/h^2)) ~ 1e-8 per step.
    assert np.abs(xg[0] - g.x0).max() <= 1e-7 * I.RBC_R0
    g.v0 = np.random.default_rng(10).standard_normal(g.v0.shape)
    _, vg, _ = run_gpu([g], 2, precision="bf16")
    assert np.allclose(vg[0].mean(axis=1), g.v0.mean(axis=1), atol=1e-6)


def test_checkpoint_resume_bitwise_bf16():
    from paper_1911_03062_gb300.npfem import Solver
    groups = make_groups([(I.rbc_type(), 3, 0.3), (I.plt_type(), 2, 0.3)])
    f = public(groups, "f_ext")

    def solver():
        s = Solver(precision="bf16")
        for g in groups:
            s.add_cells(s.create_type(g.mtype), g.x0, g.v0)
        return s

    a = solver()
    a.step(f)
    x1, v1 = a.positions(), a.velocities()
    a.step(f)
    b = solver()
    b.set_state(x1, v1)
    b.step(f)
    assert np.array_equal(a.positions(), b.positions())


def test_sampled_cells_at_50k_bf16():
    # the 50000 RBC + 5000 platelet workload in the bench's configuration (graph,
    # BF16 apply, refinement to 1e-6), 1 step, sampled cells vs the oracle
    groups = [I.materialise(g) for g in I.workload_groups("rbc50k_plt5k")]
    xg, _, st = run_gpu(groups, 1, precision="bf16")
    sample = [[0, 1, 25000, 49999], [0, 2500, 4999]]
    xo, _ = run_oracle(groups, 1, sample=sample)
    assert rel_pos_err(xg, xo, groups) <= TOL_MIXED
    assert st["max_refine_residual"] <= 1e-6


def test_late_state_step_at_50k_bf16():
    # the bench workload after 30 steps (large deformation): one step from the GPU's
    # state, sampled cells vs the oracle's step from the same state
    groups = [I.materialise(g) for g in I.workload_groups("rbc50k_plt5k")]
    err, st = one_step_parity(groups, 30, [[0, 7, 12345, 31000, 49999], [0, 1234, 4999]], precision="bf16")
    assert err <= TOL_MIXED, err
    assert st["max_refine_residual"] <= 1e-6


def test_heterogeneous_twelve_types_bf16():
    # the 12-type batch (162/642/2562-vertex meshes x k_strain {0.5,1,2,10}, dt
    # {5e-4,1e-3}), 2 cells per type, BF16 apply + refinement, vs the oracle
    groups = [I.materialise(g) for g in I.workload_groups("hetero20k", scale=0.0012)]
    assert len(groups) == 12 and {g.mtype.nV for g in groups} == {162, 642, 2562}
    xg, _, st = run_gpu(groups, 2, precision="bf16")
    xo, _ = run_oracle(groups, 2)
    assert rel_pos_err(xg, xo, groups) <= TOL_MIXED
    assert st["max_refine_residual"] <= 1e-6


def test_sampled_cells_rbc10k_plt1500_tf32():
    # the 10000 RBC + 1500 platelet workload with the TF32 apply, 1 step, sampled cells
    groups = [I.materialise(g) for g in I.workload_groups("rbc10k_plt1500")]
    xg, _, st = run_gpu(groups, 1, precision="tf32")
    xo, _ = run_oracle(groups, 1, sample=[[0, 5000, 9999], [0, 1499]])
    assert rel_pos_err(xg, xo, groups) <= TOL_MIXED
    assert st["max_refine_residual"] <= 1e-6


def test_sampled_cells_hetero20k_full_bf16():
    # the full 20000-cell, 12-type batch in one grouped launch per global step, 1 step,
    # the first and last cell of every type vs the oracle
    groups = [I.materialise(g) for g in I.workload_groups("hetero20k")]
    assert sum(g.n_cells for g in groups) == 20000
    xg, _, st = run_gpu(groups, 1, precision="bf16")
    xo, _ = run_oracle(groups, 1, sample=[[0, g.n_cells - 1] for g in groups])
    assert rel_pos_err(xg, xo, groups) <= TOL_MIXED
    assert st["max_refine_residual"] <= 1e-6


_TUNE_SCRIPT = r"""
import sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_1911_03062_gb300 import inputs as I
from paper_1911_03062_gb300.npfem import Solver
g = I.materialise(I.Group(I.rbc_type(), 40, seed=9, amp=0.3))
s = Solver(precision="bf16", autotune_cache=sys.argv[2])
s.add_cells(s.create_type(g.mtype), g.x0, g.v0)
for _ in range(2):
    s.step(g.f_ext.ravel())
np.save(sys.argv[3], s.positions())
s.close()
"""


def test_autotune_cache_file_round_trip(tmp_path):
    # a context that tunes writes its choices (one line per (mesh, operand type, row
    # bucket): the creation bucket and the bucket of its 40 cells); a second context in a
    # fresh process (empty in-process cache) reads them back, tunes nothing, and steps
    # bitwise like the first
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cache = tmp_path / "tiles.txt"
    outs = [tmp_path / "x1.npy", tmp_path / "x2.npy"]
    lines = []
    for out in outs:
        subprocess.run([sys.executable, "-c", _TUNE_SCRIPT, root, str(cache), str(out)], check=True, timeout=600)
        lines.append(cache.read_text().splitlines())
    assert len(lines[0]) == 2 and lines[1] == lines[0]
    assert any("|rows=3072" in ln for ln in lines[0]) and any("|rows=24576" in ln for ln in lines[0])
    for ln in lines[0]:
        key, nt, st, us = ln.split()
        assert int(nt) % 32 == 0 and 2 <= int(st) <= 6 and float(us) > 0
    assert np.array_equal(np.load(outs[0]), np.load(outs[1]))


@pytest.mark.parametrize("prec,graph", [("bf16", True), ("fp64", False)])
def test_host_forces_in_pieces_match_device_forces(prec, graph):
    # Host forces are copied in four pieces on a second stream and each type's predictor is
    # launched per piece as the pieces arrive; a device force array is read in place.  Two
    # types whose cells come in two batches each, so the public array interleaves them and
    # the pieces split both types' cell runs.  The steps must agree bit for bit.
    import torch
    from paper_1911_03062_gb300.npfem import Solver
    g = make_groups([(I.rbc_type(), 6, 0.3), (I.plt_type(), 5, 0.3)])
    order = [(0, slice(0, 3)), (1, slice(0, 2)), (0, slice(3, 6)), (1, slice(2, 5))]
    f_pub = np.concatenate([g[gi].f_ext[sl].ravel() for gi, sl in order])

    def run(on_device):
        s = Solver(precision=prec, use_graph=graph)
        ids = [s.create_type(gr.mtype) for gr in g]
        for gi, sl in order:
            s.add_cells(ids[gi], g[gi].x0[sl], g[gi].v0[sl])
        f = torch.from_numpy(f_pub).to("cuda") if on_device else f_pub
        for _ in range(3):
            s.step(f)
        x, v = s.positions(), s.velocities()
        s.close()
        return x, v

    xh, vh = run(False)
    xd, vd = run(True)
    assert np.all(np.isfinite(xh))
    assert np.array_equal(xh, xd) and np.array_equal(vh, vd)


@pytest.mark.parametrize("graph", [True, False])
def test_kernel_timing_mode(graph):
    # Per-kernel CUDA-event times (npfem_profile) with the step's graph and without it, host
    # forces (the predictor launched outside the graph, per force piece) and device forces:
    # every launch of the step is timed and the positions are the same bits as untimed.
    import torch
    from paper_1911_03062_gb300.npfem import Solver
    g = make_groups([(I.rbc_type(), 8, 0.3), (I.plt_type(), 4, 0.3)])
    f = public(g, "f_ext")

    def run(prof):
        s = Solver(precision="bf16", use_graph=graph)
        for gr in g:
            s.add_cells(s.create_type(gr.mtype), gr.x0, gr.v0)
        s.profile(prof)
        s.step(f)
        s.step(torch.from_numpy(f).to("cuda"))
        times = s.profile_read() if prof else {}
        x, n = s.positions(), s.stats()["launches_per_step"]
        s.close()
        return x, times, n

    x0, _, _ = run(False)
    x1, times, n = run(True)
    assert np.array_equal(x0, x1)
    assert sum(c for _, c in times.values()) == 2 * n - 2      # all but the force-pointer kernel
    assert times["predict"][1] >= 2 * 2 and times["iterate"][1] == 2 * 2 * 10
    assert all(ms > 0 for ms, _ in times.values())
