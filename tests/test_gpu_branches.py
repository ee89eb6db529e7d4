"""The step's rare branches on the GPU against the FP64 oracle, the failure paths
that can be reached without faulting a GPU, and the binding's argument checks.

Branches (Supp. Sec. 2.1, the quasi-Newton update after Eq.
(genericOptimizationNewton), and the projections of the element energies):
  - the descent fallback: an indefinite L-BFGS update (a negative-curvature pair
    admitted with curvature_tol = -inf) gives an uphill direction, the history is
    cleared and -P^{-1} grad g taken (k_fallback, k_fallback_apply);
  - the Armijo cap: c1 = 0.9 and two halvings, so most searches take the last trial;
  - collapsed triangles (sigma_2 <= tol sigma_1: the polar factor's tie-break), whose
    branch is decided by rounding, so its bar is the oracle's own sensitivity;
  - flat hinges (|b_rest| = 0) and a hinge flattened exactly (|b| ~ 0: p = b);
  - the volume projection taking several Gauss-Newton updates (squeezed cells);
  - the literal FP64 refinement residual (residual_fp64 = 1).
Each run asserts from stats() that its branch ran.  All calls go through
libnpfem.so."""
import numpy as np
import pytest

from paper_1911_03062_gb300 import inputs as I

from helpers import branch_cell, group_of, make_groups, rel_pos_err, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "bf16": 1e-6, "tf32": 1e-6}


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as G
    G.build()


def oracle_step(mt, xn, vn, f, **kw):
    from oracle import oracle as O
    T = O.OracleType.from_mesh_type(mt)
    x1, _, tr = T.step_trace(xn, vn, f, **kw)
    return x1, tr


def err_one(xg, x1, mt):
    return float(np.linalg.norm(xg.reshape(-1, 3) - x1, axis=1).max() / mt.radius)


def test_descent_fallback_matches_oracle():
    mt, xn, vn, f = branch_cell(seed=23, mirror=True)
    g = group_of(mt, xn, vn, f)
    K, m = 22, 3
    for tol, n_fb in ((1e-12, 0), (-np.inf, 1)):
        x1, tr = oracle_step(mt, xn, vn, f, K=K, m=m, curv_tol=tol)
        assert tr["fallback"].sum() == n_fb
        xg, _, st = run_gpu([g], 1, "fp64", iters=K, history=m, curvature_tol=tol)
        assert st["fallbacks"] == n_fb, (tol, st)
        assert err_one(xg[0], x1, mt) <= TOL["fp64"], (tol, err_one(xg[0], x1, mt))


def test_descent_fallback_runs_in_the_mixed_kernels():
    # The inside-out state is ill-conditioned: the oracle itself moves its result by up to
    # 1e-4 R when its input is perturbed at FP32 rounding level (6e-8 relative), so the
    # mixed forms' 1e-6 bar does not apply to it.  Here the BF16 kernels must take the
    # same branch (one fallback with every pair admitted, none with the method's rule)
    # and stay finite.
    mt, xn, vn, f = branch_cell(seed=23, mirror=True)
    g = group_of(mt, xn, vn, f)
    for tol, n_fb in ((1e-12, 0), (-np.inf, 1)):
        xg, _, st = run_gpu([g], 1, "bf16", iters=22, history=3, curvature_tol=tol)
        assert st["fallbacks"] == n_fb and np.all(np.isfinite(xg[0])), (tol, st)


@pytest.mark.parametrize("prec", ["fp64", "bf16"])
def test_line_search_cap_matches_oracle(prec):
    mt, xn, vn, f = branch_cell(seed=7)
    K, c1, cap = 8, 0.9, 2
    x1, tr = oracle_step(mt, xn, vn, f, K=K, m=3, c1=c1, max_bt=cap)
    assert tr["caps"] >= K - 2
    xg, _, st = run_gpu([group_of(mt, xn, vn, f)], 1, prec, iters=K, history=3, armijo_c1=c1,
                        max_backtracks=cap)
    assert st["capped_searches"] == tr["caps"], st
    assert st["backtracks"] == tr["backtracks"].sum(), st
    assert err_one(xg[0], x1, mt) <= TOL[prec]


def collapsed_cells(n=2):
    """Level-2 RBCs with 6 triangles each collapsed onto a segment (one vertex at the
    midpoint of the opposite edge), at rest velocity and zero force, so the first
    local step evaluates them collapsed (x^0 = y = x_n)."""
    unit, tris = I.icosphere(2)
    rest = I.rbc_shape(unit)
    mt = I.MeshType("rbc-l2", rest, tris, I.RBC_MATERIAL, I.RBC_R0)
    xs = []
    for c in range(n):
        rng = np.random.default_rng(30 + c)
        x = rest @ I.random_rotations(rng, 1)[0].T + rng.uniform(0, 50, 3)
        used, k = set(), 0
        for t in rng.permutation(len(tris)):
            a, b, cc = tris[t]
            if {a, b, cc} & used:
                continue
            x[a] = 0.5 * (x[b] + x[cc])
            used |= {a, b, cc}
            k += 1
            if k == 6:
                break
        xs.append(x)
    x = np.stack(xs)
    return mt, x, np.zeros_like(x), np.zeros_like(x)


@pytest.mark.parametrize("prec,unit", [("fp64", 1.1e-16), ("bf16", 6e-8)])
def test_collapsed_triangles_within_the_oracles_own_sensitivity(prec, unit):
    # At a collapsed triangle the polar factor is not unique (F has rank 1): sigma_2 is
    # computed as sqrt(det(F^T F)/l1), whose cancellation leaves it at ~1e-8 sigma_1 or at
    # zero depending on the last bits, so whether the tie-break branch (sigma_2 <= tol
    # sigma_1) or the generic one runs is decided by rounding -- in the oracle as on the
    # GPU.  The bar is therefore the oracle's own sensitivity: its result moves by ~1e-8 R
    # (FP64) when the input is perturbed at rounding level.  An implementation rounds at
    # each of the K = 10 iterations, so the GPU must stay within a few times the oracle's
    # response to perturbations of K rounding units of its local-step arithmetic (unit:
    # FP64 1.1e-16, FP32 6e-8).
    rel = 10 * unit
    from oracle import oracle as O
    mt, xn, vn, f = collapsed_cells()
    tris = mt.tris
    for x in xn:                           # collapsed to rounding level
        E = np.stack([x[tris[:, 1]] - x[tris[:, 0]], x[tris[:, 2]] - x[tris[:, 0]]], axis=2)
        s = np.linalg.svd(E, compute_uv=False)
        assert (s[:, 1] <= 1e-12 * s[:, 0]).sum() == 6
    T = O.OracleType.from_mesh_type(mt)
    x1, _ = T.step_cells(xn, vn, f)
    rng = np.random.default_rng(0)
    sens = max(float(np.linalg.norm(T.step_cells(xn * (1 + rel * rng.standard_normal(xn.shape)), vn, f)[0] - x1,
                                    axis=2).max()) / mt.radius for _ in range(4))
    assert sens > 1e-9                     # the branch is rounding-decided: no 1e-10 bar exists here
    xg, _, _ = run_gpu([group_of(mt, xn, vn, f)], 1, prec)
    err = float(np.linalg.norm(xg[0] - x1, axis=2).max()) / mt.radius
    assert err <= 3 * sens, (err, sens)


def tetra_split():
    """The tetrahedron with each face split 4-way (no projection): 12 flat hinges."""
    v, f = I.tetrahedron()
    verts, cache, faces = [tuple(p) for p in v], {}, []

    def mid(a, b):
        k = (min(a, b), max(a, b))
        if k not in cache:
            verts.append(tuple((np.array(verts[a]) + verts[b]) / 2))
            cache[k] = len(verts) - 1
        return cache[k]

    for a, b, c in f:
        ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
        faces += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
    return np.array(verts), np.array(faces, np.int32)


def test_flat_and_flattened_hinges_fp64():
    from oracle import oracle as O
    V, F = tetra_split()
    flat_t = I.MeshType("tet4", V, F, I.Material(1.0, 5.0, 0.5, 10.0, 1e-2), 1.7)
    rng = np.random.default_rng(41)
    x_a = V + 0.05 * rng.standard_normal(V.shape)
    g_a = group_of(flat_t, x_a, rng.standard_normal(V.shape), rng.standard_normal(V.shape))
    # a level-1 RBC with one hinge of curved rest shape made exactly flat in the current state:
    # x3 = -(c0 x0 + c1 x1 + c2 x2) / c3 gives b = 0 (to rounding), the |b| ~ 0 branch p = b
    mt, xn, vn, f = branch_cell(seed=9, dt=1e-2)
    T = O.OracleType.from_mesh_type(mt)
    hv, hc, hr = T.hinges()
    h = int(np.argmax(hr))
    i0, i1, i2, i3 = hv[h]
    xn[i3] = -(hc[h, 0] * xn[i0] + hc[h, 1] * xn[i1] + hc[h, 2] * xn[i2]) / hc[h, 3]
    vn[[i0, i1, i2, i3]] = 0.0
    f[[i0, i1, i2, i3]] = 0.0
    b = hc[h] @ xn[[i0, i1, i2, i3]]
    assert np.linalg.norm(b) <= 1e-12 * hr[h]
    g_b = group_of(mt, xn, vn, f)
    groups = [g_a, g_b]
    xg, _, _ = run_gpu(groups, 2)
    xo, _ = run_oracle(groups, 2)
    assert rel_pos_err(xg, xo, groups) <= TOL["fp64"]


def squeezed_cells(n=4, seed=7):
    """Full RBCs (642 vertices) squeezed to about 95 % of their rest volume by a random
    diagonal scaling (0.97-0.99 per axis), at rest: the volume projection of the first
    local steps needs several Gauss-Newton updates, each with the volume gradient
    recomputed at the new point."""
    mt = I.rbc_type()
    rng = np.random.default_rng(seed)
    c = mt.rest.mean(axis=0)
    x = np.stack([(mt.rest - c) @ np.diag(rng.uniform(0.97, 0.99, 3)) + c for _ in range(n)])
    return mt, x, np.zeros_like(x), np.zeros_like(x)


def gn_updates(T, x, tol):
    """Updates the volume projection of the local step takes from x when it stops at
    |V - V0| <= tol |V0| (the same iteration as the oracle's, in numpy on its V and gV)."""
    V0, p = T.volume(T.rest), x.copy()
    for j in range(9):
        V = T.volume(p)
        if abs(V - V0) <= tol * abs(V0) or j == 8:
            return j
        g = T.volume_grad(p)
        p = x + (V0 - V - np.sum(g * (x - p))) / np.sum(g * g) * g


@pytest.mark.parametrize("prec", ["fp64", "bf16"])
def test_volume_projection_with_several_updates(prec):
    # The FP64 path stops the projection at 1e-14 |V0| (here after 6-7 updates), the FP32
    # local step at 2e-6 |V0| after 2-3 updates; both recompute gV at every new point.
    # (The FP32 stop alone moves this step by 4.3e-7 R: the oracle built to stop at
    # 2e-6 |V0| lands there.  At larger volume deficits it moves it further: 3.6e-6 R
    # for cells squeezed to ~85 %.)
    from oracle import oracle as O
    mt, xn, vn, f = squeezed_cells()
    T = O.OracleType.from_mesh_type(mt)
    tol = 1e-14 if prec == "fp64" else 2e-6
    upd = [gn_updates(T, x, tol) for x in xn]
    assert min(upd) >= 2 and max(upd) >= 3, upd
    x1, _ = T.step_cells(xn, vn, f)
    xg, _, _ = run_gpu([group_of(mt, xn, vn, f)], 1, prec)
    err = float(np.linalg.norm(xg[0] - x1, axis=2).max()) / mt.radius
    assert err <= TOL[prec], err


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_fp64_refinement_residual(prec):
    # the literal FP64 residual option on 50 RBC (150 RHS rows: ragged tiles) + 7 platelets
    groups = make_groups([(I.rbc_type(), 50, 0.3), (I.plt_type(), 7, 0.3)])
    xg, _, st = run_gpu(groups, 3, prec, residual_fp64=True)
    xo, _ = run_oracle(groups, 3)
    assert rel_pos_err(xg, xo, groups) <= TOL[prec]
    assert 0 < st["max_refine_residual"] <= 1e-6


# ------------------------------------------------------------ failure paths
def test_enomem_leaves_the_context_usable():
    import torch
    from paper_1911_03062_gb300.npfem import ENOMEM, NpfemError, Solver
    mt = I.rbc_type()
    small = I.materialise(I.Group(mt, 4, seed=1))
    s = Solver(precision="bf16")
    tid = s.create_type(mt)
    s.add_cells(tid, small.x0, small.v0)
    f = small.f_ext.ravel()
    s.step(f)
    x_before = s.positions()
    # leave ~1.5 GB free, then ask for ~3.8 GB of cells: cudaMalloc refuses at once
    free, _ = torch.cuda.mem_get_info()
    hog = torch.empty(max(0, free - (3 << 29)), dtype=torch.uint8, device="cuda")
    big = I.materialise(I.Group(mt, 20000, seed=2))
    with pytest.raises(NpfemError) as e:
        s.add_cells(tid, big.x0, big.v0)
    assert e.value.code == ENOMEM
    del hog, big
    torch.cuda.empty_cache()
    # nothing changed: same cells, same state, and it still steps
    assert s.num_dofs == f.size
    assert np.array_equal(s.positions(), x_before)
    s.step(f)
    s.sync()
    more = I.materialise(I.Group(mt, 3, seed=3))
    s.add_cells(tid, more.x0, more.v0)
    s.step(np.concatenate([f, more.f_ext.ravel()]))
    assert np.all(np.isfinite(s.positions()))
    s.close()


def test_expired_wait_reports_etimeout_and_the_context_recovers():
    from paper_1911_03062_gb300.npfem import ETIMEOUT, NpfemError, Solver
    g = I.materialise(I.Group(I.plt_type(), 3, seed=4))
    s = Solver(precision="bf16")
    s.add_cells(s.create_type(g.mtype), g.x0, g.v0)
    s.check_wait(20)
    with pytest.raises(NpfemError) as e:
        s.sync()
    assert e.value.code == ETIMEOUT and "site 90" in str(e.value)
    s.sync()                               # the error word was cleared
    s.step(g.f_ext.ravel())
    assert np.all(np.isfinite(s.positions()))
    s.close()


# ------------------------------------------------------------ binding checks
def test_binding_rejects_bad_device_arguments():
    import torch
    from paper_1911_03062_gb300.npfem import Solver
    g = I.materialise(I.Group(I.plt_type(), 2, seed=5))
    s = Solver(precision="fp64")
    tid = s.create_type(g.mtype)
    s.add_cells(tid, g.x0, g.v0)
    n, nV = s.num_dofs, g.mtype.nV
    dev = lambda *shape, **kw: torch.zeros(shape, dtype=kw.get("dtype", torch.float64), device="cuda")
    bad_steps = [dev(n - 3), dev(n + 3), dev(n, dtype=torch.float32), dev(2 * n)[::2]]
    for f in bad_steps:
        with pytest.raises(ValueError):
            s.step(f)
    q = dev(6, nV)
    for qq, zz in [(dev(6, nV + 1), dev(6, nV + 1)), (q, dev(5, nV)), (q, dev(6, nV, dtype=torch.float32)),
                   (dev(6 * nV), dev(6 * nV)), (q, dev(nV, 6).t()), (q, torch.zeros(6, nV))]:
        for fn in (s.apply_pinv, s.apply_pinv_noalloc):
            with pytest.raises(ValueError):
                fn(tid, qq, zz)
    with pytest.raises(ValueError):
        s.apply_pinv(tid + 1, q, dev(6, nV))
    with pytest.raises(ValueError):
        s.positions(out=dev(n - 1))
    with pytest.raises(ValueError):
        s.add_cells(tid, g.x0.ravel()[:-1])
    with pytest.raises(ValueError):
        s.add_cells(tid, g.x0, g.v0[:1])
    with pytest.raises(ValueError):
        s.set_state(s.positions(), np.zeros(5))
    # and the good calls still work after the rejected ones, ordered on torch's stream
    f = torch.from_numpy(g.f_ext.ravel()).to("cuda")
    s.step(f)
    out = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    s.positions(out=out)
    assert torch.isfinite(out).all()
    z = s.apply_pinv(tid, torch.ones(6, nV, dtype=torch.float64, device="cuda"), dev(6, nV))
    assert torch.isfinite(z).all() and (z != 0).any()
    s.close()
