"""Particle-in-kernel collisions (paper Sec. 2.2 and the supplementary PIK
section) on the CUDA path vs the FP64 oracle's brute-force search: cells packed
into a small box so that many vertices have foreign vertices in their kernel.
Bars: FP64 1e-10 on the step map, mixed forms 1e-6 relative position error; the
number of contaminated vertices must match the oracle's exactly.

The step map with contacts amplifies input differences more than without: the
oracle against itself with 1e-13 perturbations of the positions moves by
~4e-11 (kc = 2), ~3e-10 (kc = 50), ~1e-9 (kc = 200) relative, against ~5e-12
without contacts.  The FP64 test therefore runs at kc = 2, where the collision
force still moves the cells by ~1e-4 R per step; the mixed forms run at kc = 200.
All calls go through libnpfem.so."""
import numpy as np
import pytest

from paper_1911_03062_gb300 import inputs as I

from helpers import public, split

pytestmark = pytest.mark.gpu

RK, KC, KC_FP64 = 0.5, 200.0, 2.0


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as G
    G.build()


def packed_groups(seed, n_rbc=4, n_plt=3, box=7.0):
    return [I.materialise(I.Group(I.rbc_type(), n_rbc, seed, amp=0.3, box=box)),
            I.materialise(I.Group(I.plt_type(), n_plt, seed + 1, amp=0.3, box=box))]


def _oracle_step(groups, xs, vs, Ts, kc=KC):
    """One PIK step of every cell (public order: groups in order, cells in order)."""
    from oracle import oracle as O
    cells = [(Ts[gi], xs[gi][c]) for gi, g in enumerate(groups) for c in range(g.n_cells)]
    res = O.pik(cells, RK)
    out_x, out_v, k, contacts = [], [], 0, 0
    for gi, g in enumerate(groups):
        xg, vg = np.empty_like(xs[gi]), np.empty_like(vs[gi])
        for c in range(g.n_cells):
            hc, _, p = res[k]
            hit = (hc >= 0).astype(np.int32)
            contacts += int(hit.sum())
            xo, vo = Ts[gi].step_cells_col(xs[gi][c][None], vs[gi][c][None], g.f_ext[c][None], kc, hit[None],
                                           p[None])
            xg[c], vg[c] = xo[0], vo[0]
            k += 1
        out_x.append(xg)
        out_v.append(vg)
    return out_x, out_v, contacts


def _gpu(groups, precision, kc=KC, **opts):
    from paper_1911_03062_gb300.npfem import Solver
    s = Solver(precision=precision, pik_radius=RK, collision_k=kc, **opts)
    for g in groups:
        s.add_cells(s.create_type(g.mtype), g.x0, g.v0)
    return s


def _err(xa, xb, groups):
    return max(float(np.linalg.norm(a - b, axis=2).max() / g.mtype.radius) for a, b, g in zip(xa, xb, groups))


def test_contact_fp64_step_map_matches_oracle():
    # every step: one oracle step from the GPU state, contacts counted alike
    from oracle import oracle as O
    groups = packed_groups(500)
    Ts = [O.OracleType.from_mesh_type(g.mtype) for g in groups]
    f = public(groups, "f_ext")
    s, weak = _gpu(groups, "fp64", KC_FP64), _gpu(groups, "fp64", 1e-9)
    total = 0
    for step in range(3):
        xn, vn = split(s.positions(), groups), split(s.velocities(), groups)
        s.step(f)
        x1, st = split(s.positions(), groups), s.stats()
        xo, _, contacts = _oracle_step(groups, xn, vn, Ts, kc=KC_FP64)
        assert st["contacts"] == contacts, (step, st["contacts"], contacts)
        assert _err(x1, xo, groups) <= 1e-10, step
        total += contacts
        if step == 0:
            weak.step(f)                          # the same step with a negligible collision force
            assert _err(x1, split(weak.positions(), groups), groups) > 1e-5
    s.close()
    weak.close()
    assert total > 1000


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_contact_mixed_step_matches_oracle(prec):
    # the step map from the GPU state after two steps (the search reads that state)
    from oracle import oracle as O
    groups = packed_groups(501)
    Ts = [O.OracleType.from_mesh_type(g.mtype) for g in groups]
    s = _gpu(groups, prec)
    f = public(groups, "f_ext")
    for _ in range(2):
        s.step(f)
    xn, vn = split(s.positions(), groups), split(s.velocities(), groups)
    s.step(f)
    st = s.stats()
    x1 = split(s.positions(), groups)
    s.close()
    xo, _, contacts = _oracle_step(groups, xn, vn, Ts)
    assert st["contacts"] == contacts and contacts > 50
    assert _err(x1, xo, groups) <= 1e-6, prec


def test_no_contact_is_the_plain_step():
    from paper_1911_03062_gb300.npfem import Solver
    groups = [I.materialise(I.Group(I.rbc_type(), 3, 502, amp=0.3)), I.materialise(I.Group(I.plt_type(), 2, 503, amp=0.3))]
    f = public(groups, "f_ext")
    out = []
    for opts in ({}, {"pik_radius": RK, "collision_k": KC}):
        s = Solver(precision="fp64", **opts)
        for g in groups:
            s.add_cells(s.create_type(g.mtype), g.x0, g.v0)
        s.step(f)
        out.append((s.positions(), s.stats()))
        s.close()
    assert out[1][1]["contacts"] == 0
    assert np.array_equal(out[0][0], out[1][0])


def test_contact_option_validation():
    from paper_1911_03062_gb300.npfem import EINVAL, NpfemError, Solver
    with pytest.raises(NpfemError) as e:
        Solver(precision="fp64", pik_radius=0.5, collision_k=0.0)
    assert e.value.code == EINVAL


def test_all_optional_parts_together_fp64():
    # median filter, collisions, Rayleigh damping, PBD damping and the velocity cap in one
    # step, composed in the oracle in the library's order: median of the given forces ->
    # search on x_n -> damped step with the contact term -> PBD -> cap
    import dataclasses
    from oracle import oracle as O
    from paper_1911_03062_gb300.npfem import Solver
    damp = lambda mt: dataclasses.replace(mt, material=dataclasses.replace(mt.material, rayleigh_alpha=1.0,
                                                                           rayleigh_beta=0.01))
    groups = [I.materialise(I.Group(damp(I.rbc_type()), 3, 510, amp=0.3, box=6.0)),
              I.materialise(I.Group(damp(I.plt_type()), 2, 511, amp=0.3, box=6.0))]
    kc, kappa, umax = KC_FP64, 0.7, 0.4
    s = Solver(precision="fp64", force_median=True, u_max=umax, pbd_kappa=kappa, pik_radius=RK, collision_k=kc)
    for g in groups:
        s.add_cells(s.create_type(g.mtype), g.x0, g.v0)
    s.step(public(groups, "f_ext"))
    x1, v1, st = split(s.positions(), groups), split(s.velocities(), groups), s.stats()
    s.close()
    Ts = [O.OracleType.from_mesh_type(g.mtype) for g in groups]
    res = O.pik([(Ts[gi], g.x0[c]) for gi, g in enumerate(groups) for c in range(g.n_cells)], RK)
    k, contacts = 0, 0
    for gi, g in enumerate(groups):
        T = Ts[gi]
        for c in range(g.n_cells):
            hc, _, p = res[k]
            k += 1
            hit = (hc >= 0).astype(np.int32)
            contacts += int(hit.sum())
            f = O.force_median(T, g.f_ext[c][None])
            xo, vo = T.step_cells_col(g.x0[c][None], g.v0[c][None], f, kc, hit[None], p[None])
            vo = O.velocity_cap(O.pbd_damping(T, xo, vo, kappa), umax)
            assert np.linalg.norm(x1[gi][c] - xo[0], axis=1).max() / g.mtype.radius <= 1e-10, (gi, c)
            assert np.abs(v1[gi][c] - vo[0]).max() <= 1e-5 * umax, (gi, c)
    assert st["contacts"] == contacts and contacts > 100
