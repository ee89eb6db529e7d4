"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: each test checks a closed form,
an invariant of Eq. (genericOptimizationNewton) (Supplementary Sec. 2.1), a
library routine (numpy SVD / Cholesky, scipy minimisers), finite
differences, or a brute-force computation on a tiny mesh.
"""
import numpy as np
import pytest

from paper_1911_03062_gb300 import inputs as I


@pytest.fixture(scope="module")
def O(oracle_lib):
    return oracle_lib


@pytest.fixture(scope="module")
def rbc(O):
    return I.rbc_type(), O.OracleType.from_mesh_type(I.rbc_type())


@pytest.fixture(scope="module")
def plt(O):
    return I.plt_type(), O.OracleType.from_mesh_type(I.plt_type())


def small_rbc(O, level=1, **kw):
    unit, tris = I.icosphere(level)
    mat = dict(k_strain=1.0, k_area=5.0, k_bend=0.05, k_vol=10.0, dt=1e-3)
    mat.update(kw)
    return I.rbc_shape(unit), tris, O.OracleType(I.rbc_shape(unit), tris, **mat)


def rot(seed):
    return I.random_rotations(np.random.default_rng(seed), 1)[0]


# ------------------------------------------------------------------ meshes
@pytest.mark.parametrize("level", [0, 1, 2, 3, 4])
def test_icosphere_topology(level):
    v, f = I.icosphere(level)
    nV = 10 * 4 ** level + 2
    assert v.shape == (nV, 3) and f.shape == (2 * nV - 4, 3)
    assert np.allclose(np.linalg.norm(v, axis=1), 1.0)
    # closed 2-manifold, consistently oriented: each directed edge once, its twin once
    de = {}
    for a, b, c in f:
        for e in ((a, b), (b, c), (c, a)):
            assert e not in de
            de[e] = 1
    assert all((b, a) in de for (a, b) in de)
    # outward: every face normal points away from the origin
    n = np.cross(v[f[:, 1]] - v[f[:, 0]], v[f[:, 2]] - v[f[:, 0]])
    assert np.all(np.einsum("ij,ij->i", n, v[f].mean(axis=1)) > 0)


def test_evans_fung_profile():
    # centre thickness R0*C0, maximum thickness of the published profile
    r2 = np.linspace(0, 1, 200001)
    t = I.RBC_R0 * np.sqrt(1 - r2) * (I.RBC_C0 + I.RBC_C1 * r2 + I.RBC_C2 * r2 ** 2)
    assert t[0] == pytest.approx(0.810, abs=5e-4)
    assert t.max() == pytest.approx(2.566, abs=5e-4)
    assert r2[np.argmax(t)] == pytest.approx(0.490, abs=5e-3)
    rest = I.rbc_type().rest
    assert np.ptp(rest[:, 0]) == pytest.approx(2 * I.RBC_R0, rel=1e-12)


# ------------------------------------------------------------- projections
def test_polar_matches_library_svd(O):
    rng = np.random.default_rng(0)
    for _ in range(200):
        F = rng.standard_normal((3, 2))
        T, s = O.polar(F)
        U, S, Vt = np.linalg.svd(F, full_matrices=False)
        assert np.allclose(s, S, rtol=1e-12, atol=1e-14)
        assert np.allclose(T, U @ Vt, atol=1e-11)
        assert np.allclose(T.T @ T, np.eye(2), atol=1e-12)


def test_polar_special_cases(O):
    Q = np.linalg.qr(np.random.default_rng(1).standard_normal((3, 3)))[0][:, :2]
    T, s = O.polar(Q)                        # already a rotation: fixed point
    assert np.allclose(T, Q, atol=1e-14) and np.allclose(s, 1)
    T, s = O.polar(3.0 * Q)                  # uniform scale: same polar factor
    assert np.allclose(T, Q, atol=1e-14) and np.allclose(s, 3)
    F = np.outer([0.0, 0.0, 2.0], [1.0, 0.0])   # rank-1: degenerate triangle branch
    T, s = O.polar(F)
    assert s[1] == 0 and np.allclose(T.T @ T, np.eye(2), atol=1e-14)


def brute_area(s1, s2):
    """Global minimiser of (d1-s1)^2 + (1/d1-s2)^2 over d1 > 0 by grid + golden section."""
    from scipy.optimize import minimize_scalar
    phi = lambda d: (d - s1) ** 2 + (1.0 / d - s2) ** 2
    grid = np.exp(np.linspace(np.log(1e-3), np.log(1e3), 200001))
    i = int(np.argmin(phi(grid)))
    r = minimize_scalar(phi, bounds=(grid[max(i - 1, 0)], grid[min(i + 1, len(grid) - 1)]),
                        method="bounded", options=dict(xatol=1e-14))
    return np.array([r.x, 1.0 / r.x])


def test_area_target_brute_force(O):
    rng = np.random.default_rng(2)
    cases = [(1.0, 1.0), (1.3, 1.3), (0.7, 0.7), (1.5, 0.9), (1.2, 0.3), (3.0, 2.0), (0.2, 0.1),
             (1.0, 1e-9)]
    cases += [tuple(sorted(rng.uniform(0.2, 2.5, 2), reverse=True)) for _ in range(40)]
    for s1, s2 in cases:
        d = O.area_target(s1, s2)
        assert d[0] * d[1] == pytest.approx(1.0, rel=1e-12)
        db = brute_area(s1, s2)
        f = lambda dd: (dd[0] - s1) ** 2 + (dd[1] - s2) ** 2
        assert f(d) <= f(db) + 1e-12, (s1, s2, d, db)
        assert np.allclose(d, db, rtol=1e-6), (s1, s2, d, db)


def test_area_target_equal_singular_values(O):
    for s in (0.3, 0.9, 1.0, 1.1, 1.9):
        assert np.allclose(O.area_target(s, s), [1.0, 1.0], atol=1e-14)


def test_area_projection_keeps_singular_vectors(O):
    rng = np.random.default_rng(3)
    for _ in range(100):
        F = rng.standard_normal((3, 2))
        Pa, d = O.area_project(F)
        U, S, Vt = np.linalg.svd(F, full_matrices=False)
        assert np.allclose(Pa, U @ np.diag(d) @ Vt, atol=1e-10)
        assert np.prod(np.linalg.svd(Pa, compute_uv=False)) == pytest.approx(1.0, rel=1e-12)


# ------------------------------------------------------------ volume, hinges
def test_volume_closed_forms(O):
    v, f = I.tetrahedron()
    T = O.OracleType(v, f, 1, 1, 1, 1, 1e-3)
    assert T.V0 == pytest.approx(8.0 / 3.0, rel=1e-14)          # regular tet of edge 2*sqrt(2)
    assert T.volume(v * 2.0 + 7.0) == pytest.approx(8.0 * 8.0 / 3.0, rel=1e-13)
    u, t = I.icosphere(4)
    S = O.OracleType(u, t, 1, 1, 1, 1, 1e-3)
    assert S.V0 == pytest.approx(4.0 / 3.0 * np.pi, rel=5e-3)
    assert S.V0 < 4.0 / 3.0 * np.pi                               # inscribed polyhedron


def test_volume_gradient_fd(O):
    rest, tris, T = small_rbc(O, 2)
    x = rest + 0.05 * np.random.default_rng(4).standard_normal(rest.shape)
    g = T.volume_grad(x)
    h = 1e-6
    fd = np.zeros_like(x)
    for i in range(x.shape[0]):
        for c in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, c] += h
            xm[i, c] -= h
            fd[i, c] = (T.volume(xp) - T.volume(xm)) / (2 * h)
    assert np.allclose(g, fd, atol=1e-8 * np.abs(g).max())
    assert np.allclose(g.sum(axis=0), 0, atol=1e-12)               # translation invariance


def test_volume_projection_kkt(O, rbc):
    # The projection is the Gauss-Newton closest-point iteration stopped once
    # the constraint holds; for a small violation that is also (to first
    # order) the KKT point: x - p parallel to grad V(p).
    mt, T = rbc
    rng = np.random.default_rng(5)
    x = mt.rest * np.array([1.001, 1.0, 1.0]) + 0.02 * rng.standard_normal(mt.rest.shape)
    p, it = T.volume_project(x)
    assert 1 <= it <= 8
    assert T.volume(p) == pytest.approx(T.V0, rel=1e-14)
    gV = T.volume_grad(p).ravel()
    r = (x - p).ravel()
    lam = r @ gV / (gV @ gV)
    assert np.linalg.norm(r - lam * gV) <= 1e-7 * np.linalg.norm(r)
    # p is no farther from x than other points of the constraint surface nearby
    for k in range(20):
        w = rng.standard_normal(r.shape)
        w -= (w @ gV) / (gV @ gV) * gV                 # tangent direction
        q = p.ravel() + 1e-3 * w / np.linalg.norm(w)
        gq = T.volume_grad(q.reshape(-1, 3)).ravel()
        q = q + (T.V0 - T.volume(q.reshape(-1, 3))) / (gq @ gq) * gq   # back onto V = V0
        assert np.linalg.norm(x.ravel() - q) >= np.linalg.norm(r) - 1e-12
    # a large violation: the iteration stops at its cap, close to the surface
    x2 = mt.rest * np.array([1.05, 0.97, 1.1])
    p2, it2 = T.volume_project(x2)
    assert it2 == 8 and T.volume(p2) == pytest.approx(T.V0, rel=1e-11)


def test_hinge_stencil_properties(O, rbc):
    mt, T = rbc
    hv, hc, hr = T.hinges()
    assert T.nH == 3 * mt.tris.shape[0] // 2
    assert np.allclose(hc.sum(axis=1), 0, atol=1e-12)              # kills translations
    # on the sphere the hinge vector is normal to the surface
    u, tris = I.icosphere(3)
    S = O.OracleType(u, tris, 1, 1, 1, 1, 1e-3)
    hv, hc, hr = S.hinges()
    b = np.einsum("hj,hjd->hd", hc, u[hv])
    nrm = u[hv[:, 0]] + u[hv[:, 1]]
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    cosang = np.abs(np.einsum("hd,hd->h", b, nrm)) / np.linalg.norm(b, axis=1)
    assert cosang.min() > 0.99
    # rotation + translation leave |b| unchanged
    R = rot(6)
    X2 = u @ R.T + 3.0
    b2 = np.einsum("hj,hjd->hd", hc, X2[hv])
    assert np.allclose(np.linalg.norm(b2, axis=1), hr, rtol=1e-12)


def test_flat_hinges_have_zero_rest_vector(O):
    # one 4-way split of the tetrahedron without projection: the edges inside
    # each original face are flat hinges
    v, f = I.tetrahedron()
    verts = [tuple(p) for p in v]
    cache, faces = {}, []

    def mid(a, b):
        k = (min(a, b), max(a, b))
        if k not in cache:
            verts.append(tuple((np.array(verts[a]) + verts[b]) / 2))
            cache[k] = len(verts) - 1
        return cache[k]

    for a, b, c in f:
        ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
        faces += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
    V, F = np.array(verts), np.array(faces, np.int32)
    T = O.OracleType(V, F, 1, 1, 1, 1, 1e-3)
    hv, hc, hr = T.hinges()
    flat = np.isclose(hr, 0, atol=1e-12)
    assert flat.sum() == 12                      # 3 inner edges per original face
    assert np.all(hr[~flat] > 0.1)


# --------------------------------------------------------------- matrix P
def test_P_structure_and_solve(O, rbc):
    mt, T = rbc
    P = T.P_dense()
    nV = mt.nV
    m = 1.0 / nV
    assert np.allclose(P, P.T, atol=0)
    # elastic parts annihilate constants: P 1 = (m/h^2 + k_vol) 1
    assert np.allclose(P.sum(axis=1), m / mt.material.dt ** 2 + mt.material.k_vol, rtol=1e-12)
    # library Cholesky + solve of the same matrix
    L = np.linalg.cholesky(P)
    b = np.random.default_rng(7).standard_normal((nV, 3))
    ref = np.linalg.solve(L.T, np.linalg.solve(L, b))
    x = T.solve(b)
    assert np.allclose(x, ref, rtol=1e-12, atol=1e-14 * np.abs(ref).max())
    assert np.linalg.norm(P @ x - b) <= 1e-12 * np.linalg.norm(b)
    assert T.nnzL < nV * nV / 4                  # the RCM envelope is sparse


def test_P_quadratic_form_at_rest(O, rbc):
    # F(rest) has orthonormal columns, so x^T A_t^T A_t x summed over xyz = 2 per
    # triangle: sum_c X_c^T P X_c = sum_t 2 (ks+ka) A_t + kb sum_e |b_rest|^2 + (m/h^2 + kv)|X|^2
    mt, T = rbc
    P = T.P_dense()
    X = mt.rest
    mat = mt.material
    e = X[mt.tris[:, 1]] - X[mt.tris[:, 0]]
    f = X[mt.tris[:, 2]] - X[mt.tris[:, 0]]
    area = 0.5 * np.linalg.norm(np.cross(e, f), axis=1)
    hv, hc, hr = T.hinges()
    expect = (2 * (mat.k_strain + mat.k_area) * area.sum() + mat.k_bend * (hr ** 2).sum()
              + (1.0 / mt.nV / mat.dt ** 2 + mat.k_vol) * (X ** 2).sum())
    got = np.einsum("vc,vw,wc->", X, P, X)
    assert got == pytest.approx(expect, rel=1e-12)


# ------------------------------------------------------------------ energy
def test_rest_state_is_stationary(O, rbc):
    mt, T = rbc
    R, t = rot(8), np.array([50.0, 120.0, 7.0])
    x = mt.rest @ R.T + t
    e, g, terms = T.energy(x, x)
    assert e < 1e-24 and np.abs(g).max() < 1e-12
    xo, vo = T.step(x, np.zeros_like(x), np.zeros_like(x))
    assert np.abs(xo - x).max() < 1e-13 * np.abs(x).max()
    assert np.abs(vo).max() < 1e-9


@pytest.mark.parametrize("term", [1, 2, 4, 8, 16])
def test_gradient_central_differences(O, term):
    rest, tris, T = small_rbc(O, 1)
    rng = np.random.default_rng(9 + term)
    x = rest * 1.08 + 0.08 * rng.standard_normal(rest.shape)
    y = rest + 0.05 * rng.standard_normal(rest.shape)
    e, g, _ = T.energy(x, y, mask=term)
    h = 1e-6
    fd = np.zeros_like(x)
    for i in range(x.shape[0]):
        for c in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, c] += h
            xm[i, c] -= h
            fd[i, c] = (T.energy(xp, y, term, grad=False)[0] - T.energy(xm, y, term, grad=False)[0]) / (2 * h)
    assert np.linalg.norm(g - fd) <= 1e-6 * np.linalg.norm(g), term


def test_energy_rigid_invariance(O, plt):
    mt, T = plt
    rng = np.random.default_rng(10)
    x = mt.rest * 1.1 + 0.05 * rng.standard_normal(mt.rest.shape)
    y = mt.rest + 0.03 * rng.standard_normal(mt.rest.shape)
    R, t = rot(11), np.array([-3.0, 40.0, 2.5])
    e1, g1, t1 = T.energy(x, y)
    e2, g2, t2 = T.energy(x @ R.T + t, y @ R.T + t)
    assert np.allclose(t1, t2, rtol=1e-10, atol=1e-14)
    assert np.allclose(g1 @ R.T, g2, atol=1e-10 * np.abs(g1).max())


# -------------------------------------------------------------- time step
def seeded_cell(mt, seed, amp=0.1):
    g = I.materialise(I.Group(mt, 1, seed, amp=amp))
    return g.x0[0], g.v0[0], g.f_ext[0]


def test_step_rigid_motion_invariance(O, rbc):
    mt, T = rbc
    xn, vn, f = seeded_cell(mt, 12, amp=2.0)
    vn = vn + 0.5 * np.random.default_rng(13).standard_normal(vn.shape)
    x1, v1 = T.step(xn, vn, f)
    R, t = rot(14), np.array([10.0, -20.0, 30.0])
    x2, v2 = T.step(xn @ R.T + t, vn @ R.T, f @ R.T)
    assert np.abs(x1 @ R.T + t - x2).max() < 1e-9 * mt.radius
    assert np.abs(v1 @ R.T - v2).max() < 1e-6


def test_step_conserves_linear_momentum(O, rbc):
    mt, T = rbc
    rng = np.random.default_rng(15)
    xn = mt.rest * np.array([1.1, 0.95, 1.2]) + 0.03 * rng.standard_normal(mt.rest.shape)
    vn = rng.standard_normal(mt.rest.shape)
    x1, v1 = T.step(xn, vn, np.zeros_like(xn))
    assert np.allclose(v1.mean(axis=0), vn.mean(axis=0), atol=1e-9)
    assert not np.allclose(v1, vn)


def test_step_energy_monotone(O, rbc):
    mt, T = rbc
    xn, vn, f = seeded_cell(mt, 16, amp=5.0)
    vn = vn + np.random.default_rng(17).standard_normal(vn.shape)
    for m in (5, 0):
        x1, v1, tr = T.step(xn, vn, f, m=m, trace=True)
        assert tr["caps"] == 0
        assert np.all(np.diff(tr["g"]) <= 0), tr["g"]
        assert tr["g"][-1] < tr["g"][0]


def test_pure_pd_is_local_global_iteration(O):
    # with no history and alpha = 1 accepted, x^{k+1} = P^{-1}(P x^k - grad g(x^k))
    rest, tris, T = small_rbc(O, 2)
    rng = np.random.default_rng(18)
    xn = rest * 1.05 + 0.02 * rng.standard_normal(rest.shape)
    vn = 0.1 * rng.standard_normal(rest.shape)
    f = 0.1 * rng.standard_normal(rest.shape)
    x1, _, tr = T.step(xn, vn, f, K=1, m=0, trace=True)
    assert tr["alpha"][0] == 1.0
    y = xn + T.dt * vn + T.dt ** 2 * rest.shape[0] * f
    _, g, _ = T.energy(y, y)
    P = T.P_dense()
    assert np.allclose(x1, np.linalg.solve(P, P @ y - g), atol=1e-12)


def test_step_converges_to_stationary_point_newtons_law(O, rbc):
    # Eq. (Newton2nd) with C = 0:  M (v_{n+1} - v_n)/h = F_int(x_{n+1}) + F_ext
    mt, T = rbc
    xn, vn, f = seeded_cell(mt, 19, amp=20.0)
    vn = vn + 2.0 * np.random.default_rng(20).standard_normal(vn.shape)
    x1, v1 = T.step(xn, vn, f, K=40)
    h, m = mt.material.dt, 1.0 / mt.nV
    _, gint, _ = T.energy(x1, x1, mask=30)          # sum_i grad E_i = -F_int
    resid = m * (v1 - vn) / h - (-gint + f)
    assert np.abs(resid).max() < 1e-7 * np.abs(m * (v1 - vn) / h).max()


def test_tetrahedron_matches_brute_force_newton(O):
    v, tris = I.tetrahedron()
    T = O.OracleType(v, tris, 1.0, 5.0, 0.05, 10.0, 0.05)
    rng = np.random.default_rng(21)
    xn = v + 0.05 * rng.standard_normal(v.shape)
    vn = 2.0 * rng.standard_normal(v.shape)
    f = 5.0 * rng.standard_normal(v.shape)
    x_orc, _ = T.step(xn, vn, f, K=200)
    y = xn + T.dt * vn + T.dt ** 2 * 4 * f
    # damped Newton with a finite-difference Hessian of the analytic gradient
    x = y.copy()
    for _ in range(100):
        e, g, _ = T.energy(x, y)
        if np.linalg.norm(g) < 1e-13:
            break
        H = np.zeros((12, 12))
        hh = 1e-6
        for i in range(12):
            xp, xm = x.ravel().copy(), x.ravel().copy()
            xp[i] += hh
            xm[i] -= hh
            H[:, i] = (T.energy(xp, y)[1].ravel() - T.energy(xm, y)[1].ravel()) / (2 * hh)
        H = 0.5 * (H + H.T)
        w = np.linalg.eigvalsh(H)
        mu = max(0.0, 1e-8 - w.min())
        d = -np.linalg.solve(H + mu * np.eye(12), g.ravel()).reshape(4, 3)
        a = 1.0
        while T.energy(x + a * d, y, grad=False)[0] > e and a > 1e-12:
            a *= 0.5
        x = x + a * d
    assert np.abs(x - x_orc).max() < 1e-9
    assert np.abs(x - y).max() > 1e-3             # a non-trivial minimiser


# ------------------------------------------- quasi-Newton control flow
# The update after Eq. (genericOptimizationNewton), x^{k+1} = x^k - alpha H grad g,
# with H the L-BFGS operator of initial matrix P^{-1}.  The oracle evaluates H grad g
# by the two-loop recursion; these tests rebuild H densely by the BFGS inverse update
# (Nocedal & Wright, Numerical Optimization, Eq. 6.17):
#     H <- (I - rho s y^T) H (I - rho y s^T) + rho s s^T,   rho = 1 / (s . y),
# from H_0 = P^{-1} (per component: kron(P^{-1}, I_3) in the [nV][3] layout) over the
# last min(k, m) kept pairs, oldest first, and check every iteration's direction,
# the history's curvature rule, the descent fallback and the Armijo acceptance
# against the step's own record (orc_step_trace).

def slow_cell(O, seed=5, dt=0.05, mirror=False):
    """A level-1 RBC at dt = 0.05 (inertia no longer dominant, so the iterations stay
    far from convergence for K > 15) in a deformed state with velocities and forces;
    mirror: inside out (large non-convex projections, a negative-curvature pair)."""
    from helpers import branch_cell
    mt, xn, vn, f = branch_cell(seed, dt, mirror)
    return O.OracleType.from_mesh_type(mt), xn, vn, f


def bfgs_directions(T, tr, m, curv_tol=1e-12):
    """Per iteration k of a traced step: (the direction the method prescribes, whether
    the descent fallback applies, the L-BFGS direction before that test), from the
    dense BFGS inverse update over the pairs of the recorded iterates."""
    n3 = 3 * T.nV
    H0 = np.kron(np.linalg.inv(T.P_dense()), np.eye(3))
    pairs, out = [], []
    for k in range(len(tr["d"])):
        g = tr["grad"][k].ravel()
        H = H0
        for s, y in pairs[-m:]:
            rho = 1.0 / (s @ y)
            V = np.eye(n3) - rho * np.outer(y, s)
            H = V.T @ H @ V + rho * np.outer(s, s)
        d_lbfgs = -H @ g
        fallback = bool(pairs) and g @ d_lbfgs >= 0
        if fallback:
            pairs = []
        out.append((-H0 @ g if fallback else d_lbfgs, fallback, d_lbfgs))
        s = (tr["x"][k + 1] - tr["x"][k]).ravel()
        y = (tr["grad"][k + 1] - tr["grad"][k]).ravel()
        if m > 0 and s @ y > curv_tol * np.linalg.norm(s) * np.linalg.norm(y):
            pairs.append((s, y))
    return out


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(b)


@pytest.mark.parametrize("m", [1, 3, 5])
def test_lbfgs_direction_is_the_dense_bfgs_inverse_update(O, m):
    T, xn, vn, f = slow_cell(O)
    K = 18
    x1, _, tr = T.step_trace(xn, vn, f, K=K, m=m)
    assert tr["kept"].all() and not tr["fallback"].any()
    dirs = bfgs_directions(T, tr, m)
    for k, (d, fb, _) in enumerate(dirs):
        assert rel(tr["d"][k], d) < 1e-10, (k, rel(tr["d"][k], d))
    # far from convergence to the end: the ring wraps with meaningful pairs
    assert np.linalg.norm(tr["d"][-1]) > 1e-5 * np.linalg.norm(tr["d"][0])
    # the history matters: a step with another m is a different step
    x1b, _ = T.step(xn, vn, f, K=K, m=m + 1)
    assert np.abs(x1 - x1b).max() > 1e-8
    # and the recorded iterates chain: x^{k+1} = x^k + alpha_k d_k, x_{n+1} = x^K
    for k in range(K):
        assert np.allclose(tr["x"][k + 1], tr["x"][k] + tr["alpha"][k] * tr["d"][k], rtol=0, atol=1e-13)
    assert np.array_equal(x1, tr["x"][K])


def test_curvature_rule_and_descent_fallback(O):
    T, xn, vn, f = slow_cell(O, seed=23, mirror=True)
    K, m = 22, 3
    # the method's threshold (s.y > 1e-12 |s||y|) rejects the negative-curvature pair
    _, _, tr = T.step_trace(xn, vn, f, K=K, m=m)
    sy = np.array([np.dot((tr["x"][k + 1] - tr["x"][k]).ravel(), (tr["grad"][k + 1] - tr["grad"][k]).ravel())
                   for k in range(K)])
    assert (sy < 0).sum() == 1 and not tr["kept"][sy < 0].any() and tr["kept"][sy > 0].all()
    for k, (d, fb, _) in enumerate(bfgs_directions(T, tr, m)):
        assert not fb and rel(tr["d"][k], d) < 1e-10, k
    # with every pair kept, the update after the indefinite one is not a descent
    # direction: the step clears its history and takes -P^{-1} grad instead
    _, _, tr = T.step_trace(xn, vn, f, K=K, m=m, curv_tol=-np.inf)
    dirs = bfgs_directions(T, tr, m, curv_tol=-np.inf)
    fbs = [fb for _, fb, _ in dirs]
    assert fbs == [bool(b) for b in tr["fallback"]] and sum(fbs) == 1
    k_fb = fbs.index(True)
    g = tr["grad"][k_fb].ravel()
    d_l = dirs[k_fb][2]
    assert g @ d_l > 0.05 * np.linalg.norm(g) * np.linalg.norm(d_l)      # decisively uphill
    assert rel(tr["d"][k_fb], -T.solve(tr["grad"][k_fb])) < 1e-12
    for k, (d, _, _) in enumerate(dirs):
        assert rel(tr["d"][k], d) < 1e-10, k
    # after the reset the history restarts from the fallback's own pair
    assert k_fb + 3 < K and all(tr["kept"][k_fb:])


def armijo_trials(T, tr, k, c1):
    """(energy at each halving j = 0..bt of iteration k, the Armijo right-hand sides)."""
    y = tr["x"][0]                      # x^0 = y, the inertia term's centre
    x, d, g0 = tr["x"][k], tr["d"][k], tr["g"][k]
    gd = float(np.dot(tr["grad"][k].ravel(), d.ravel()))
    e, rhs = [], []
    for j in range(tr["backtracks"][k] + 1):
        a = 0.5 ** j
        e.append(T.energy(x + a * d, y, grad=False)[0])
        rhs.append(g0 + c1 * a * gd)
    return np.array(e), np.array(rhs), gd


def test_armijo_takes_the_first_sufficient_halving(O):
    T, xn, vn, f = slow_cell(O, seed=7)
    K, c1 = 12, 0.9                     # c1 = 0.9: alpha = 1 rarely suffices
    x1, _, tr = T.step_trace(xn, vn, f, K=K, m=3, c1=c1, max_bt=8)
    assert tr["caps"] == 0 and tr["backtracks"].sum() >= K and tr["backtracks"].max() >= 2
    for k in range(K):
        e, rhs, gd = armijo_trials(T, tr, k, c1)
        assert gd < 0
        assert np.all(e[:-1] > rhs[:-1]), k            # every earlier halving fails
        assert e[-1] <= rhs[-1], k                     # the accepted one satisfies it
        assert tr["alpha"][k] == 0.5 ** tr["backtracks"][k]
        assert tr["g"][k + 1] == e[-1]                 # the energy of the accepted trial
    assert np.all(np.diff(tr["g"]) < 0)


def test_armijo_cap_takes_the_last_trial(O):
    T, xn, vn, f = slow_cell(O, seed=7)
    K, c1, cap = 8, 0.9, 2
    _, _, tr = T.step_trace(xn, vn, f, K=K, m=3, c1=c1, max_bt=cap)
    capped = 0
    for k in range(K):
        e, rhs, _ = armijo_trials(T, tr, k, c1)
        assert np.all(e[:-1] > rhs[:-1]), k
        assert tr["g"][k + 1] == e[-1]                 # the last trial evaluated is the one taken
        if e[-1] > rhs[-1]:                            # no trial met the condition: the cap
            capped += 1
            assert tr["backtracks"][k] == cap and tr["alpha"][k] == 0.5 ** cap
            assert np.allclose(tr["x"][k + 1], tr["x"][k] + 0.25 * tr["d"][k], rtol=0, atol=1e-13)
    assert capped == tr["caps"] and capped >= K - 2


def test_dynamics_amplify_rounding_level_perturbations(O):
    # The stepped dynamics of the amplitude-0.3 suspension amplify a 1e-12 R
    # perturbation of the initial positions by more than 100x within 40 steps, so two
    # implementations that differ only in rounding order separate at this rate; late
    # states are therefore compared on one step from a shared state.
    g = I.materialise(I.workload_groups("rbc50k_plt5k", scale=0.0002)[0])
    T = O.OracleType.from_mesh_type(g.mtype)
    rng = np.random.default_rng(3)
    xa, va = g.x0.copy(), g.v0.copy()
    xb, vb = g.x0 + 1e-12 * g.mtype.radius * rng.standard_normal(g.x0.shape), g.v0.copy()
    d0 = np.linalg.norm(xa - xb, axis=2).max()
    for _ in range(40):
        xa, va = T.step_cells(xa, va, g.f_ext, K=10, m=5, threads=4)
        xb, vb = T.step_cells(xb, vb, g.f_ext, K=10, m=5, threads=4)
    assert np.linalg.norm(xa - xb, axis=2).max() > 100 * d0


# ------------------------------------------------------- f2: force filter, velocity cap
def _closed_one_rings(tris, nV):
    ring = [set([v]) for v in range(nV)]
    for a, b, c in tris:
        for u, w in ((a, b), (b, c), (c, a)):
            ring[u].add(w)
            ring[w].add(u)
    return [sorted(r) for r in ring]


def test_force_median_matches_library_median(O, rbc):
    # component-wise median over {v} + one-ring (valence 5 -> 6 values: mean of the two
    # middle ones; valence 6 -> 7 values), against numpy's median on an independently
    # built neighbourhood
    mt, T = rbc
    f = np.random.default_rng(21).standard_normal((2, mt.nV, 3))
    got = O.force_median(T, f)
    rings = _closed_one_rings(mt.tris, mt.nV)
    assert {len(r) for r in rings} == {6, 7}
    ref = np.stack([np.stack([np.median(fc[r], axis=0) for r in rings]) for fc in f])
    assert np.array_equal(got, ref)


def test_force_median_constant_field_and_spike(O, rbc):
    mt, T = rbc
    f = np.tile(np.array([0.3, -1.2, 2.5]), (mt.nV, 1))
    assert np.array_equal(O.force_median(T, f), f)
    g = f.copy()
    g[100] = [1e6, -1e6, 3e3]                      # one spike: removed, neighbours untouched
    assert np.array_equal(O.force_median(T, g), f)


def test_velocity_cap_closed_form(O):
    rng = np.random.default_rng(22)
    v = rng.standard_normal((500, 3)) * rng.uniform(0.0, 0.2, (500, 1))
    umax = 0.05
    w = O.velocity_cap(v, umax)
    n, m = np.linalg.norm(v, axis=1), np.linalg.norm(w, axis=1)
    below = n <= umax
    assert np.array_equal(w[below], v[below])
    assert np.allclose(m[~below], umax, rtol=1e-15, atol=0)
    assert np.allclose(w[~below] / m[~below, None], v[~below] / n[~below, None], rtol=0, atol=1e-15)


# ------------------------------------------------------- f1: PBD velocity damping
def test_pbd_damping_keeps_rigid_motion_and_scales_the_rest(O, rbc):
    mt, T = rbc
    rng = np.random.default_rng(23)
    R = rot(5)
    x = mt.rest @ R.T + np.array([3.0, -1.0, 2.0])
    vcm, w = np.array([0.2, -0.1, 0.05]), np.array([0.3, 0.7, -0.4])
    xc = x.mean(axis=0)                                  # uniform masses
    rigid = vcm + np.cross(w, x - xc)
    # a rigid velocity field is left unchanged
    assert np.allclose(O.pbd_damping(T, x, rigid, 0.8), rigid, rtol=0, atol=1e-12)
    # a field with zero momentum and zero angular momentum is scaled by (1 - kappa)
    u = rng.standard_normal(x.shape)
    u -= u.mean(axis=0)
    r = x - xc
    Iten = (np.sum(r * r) * np.eye(3) - r.T @ r)
    Lmom = np.cross(r, u).sum(axis=0)
    u -= np.cross(np.linalg.solve(Iten, Lmom), r)        # remove the rigid rotation part
    assert np.allclose(O.pbd_damping(T, x, u, 0.7), 0.3 * u, rtol=0, atol=1e-12)
    # linear superposition: rigid part kept, the rest scaled
    assert np.allclose(O.pbd_damping(T, x, rigid + u, 0.5), rigid + 0.5 * u, rtol=0, atol=1e-12)
    # linear and angular momentum are conserved
    v0 = rigid + rng.standard_normal(x.shape)
    d = O.pbd_damping(T, x, v0, 0.9)
    assert np.allclose(d.sum(axis=0), v0.sum(axis=0), rtol=1e-12, atol=1e-12)
    assert np.allclose(np.cross(r, d).sum(axis=0), np.cross(r, v0).sum(axis=0), rtol=1e-12, atol=1e-10)


# ------------------------------------------------------------------ Rayleigh damping
ALPHA, BETA = 2.0, 0.01          # beta_D = 0.01 as in the paper's parameter table; alpha > 0 to pin both


def damped(mt, O, alpha=ALPHA, beta=BETA):
    return O.OracleType.from_mesh_type(mt).set_damping(alpha, beta)


def test_damping_zero_is_the_undamped_type(O, rbc):
    mt, T = rbc
    xn, vn, f = seeded_cell(mt, 40, amp=5.0)
    x1, v1 = T.step(xn, vn, f)
    x2, v2 = damped(mt, O, 0.0, 0.0).step(xn, vn, f)
    assert np.array_equal(x1, x2) and np.array_equal(v1, v2)
    with pytest.raises(ValueError):
        damped(mt, O, -1.0, 0.0)


def test_damped_P_is_Mt_over_h2_plus_L(O, rbc):
    # P = Mt/h^2 + L with Mt = M + h (alpha M + beta L), L = P_undamped - M/h^2
    mt, T = rbc
    h, m = mt.material.dt, 1.0 / mt.nV
    P0 = T.P_dense()
    L = P0 - np.eye(mt.nV) * m / h ** 2
    expect = P0 + (ALPHA * m * np.eye(mt.nV) + BETA * L) / h
    assert np.allclose(damped(mt, O).P_dense(), expect, rtol=1e-13, atol=1e-13 * np.abs(expect).max())


def test_damped_inertia_gradient_central_differences(O):
    rest, tris, T = small_rbc(O, 1)
    T.set_damping(ALPHA, 0.5)                        # large beta so the L term is not swamped
    rng = np.random.default_rng(41)
    x = rest * 1.08 + 0.08 * rng.standard_normal(rest.shape)
    y = rest + 0.05 * rng.standard_normal(rest.shape)
    e, g, _ = T.energy(x, y, mask=1)
    hh = 1e-6
    fd = np.zeros_like(x)
    for i in range(x.shape[0]):
        for c in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, c] += hh
            xm[i, c] -= hh
            fd[i, c] = (T.energy(xp, y, 1, grad=False)[0] - T.energy(xm, y, 1, grad=False)[0]) / (2 * hh)
    assert np.linalg.norm(g - fd) <= 1e-7 * np.linalg.norm(g)
    # and the quadratic form itself: e = 1/(2h^2) d^T Mt d, Mt from the undamped P
    _, _, T0 = small_rbc(O, 1)
    h, m = T.dt, 1.0 / rest.shape[0]
    L = T0.P_dense() - np.eye(rest.shape[0]) * m / h ** 2
    Mt = (1 + h * ALPHA) * m * np.eye(rest.shape[0]) + h * 0.5 * L
    d = x - y
    assert e == pytest.approx(np.einsum("vc,vw,wc->", d, Mt, d) / (2 * h ** 2), rel=1e-12)


def test_damped_step_converges_to_newtons_law(O, rbc):
    # Eq. (Newton2nd) with C = alpha M + beta L:  M (v1 - v0)/h + C v1 = F_int(x1) + F_ext
    mt, T = rbc
    xn, vn, f = seeded_cell(mt, 42, amp=20.0)
    vn = vn + 2.0 * np.random.default_rng(43).standard_normal(vn.shape)
    x1, v1 = damped(mt, O).step(xn, vn, f, K=40)
    h, m = mt.material.dt, 1.0 / mt.nV
    L = T.P_dense() - np.eye(mt.nV) * m / h ** 2
    _, gint, _ = T.energy(x1, x1, mask=30)
    lhs = m * (v1 - vn) / h + ALPHA * m * v1 + BETA * (L @ v1)
    assert np.abs(lhs - (-gint + f)).max() < 1e-7 * np.abs(m * (v1 - vn) / h).max()
    # the damping force is not negligible at this state
    assert np.abs(ALPHA * m * v1 + BETA * (L @ v1)).max() > 1e-3 * np.abs(m * (v1 - vn) / h).max()


def test_damped_step_mean_velocity_closed_form(O, rbc):
    # F_ext summing to zero: 1^T L = k_vol 1^T (elastic parts annihilate constants),
    # so at every iterate mean(v1) = mean(v0) / (1 + h alpha + h beta k_vol / m)
    mt, T = rbc
    xn, vn, _ = seeded_cell(mt, 44, amp=5.0)
    vn = vn + np.random.default_rng(45).standard_normal(vn.shape)
    f = np.random.default_rng(46).standard_normal(vn.shape)
    f -= f.mean(axis=0)
    x1, v1 = damped(mt, O).step(xn, vn, f)
    h, m, kv = mt.material.dt, 1.0 / mt.nV, mt.material.k_vol
    expect = vn.mean(axis=0) / (1 + h * ALPHA + h * BETA * kv / m)
    assert np.allclose(v1.mean(axis=0), expect, rtol=1e-9, atol=1e-12)


# ------------------------------------------------------------------ PIK collisions
RK, KC = 0.5, 200.0


def octahedron():
    v = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], float)
    t = []
    for sx in (0, 1):
        for sy in (2, 3):
            for sz in (4, 5):
                tri = [sx, sy, sz]
                a, b, c = v[tri]
                if np.dot(np.cross(b - a, c - a), a + b + c) < 0:
                    tri = [sx, sz, sy]
                t.append(tri)
    return v, np.array(t, np.int32)


def test_vertex_normals_of_regular_solids(O):
    # by symmetry the area-weighted normal of a regular polyhedron's vertex is radial
    v, t = octahedron()
    T = O.OracleType(v, t, 1.0, 5.0, 0.05, 10.0, 1e-3)
    assert np.array_equal(T.normals(v), v)
    unit, tris = I.icosphere(0)
    Ti = O.OracleType(unit * 2.0, tris, 1.0, 5.0, 0.05, 10.0, 1e-3)
    R = rot(50)
    x = unit @ R.T * 2.0 + np.array([3.0, -1.0, 7.0])
    assert np.allclose(Ti.normals(x), unit @ R.T, atol=1e-14)


def test_pik_head_on_closed_form(O):
    # A's vertex (0,0,1) faces B's vertex (0,0,1+d) whose normal is (0,0,-1):
    # s = d, p = x_i + (rk - d)(0,0,-1); every other pair is farther than rk
    v, t = octahedron()
    T = O.OracleType(v, t, 1.0, 5.0, 0.05, 10.0, 1e-3)
    d = 0.2
    xa, xb = v.copy(), v * np.array([1.0, -1.0, -1.0]) + np.array([0.0, 0.0, 2.0 + d])   # B: A turned about x
    (hca, hva, pa), (hcb, hvb, pb) = O.pik([(T, xa), (T, xb)], RK)
    assert (hca >= 0).sum() == 1 and hca[4] == 1 and hva[4] == 4      # B's vertex 4 sits at (0,0,1+d)
    assert np.allclose(pa[4], [0.0, 0.0, 1.0 - (RK - d)], atol=1e-15)
    assert hcb[4] == 0 and hvb[4] == 4 and np.allclose(pb[4], [0.0, 0.0, 1.0 + d + (RK - d)], atol=1e-15)
    free = hca < 0
    assert np.array_equal(pa[free], xa[free])


def _overlapping_cells(seed, n=3, level=1):
    unit, tris = I.icosphere(level)
    rest = I.rbc_shape(unit) * 0.5
    rng = np.random.default_rng(seed)
    xs = [rest @ rot(seed + i).T + rng.uniform(-1.0, 1.0, 3) for i in range(n)]
    return rest, tris, xs


def test_pik_matches_kdtree_and_projects_onto_the_plane(O):
    spatial = pytest.importorskip("scipy.spatial")
    rest, tris, xs = _overlapping_cells(51)
    T = O.OracleType(rest, tris, 1.0, 5.0, 0.05, 10.0, 1e-3)
    res = O.pik([(T, x) for x in xs], RK)
    nrm = [T.normals(x) for x in xs]
    hits = 0
    for a, (hc, hv, p) in enumerate(res):
        others = [b for b in range(len(xs)) if b != a]
        pts = np.vstack([xs[b] for b in others])
        owner = np.concatenate([[b] * len(xs[b]) for b in others])
        vert = np.concatenate([np.arange(len(xs[b])) for b in others])
        dist, idx = spatial.cKDTree(pts).query(xs[a], distance_upper_bound=RK)
        found = np.isfinite(dist)
        assert np.array_equal(hc >= 0, found)
        assert np.array_equal(hc[found], owner[idx[found]]) and np.array_equal(hv[found], vert[idx[found]])
        for i in np.flatnonzero(found):
            xj, nj = xs[hc[i]][hv[i]], nrm[hc[i]][hv[i]]
            assert np.dot(p[i] - xj, nj) == pytest.approx(RK, abs=1e-13)          # on the plane
            assert np.linalg.norm(np.cross(p[i] - xs[a][i], nj)) < 1e-13          # moved along n_j
        hits += found.sum()
    assert hits > 20


def test_collision_gradient_central_differences(O):
    rest, tris, T = small_rbc(O, 1)
    rng = np.random.default_rng(52)
    x = rest * 1.05 + 0.05 * rng.standard_normal(rest.shape)
    y = rest + 0.05 * rng.standard_normal(rest.shape)
    hit = (rng.uniform(size=rest.shape[0]) < 0.3).astype(np.int32)
    p = x + 0.2 * rng.standard_normal(rest.shape)
    e, g, _ = T.energy_col(x, y, KC, hit, p)
    e0, g0, _ = T.energy(x, y)
    assert e - e0 == pytest.approx(0.5 * KC * (((x - p) ** 2).sum(axis=1) * hit).sum(), rel=1e-12)
    hh = 1e-6
    fd = np.zeros_like(x)
    for i in range(x.shape[0]):
        for c in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, c] += hh
            xm[i, c] -= hh
            fd[i, c] = (T.energy_col(xp, y, KC, hit, p, grad=False)[0] - T.energy_col(xm, y, KC, hit, p, grad=False)[0]) / (2 * hh)
    assert np.linalg.norm(g - fd) <= 1e-6 * np.linalg.norm(g)


def test_collision_step_converges_to_newtons_law(O, rbc):
    # M (v1 - v0)/h = F_int(x1) + F_ext (zero at contaminated vertices) + kc (p - x1)
    mt, T = rbc
    xn, vn, f = seeded_cell(mt, 53, amp=5.0)
    rng = np.random.default_rng(54)
    hit = (rng.uniform(size=mt.nV) < 0.2).astype(np.int32)
    p = xn + 0.05 * rng.standard_normal(xn.shape)
    x1, v1 = T.step_cells_col(xn[None], vn[None], f[None], KC, hit[None], p[None], K=40)
    x1, v1 = x1[0], v1[0]
    h, m = mt.material.dt, 1.0 / mt.nV
    _, gint, _ = T.energy(x1, x1, mask=30)
    fext = f * (1 - hit)[:, None]
    fcol = KC * (p - x1) * hit[:, None]
    resid = m * (v1 - vn) / h - (-gint + fext + fcol)
    assert np.abs(resid).max() < 1e-7 * np.abs(m * (v1 - vn) / h).max()
    assert np.abs(fcol).max() > 1e-2 * np.abs(m * (v1 - vn) / h).max()


def test_pik_without_contact_is_the_plain_step(O, rbc):
    mt, T = rbc
    g = I.materialise(I.Group(mt, 2, 55, amp=0.3))
    g.x0[1] += 50.0
    cells = [(T, g.x0[c], g.v0[c]) for c in range(2)]
    out = O.pik_step(cells, [g.f_ext[0], g.f_ext[1]], RK, KC)
    for c in range(2):
        x1, v1 = T.step(g.x0[c], g.v0[c], g.f_ext[c])
        assert np.array_equal(out[c][0], x1) and np.array_equal(out[c][1], v1)


def test_collisions_keep_approaching_cells_apart(O):
    unit, tris = I.icosphere(2)
    rest = unit * 1.0
    T = O.OracleType(rest, tris, 1.0, 5.0, 0.05, 10.0, 1e-3)
    xa, xb = rest.copy(), rest + np.array([2.3, 0.0, 0.0])
    va, vb = np.tile([20.0, 0, 0], (len(rest), 1)), np.tile([-20.0, 0, 0], (len(rest), 1))
    zero = np.zeros_like(rest)

    def gap(col):
        cells = [(T, xa.copy(), va.copy()), (T, xb.copy(), vb.copy())]
        for _ in range(15):
            if col:
                out = O.pik_step(cells, [zero, zero], RK, 5000.0)
            else:
                out = [T.step(x, v, zero) for _, x, v in cells]
            cells = [(T, o[0], o[1]) for o in out]
        return cells[1][1][:, 0].min() - cells[0][1][:, 0].max()

    assert gap(False) < 0.0          # without collisions the surfaces pass through each other
    assert gap(True) > 0.1           # with them they stay apart


def test_pik_ties_and_kernel_boundary(O):
    # exact ties go to the lower cell index; a foreign vertex exactly rk away is outside
    v, t = octahedron()
    T = O.OracleType(v, t, 1.0, 5.0, 0.05, 10.0, 1e-3)
    turn = np.array([1.0, -1.0, -1.0])          # B's vertex 4 becomes its lowest point
    xa = v.copy()
    xb = v * turn + np.array([0.25, 0.0, 2.25])   # vertex 4 at (0.25, 0, 1.25)
    xc = v * turn + np.array([-0.25, 0.0, 2.25])  # vertex 4 at (-0.25, 0, 1.25): same distance to A's top
    (hca, hva, _), (hcb, _, _), (hcc, _, _) = O.pik([(T, xa), (T, xb), (T, xc)], RK)
    assert hca[4] == 1 and hva[4] == 4
    assert hcb[4] == 0 and hcc[4] == 0            # B and C tops are exactly rk apart: not each other's
    xd = v * turn + np.array([0.0, 0.0, 2.0 + RK])  # vertex 4 exactly rk above A's top
    (hca, _, _), (hcd, _, _) = O.pik([(T, xa), (T, xd)], RK)
    assert (hca >= 0).sum() == 0 and (hcd >= 0).sum() == 0


# ------------------------------------------------------------------ IBM (multi-direct forcing)
def test_phi4_is_peskins_four_point_function(O):
    # textbook values and moments: partition of unity, zero first moment, sum of squares 3/8
    assert (O.phi4(0.0), O.phi4(1.0), O.phi4(2.0), O.phi4(2.5)) == (0.5, 0.25, 0.0, 0.0)
    assert O.phi4(-0.7) == O.phi4(0.7)
    for r in np.random.default_rng(60).uniform(0.0, 1.0, 25):
        w = np.array([O.phi4(r - j) for j in (-1, 0, 1, 2)])
        assert w.sum() == pytest.approx(1.0, abs=1e-15)
        assert (w * (r - np.array([-1, 0, 1, 2]))).sum() == pytest.approx(0.0, abs=1e-15)
        assert (w ** 2).sum() == pytest.approx(3.0 / 8.0, abs=1e-15)
    for a in (1.0 - 1e-9, 1.0 + 1e-9):                        # continuous where the branches meet
        assert O.phi4(a) == pytest.approx(0.25, abs=1e-8)


def test_vertex_areas(O, rbc):
    v, t = octahedron()
    T = O.OracleType(v, t, 1.0, 5.0, 0.05, 10.0, 1e-3)
    assert np.allclose(T.vertex_areas(v), 4 * (np.sqrt(3) / 2) / 3, atol=1e-15)
    mt, Tr = rbc
    x = seeded_cell(mt, 61, amp=2.0)[0]
    e1, e2 = x[mt.tris[:, 1]] - x[mt.tris[:, 0]], x[mt.tris[:, 2]] - x[mt.tris[:, 0]]
    assert Tr.vertex_areas(x).sum() == pytest.approx(0.5 * np.linalg.norm(np.cross(e1, e2), axis=1).sum(), rel=1e-13)


def _lattice(n=12, dx=0.5, origin=(-3.0, -2.0, -1.0)):
    return n, dx, np.array(origin)


def test_ibm_interpolates_linear_fields_exactly_and_conserves_force(O):
    n, dx, o = _lattice()
    idx = np.indices((n, n, n))[::-1].astype(float)             # (x, y, z) index of node [z][y][x]
    nodes = o[:, None, None, None] + dx * idx
    a, B = np.array([0.3, -0.2, 0.1]), np.random.default_rng(62).standard_normal((3, 3))
    u = a[:, None, None, None] + np.einsum("cd,dzyx->czyx", B, nodes)
    rng = np.random.default_rng(63)
    X = o + dx * rng.uniform(2.0, n - 3.0, (40, 3))             # stencils inside the lattice
    A = rng.uniform(0.1, 0.3, 40)
    f, F = O.ibm(X, np.zeros_like(X), A, u, o, dx, dt=0.5, cycles=0)
    assert np.allclose(f, -(a + X @ B.T) * A[:, None] / 0.5, rtol=1e-12, atol=1e-12)
    # spread: sum_x F dx^3 = sum_k f_k dx
    assert np.allclose(F.reshape(3, -1).sum(axis=1) * dx ** 3, f.sum(axis=0) * dx, rtol=1e-12)


def test_ibm_single_point_cycle_closed_form(O):
    # uniform u0: a cycle sees u_c(X) = u0 + dt f_{c-1} (3/8)^3 / dx^2, so with
    # g = 1 - A (3/8)^3 / dx^2, f_c = g f_{c-1} + f0 = f0 (1 + g + ... + g^c),
    # for any position of the point
    n, dx, o = _lattice()
    u0, U, A, dt = np.array([0.2, -0.1, 0.05]), np.array([[0.5, 0.3, -0.2]]), np.array([0.7]), 0.25
    u = np.broadcast_to(u0[:, None, None, None], (3, n, n, n)).copy()
    for X in (o + dx * np.array([[5.0, 6.0, 5.0]]), o + dx * np.array([[5.3, 6.71, 4.2]])):
        f0 = (U - u0) * A / dt
        g = 1 - A * (3 / 8) ** 3 / dx ** 2
        for c in (1, 2, 3):
            fc, _ = O.ibm(X, U, A, u, o, dx, dt, cycles=c)
            assert np.allclose(fc, f0 * sum(g ** i for i in range(c + 1)), rtol=1e-13, atol=1e-14), c


def test_damped_collision_step_converges_to_newtons_law(O, rbc):
    # both optional terms at once: M (v1 - v0)/h + C v1 = F_int(x1) + F_ext (zero at
    # contaminated vertices) + kc (p - x1), C = alpha M + beta L
    mt, T = rbc
    xn, vn, f = seeded_cell(mt, 64, amp=5.0)
    vn = vn + np.random.default_rng(65).standard_normal(vn.shape)
    rng = np.random.default_rng(66)
    hit = (rng.uniform(size=mt.nV) < 0.2).astype(np.int32)
    p = xn + 0.05 * rng.standard_normal(xn.shape)
    Td = damped(mt, O)
    x1, v1 = Td.step_cells_col(xn[None], vn[None], f[None], KC, hit[None], p[None], K=60)
    x1, v1 = x1[0], v1[0]
    h, m = mt.material.dt, 1.0 / mt.nV
    L = T.P_dense() - np.eye(mt.nV) * m / h ** 2
    _, gint, _ = T.energy(x1, x1, mask=30)
    lhs = m * (v1 - vn) / h + ALPHA * m * v1 + BETA * (L @ v1)
    rhs = -gint + f * (1 - hit)[:, None] + KC * (p - x1) * hit[:, None]
    assert np.abs(lhs - rhs).max() < 1e-7 * np.abs(m * (v1 - vn) / h).max()
