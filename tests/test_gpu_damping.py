"""Rayleigh damping C = alpha M + beta L (paper Sec. 2.1, Eq. (Newton2nd)) on the
CUDA path vs the damped FP64 oracle: Mt = M + h C in the inertia term and the
predictor y = x_n + h Mt^{-1}(M v_n + h F_ext).  Bars: FP64 1e-10, mixed forms
1e-6 relative position error.  All calls go through libnpfem.so."""
import dataclasses

import numpy as np
import pytest

from paper_1911_03062_gb300 import inputs as I

from helpers import make_groups, public, rel_pos_err, run_gpu, run_oracle, split

pytestmark = pytest.mark.gpu

BETA = 0.01          # the paper's parameter table (alpha_D = 0, beta_D = 0.01)


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as G
    G.build()


def damped(mt, alpha=0.0, beta=BETA):
    return dataclasses.replace(mt, material=dataclasses.replace(mt.material, rayleigh_alpha=alpha,
                                                                rayleigh_beta=beta))


def _opts(prec):
    if prec == "bf16-plain":
        return "bf16", {"refine_split": False}
    return prec, {}


@pytest.mark.parametrize("alpha,beta", [(0.0, BETA), (2.0, BETA), (2.0, 0.0)])
def test_damped_fp64_matches_oracle(alpha, beta):
    groups = make_groups([(damped(I.rbc_type(), alpha, beta), 5, 0.3),
                          (damped(I.plt_type(), alpha, beta), 3, 0.3)], seed=400)
    xg, _, _ = run_gpu(groups, 3, "fp64")
    xo, _ = run_oracle(groups, 3)
    assert rel_pos_err(xg, xo, groups) <= 1e-10


@pytest.mark.parametrize("prec", ["bf16", "bf16-plain", "tf32"])
def test_damped_mixed_matches_oracle(prec):
    # 131 red cells: two 128-row tiles of the predictor apply, the second ragged;
    # undamped platelets beside them (one damped item in the grouped apply)
    groups = make_groups([(damped(I.rbc_type(), 2.0, BETA), 131, 0.3), (I.plt_type(), 4, 0.3)], seed=401)
    p, kw = _opts(prec)
    xg, _, st = run_gpu(groups, 3, p, **kw)
    sample = [np.array([0, 1, 64, 127, 128, 130]), np.arange(4)]
    xo, _ = run_oracle(groups, 3, sample=sample)
    assert rel_pos_err(xg, xo, groups) <= 1e-6, prec
    assert st["max_refine_residual"] <= 1e-6


def test_damping_changes_the_step_and_the_mean_velocity_closed_form():
    # zero net force per cell: 1^T L = k_vol 1^T, so the cell's mean velocity after
    # one step is m v0 / ((1 + h alpha) m + h beta k_vol) exactly (any iterate)
    from paper_1911_03062_gb300.npfem import Solver
    alpha = 2.0
    mt0 = I.rbc_type()
    groups = make_groups([(mt0, 4, 0.3)], seed=402)
    g = groups[0]
    f = g.f_ext - g.f_ext.mean(axis=1, keepdims=True)
    out = {}
    for name, mt in (("plain", mt0), ("damped", damped(mt0, alpha, BETA))):
        s = Solver(precision="fp64")
        s.add_cells(s.create_type(mt), g.x0, g.v0)
        s.step(f.ravel())
        out[name] = (s.positions().reshape(g.x0.shape), s.velocities().reshape(g.x0.shape))
        s.close()
    assert np.abs(out["plain"][0] - out["damped"][0]).max() > 1e-6
    m, h, kv = 1.0 / mt0.nV, mt0.material.dt, mt0.material.k_vol
    expect = g.v0.mean(axis=1) / (1 + h * alpha + h * BETA * kv / m)
    assert np.allclose(out["damped"][1].mean(axis=1), expect, rtol=1e-9, atol=1e-12)


def test_damping_rejects_negative_coefficients():
    from paper_1911_03062_gb300.npfem import EINVAL, NpfemError, Solver
    s = Solver(precision="fp64")
    with pytest.raises(NpfemError) as e:
        s.create_type(damped(I.plt_type(), -1.0, 0.0))
    assert e.value.code == EINVAL and "Rayleigh" in str(e.value)
    s.close()
