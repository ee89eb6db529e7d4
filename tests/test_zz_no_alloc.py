"""The allocation-free apply (npfem_apply_pinv_noalloc) against the
allocating one (npfem_apply_pinv), through the C ABI.

Some callers cannot let the library allocate device memory -- their GPU
memory is owned by another allocator, or a cudaMalloc/cudaFree
synchronisation would stall their loop -- so this entry point takes its
temporaries from one static device array.  The array is shared by all calls
and keeps the previous call's contents, so the second call below uses fewer
columns than the first: stale rows from the first call must not leak into
the ragged last cell of the second.  Collected last (file name) so that a
run stopping at the first failure has already run every other test."""
import numpy as np
import pytest

from paper_1911_03062_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as G
    G.build()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("bf16", 2e-6), ("tf32", 2e-6)])
def test_noalloc_apply_matches_allocating_apply(prec, tol):
    import torch
    from paper_1911_03062_gb300.npfem import Solver
    mt = I.rbc_type()
    s = Solver(precision=prec)
    tid = s.create_type(mt)
    rng = np.random.default_rng(11)
    for n_cols in (131, 100):            # two calls in a row, the second smaller and ragged
        q = torch.tensor(rng.standard_normal((n_cols, mt.nV)), device="cuda")
        z_ref = s.apply_pinv(tid, q, torch.empty_like(q)).cpu().numpy()
        z = s.apply_pinv_noalloc(tid, q, torch.full_like(q, np.nan)).cpu().numpy()
        assert np.all(np.isfinite(z))
        assert np.abs(z - z_ref).max() <= tol * np.abs(z_ref).max(), (prec, n_cols)
    s.close()


def test_noalloc_rejects_oversize_request():
    import torch
    from paper_1911_03062_gb300.npfem import EINVAL, NpfemError, Solver
    mt = I.rbc_type()
    s = Solver(precision="bf16")
    tid = s.create_type(mt)
    n_cols = (1 << 21) // mt.nV + 30     # beyond the 2^21-element static scratch
    q = torch.zeros((n_cols, mt.nV), dtype=torch.float64, device="cuda")
    with pytest.raises(NpfemError) as e:
        s.apply_pinv_noalloc(tid, q, torch.empty_like(q))
    assert e.value.code == EINVAL and "static scratch" in str(e.value)
    s.close()
