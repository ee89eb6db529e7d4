"""CPU checks of the C-ABI library: it builds for sm_103a, exports every
function include/npfem.h declares, and refuses to run without a GPU (no CPU
fallback)."""
import ctypes

import pytest

from paper_1911_03062_gb300 import build as B
from paper_1911_03062_gb300 import npfem as N


@pytest.fixture(scope="module")
def lib_path():
    return B.build()


def test_header_symbols_exported(lib_path):
    names = N.header_functions()
    assert "npfem_step" in names and "npfem_create_mesh_type" in names
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_default_options_match_header(lib_path):
    o = N.default_options()
    assert (o.precision, o.iters, o.history, o.max_backtracks, o.refine_max) == (0, 10, 5, 8, 3)
    assert o.armijo_c1 == 1e-4 and o.refine_tol == 1e-6 and o.use_graph == 1


def test_no_cpu_fallback(lib_path):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(N.NpfemError) as e:
        N.Solver()
    assert e.value.code in (N.ECUDA, N.EINVAL)


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    monkeypatch.setattr(N, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        N.load(str(tmp_path / "libnpfem.so"))
