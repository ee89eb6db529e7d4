"""CPU checks of the C-ABI library: it builds for sm_103a, exports every
function include/npfem.h declares, the Python binding's struct mirrors have the
header's layouts, and it refuses to run without a GPU (no CPU fallback)."""
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


def test_struct_layouts_match_header(tmp_path):
    # the ctypes mirrors of the header's structs: size and every field offset, as a C
    # compiler lays them out
    import os
    import subprocess
    structs = {"npfem_options": N.Options, "npfem_material": N.Material, "npfem_step_stats": N.StepStats,
               "npfem_kernel_times": N.KernelTimes, "npfem_lattice": N.Lattice}
    inc = os.path.join(os.path.dirname(B.LIB), os.pardir, "include")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "npfem.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["return 0;", "}"]
    src, exe = tmp_path / "layout.c", tmp_path / "layout"
    src.write_text("\n".join(lines))
    subprocess.check_call(["gcc", "-std=c99", "-I", os.path.abspath(inc), str(src), "-o", str(exe)])
    got = {}
    for line in subprocess.check_output([str(exe)], text=True).splitlines():
        cname, field, val = line.split()
        got[(cname, field)] = int(val)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


class _FakeCuda:
    """Stands in for a CUDA tensor (no GPU here): what the binding's checks read."""
    is_cuda = True

    def __init__(self, shape, dtype="torch.float64", device=0, contiguous=True):
        import types
        self.shape, self.dtype, self._c = tuple(shape), dtype, contiguous
        self.device = types.SimpleNamespace(index=device)

    def is_contiguous(self):
        return self._c

    def numel(self):
        import numpy as np
        return int(np.prod(self.shape))

    def dim(self):
        return len(self.shape)

    def data_ptr(self):
        return 0


def test_binding_checks_device_arguments_before_the_library():
    import numpy as np
    import torch
    F = _FakeCuda
    with pytest.raises(ValueError, match="CUDA tensor"):
        N._dev_ptr(torch.zeros(4, dtype=torch.float64), 0)
    for bad in (F((4,), dtype="torch.float32"), F((4,), contiguous=False), F((4,), device=1)):
        with pytest.raises(ValueError):
            N._dev_ptr(bad, 0, numel=4)
    with pytest.raises(ValueError):
        N._dev_ptr(F((5,)), 0, numel=4)
    with pytest.raises(ValueError):
        N._dev_ptr(F((3, 4)), 0, shape=(3, 5))
    assert N._dev_ptr(F((3, 4)), 0, shape=(3, 4)).value is None      # accepted (null pointer of the fake)
    with pytest.raises(ValueError):
        N._host(np.zeros(5), 6, "f_ext")
    # the Solver's own checks, without a context: apply shapes and type ids, step sizes
    s = N.Solver.__new__(N.Solver)
    s.device, s.types = 0, [642]

    class _Lib:
        @staticmethod
        def npfem_num_dofs(ctx):
            return 3 * 642
    s._L, s._ctx = _Lib(), None
    with pytest.raises(ValueError):
        s._apply_args(0, F((6, 641)), F((6, 641)))
    with pytest.raises(ValueError):
        s._apply_args(0, F((6, 642)), F((5, 642)))
    with pytest.raises(ValueError):
        s._apply_args(1, F((6, 642)), F((6, 642)))
    with pytest.raises(ValueError):
        s._apply_args(0, F((6 * 642,)), F((6 * 642,)))
    with pytest.raises(ValueError):
        s.step(F((3 * 642 + 3,)))
    with pytest.raises(ValueError):
        s.step(np.zeros(3 * 642 - 1))
    with pytest.raises(ValueError):
        s.add_cells(0, np.zeros(3 * 642 + 1))
    with pytest.raises(ValueError):
        s.add_cells(0, np.zeros(3 * 642), np.zeros(3))
