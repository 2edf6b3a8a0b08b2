"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point declared in include/tdks.h (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "tdks.h")).read()
    return sorted(set(re.findall(r"^\s*(?:tdks_status|const char\*)\s+(tdks_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1810_13130_gb300.build import build
    return build()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("tdks_create", "tdks_apply_H", "tdks_density", "tdks_dipole", "tdks_hartree",
              "tdks_expm", "tdks_magnus_step", "tdks_set_potential", "tdks_propagate_host"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(libpath):
    from paper_1810_13130_gb300 import tdks
    assert set(_declared()) <= set(tdks.exported_symbols())
    lib = tdks.lib()
    assert lib.tdks_status_string(-4).decode() == "not converged"


def test_create_rejects_bad_descriptors_without_gpu(libpath):
    """Argument validation happens before any CUDA call."""
    from paper_1810_13130_gb300 import tdks
    L = tdks.lib()
    import numpy as np
    X = np.array([0.0, 1.0, 0.5])          # not increasing
    occ = np.array([2.0])
    m = tdks.MeshDesc(2, 2, 2, X.ctypes.data_as(tdks._dp), X.ctypes.data_as(tdks._dp),
                      X.ctypes.data_as(tdks._dp), 3, 0)
    s = tdks.SystemDesc(1, occ.ctypes.data_as(tdks._dp), 0, None, None, 0, 0.0, 1, 1)
    h = ctypes.c_void_p()
    assert L.tdks_create(ctypes.byref(m), ctypes.byref(s), None, ctypes.byref(h)) == -1
    Xg = np.array([0.0, 1.0, 2.0])
    m = tdks.MeshDesc(2, 2, 2, Xg.ctypes.data_as(tdks._dp), Xg.ctypes.data_as(tdks._dp),
                      Xg.ctypes.data_as(tdks._dp), 9, 0)          # p = 9 unsupported
    assert L.tdks_create(ctypes.byref(m), ctypes.byref(s), None, ctypes.byref(h)) == -1
    m = tdks.MeshDesc(2, 2, 2, Xg.ctypes.data_as(tdks._dp), Xg.ctypes.data_as(tdks._dp),
                      Xg.ctypes.data_as(tdks._dp), 3, 5)          # nq != p+1
    assert L.tdks_create(ctypes.byref(m), ctypes.byref(s), None, ctypes.byref(h)) == -1


def test_binding_has_no_cpu_fallback(libpath):
    """Host tensors are refused before any library call: there is no CPU path."""
    import numpy as np
    import torch
    from paper_1810_13130_gb300 import tdks
    rho = torch.zeros(8 * 27, dtype=torch.float64)                  # a host tensor
    b = np.array([0.0, 1.0, 2.0])
    with pytest.raises(tdks.TDKSError, match="CUDA tensor"):
        tdks.dipole_noalloc(rho, b, b, b, 2)
    with pytest.raises(tdks.TDKSError):
        tdks._dev(torch.zeros(4, dtype=torch.complex64), torch.complex128, "psi")


def test_dipole_noalloc_rejects_a_short_density_before_the_library(monkeypatch):
    """The allocation-free dipole reads nx*ny*nz*(p+1)^3 doubles with no length
    argument: the binding must refuse a density of any other length before any call
    into the library (none could then read past the tensor)."""
    import numpy as np
    import torch
    from paper_1810_13130_gb300 import tdks

    def no_library():
        raise AssertionError("the library was reached")

    monkeypatch.setattr(tdks, "lib", no_library)
    X = np.linspace(-1.0, 1.0, 3)               # 2 x 2 x 2 elements, p = 2: 216 values
    for n in (215, 217, 0):
        with pytest.raises(tdks.TDKSError, match="nx\\*ny\\*nz"):
            tdks.dipole_noalloc(torch.zeros(n, dtype=torch.float64), X, X, X, 2)
    # the right length passes the length check and stops at the device check (CPU tensor)
    with pytest.raises(tdks.TDKSError, match="CUDA tensor"):
        tdks.dipole_noalloc(torch.zeros(216, dtype=torch.float64), X, X, X, 2)
