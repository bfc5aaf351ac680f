"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/rqmc.h declares; argument validation answers before any CUDA call."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "rqmc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*([a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while")))


@pytest.fixture(scope="module")
def lib():
    from paper_1408_5526_gb300 import _build, rqmc
    _build.build()
    return rqmc.load()


def test_every_declared_symbol_is_exported(lib):
    from paper_1408_5526_gb300 import rqmc
    decl = _declared()
    assert len(decl) >= 20
    assert sorted(rqmc.EXPORTS) == decl
    for name in decl:
        assert getattr(lib, name) is not None


def test_abi_version_and_status_strings(lib):
    assert lib.rqmc_abi_version() == 1
    assert lib.rqmc_status_string(0) == b"ok"
    assert lib.rqmc_status_string(1) == b"invalid argument"


def test_validation_before_any_launch(lib):
    from paper_1408_5526_gb300 import rqmc
    th = np.zeros(4)
    dp = th.ctypes.data_as(C.POINTER(C.c_double))
    # NULL parameters / bad sizes are rejected without touching the device
    assert lib.price_caplets(None, dp, 1, 16, 1, 0, 1, 0, dp, dp, dp, None) == 1
    assert lib.price_mbs(None, 16, 1, 0, 1, 0, dp, dp, dp, None) == 1
    assert lib.rqmc_points(8, 16, 1, 0, 1, 0, 1, 0, None, None) == 1
    bad = rqmc.MbsParams(0, 0, 0.007, 0.01, -0.005, 10.0, 0.5, 0.02, 1.0)
    assert lib.price_mbs(C.byref(bad), 16, 1, 0, 1, 0, dp, dp, dp, None) == 1
    assert b"months" in lib.rqmc_last_error()


def test_sobol_table_recurrence_rejects_even_direction_numbers(lib):
    poly = np.array([1, 3], dtype=np.int64)
    vinit = np.array([[1] + [0] * 17, [2] + [0] * 17], dtype=np.int64)   # m_1 = 2 is not odd
    st = lib.rqmc_set_sobol_table(poly.ctypes.data_as(C.POINTER(C.c_int64)),
                                  vinit.ctypes.data_as(C.POINTER(C.c_int64)), 2, 18)
    assert st == 1
    from paper_1408_5526_gb300 import inputs
    p, v = inputs.joe_kuo_table()
    assert lib.rqmc_set_sobol_table(p.ctypes.data_as(C.POINTER(C.c_int64)),
                                    v.ctypes.data_as(C.POINTER(C.c_int64)), 4096, v.shape[1]) == 0


def test_binding_refuses_output_tensors_it_cannot_write_safely():
    # the C ABI writes through a raw pointer; the binding checks size, dtype, device and
    # layout of a caller's tensor first
    import pytest
    import torch
    from paper_1408_5526_gb300 import rqmc
    with pytest.raises(TypeError):
        rqmc._check_out(np.zeros(8), 8, torch.float64, "t")
    with pytest.raises(ValueError):                       # host tensor
        rqmc._check_out(torch.zeros(8, dtype=torch.float64), 8, torch.float64, "t")
    with pytest.raises(ValueError):                       # wrong dtype (checked before the device)
        rqmc._check_out(torch.zeros(8, dtype=torch.float32), 8, torch.float64, "t")
