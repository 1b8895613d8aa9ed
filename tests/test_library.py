"""CPU checks of the C ABI: the library builds, loads, and exports every symbol include/kpp.h declares.

No compute call is made here (there is no GPU); only host-only entry points are called.
"""
import ctypes
import os
import re

import pytest

from paper_2501_11673_gb300 import build as kbuild
from paper_2501_11673_gb300 import kpp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "kpp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*([a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n.startswith(("kpp_", "cdpp_"))))


@pytest.fixture(scope="module")
def lib():
    path = kbuild.build()
    return kpp.load(path)


def test_header_declarations_are_all_exported(lib):
    declared = _declared_functions()
    assert "kpp_solve" in declared and "cdpp_solve" in declared and "kpp_factor_blocks" in declared
    assert "kpp_partition" in declared
    for name in declared:
        assert hasattr(lib, name), f"{name} declared in kpp.h but not exported"
    assert sorted(kpp.EXPORTS) == declared


def test_host_only_entry_points(lib):
    p = lib.kpp_params_default()
    assert p.tol == 1e-8 and p.adaptive_rho == 1 and p.max_outer == 20
    assert lib.kpp_status_string(0) == b"KPP_OK"
    assert lib.kpp_status_string(4) == b"KPP_ERR_NOT_SPD"
    P = kpp.Partition(103, 10)
    assert P.nb == 11
    h = ctypes.c_void_p()
    assert lib.kpp_partition(0, 10, ctypes.byref(h)) == kpp.ERR_ARG
    assert lib.kpp_partition(10, 0, ctypes.byref(h)) == kpp.ERR_ARG
    assert "kpp_partition" in kpp.last_error()
    assert kpp.build_info().startswith("sm_103a")


def test_build_targets_sm_103a_only():
    assert kbuild.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
