"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, loads, exports every entry point declared in include/ftcc.h, and
reports the absence of a device instead of falling back to the CPU."""
import ctypes
import os
import re

import pytest

from paper_2004_01729_gb300 import build, ftcc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ftcc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(", src, re.M)
    return sorted(set(n for n in names if re.match(r"^(ftcc_|ft_ccsd_|build_integrals$)", n)))


@pytest.fixture(scope="module")
def lib():
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("build_integrals", "ft_ccsd_solve", "ft_ccsd_adjoint", "ftcc_create", "ftcc_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_symbol():
    bound = {n for n, _, _ in ftcc._SIGS}
    assert bound == set(declared_functions())


def test_status_strings(lib):
    ftcc._lib = None
    L = ftcc.load()
    assert L.ftcc_status_string(0) == b"ok"
    assert L.ftcc_status_string(ftcc.ERR_NO_DEVICE) == b"no CUDA device"
    assert L.ftcc_status_string(99) == b"unknown status"


def test_no_device_is_reported_not_emulated():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    L = ftcc.load()
    h = ctypes.c_void_p()
    s = L.ftcc_create(0, None, None, ctypes.byref(h))
    assert s == ftcc.ERR_NO_DEVICE
    assert not h.value


def test_null_arguments_are_rejected():
    L = ftcc.load()
    assert L.ftcc_create(0, None, None, None) == ftcc.ERR_INVALID_ARG
    assert L.build_integrals(None, None) == ftcc.ERR_INVALID_ARG
    assert L.ft_ccsd_iterate(None, 1, None) == ftcc.ERR_INVALID_ARG
    assert L.ft_ccsd_adjoint(None, None, None) == ftcc.ERR_INVALID_ARG
    st = (ctypes.c_int * 2)()
    out = (ftcc.AdjointResult * 2)()
    assert L.ft_ccsd_adjoint_batched(None, 2, out, st) == ftcc.ERR_INVALID_ARG
    hs = (ctypes.c_void_p * 2)(None, None)   # a NULL context: nothing runs
    assert L.ft_ccsd_adjoint_batched(hs, 2, out, st) == ftcc.ERR_INVALID_ARG
    assert L.ft_ccsd_adjoint_batched(hs, 0, out, st) == ftcc.ERR_INVALID_ARG
    L.ftcc_destroy(None)
