"""The C-ABI library builds for sm_103a, loads, and exports every entry point
include/gpuns.h declares (no compute calls: no GPU needed)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "gpuns.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z_0-9]*\s*\*?\s*([a-z_][a-z_0-9]*)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2509_13307_gb300.build import build
    path = build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["ns_init", "ns_step", "ns_evidence", "loglike_batch", "loglike_grad_batch",
                     "ns_problem_create", "ns_free", "ns_problem_free", "ns_strerror"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_lists_every_export():
    from paper_2509_13307_gb300 import _lib
    assert sorted(_lib.EXPORTS) == declared_functions()


def test_strerror_is_static_and_total(lib):
    lib.ns_strerror.restype = ctypes.c_char_p
    for code in range(-8, 1):
        assert isinstance(lib.ns_strerror(code), bytes)


def test_null_arguments_are_rejected_without_a_device(lib):
    # argument validation happens before any CUDA call
    assert lib.ns_problem_create(None, None) == -1
    assert lib.ns_init(None, None, None, None) == -1
    assert lib.ns_step(None, 1, None) == -1
    assert lib.ns_evidence(None, 0, None, None, None, None, None) == -1
