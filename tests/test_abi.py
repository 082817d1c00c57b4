"""The C-ABI library loads and exports every entry point include/vpm.h declares (no GPU
needed), and argument checks that precede any CUDA call reject bad input."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "vpm.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2511_11430_gb300 import _lib, build

    build.build()
    return _lib.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while", "for")))


def test_header_declares_the_six_entry_points():
    names = declared_functions()
    for n in ("vpm_induce", "vpm_segments_induce", "vpm_rhs", "vpm_step", "aic_solve", "vpm_induce_backward"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 9
    for n in names:
        assert hasattr(lib, n), n


def test_binding_signatures_cover_header(lib):
    from paper_2511_11430_gb300 import _lib

    assert set(declared_functions()) == set(_lib.SIGNATURES)


def test_version_and_invalid_arguments_without_gpu(lib):
    from paper_2511_11430_gb300 import _lib

    assert lib.vpm_version() == 10100
    # sigma <= 0 is rejected before anything touches the device
    st = lib.vpm_induce(None, None, 10, None, 10, ctypes.c_float(-1.0), 0, None, None, None, 0, None)
    assert st == _lib.VPM_ERR_INVALID_ARG
    assert b"sigma" in lib.vpm_last_error()
    st = lib.vpm_induce(None, None, -1, None, 10, ctypes.c_float(1.0), 0, None, None, None, 0, None)
    assert st == _lib.VPM_ERR_INVALID_ARG
    st = lib.vpm_induce(None, None, 1 << 31, None, 10, ctypes.c_float(1.0), 0, None, None, None, 0, None)
    assert st == _lib.VPM_ERR_LIMIT
    st = lib.vpm_segments_induce(None, None, 4, None, 4, ctypes.c_float(0.1), 3, 0, None, None, None, 0, None)
    assert st == _lib.VPM_ERR_INVALID_ARG  # Vatistas exponent must be 1 or 2
    p = _lib.VpmParams()
    p.sigma = 0.0
    st = lib.vpm_rhs(None, None, 10, None, None, 0, ctypes.byref(p), None, None, None, None, 0, None)
    assert st == _lib.VPM_ERR_INVALID_ARG
    st = lib.vpm_rhs(None, None, 10, None, None, 0, None, None, None, None, None, 0, None)
    assert st == _lib.VPM_ERR_INVALID_ARG
    st = lib.aic_solve(None, None, None, VPM_MAX_AIC_PLUS_ONE, ctypes.c_double(1e-12), 5, None, None, None, 0, None)
    assert st == _lib.VPM_ERR_INVALID_ARG
    # the treecode entries check theta, order and sigma before any CUDA call
    F = ctypes.c_float
    st = lib.vpm_tree_induce(None, None, 10, F(0.1), F(1.5), 4, None, None, None, 0, None)
    assert st == _lib.VPM_ERR_INVALID_ARG and b"theta" in lib.vpm_last_error()
    st = lib.vpm_tree_induce(None, None, 10, F(0.1), F(0.5), 5, None, None, None, 0, None)
    assert st == _lib.VPM_ERR_INVALID_ARG and b"order" in lib.vpm_last_error()
    st = lib.vpm_tree_induce(None, None, 10, F(0.0), F(0.5), 4, None, None, None, 0, None)
    assert st == _lib.VPM_ERR_INVALID_ARG and b"sigma" in lib.vpm_last_error()
    p.sigma = 0.1
    p.vatistas_n = 2
    st = lib.vpm_rhs_tree(None, None, 10, None, None, 0, ctypes.byref(p), F(-0.1), 4, None, None, None, None, 0,
                          None)
    assert st == _lib.VPM_ERR_INVALID_ARG and b"theta" in lib.vpm_last_error()
    st = lib.vpm_step_tree(None, None, None, 10, None, None, 0, ctypes.byref(p), F(0.5), 1, ctypes.c_double(1e-3),
                           None, 0, None)
    assert st == _lib.VPM_ERR_INVALID_ARG and b"order" in lib.vpm_last_error()
    # zero-size calls are no-ops that succeed
    assert lib.vpm_tree_induce(None, None, 0, F(0.1), F(0.5), 4, None, None, None, 0, None) == 0
    assert lib.vpm_induce(None, None, 5, None, 0, ctypes.c_float(1.0), 0, None, None, None, 0, None) == 0
    assert lib.aic_solve(None, None, None, 0, ctypes.c_double(1e-12), 5, None, None, None, 0, None) == 0


VPM_MAX_AIC_PLUS_ONE = 8193


def test_product_package_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_2511_11430_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "vpm_oracle" not in txt and "liboracle" not in txt, f
