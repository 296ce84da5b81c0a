"""The C-ABI library loads and exports every symbol include/lmfmm.h declares;
argument validation that needs no GPU."""
import ctypes
import os
import re

import pytest

from paper_2507_18491_gb300 import build, lmfmm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "lmfmm.h")).read()
    return sorted(set(re.findall(r"\b(lmfmm_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return lmfmm.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(lmfmm.EXPORTS)


def test_default_params(lib):
    prm = lmfmm.default_params()
    assert prm.p == 8 and prm.depth == -1 and prm.precision == lmfmm.FP64
    assert 0 < prm.theta < 1


def test_bad_params_rejected_before_device_use(lib):
    prm = lmfmm.default_params()
    prm.p = 0
    h = ctypes.c_void_p()
    rc = lib.lmfmm_create(ctypes.byref(h), ctypes.byref(prm), 0)
    assert rc == lmfmm.ERR_ARG
    assert b"parameter" in lib.lmfmm_last_error(None)
    prm = lmfmm.default_params()
    prm.theta = 1.5
    assert lib.lmfmm_create(ctypes.byref(h), ctypes.byref(prm), 0) == lmfmm.ERR_ARG
    assert lib.lmfmm_create(None, ctypes.byref(prm), 0) == lmfmm.ERR_ARG
    for bad in (-1, 4):
        prm = lmfmm.default_params()
        prm.precision = lmfmm.MIXED
        prm.tensor_cores = bad
        assert lib.lmfmm_create(ctypes.byref(h), ctypes.byref(prm), 0) == lmfmm.ERR_ARG
        assert b"tensor_cores" in lib.lmfmm_last_error(None)


def test_quad_node_cap_default_and_range(lib):
    prm = lmfmm.default_params()
    assert prm.quad_node_cap == 1 << 20 and prm.tensor_cores == 1
    prm.quad_node_cap = 10
    h = ctypes.c_void_p()
    assert lib.lmfmm_create(ctypes.byref(h), ctypes.byref(prm), 0) == lmfmm.ERR_ARG
    assert b"quad_node_cap" in lib.lmfmm_last_error(None)


def test_null_context_is_an_argument_error(lib):
    assert lib.lmfmm_check(None, None) == lmfmm.ERR_ARG
    assert lib.lmfmm_test_set_status(None, 4) == lmfmm.ERR_ARG
    assert lib.lmfmm_matvec(None, None, lmfmm.C128, None, None) == lmfmm.ERR_ARG
    assert lib.lmfmm_set_points_device(None, 1, None, None) == lmfmm.ERR_ARG


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    """No fallback: without the compiled library every entry point raises."""
    monkeypatch.setattr(lmfmm, "_lib", None)
    monkeypatch.setattr(lmfmm, "library_path", lambda: str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        lmfmm.load()
    with pytest.raises(RuntimeError, match="not built"):
        lmfmm.default_params()
    with pytest.raises(RuntimeError, match="not built"):
        lmfmm.plan_check([0.0], [1, 2], [[0.1, 0.2, 0.3]])
