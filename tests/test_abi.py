"""CPU checks of the C-ABI library: it loads, exports every entry point that
include/gbfmm.h declares, and reports errors without needing a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "gbfmm.h")).read()
    return sorted(set(re.findall(r"^GBFMM_API[^(]*?\b(fmm_\w+)\s*\(", txt, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2107_07166_gb300 import build, fmm
    build.build()
    return fmm.load()


def test_header_declares_the_api():
    syms = declared_symbols()
    for s in ("fmm_create", "fmm_build", "fmm_forces", "fmm_diagnostics", "fmm_destroy"):
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    for s in declared_symbols():
        assert hasattr(lib, s), s
    from paper_2107_07166_gb300 import fmm
    assert sorted(fmm.EXPORTS) == declared_symbols()


def test_strerror_names_every_code(lib):
    for code in range(0, -7, -1):
        msg = lib.fmm_strerror(code).decode()
        assert msg and msg != "unknown status"
    assert lib.fmm_strerror(-99).decode() == "unknown status"


def test_null_context_is_rejected(lib):
    x = np.zeros((4, 3))
    m = np.ones(4)
    P = ctypes.c_void_p
    assert lib.fmm_build(None, x.ctypes.data_as(P), m.ctypes.data_as(P), 4, 8) == -1
    assert lib.fmm_forces(None, 2, 0.5, 0, x.ctypes.data_as(P), None) == -1
    assert lib.fmm_destroy(None) == 0
    assert "NULL" in lib.fmm_last_error().decode()


def test_create_reports_missing_device(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    rc = lib.fmm_create(ctypes.byref(h), 0, 0, None)
    assert rc == -3                      # FMM_ERR_CUDA, no device


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2107_07166_gb300 import fmm
    saved = fmm._lib
    try:
        fmm._lib = None
        with pytest.raises(OSError):
            fmm.load(str(tmp_path / "missing.so"))
    finally:
        fmm._lib = saved


def test_generated_index_closed_form():
    """The generator's closed-form multi-index position equals its enumeration order."""
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "gen_expansion", os.path.join(ROOT, "paper_2107_07166_gb300", "csrc", "gen_expansion.py"))
    g = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(g)
    for p in range(0, 9):
        for k, a in enumerate(g.mis(p)):
            assert g.idx(a) == k
        assert len(g.mis(p)) == g.nmi(p)
