"""libgfm builds for sm_103a, loads, and exports every entry point that
include/gfm.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "gfm.h")) as fh:
        src = fh.read()
    return sorted(set(re.findall(r"^(?:gfm_status|const char \*)\s*(gfm_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("gfm_create", "gfm_assemble", "gfm_solve", "gfm_solve_adjoint", "gfm_destroy"):
        assert must in names


def test_library_loads_and_exports_every_declared_symbol():
    import paper_1804_01130_gb300 as gfm
    lib = gfm.load_library()
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(_declared()) == set(gfm.EXPORTED_SYMBOLS)


def test_status_strings_without_gpu():
    import paper_1804_01130_gb300 as gfm
    lib = gfm.load_library()
    assert lib.gfm_status_string(0) == b"GFM_OK"
    assert lib.gfm_status_string(6) == b"GFM_ERR_TIMEOUT"
    assert lib.gfm_last_error(None) == b"NULL handle"


def test_null_arguments_are_rejected_on_the_host():
    import paper_1804_01130_gb300 as gfm
    lib = gfm.load_library()
    h = ctypes.c_void_p()
    assert lib.gfm_create(None, 0, None, ctypes.byref(h)) == gfm.GFM_ERR_ARG
    assert lib.gfm_destroy(None) == gfm.GFM_ERR_ARG
    assert lib.gfm_default_opts(None) == gfm.GFM_ERR_ARG


def test_no_cpu_fallback_without_cuda():
    import torch

    import paper_1804_01130_gb300 as gfm
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(gfm.GFMError):
        gfm.GFM([0], [1], [[1.0], [0.0], [0.0]], [[0.0, 1.0], [0.0, 0.0], [0.0, 0.0]])
