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


def test_noalloc_wrapper_checks_sizes_before_any_device_call():
    """solve_csr_noalloc rejects inconsistent tensor sizes, dtypes and
    devices on the host, before it reaches the library (CPU tensors here:
    each mismatch is caught ahead of the device check)."""
    import torch

    import paper_1804_01130_gb300 as gfm
    n, nnz = 10, 28

    def call(rp=n + 1, col=nnz, val=nnz, b=n, x=n, info=32, rp_dtype=torch.int32):
        return gfm.solve_csr_noalloc(torch.zeros(rp, dtype=rp_dtype), torch.zeros(col, dtype=torch.int32),
                                     torch.zeros(val, dtype=torch.float64), torch.zeros(b, dtype=torch.float64),
                                     x=torch.zeros(x, dtype=torch.float64), info=torch.zeros(info, dtype=torch.uint8))

    for bad, match in ((dict(rp=n), "row_ptr"), (dict(val=nnz - 1), "val"), (dict(x=n + 1), "x has"),
                       (dict(info=16), "info"), (dict(col=n - 1, val=n - 1), "nnz"),
                       (dict(rp_dtype=torch.int64), "int32"),
                       (dict(rp=gfm.NOALLOC_MAX_CELLS + 2, b=gfm.NOALLOC_MAX_CELLS + 1,
                             x=gfm.NOALLOC_MAX_CELLS + 1), "capacity")):
        with pytest.raises(gfm.GFMError, match=match) as e:
            call(**bad)
        assert e.value.status == gfm.GFM_ERR_ARG
    # consistent sizes get as far as the device check: CPU tensors are refused
    with pytest.raises(gfm.GFMError, match="CUDA"):
        call()


STRUCTS = (("gfm_mesh", "_Mesh"), ("gfm_phys", "_Phys"), ("gfm_solve_opts", "_Opts"), ("gfm_solve_info", "_Info"),
           ("gfm_tuning", "_Tuning"), ("gfm_profile", "_Profile"))


def test_binding_structs_match_the_header_layout(tmp_path):
    """The ctypes structures of the binding have the size and field offsets
    of the header's structs, as a C compiler lays them out (gcc, host only)."""
    import shutil
    import subprocess
    import paper_1804_01130_gb300 as gfm
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "gfm.h"', "int main(void) {"]
    for cname, pyname in STRUCTS:
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in getattr(gfm, pyname)._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, pyname in STRUCTS:
        st = getattr(gfm, pyname)
        assert got[(cname, "size")] == ctypes.sizeof(st), cname
        for fname, _ in st._fields_:
            assert got[(cname, fname)] == getattr(st, fname).offset, (cname, fname)
