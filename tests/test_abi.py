"""Host-side checks of the C ABI (no GPU needed): the library builds and
loads, exports every function include/mm.h declares, and rejects invalid
arguments before touching the GPU."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mm.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mm_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1406_7459_gb300 import mm
    if not os.path.exists(mm.LIB_PATH):
        if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
            pytest.skip("libmm.so not built and nvcc unavailable")
        from paper_1406_7459_gb300 import build
        build.build()
    return mm.lib()


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("mm_create", "mm_destroy", "mm_set_field", "mm_set_m", "mm_get_m",
                 "mm_demag_field", "mm_step", "mm_energy", "mm_last_error"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1406_7459_gb300 import mm
    for name in _declared():
        assert hasattr(lib, name), name
        assert name in mm._PROTOS, "binding lacks %s" % name


def _create(lib, grid, cell=(1e-9, 1e-9, 1e-9), Ms=8e5, A=1e-11, Ku=0.0, alpha=0.1, gamma=2.2e5):
    out = ctypes.c_void_p(123)
    g = (ctypes.c_int * 3)(*grid)
    c = (ctypes.c_double * 3)(*cell)
    rc = lib.mm_create(ctypes.byref(out), g, c, Ms, A, Ku, alpha, gamma, None)
    return rc, out


@pytest.mark.parametrize("kw", [dict(grid=(0, 4, 1)), dict(grid=(4, -1, 1)),
                                dict(grid=(4, 4, 1), cell=(1e-9, 0.0, 1e-9)),
                                dict(grid=(4, 4, 1), Ms=0.0), dict(grid=(4, 4, 1), A=-1.0),
                                dict(grid=(4, 4, 1), alpha=-0.1), dict(grid=(4, 4, 1), gamma=0.0),
                                dict(grid=(4, 4, 1), Ku=float("nan"))])
def test_create_rejects_bad_arguments_without_a_gpu(lib, kw):
    rc, out = _create(lib, **kw)
    assert rc == -1
    assert out.value is None
    assert len(lib.mm_last_error(None)) > 0


def test_null_handling(lib):
    assert lib.mm_destroy(None) == 0
    assert lib.mm_step(None, 1, 1e-13) == -1
    assert lib.mm_set_field(None, None) == -1
    assert lib.mm_sync(None) == -1
    assert lib.mm_create(None, None, None, 1.0, 1.0, 1.0, 1.0, 1.0, None) == -1
    # mm_gemm_bf16 rejects a null C or null operands before any CUDA call
    assert lib.mm_gemm_bf16(None, None, None, 4, 4, 4, 4, 1, 4, 1, 4, 1, 1, 0, 0, 0, 1.0, 0.0, 0, None) == -1


def test_python_binding_names_match_c_names():
    from paper_1406_7459_gb300 import mm
    for name in _declared():
        assert callable(getattr(mm, name)), name
