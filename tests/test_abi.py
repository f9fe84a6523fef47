"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point include/*.h declares (no device calls are made here)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?(?:int|void|char|double|int64_t)\s*\*?\s*(\w+)\s*\(",
                             text, flags=re.M):
            names.append(m.group(1))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_1505_07630_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = set(declared_functions())
    for required in ("ldu_create", "ldu_update_values", "ldu_set_face_coeffs", "ldu_spmv",
                     "pcg_solve", "pipecg_solve", "ldu_face_grad", "ldu_destroy",
                     "ldu_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_calls_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.ldu_status_string.restype = ctypes.c_char_p
    assert lib.ldu_status_string(-5) == b"grid barrier timed out"
    assert lib.ldu_status_string(0) == b"ok"
    # argument checks happen on the host before any CUDA call
    lib.ldu_create.restype = ctypes.c_int
    assert lib.ldu_create(ctypes.c_int64(4), ctypes.c_int64(0), None, None, None, None, None,
                          None, None, None) == -1
    # sizes the 32-bit layout cannot index are refused before any allocation
    # (the array pointers are only tested for null, never read, on this path)
    h = ctypes.c_void_p()
    fake = ctypes.c_void_p(256)
    assert lib.ldu_create(ctypes.c_int64(1 << 31), ctypes.c_int64(0), None, None, fake, None, None,
                          None, None, ctypes.byref(h)) == -7
    assert lib.ldu_create(ctypes.c_int64(8), ctypes.c_int64(1 << 30), fake, fake, fake, fake, fake,
                          None, None, ctypes.byref(h)) == -7
    assert h.value is None
    lib.ldu_destroy(None)


def test_binding_names_match_the_abi():
    """Every entry point of the header has a binding of the same name
    (handle queries are methods of the handle object instead)."""
    import paper_1505_07630_gb300 as pkg
    as_methods = {"ldu_last_stats", "ldu_get_info", "ldu_status_string"}
    missing = [n for n in declared_functions()
               if n not in as_methods and not callable(getattr(pkg, n, None))]
    assert not missing, missing


def test_product_path_does_not_import_the_oracle():
    pkg_dir = os.path.join(ROOT, "paper_1505_07630_gb300")
    for path in glob.glob(os.path.join(pkg_dir, "**", "*.*"), recursive=True):
        if path.endswith((".py", ".cu", ".cuh", ".h")):
            text = open(path).read()
            assert "import oracle" not in text and "from oracle" not in text, path
            assert "ldu_oracle" not in text, path
