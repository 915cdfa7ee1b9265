"""The C-ABI library builds, loads and exports every symbol include/pasta.h
declares; host-side argument checks answer without touching a GPU."""
import ctypes
import os
import re

import pytest

from paper_1902_03317_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w\s\*]*?\b(pasta_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("pasta_coo_create", "pasta_coo_sort_by_mode", "pasta_mttkrp",
                     "pasta_cp_loss_fwd", "pasta_cp_loss_bwd", "pasta_coo_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(declared_functions()) <= set(_lib.SIGNATURES)


def test_version_and_status_strings(lib):
    assert lib.pasta_version() == 3
    for code, name in _lib.STATUS.items():
        assert lib.pasta_status_str(code).decode() == name


def test_host_side_argument_errors(lib):
    h = ctypes.c_void_p()
    dims = _lib.u64_array([4, 4, 4])
    # order out of range, zero dim, unknown flag, NULL out: rejected before any CUDA call
    assert lib.pasta_coo_create(ctypes.byref(h), 1, dims, 0, None, None, 0, None) == 1
    assert lib.pasta_coo_create(ctypes.byref(h), 3, _lib.u64_array([4, 0, 4]), 0, None, None, 0, None) == 1
    assert lib.pasta_coo_create(ctypes.byref(h), 3, dims, 0, None, None, 8, None) == 1
    assert lib.pasta_coo_create(None, 3, dims, 0, None, None, 0, None) == 1
    assert lib.pasta_coo_create(ctypes.byref(h), 3, dims, 5, None, None, 0, None) == 1
    assert "NULL" in lib.pasta_last_error().decode()
    # NULL handle everywhere
    assert lib.pasta_mttkrp(None, None, 0, 0, 16, None, None) == 1
    assert lib.pasta_cp_loss_fwd(None, None, 0, 16, -1, None, None, None) == 1
    assert lib.pasta_cp_loss_bwd(None, None, 0, 16, -1, None, None, None) == 1
    assert lib.pasta_coo_sort_by_mode(None, 0, None) == 1
    assert lib.pasta_coo_view(None, 0, None, None, None) == 1
    assert lib.pasta_coo_copy_out(None, 0, None, None, None, None) == 1
    assert lib.pasta_coo_info(None, None, None, None) == 1
    assert lib.pasta_coo_destroy(None) == 0
    assert lib.pasta_convert(None, 9, None, 0, 4, None) == 1


def test_product_path_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        _lib.lib()


def test_set_allocator_argument_checks():
    """Both callbacks or neither; resetting to the default always works when
    no block is held (no GPU needed: nothing is allocated)."""
    import ctypes
    from paper_1902_03317_gb300 import _lib
    L = _lib.lib()
    ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p)
    FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)
    a = ALLOC(lambda n, d, s, c: None)
    f = FREE(lambda p, c: None)
    assert L.pasta_set_allocator(ctypes.cast(a, ctypes.c_void_p), None, None) == 1
    assert L.pasta_set_allocator(None, ctypes.cast(f, ctypes.c_void_p), None) == 1
    assert L.pasta_set_allocator(ctypes.cast(a, ctypes.c_void_p), ctypes.cast(f, ctypes.c_void_p), None) == 0
    assert L.pasta_set_allocator(None, None, None) == 0


def test_cp_als_rejects_a_null_handle():
    """pasta_cp_als checks its arguments before any device work."""
    import ctypes
    from paper_1902_03317_gb300 import _lib
    L = _lib.lib()
    fits = (ctypes.c_double * 4)()
    done = ctypes.c_int(7)
    assert L.pasta_cp_als(None, None, 4, 4, 0.0, None, ctypes.cast(fits, ctypes.c_void_p),
                          ctypes.cast(ctypes.pointer(done), ctypes.c_void_p), None) == 1
    assert b"NULL" in L.pasta_last_error()
