"""CPU checks of the C-ABI boundary: librsk.so builds, loads without a GPU, and exports every
entry point include/rsk.h declares with the signature the Python binding marshals."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rsk.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2508_21189_gb300 import build as b
    b.build()
    from paper_2508_21189_gb300 import _lib
    return _lib.load()


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return re.findall(r"^\s*(?:rsk_status|const char\*|int32_t)\s+(rsk_\w+)\s*\(", src, flags=re.M)


def test_header_declares_entry_points():
    names = declared()
    assert "rsk_sparse_sign_apply" in names and "rsk_create" in names
    assert len(names) == len(set(names))


def test_every_declared_symbol_is_exported(lib):
    from paper_2508_21189_gb300 import _lib
    for name in declared():
        assert hasattr(lib, name), f"{name} declared in rsk.h but not exported"
        assert name in _lib.SIGNATURES, f"{name} has no Python marshalling"
    for name in _lib.SIGNATURES:
        assert name in declared(), f"binding marshals {name} which rsk.h does not declare"


def test_argument_counts_match_header(lib):
    from paper_2508_21189_gb300 import _lib
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    for name in declared():
        m = re.search(name + r"\s*\(([^)]*)\)", src)
        args = [a for a in m.group(1).split(",") if a.strip() and a.strip() != "void"]
        assert len(args) == len(_lib.SIGNATURES[name]), name


def test_host_only_calls(lib):
    assert lib.rsk_version() == 200
    c, m, p = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    args = (ctypes.byref(c), ctypes.byref(m), ctypes.byref(p))
    assert lib.rsk_sparse_sign_index_dims(20000, 400, 8, *args) == 0
    assert m.value == (20000 + c.value - 1) // c.value and p.value >= 401
    assert c.value * 8 <= 6144
    assert lib.rsk_sparse_sign_index_dims(20000, 400, 32, *args) == 0 and c.value * 32 <= 6144
    # invalid shapes are rejected before any device work
    assert lib.rsk_sparse_sign_index_dims(100, 4, 8, *args) == 1
    assert lib.rsk_sparse_sign_index_dims(100, 9000, 8, *args) == 1
    assert lib.rsk_sparse_sign_index_dims(100, 64, 33, *args) == 1
    assert lib.rsk_sparse_sign_apply(None, None, 0, 10, 1, 1, 4, 2, 0, None, 0, 1, None) == 1
    assert lib.rsk_destroy(None) == 1
    assert lib.rsk_set_wait_limit(None, 1) == 1


def test_noalloc_rejects_invalid_sizes_before_any_device_work(lib):
    # every argument is validated before the fixed scratch array is sized or the device is touched:
    # d that does not fit in 32 bits, zeta > d, d > 8192, an unknown dtype and lda < k all return
    # RSK_ERR_INVALID_ARG (never a division by zero in the sizing, never RSK_ERR_UNSUPPORTED)
    fake = ctypes.c_void_p(256)  # never dereferenced: the checks come first
    call = lib.rsk_sparse_sign_apply_noalloc
    assert call(fake, 2, 1 << 20, 256, 256, (1 << 32) - 3, 8, 0, fake, 1, 256, None) == 1
    assert call(fake, 2, 1 << 20, 256, 256, 4, 8, 0, fake, 1, 256, None) == 1
    assert call(fake, 2, 1 << 20, 256, 256, 9000, 8, 0, fake, 1, 256, None) == 1
    assert call(fake, 7, 1 << 20, 256, 256, 2048, 8, 0, fake, 1, 256, None) == 1
    assert call(fake, 2, 1 << 20, 256, 100, 2048, 8, 0, fake, 1, 256, None) == 1
    assert call(None, 2, 1 << 20, 256, 256, 2048, 8, 0, fake, 1, 256, None) == 1
