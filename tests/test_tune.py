"""The autotuner's table and on-disk cache on the host (no GPU): set / get, the text format, load
merging and overriding, clearing, rejection of invalid entries, and the lazy load of the file named
by RSK_TUNE_CACHE in a fresh process."""
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LINE = re.compile(r"^rsk-tune v1 kernel=\d+ dtype=-?\d+ n=\d+ k=\d+ d=\d+ sms=\d+ value=\d+$")


@pytest.fixture()
def lib():
    from paper_2508_21189_gb300 import build as b
    b.build()
    from paper_2508_21189_gb300 import _lib
    L = _lib.load()
    assert L.rsk_tune_cache_clear() == 0
    yield L
    L.rsk_tune_cache_clear()


def get(L, *key):
    import ctypes
    v = ctypes.c_int32(-1)
    assert L.rsk_tune_cache_get(*key, ctypes.byref(v)) == 0
    return v.value


def test_set_get_save_load(lib, tmp_path):
    key = (0, 2, 1 << 22, 256, 2048, 152)
    assert get(lib, *key) == 0
    assert lib.rsk_tune_cache_set(*key, 38) == 0
    assert lib.rsk_tune_cache_set(1, 1, 1 << 22, 256, 2048, 152, 19) == 0
    assert lib.rsk_tune_cache_set(2, 1, 33411882, 512, 0, 152, 4096) == 0
    assert get(lib, *key) == 38
    path = str(tmp_path / "tune.txt")
    assert lib.rsk_tune_cache_save(path.encode()) == 0
    lines = [x for x in open(path).read().splitlines() if x and not x.startswith("#")]
    assert len(lines) == 3 and all(LINE.match(x) for x in lines)
    assert lib.rsk_tune_cache_clear() == 0 and get(lib, *key) == 0
    # later lines override earlier ones; comments and junk are skipped
    with open(path, "a") as f:
        f.write("# a comment\nnot a tuning line\nrsk-tune v1 kernel=0 dtype=2 n=4194304 k=256 d=2048 sms=152 value=76\n")
    assert lib.rsk_tune_cache_load(path.encode()) == 0
    assert get(lib, *key) == 76
    assert get(lib, 2, 1, 33411882, 512, 0, 152) == 4096
    # a different SM count is a different key
    assert get(lib, 0, 2, 1 << 22, 256, 2048, 148) == 0


def test_rejects_invalid(lib, tmp_path):
    assert lib.rsk_tune_cache_set(3, 0, 1, 1, 1, 1, 5) == 1
    assert lib.rsk_tune_cache_set(0, 0, 1, 1, 1, 1, 0) == 1
    assert lib.rsk_tune_cache_load(str(tmp_path / "missing.txt").encode()) == 1
    assert lib.rsk_tune_cache_load(None) == 1


def test_environment_cache_is_read_lazily(tmp_path):
    path = tmp_path / "env_tune.txt"
    path.write_text("rsk-tune v1 kernel=1 dtype=2 n=65536 k=40 d=1000 sms=152 value=3\n")
    code = ("import ctypes, sys; sys.path.insert(0, %r)\n"
            "from paper_2508_21189_gb300 import _lib\n"
            "L = _lib.load(); v = ctypes.c_int32()\n"
            "L.rsk_tune_cache_get(1, 2, 65536, 40, 1000, 152, ctypes.byref(v)); print(v.value)\n") % ROOT
    out = subprocess.run([sys.executable, "-c", code], env=dict(os.environ, RSK_TUNE_CACHE=str(path)),
                         capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == "3"
