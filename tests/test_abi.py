"""The C ABI library loads and exports what include/algsig.h declares.  No
compute calls here: only host-side queries and argument checks that fail
before any device work."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "algsig.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(as_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import paper_2411_18183_gb300 as ag
    if not os.path.exists(ag.LIB_PATH):
        from paper_2411_18183_gb300 import build
        build.build()
    return ag.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared()
    assert len(names) >= 9
    for name in names:
        assert hasattr(lib, name), name
    import paper_2411_18183_gb300 as ag
    assert set(ag.EXPORTS) <= set(names)


def test_host_queries(lib):
    assert lib.as_version() >= 100
    assert lib.as_status_string(3) == b"AS_ERR_CAPACITY"
    # cap = next power of two >= m / lf (at least 64); slots + signatures + flags
    assert lib.as_join_table_bytes(1000, 0.5) == 2048 * 16 + ((1000 * 8 + 255) // 256) * 256 + 256
    assert lib.as_join_table_bytes(10, 0.0) == 0
    assert lib.as_join_table_bytes(10, 1.5) == 0
    assert lib.as_join_probe_ws_bytes(5000) == (5000 * 8 + 255) // 256 * 256 + 256
    assert lib.as_join_ws_bytes(1000, 5000, 0.5) == (lib.as_join_table_bytes(1000, 0.5) + 256
                                                     + lib.as_join_probe_ws_bytes(5000))


def test_argument_errors_before_any_device_work(lib):
    assert lib.as_sig_compute(None, None, 5, None, None) == 1
    assert b"null" in lib.as_last_error()
    buf = (ctypes.c_uint8 * 64)()
    base = (ctypes.addressof(buf) + 15) // 16 * 16
    assert lib.as_sig_compute(base + 1, base, 1, base, None) == 1
    assert b"aligned" in lib.as_last_error()
    import paper_2411_18183_gb300 as ag
    t = ag.Table()
    assert lib.as_join_build(base, 64, base, base, None, 4, None, ctypes.c_float(2.0), ctypes.byref(t), None) == 1
