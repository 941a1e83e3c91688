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
    # cap = next power of two >= m / lf (at least 64); slots + signatures + flags + R-row bitmap
    assert lib.as_join_table_bytes(1000, 0.5) == (2048 * 16 + ((1000 * 8 + 255) // 256) * 256 + 256
                                                  + ((1000 + 31) // 32 * 4 + 255) // 256 * 256)
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


def r256(x):
    return (x + 255) // 256 * 256


def test_partitioned_and_prefix_workspace_queries(lib):
    """Workspace sizes of the partitioned and prefix joins are host arithmetic:
    they follow the documented layouts, reject what the calls would reject, and
    the automatic partition count keeps about 1024 R rows per partition."""
    import paper_2411_18183_gb300 as ag
    m, n, lf = 100_000, 400_000, 0.5
    # prefix join: the one-table join's slots, R's and S's signatures, flags and counter
    assert ag.join_prefix_ws_bytes(m, n, lf) == 262144 * 16 + r256(m * 8) + r256(n * 8) + 512
    assert ag.join_prefix_ws_bytes(m, n, 0.0) == 0
    # partitioned join: signatures, entries, 7 per-partition arrays, slots (< 2 m / lf + 65 per partition)
    for bits in (0, 4, 12):
        P = 1 << bits
        slots = int(2.0 * m / lf) + 64 * P + P
        want = (r256(m * 8) + r256(n * 8) + r256(m * 16) + r256(n * 16) + 7 * r256((P + 1) * 8)
                + r256(slots * 16) + 512)
        assert ag.join_part_ws_bytes(m, n, lf, bits) == want, bits
    assert ag.join_part_ws_bytes(m, n, lf, 13) == 0
    assert ag.join_part_ws_bytes(m, n, 1e-9) == 0                      # beyond 2^40 slots
    assert ag.join_part_ws_bytes(2 ** 32, n, lf) == 0
    # automatic bits: the smallest b with m >> (b + 10) == 0 (at most 12)
    for mm, bits in ((1000, 0), (1024, 1), (100_000, 7), (10 ** 9, 12)):
        assert ag.join_part_ws_bytes(mm, 10, lf) == ag.join_part_ws_bytes(mm, 10, lf, bits), mm


def test_new_join_argument_errors_before_any_device_work(lib):
    import paper_2411_18183_gb300 as ag
    buf = (ctypes.c_uint8 * 64)()
    base = (ctypes.addressof(buf) + 15) // 16 * 16
    # misaligned arena, null pointers, oversize prefix: rejected on the host
    assert lib.as_join_prefix(base + 1, base, None, 1, base, base, None, 1, 16, ctypes.c_float(0.5), base, 64,
                              base, 1, None, None, None) == 1
    assert lib.as_join_prefix(base, base, None, 1, base, base, None, 1, 2 ** 40, ctypes.c_float(0.5), base, 64,
                              base, 1, None, None, None) == 1
    assert lib.as_join_partitioned(None, None, None, 5, base, base, None, 1, ctypes.c_float(0.5), ag.PART_BITS_AUTO,
                                   base, 64, base, 1, None, None, None) == 1
    assert lib.as_join_partitioned(base, base, None, 1, base, base, None, 1, ctypes.c_float(0.5), 13, base, 64,
                                   base, 1, None, None, None) == 1
