"""as_join_probe_noalloc (probe with the library's fixed signature scratch, no
workspace): same pairs and count as as_join_probe on two calls in a row, and
sizes beyond the scratch are rejected before any device work.  Collected last
so that it also runs after every other test has used the library."""
import ctypes
import re
from pathlib import Path

import numpy as np
import pytest
import torch

import oracle
import workloads

HEADER = Path(__file__).resolve().parents[1] / "include" / "algsig.h"


def header_max_keys() -> int:
    m = re.search(r"#define\s+AS_PROBE_NOALLOC_MAX_KEYS\s+\(1u\s*<<\s*(\d+)\)", HEADER.read_text())
    return 1 << int(m.group(1))


def test_binding_constant_matches_header():
    import paper_2411_18183_gb300 as ag
    assert ag.PROBE_NOALLOC_MAX_KEYS == header_max_keys()


def test_rejects_more_keys_than_the_scratch():
    import paper_2411_18183_gb300 as ag
    lib = ag.load()
    lib.as_join_probe_noalloc.restype = ctypes.c_int
    t = ag.Table()
    st = lib.as_join_probe_noalloc(ctypes.byref(t), None, None, None, ctypes.c_uint64(header_max_keys() + 1),
                                   None, ctypes.c_uint64(0), None, None, None)
    assert st == ag.AS_ERR_INVALID
    assert b"fixed scratch" in lib.as_last_error()
    # argument errors past the size check name this entry point, not as_join_probe
    st = lib.as_join_probe_noalloc(ctypes.byref(t), None, None, None, ctypes.c_uint64(4), None,
                                   ctypes.c_uint64(0), None, None, None)
    assert st == ag.AS_ERR_INVALID
    assert lib.as_last_error().startswith(b"as_join_probe_noalloc:")


def sorted_pairs(pairs, cnt):
    return oracle.sort_pairs(pairs[: 2 * cnt].cpu().numpy().view(np.uint32))


@pytest.mark.gpu
def test_noalloc_probe_matches_probe_twice(cuda):
    ag = cuda
    spec = workloads.CONFIGS["plain"].scaled(3000, 40000)
    wl = workloads.generate(spec)
    R = ag.DeviceRelation.from_host(wl.R.arena, wl.R.off, wl.R.ids)
    S = ag.DeviceRelation.from_host(wl.S.arena, wl.S.off, wl.S.ids)
    tb = ag.join_table_bytes(R.n, 0.5)
    ws = ag.alloc_ws(tb)
    t = ag.join_build(R, ws, 0.5)
    cap = wl.expected_pairs() + 1024
    pairs = torch.zeros(2 * cap, dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    pws = ag.alloc_ws(ag.join_probe_ws_bytes(S.n))
    n0 = ag.join_probe(t, S, pairs, count, ws=pws)
    want = sorted_pairs(pairs, n0)
    assert n0 == wl.expected_pairs()
    for _ in range(2):
        pairs.zero_()
        count.fill_(12345)                   # the call clears the counter itself
        n1 = ag.join_probe_noalloc(t, S, pairs, count)
        assert n1 == n0 == int(count.item())
        assert np.array_equal(sorted_pairs(pairs, n1), want)
    # the oracle agrees as well
    assert np.array_equal(want, oracle.sort_pairs(oracle.join_simple(wl.R, wl.S)))


@pytest.mark.gpu
def test_noalloc_probe_at_the_scratch_limit(cuda):
    """S with exactly AS_PROBE_NOALLOC_MAX_KEYS rows (short keys): the whole
    scratch is written and read; pairs and count as as_join_probe's, twice."""
    ag = cuda
    n = header_max_keys()
    wl = workloads.generate(workloads.CONFIGS["plain"].scaled(n // 10, n))
    assert wl.S.n == n
    R = ag.DeviceRelation.from_host(wl.R.arena, wl.R.off, wl.R.ids)
    S = ag.DeviceRelation.from_host(wl.S.arena, wl.S.off, wl.S.ids)
    ws = ag.alloc_ws(ag.join_table_bytes(R.n, 0.5))
    t = ag.join_build(R, ws, 0.5)
    cap = wl.expected_pairs() + 4096
    pairs = torch.zeros(2 * cap, dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    n0 = ag.join_probe(t, S, pairs, count, ws=ag.alloc_ws(ag.join_probe_ws_bytes(S.n)))
    want = sorted_pairs(pairs, n0)
    for _ in range(2):
        pairs.zero_()
        n1 = ag.join_probe_noalloc(t, S, pairs, count)
        assert n1 == n0
        assert np.array_equal(sorted_pairs(pairs, n1), want)
