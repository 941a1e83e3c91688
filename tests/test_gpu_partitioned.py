"""Radix-partitioned signature join (as_join_partitioned through the C ABI)
against the CPU oracle: sorted (r_id, s_id) pairs, bit-exact, for every number
of partition bits, with empty, skewed and colliding inputs."""
import random

import numpy as np
import pytest
import torch

import oracle
import workloads
from cases import edge_keys, five_symbol_collision
from packing import relation_garbage_tail

pytestmark = pytest.mark.gpu


def dev(ag, rel):
    return ag.DeviceRelation.from_host(rel.arena, rel.off, rel.ids)


def gpu_part(ag, R, S, bits, lf=0.5):
    pairs = ag.join_partitioned(dev(ag, R), dev(ag, S), load_factor=lf, part_bits=bits)
    return oracle.sort_pairs(pairs.cpu().numpy().view(np.uint32))


def check(ag, R, S, bits, lf=0.5):
    got = gpu_part(ag, R, S, bits, lf)
    want = oracle.join_simple(R, S)
    assert got.shape == want.shape, (bits, got.shape, want.shape)
    assert np.array_equal(got, want), bits
    return want


@pytest.mark.parametrize("bits", [0, 1, 5, 12, "auto"])
def test_edge_keys_and_collisions(cuda, bits):
    b = cuda.PART_BITS_AUTO if bits == "auto" else bits
    keys = edge_keys()
    x, y = five_symbol_collision()
    R = relation_garbage_tail(keys + [x, b"A", b"\0"], seed=1)
    S = relation_garbage_tail(list(reversed(keys)) + keys + [y, b"A\0", b"\0\0", x], seed=2)
    check(cuda, R, S, b)


def test_duplicates_ids_and_load_factors(cuda):
    rng = random.Random(5)
    pool = [bytes(rng.randrange(4) for _ in range(rng.randrange(0, 40))) for _ in range(60)]
    rkeys = [rng.choice(pool) for _ in range(1000)]
    skeys = [rng.choice(pool) for _ in range(3000)]
    R = relation_garbage_tail(rkeys, seed=6, ids=[rng.randrange(2 ** 32) for _ in rkeys])
    S = relation_garbage_tail(skeys, seed=7, ids=[rng.randrange(2 ** 32) for _ in skeys])
    for lf in (1.0, 0.5, 0.25):
        for bits in (0, 3, 8):
            check(cuda, R, S, bits, lf)


def test_one_hot_key(cuda):
    # every R and S row has the same key: one partition holds everything, the others are empty
    k = b"the same key" * 9
    R = workloads.relation_from_keys([k] * 300)
    S = workloads.relation_from_keys([k] * 50 + [b"other"] * 20)
    want = check(cuda, R, S, 6)
    assert len(want) == 300 * 50


def test_empty_relations(cuda):
    E = workloads.relation_from_keys([])
    X = workloads.relation_from_keys([b"x", b""])
    for R, S in ((E, X), (X, E), (E, E)):
        assert gpu_part(cuda, R, S, 4).shape == (0, 2)
    assert gpu_part(cuda, X, X, 4).tolist() == [[0, 0], [1, 1]]


@pytest.mark.parametrize("name,scale", [("plain", None), ("large", (20_000, 200_000)),
                                        ("collision", (2_000, 20_000))])
def test_configs_match_the_unpartitioned_join(cuda, name, scale):
    spec = workloads.CONFIGS[name] if scale is None else workloads.CONFIGS[name].scaled(*scale)
    wl = workloads.generate(spec)
    want = check(cuda, wl.R, wl.S, cuda.PART_BITS_AUTO)
    assert len(want) == wl.expected_pairs()
    other = cuda.join(dev(cuda, wl.R), dev(cuda, wl.S))
    assert np.array_equal(oracle.sort_pairs(other.cpu().numpy().view(np.uint32)), want)


def test_capacity_overflow_reports_exact_count(cuda):
    ag = cuda
    wl = workloads.generate(workloads.CONFIGS["plain"].scaled(1000, 10_000))
    R, S = dev(ag, wl.R), dev(ag, wl.S)
    ws = ag.alloc_ws(ag.join_part_ws_bytes(R.n, S.n, 0.5))
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    pairs = torch.full((2 * 100,), -1, dtype=torch.int32, device="cuda")
    st, cnt = ag.join_partitioned_into(R, S, ws, pairs, count, 0.5, sync=True, allow_capacity=True)
    want = oracle.join_simple(wl.R, wl.S)
    assert st == ag.AS_ERR_CAPACITY and cnt == len(want) == 3000
    got = pairs.cpu().numpy().view(np.uint32).reshape(-1, 2)
    wantset = {tuple(p) for p in want.tolist()}
    assert all(tuple(p) in wantset for p in got.tolist())


def test_bad_arguments_are_rejected(cuda):
    ag = cuda
    assert ag.join_part_ws_bytes(10, 10, 0.5, 13) == 0
    assert ag.join_part_ws_bytes(10, 10, 0.0) == 0
    X = dev(ag, workloads.relation_from_keys([b"x"]))
    small = ag.alloc_ws(256)
    pairs = torch.empty(2, dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(ag.AlgsigError):
        ag.join_partitioned_into(X, X, small, pairs, count, 0.5)
