"""Prefix join (as_join_prefix through the C ABI): the join on the keys' first L
bytes against the oracle's definition, for L below, at and above the key
lengths, with odd starts, empty keys and duplicates."""
import random

import numpy as np
import pytest

import oracle
import workloads
from cases import edge_keys
from packing import relation_garbage_tail

pytestmark = pytest.mark.gpu


def dev(ag, rel):
    return ag.DeviceRelation.from_host(rel.arena, rel.off, rel.ids)


def check(ag, R, S, L):
    got = oracle.sort_pairs(ag.join_prefix(dev(ag, R), dev(ag, S), L).cpu().numpy().view(np.uint32))
    want = oracle.join_prefix(R, S, L)
    assert got.shape == want.shape, (L, got.shape, want.shape)
    assert np.array_equal(got, want), L
    return want


def test_shared_prefixes_every_length(cuda):
    rng = random.Random(31)
    stems = [bytes(rng.randrange(256) for _ in range(rng.randrange(0, 300))) for _ in range(12)]
    keys = [st + bytes(rng.randrange(4) for _ in range(rng.randrange(0, 40))) for st in stems for _ in range(6)]
    R = relation_garbage_tail([rng.choice(keys) for _ in range(150)], seed=32,
                              ids=[rng.randrange(2 ** 32) for _ in range(150)])
    S = relation_garbage_tail([rng.choice(keys) for _ in range(400)], seed=33)
    for L in (1, 2, 15, 16, 17, 33, 100, 255, 256, 257, 300, 340, 10_000):
        check(cuda, R, S, L)


def test_edge_keys_and_the_two_ends(cuda):
    keys = edge_keys()
    R = relation_garbage_tail(keys, seed=34)
    S = relation_garbage_tail(list(reversed(keys)) + keys[:20], seed=35)
    check(cuda, R, S, 7)
    longest = max(len(k) for k in keys)
    want = check(cuda, R, S, longest)
    assert np.array_equal(want, oracle.join_simple(R, S))
    small_R = workloads.relation_from_keys([b"ab", b"", b"abc"])
    small_S = workloads.relation_from_keys([b"x", b"abd"])
    assert len(check(cuda, small_R, small_S, 0)) == 6          # every pair joins at L = 0


def test_large_config_scaled_at_256_bytes(cuda):
    wl = workloads.generate(workloads.CONFIGS["large"].scaled(5_000, 50_000))
    want = check(cuda, wl.R, wl.S, 256)
    assert len(want) >= wl.expected_pairs()


def test_bad_prefix_length_rejected(cuda):
    ag = cuda
    X = dev(ag, workloads.relation_from_keys([b"x"]))
    with pytest.raises(ag.AlgsigError):
        ag.join_prefix(X, X, 2 ** 33)
