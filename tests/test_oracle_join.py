"""Pins of the oracle's joins: nested loop (brute force) = simple hash join =
Grace hash join (Section 2), plus the ground truth of the input generator."""
import random

import numpy as np
import pytest

import oracle
import workloads
from cases import edge_keys, five_symbol_collision
from workloads import relation_from_keys


def brute(rkeys, skeys, rids=None, sids=None):
    rids = rids if rids is not None else list(range(len(rkeys)))
    sids = sids if sids is not None else list(range(len(skeys)))
    out = [(rids[r], sids[s]) for r in range(len(rkeys)) for s in range(len(skeys)) if rkeys[r] == skeys[s]]
    return np.array(sorted(out), dtype=np.uint32).reshape(-1, 2)


def run_all(R, S):
    a = oracle.join_nested(R, S)
    b = oracle.join_simple(R, S)
    c = oracle.join_grace(R, S, log2_parts=3, nthreads=3)
    assert np.array_equal(a, b) and np.array_equal(b, c)
    return a


def test_edge_keys_join():
    keys = edge_keys()
    R = workloads.relation_from_keys(keys)
    S = workloads.relation_from_keys(list(reversed(keys)))
    got = run_all(R, S)
    assert np.array_equal(got, brute(keys, list(reversed(keys))))
    # "A" and "A\0" share a signature but are different keys
    ia, ia0 = keys.index(b"A"), keys.index(b"A\0")
    assert oracle.sig(keys[ia]) == oracle.sig(keys[ia0])
    pairs = {tuple(p) for p in got.tolist()}
    rev = list(reversed(keys))
    assert (ia, rev.index(b"A\0")) not in pairs


def test_collision_pair_does_not_join():
    a, b = five_symbol_collision()
    R = workloads.relation_from_keys([a])
    S = workloads.relation_from_keys([b, a])
    got = run_all(R, S)
    assert got.tolist() == [[0, 1]]


def test_random_small_with_duplicates_and_ids():
    rng = random.Random(10)
    pool = [bytes(rng.randrange(3) for _ in range(rng.randrange(0, 5))) for _ in range(30)]
    rkeys = [rng.choice(pool) for _ in range(300)]
    skeys = [rng.choice(pool) for _ in range(500)]
    rids = [rng.randrange(2 ** 32) for _ in rkeys]
    sids = [rng.randrange(2 ** 32) for _ in skeys]
    R = workloads.relation_from_keys(rkeys, rids)
    S = workloads.relation_from_keys(skeys, sids)
    got = run_all(R, S)
    assert np.array_equal(got, brute(rkeys, skeys, rids, sids))


def test_empty_relations():
    R = workloads.relation_from_keys([])
    S = workloads.relation_from_keys([b"x"])
    assert run_all(R, S).shape == (0, 2)
    assert run_all(S, R).shape == (0, 2)


def test_plain_workload_ground_truth():
    wl = workloads.generate(workloads.CONFIGS["plain"])
    got = oracle.join_simple(wl.R, wl.S)
    assert len(got) == wl.expected_pairs() == 30_000
    g2 = oracle.join_grace(wl.R, wl.S, log2_parts=6, nthreads=4)
    assert np.array_equal(got, g2)
    # every pair is an exact copy made by the generator
    src = wl.s_src[got[:, 1]]
    assert np.array_equal(src, got[:, 0].astype(np.int64))


def test_collision_workload_ground_truth():
    spec = workloads.CONFIGS["collision"].scaled(500, 5_000)
    wl = workloads.generate(spec)
    got = oracle.join_simple(wl.R, wl.S)
    assert len(got) == wl.expected_pairs() == int((wl.s_kind == 1).sum()) == 2_000
    assert set(wl.s_kind[got[:, 1]].tolist()) == {1}
    # near-duplicates exist, share no signature with their source (<= 6 byte changes
    # touch <= 6 symbols; equal signatures would need a 2^-64 event) and do not join
    near = np.nonzero(wl.s_kind == 2)[0][:200]
    sS = oracle.sig_batch(wl.S.arena, wl.S.off)
    sR = oracle.sig_batch(wl.R.arena, wl.R.off)
    assert len(near) == 200 and not np.any(sS[near] == sR[wl.s_src[near]])


def test_large_workload_ground_truth_scaled():
    spec = workloads.CONFIGS["large"].scaled(20_000, 200_000)
    wl = workloads.generate(spec)
    got = oracle.join_grace(wl.R, wl.S, log2_parts=8, nthreads=4)
    assert len(got) == wl.expected_pairs()
    assert (wl.r_mult > 1).any()


def test_join_modes_by_definition_and_brute_force():
    """semi / anti / outer_s and their R-side counterparts (semi_r / anti_r /
    outer_r) of the oracle against a brute-force statement on small relations
    with duplicates, empty keys and ids that are not rows."""
    import random
    rng = random.Random(11)
    pool = [b"", b"a", b"ab", b"abc", b"xyz" * 5, bytes(range(40))]
    rk = [rng.choice(pool) for _ in range(25)]
    sk = [rng.choice(pool + [b"q", b"zz"]) for _ in range(40)]
    R = workloads.relation_from_keys(rk, ids=[1000 + i for i in range(len(rk))])
    S = workloads.relation_from_keys(sk, ids=[7 * i + 3 for i in range(len(sk))])
    NO = oracle.NO_ROW
    inner = sorted((1000 + i, 7 * j + 3) for j, s in enumerate(sk) for i, r in enumerate(rk) if r == s)
    has = {j for j, s in enumerate(sk) if s in rk}
    r_has = {i for i, r in enumerate(rk) if r in sk}
    want = {
        "inner": inner,
        "semi": sorted((NO, 7 * j + 3) for j in range(len(sk)) if j in has),
        "anti": sorted((NO, 7 * j + 3) for j in range(len(sk)) if j not in has),
        "outer_s": sorted(inner + [(NO, 7 * j + 3) for j in range(len(sk)) if j not in has]),
        "semi_r": sorted((1000 + i, NO) for i in range(len(rk)) if i in r_has),
        "anti_r": sorted((1000 + i, NO) for i in range(len(rk)) if i not in r_has),
        "outer_r": sorted(inner + [(1000 + i, NO) for i in range(len(rk)) if i not in r_has]),
    }
    # the R-side modes partition R, and every R row appears once
    assert len(want["semi_r"]) + len(want["anti_r"]) == len(rk)
    for mode, w in want.items():
        got = [tuple(int(x) for x in row) for row in oracle.join_mode(R, S, mode)]
        assert got == w, mode


def test_signature_only_join_by_definition():
    """The signature-only join of Figure 2 (no byte comparison) equals the
    exact join when no two different keys share a signature and length, and
    adds exactly the colliding pairs otherwise: the five-symbol collision for
    four components, a three-symbol collision for the paper's two components
    (which four components separate).  Checked against a nested loop over
    (signature, length)."""
    from cases import symbol_collision
    rng = random.Random(31)
    keys = [bytes(rng.randrange(256) for _ in range(rng.randrange(0, 40))) for _ in range(80)]
    R = relation_from_keys(keys + keys[:10])
    S = relation_from_keys(keys[5:] + [b"", b"\0"])
    assert np.array_equal(oracle.join_sig_only(R, S), oracle.join_simple(R, S))
    assert np.array_equal(oracle.join_sig_only(R, S, 2), oracle.join_simple(R, S))
    a4, b4 = five_symbol_collision()
    a2, b2 = symbol_collision(2, 12, (0, 5, 11), seed=3)
    R = relation_from_keys([a4, a2])
    S = relation_from_keys([b4, b2, a4])
    assert oracle.join_simple(R, S).tolist() == [[0, 2]]
    assert oracle.join_sig_only(R, S, 4).tolist() == [[0, 0], [0, 2]]
    assert oracle.join_sig_only(R, S, 2).tolist() == [[0, 0], [0, 2], [1, 1]]
    # brute force over (signature, length)
    sR, sS = oracle.sig_batch(R.arena, R.off), oracle.sig_batch(S.arena, S.off)
    lR, lS = np.diff(R.off), np.diff(S.off)
    for n in (2, 4):
        m = np.uint64(oracle.component_mask(n))
        brute = [[i, j] for i in range(R.n) for j in range(S.n) if (sR[i] & m) == (sS[j] & m) and lR[i] == lS[j]]
        assert oracle.join_sig_only(R, S, n).tolist() == brute


def test_prefix_join_by_definition_and_brute_force():
    """The prefix join against what fixes it: with L at least the longest key it
    is the exact join; at L = 0 every pair joins; and a nested loop over
    truncated keys on small random inputs, for lengths around the keys'."""
    rng = random.Random(21)
    pool = [bytes(rng.randrange(3) for _ in range(rng.randrange(0, 12))) for _ in range(25)]
    rkeys = [rng.choice(pool) for _ in range(70)]
    skeys = [rng.choice(pool) for _ in range(90)]
    R = relation_from_keys(rkeys, ids=[rng.randrange(2 ** 32) for _ in rkeys])
    S = relation_from_keys(skeys, ids=[rng.randrange(2 ** 32) for _ in skeys])
    assert np.array_equal(oracle.join_prefix(R, S, 12), oracle.join_simple(R, S))
    everything = oracle.sort_pairs(np.array([(int(r), int(s)) for r in R.ids for s in S.ids], dtype=np.uint32))
    assert np.array_equal(oracle.join_prefix(R, S, 0), everything)
    for L in (1, 2, 3, 5, 8):
        want = [(int(R.ids[i]), int(S.ids[j])) for i, a in enumerate(rkeys) for j, b in enumerate(skeys)
                if a[:L] == b[:L]]
        assert np.array_equal(oracle.join_prefix(R, S, L), oracle.sort_pairs(np.array(want, dtype=np.uint32))), L
