"""GPU signature join (as_join / as_join_build / as_join_probe through the C
ABI) against the CPU oracle: sorted (r_id, s_id) pairs, bit-exact."""
import dataclasses
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


def gpu_join(ag, R, S, lf=0.5):
    pairs = ag.join(dev(ag, R), dev(ag, S), load_factor=lf)
    return oracle.sort_pairs(pairs.cpu().numpy().view(np.uint32))


def check(ag, R, S, lf=0.5):
    got = gpu_join(ag, R, S, lf)
    want = oracle.join_simple(R, S)
    assert got.shape == want.shape, (got.shape, want.shape)
    assert np.array_equal(got, want)
    return want


def test_edge_keys(cuda):
    keys = edge_keys()
    R = relation_garbage_tail(keys, seed=1)
    S = relation_garbage_tail(list(reversed(keys)) + keys, seed=2)
    check(cuda, R, S)


def test_collision_pair_and_padding_twins(cuda):
    a, b = five_symbol_collision()
    R = relation_garbage_tail([a, b"A", b"\0"], seed=3)
    S = relation_garbage_tail([b, b"A\0", b"", b"\0\0", a], seed=4)
    got = check(cuda, R, S)
    assert got.tolist() == [[0, 4]]


def test_random_small_duplicates_ids_and_load_factors(cuda):
    rng = random.Random(5)
    pool = [bytes(rng.randrange(4) for _ in range(rng.randrange(0, 40))) for _ in range(60)]
    rkeys = [rng.choice(pool) for _ in range(1000)]
    skeys = [rng.choice(pool) for _ in range(3000)]
    R = relation_garbage_tail(rkeys, seed=6, ids=[rng.randrange(2 ** 32) for _ in rkeys])
    S = relation_garbage_tail(skeys, seed=7, ids=[rng.randrange(2 ** 32) for _ in skeys])
    for lf in (1.0, 0.5, 0.25):
        check(cuda, R, S, lf)


def test_full_table_load_factor_one(cuda):
    # m = cap = 64: every slot used, probes of absent keys walk the whole table
    rng = random.Random(8)
    rkeys = [bytes(rng.randrange(256) for _ in range(20)) for _ in range(64)]
    skeys = [rng.choice(rkeys) for _ in range(100)] + [b"absent"] * 10
    check(cuda, workloads.relation_from_keys(rkeys), workloads.relation_from_keys(skeys), lf=1.0)


def test_empty_relations(cuda):
    E = workloads.relation_from_keys([])
    X = workloads.relation_from_keys([b"x", b""])
    for R, S in ((E, X), (X, E), (E, E)):
        got = gpu_join(cuda, R, S)
        assert got.shape == (0, 2)
    got = gpu_join(cuda, X, X)
    assert got.tolist() == [[0, 0], [1, 1]]


def test_capacity_overflow_reports_exact_count(cuda):
    ag = cuda
    wl = workloads.generate(workloads.CONFIGS["plain"].scaled(1000, 10_000))
    R, S = dev(ag, wl.R), dev(ag, wl.S)
    ws = ag.alloc_ws(ag.join_ws_bytes(R.n, S.n, 0.5))
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    pairs = torch.full((2 * 100,), -1, dtype=torch.int32, device="cuda")
    st, cnt = ag.join_into(R, S, ws, pairs, count, 0.5, sync=True, allow_capacity=True)
    want = oracle.join_simple(wl.R, wl.S)
    assert st == ag.AS_ERR_CAPACITY and cnt == len(want) == 3000
    part = pairs.cpu().numpy().view(np.uint32).reshape(-1, 2)
    wantset = {tuple(p) for p in want.tolist()}
    assert all(tuple(p) in wantset for p in part.tolist())


def test_build_probe_split_and_signature_output(cuda):
    ag = cuda
    wl = workloads.generate(workloads.CONFIGS["plain"].scaled(3000, 30_000))
    R, S = dev(ag, wl.R), dev(ag, wl.S)
    ws = ag.alloc_ws(ag.join_table_bytes(R.n, 0.5))
    sigR = ag.sig_compute(R)
    t = ag.join_build(R, ws, 0.5, sigR=sigR)
    pairs = torch.empty(2 * 20_000, dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    sigS = torch.empty(S.n, dtype=torch.int64, device="cuda")
    cnt = ag.join_probe(t, S, pairs, count, sigS_out=sigS)
    pws = ag.alloc_ws(ag.join_probe_ws_bytes(S.n))
    cnt2 = ag.join_probe(t, S, pairs, count, ws=pws)
    assert cnt2 == cnt
    got = oracle.sort_pairs(pairs[: 2 * cnt].cpu().numpy().view(np.uint32))
    assert np.array_equal(got, oracle.join_simple(wl.R, wl.S))
    assert np.array_equal(sigS.cpu().numpy().view(np.uint64), oracle.sig_batch(wl.S.arena, wl.S.off, nthreads=8))


def test_plain_config_full(cuda):
    wl = workloads.generate(workloads.CONFIGS["plain"])
    want = check(cuda, wl.R, wl.S)
    assert len(want) == 30_000


def test_collision_config_scaled(cuda):
    wl = workloads.generate(workloads.CONFIGS["collision"].scaled(2_000, 20_000))
    want = check(cuda, wl.R, wl.S)
    assert len(want) == 8_000


def test_large_config_scaled(cuda):
    wl = workloads.generate(workloads.CONFIGS["large"].scaled(20_000, 200_000))
    want = check(cuda, wl.R, wl.S)
    assert len(want) == wl.expected_pairs()


# ----------------------------------------------------------------------------- the comparison join

def gpu_baseline(ag, R, S, tagged, lf=0.5):
    pairs = ag.baseline_join(dev(ag, R), dev(ag, S), load_factor=lf, tagged=tagged)
    return oracle.sort_pairs(pairs.cpu().numpy().view(np.uint32))


@pytest.mark.parametrize("tagged", [False, True])
def test_baseline_join_matches_oracle(cuda, tagged):
    keys = edge_keys()
    R = relation_garbage_tail(keys, seed=11)
    S = relation_garbage_tail(list(reversed(keys)) + keys, seed=12)
    assert np.array_equal(gpu_baseline(cuda, R, S, tagged), oracle.join_simple(R, S))
    rng = random.Random(13)
    pool = [bytes(rng.randrange(4) for _ in range(rng.randrange(0, 40))) for _ in range(60)]
    R = relation_garbage_tail([rng.choice(pool) for _ in range(800)], seed=14)
    S = relation_garbage_tail([rng.choice(pool) for _ in range(2000)], seed=15)
    for lf in (1.0, 0.5):
        assert np.array_equal(gpu_baseline(cuda, R, S, tagged, lf), oracle.join_simple(R, S))
    wl = workloads.generate(workloads.CONFIGS["large"].scaled(5_000, 50_000))
    assert np.array_equal(gpu_baseline(cuda, wl.R, wl.S, tagged), oracle.join_simple(wl.R, wl.S))


def test_probe_with_given_signatures(cuda):
    """as_join_probe_sigs with signatures from as_sig_compute gives the join;
    signatures that are wrong for some rows only lose those rows' matches."""
    ag = cuda
    wl = workloads.generate(workloads.CONFIGS["plain"].scaled(2000, 25_000))
    R, S = dev(ag, wl.R), dev(ag, wl.S)
    ws = ag.alloc_ws(ag.join_table_bytes(R.n, 0.5))         # the table lives in ws: keep it
    t = ag.join_build(R, ws, 0.5)
    pairs = torch.empty(2 * 20_000, dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    sigS = ag.sig_compute(S)
    cnt = ag.join_probe_sigs(t, S, sigS, pairs, count)
    want = oracle.join_simple(wl.R, wl.S)
    assert np.array_equal(oracle.sort_pairs(pairs[: 2 * cnt].cpu().numpy().view(np.uint32)), want)
    bad = sigS.clone()
    bad[::2] ^= 1                                   # corrupt even rows' signatures
    cnt = ag.join_probe_sigs(t, S, bad, pairs, count)
    got = oracle.sort_pairs(pairs[: 2 * cnt].cpu().numpy().view(np.uint32))
    assert np.array_equal(got, want[want[:, 1] % 2 == 1])


@pytest.mark.parametrize("mode", ["inner", "semi", "anti", "outer_s", "outer_r", "semi_r", "anti_r"])
def test_probe_modes_match_oracle(cuda, mode):
    """as_join_probe_mode against the oracle's definitions, on a scaled large-workload
    relation pair (duplicate R keys) and on the edge keys; the R-side modes twice on one
    table (the row bitmap is cleared by each call)."""
    ag = cuda
    cases = []
    wl = workloads.generate(workloads.CONFIGS["large"].scaled(3000, 20_000))
    cases.append((wl.R, wl.S))
    keys = edge_keys()
    cases.append((workloads.relation_from_keys(keys[::2] + keys[:5]),
                  workloads.relation_from_keys(keys, ids=[5 * i + 1 for i in range(len(keys))])))
    for Rh, Sh in cases:
        R, S = dev(ag, Rh), dev(ag, Sh)
        ws = ag.alloc_ws(ag.join_table_bytes(R.n, 0.5))
        t = ag.join_build(R, ws, 0.5)
        sigS = ag.sig_compute(S)
        want = oracle.join_mode(Rh, Sh, mode)
        pairs = torch.zeros(2 * (len(want) + 64), dtype=torch.int32, device="cuda")
        count = torch.zeros(1, dtype=torch.int64, device="cuda")
        for _ in range(2 if mode.endswith("_r") else 1):
            cnt = ag.join_probe_mode(t, S, sigS, pairs, count, mode=mode)
            got = oracle.sort_pairs(pairs[: 2 * cnt].cpu().numpy().view(np.uint32))
            assert np.array_equal(got, want), (mode, Rh.n, Sh.n)


@pytest.mark.parametrize("seed", range(4))
def test_signature_collisions_rejected_at_every_alignment(cuda, seed):
    """Equal-length keys that share all four signature components but differ
    in five symbols reach the byte comparison as candidates; at any start
    alignment of either key (random gap keys of 0..16 bytes before each key),
    with differences in the first and last symbols and across 512-byte
    comparison steps, and at odd lengths, only exact copies may join."""
    from packing import interleave_gaps
    rng = random.Random(1000 + seed)
    shapes = [(5, (0, 1, 2, 3, 4)), (8, (0, 2, 4, 6, 7)), (24, (1, 4, 9, 15, 22)),
              (256, (0, 100, 200, 254, 255)), (257, (3, 255, 256, 100, 7)), (520, (0, 255, 256, 511, 519)),
              (700, (10, 300, 512, 600, 650))]
    rkeys, skeys = [], []
    for n_sym, pos in shapes:
        a, b = five_symbol_collision(n_sym, pos, seed=rng.randrange(1 << 30))
        rkeys += [a]
        skeys += [b, a]
        if max(pos) < n_sym - 1:                      # odd length: drop the last (equal) byte of both
            rkeys += [a[:-1]]
            skeys += [b[:-1], a[:-1]]
    R = relation_garbage_tail(interleave_gaps(rkeys, seed=rng.randrange(1 << 30)), seed=seed)
    S = relation_garbage_tail(interleave_gaps(skeys, seed=rng.randrange(1 << 30)), seed=seed + 1)
    check(cuda, R, S)


@pytest.mark.parametrize("n_components", [4, 2])
def test_signature_only_probe_matches_oracle(cuda, n_components):
    """AS_JOIN_SIG_ONLY (the probe of Figure 2 without byte verification) with
    n-component signatures on both sides against the oracle's definition: the
    exact pairs plus the constructed collisions (five symbols for n = 4, three
    for n = 2), and the exact join still rejects them."""
    from cases import symbol_collision
    ag = cuda
    a4, b4 = five_symbol_collision()
    a2, b2 = symbol_collision(2, 12, (0, 5, 11), seed=3)
    wl = workloads.generate(workloads.CONFIGS["large"].scaled(2000, 10_000))
    keys_r = [wl.R.key(i) for i in range(wl.R.n)] + [a4, a2]
    keys_s = [wl.S.key(i) for i in range(wl.S.n)] + [b4, b2, a4]
    Rh = relation_garbage_tail(keys_r, seed=1)
    Sh = relation_garbage_tail(keys_s, seed=2)
    R, S = dev(ag, Rh), dev(ag, Sh)
    sigR = ag.sig_compute(R, n_components=n_components)
    sigS = ag.sig_compute(S, n_components=n_components)
    ws = ag.alloc_ws(ag.join_table_bytes(R.n, 0.5))
    t = ag.join_build(R, ws, 0.5, sigR=sigR)
    for mode, want in (("sig_only", oracle.join_sig_only(Rh, Sh, n_components)),
                       ("inner", oracle.join_simple(Rh, Sh))):
        pairs = torch.zeros(2 * (len(want) + 64), dtype=torch.int32, device="cuda")
        count = torch.zeros(1, dtype=torch.int64, device="cuda")
        cnt = ag.join_probe_mode(t, S, sigS, pairs, count, mode=mode)
        got = oracle.sort_pairs(pairs[: 2 * cnt].cpu().numpy().view(np.uint32))
        assert np.array_equal(got, want), (mode, n_components)
    extra = len(oracle.join_sig_only(Rh, Sh, n_components)) - len(oracle.join_simple(Rh, Sh))
    assert extra == (1 if n_components == 4 else 2)


def test_byte_symbol_join_exact_and_signature_only(cuda):
    """The join on GF(2^8) signatures (as_sig_compute_gf8 on both sides): exact
    with verification, and the signature-only probe adds exactly the
    constructed five-byte collision (and the pair past the 255-byte wrap)."""
    from gfpoly import gpow8, solve8
    ag = cuda
    rng = random.Random(808)
    pos = [2, 9, 40, 100, 200]
    M = [[gpow8(2, k * pos[j]) for j in range(4)] for k in range(1, 5)]
    d = solve8(M, [gpow8(2, k * pos[4]) for k in range(1, 5)]) + [1]
    a = bytes(rng.randrange(32, 127) for _ in range(230))
    b = bytearray(a)
    for p_, dj in zip(pos, d):
        b[p_] ^= dj
    w = bytes(rng.randrange(32, 127) for _ in range(300))
    w2 = bytearray(w)
    w2[0] ^= 0x5A
    w2[255] ^= 0x5A
    wl = workloads.generate(workloads.CONFIGS["large"].scaled(2000, 10_000))
    Rh = relation_garbage_tail([wl.R.key(i) for i in range(wl.R.n)] + [a, w], seed=5)
    Sh = relation_garbage_tail([wl.S.key(i) for i in range(wl.S.n)] + [bytes(b), bytes(w2), a], seed=6)
    R, S = dev(ag, Rh), dev(ag, Sh)
    sigR, sigS = ag.sig_compute_gf8(R), ag.sig_compute_gf8(S)
    ws = ag.alloc_ws(ag.join_table_bytes(R.n, 0.5))
    t = ag.join_build(R, ws, 0.5, sigR=sigR)
    for mode, want in (("sig_only", oracle.join_sig_only(Rh, Sh, field=8)), ("inner", oracle.join_simple(Rh, Sh))):
        pairs = torch.zeros(2 * (len(want) + 64), dtype=torch.int32, device="cuda")
        count = torch.zeros(1, dtype=torch.int64, device="cuda")
        cnt = ag.join_probe_mode(t, S, sigS, pairs, count, mode=mode)
        got = oracle.sort_pairs(pairs[: 2 * cnt].cpu().numpy().view(np.uint32))
        assert np.array_equal(got, want), mode
    assert len(oracle.join_sig_only(Rh, Sh, field=8)) - len(oracle.join_simple(Rh, Sh)) >= 2


def test_output_buffers_never_written_past_their_capacity(cuda):
    """Canary words after every output buffer: the pairs buffer of a join that
    overflows its capacity, the batch's per-join regions (each join's region
    is followed by the next join's canaried gap) and the signature output stay
    untouched past their ends."""
    ag = cuda
    CANARY = 0x5A5A5A5A
    wl = workloads.generate(workloads.CONFIGS["plain"].scaled(1000, 10_000))
    R, S = dev(ag, wl.R), dev(ag, wl.S)
    ws = ag.alloc_ws(ag.join_ws_bytes(R.n, S.n, 0.5))
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    for cap in (0, 1, 100, 2999, 3000):
        buf = torch.full((2 * cap + 64,), CANARY, dtype=torch.int32, device="cuda")
        st, cnt = ag.join_into(R, S, ws, buf[: 2 * cap], count, 0.5, sync=True, allow_capacity=True)
        assert cnt == 3000 and st == (ag.AS_OK if cap >= 3000 else ag.AS_ERR_CAPACITY)
        assert bool((buf[2 * cap:] == CANARY).all()), cap
    sig = torch.full((S.n + 16,), CANARY, dtype=torch.int64, device="cuda")
    ag.sig_compute(S, sig[: S.n])
    torch.cuda.synchronize()
    assert bool((sig[S.n:] == CANARY).all())
    # batch: join j's region of pair_cap pairs is followed by a gap of canaries
    keys_r = [wl.R.key(i) for i in range(200)]
    keys_s = [wl.S.key(i) for i in range(2000)]
    Rb = ag.DeviceRelation.from_host(*_pack(keys_r + keys_r))
    Sb = ag.DeviceRelation.from_host(*_pack(keys_s + keys_s))
    caps = [5, 3]
    descs = ag.make_descs([(0, 200, 0, 2000), (200, 400, 2000, 4000)], caps)
    gap = 32
    descs[1].pair_offset = caps[0] + gap
    total = caps[0] + gap + caps[1] + gap
    pairs = torch.full((2 * total,), CANARY, dtype=torch.int32, device="cuda")
    counts = torch.zeros(2, dtype=torch.int64, device="cuda")
    bws = ag.alloc_ws(ag.join_batch_ws_bytes(descs, Rb.n, Sb.n, 0.5))
    b = ag.join_batch_prepare(descs, Rb, Sb, bws, 0.5)
    ag.join_batch_run(b, Rb, Sb, pairs, counts)
    torch.cuda.synchronize()
    assert counts.tolist()[0] > caps[0] and counts.tolist()[1] > caps[1]
    p = pairs.view(-1, 2)
    assert bool((p[caps[0]: caps[0] + gap] == CANARY).all())
    assert bool((p[caps[0] + gap + caps[1]:] == CANARY).all())


def _pack(keys):
    rel = workloads.relation_from_keys(keys)
    return rel.arena, rel.off, rel.ids


@pytest.mark.parametrize("which", ["signature", "fullstring"])
def test_whole_join_on_a_stream_and_in_a_cuda_graph(cuda, which):
    """as_join and as_baseline_join fork S's signatures (hashes) onto a side
    stream and join it back: on a non-default stream, back to back without a
    synchronisation, and captured in a CUDA graph and replayed, every run
    gives the oracle's pairs."""
    ag = cuda
    wl = workloads.generate(workloads.CONFIGS["large"].scaled(3_000, 30_000))
    R = ag.DeviceRelation.from_host(wl.R.arena, wl.R.off, wl.R.ids)
    S = ag.DeviceRelation.from_host(wl.S.arena, wl.S.off, wl.S.ids)
    want = oracle.join_simple(wl.R, wl.S)
    cap = len(want) + 1024
    stream = torch.cuda.Stream()
    if which == "signature":
        ws = ag.alloc_ws(ag.join_ws_bytes(R.n, S.n, 0.5))
        run = lambda pairs, count: ag.join_into(R, S, ws, pairs, count, 0.5, sync=False, stream=stream)
    else:
        ws = ag.alloc_ws(ag.baseline_ws_bytes(R.n, S.n, 0.5))
        run = lambda pairs, count: ag.baseline_join_into(R, S, ws, pairs, count, 0.5, tagged=True, sync=False,
                                                         stream=stream)
    pairs = torch.empty(2 * cap, dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    with torch.cuda.stream(stream):
        for _ in range(3):
            run(pairs, count)
    stream.synchronize()
    n = int(count.item())
    assert np.array_equal(oracle.sort_pairs(pairs[: 2 * n].cpu().numpy().view(np.uint32)), want)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        run(pairs, count)
    for _ in range(2):
        pairs.zero_()
        count.zero_()
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        n = int(count.item())
        assert np.array_equal(oracle.sort_pairs(pairs[: 2 * n].cpu().numpy().view(np.uint32)), want)


def test_whole_join_fused_pass_matches_oracle(cuda):
    """From 2^19 S keys as_join probes each group of S keys inside the signature
    kernel; with edge keys at both ends of the arena, duplicates and ids, its
    pairs and signatures equal the oracle's (and those of the separate calls)."""
    ag = cuda
    spec = dataclasses.replace(workloads.CONFIGS["large"], m=20_000, n=(1 << 20) + 777, r_len=(1, 300),
                               s_len=(1, 300))
    wl = workloads.generate(spec)
    ids_r = (np.arange(wl.R.n, dtype=np.uint32) * 7 + 3).astype(np.uint32)
    ids_s = (np.arange(wl.S.n, dtype=np.uint32) * 5 + 1).astype(np.uint32)
    R = ag.DeviceRelation.from_host(wl.R.arena, wl.R.off, ids_r)
    S = ag.DeviceRelation.from_host(wl.S.arena, wl.S.off, ids_s)
    from workloads import Relation
    # (keys of one or two bytes also join by chance, so the oracle, not the generator, gives the count)
    want = oracle.join_grace(Relation(wl.R.arena, wl.R.off, ids_r), Relation(wl.S.arena, wl.S.off, ids_s), nthreads=8)
    ws = ag.alloc_ws(ag.join_ws_bytes(R.n, S.n, 0.5))
    pairs = torch.empty(2 * (len(want) + 4096), dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    st, cnt = ag.join_into(R, S, ws, pairs, count, 0.5, sync=True)
    assert cnt == len(want)
    got = oracle.sort_pairs(pairs[: 2 * cnt].cpu().numpy().view(np.uint32))
    assert np.array_equal(got, want)


def _pair_keys(p):
    p = np.asarray(p, dtype=np.uint32).reshape(-1, 2)
    return (p[:, 0].astype(np.uint64) << np.uint64(32)) | p[:, 1].astype(np.uint64)


def test_fused_pass_capacity_and_split_probe(cuda):
    """The fused signature-and-probe pass (from 2^19 S keys) when the pair
    buffer is too small, through as_join and through as_join_build +
    as_join_probe: the exact count with AS_ERR_CAPACITY below it, canary words
    after the buffer untouched, every pair written distinct and one of the
    oracle's (all of them at the exact capacity), and the S signatures that
    as_join_probe returns equal to the oracle's."""
    ag = cuda
    CANARY = 0x5A5A5A5A
    wl = workloads.generate(workloads.CONFIGS["plain"].scaled(20_000, (1 << 19) + 100))
    R, S = dev(ag, wl.R), dev(ag, wl.S)
    want = oracle.join_grace(wl.R, wl.S, nthreads=8)
    exact = len(want)
    assert exact == wl.expected_pairs()
    wantk = _pair_keys(want)
    count = torch.zeros(1, dtype=torch.int64, device="cuda")

    def check_buffer(buf, cap, st, cnt):
        assert cnt == exact and st == (ag.AS_OK if cap >= exact else ag.AS_ERR_CAPACITY), cap
        assert bool((buf[2 * cap:] == CANARY).all()), cap
        got = _pair_keys(buf[: 2 * min(cap, exact)].cpu().numpy().view(np.uint32))
        assert np.unique(got).size == got.size and np.isin(got, wantk).all(), cap
        if cap >= exact:
            assert np.array_equal(np.sort(got), np.sort(wantk))

    ws = ag.alloc_ws(ag.join_ws_bytes(R.n, S.n, 0.5))
    for cap in (0, 1, 4099, exact - 1, exact):
        buf = torch.full((2 * cap + 64,), CANARY, dtype=torch.int32, device="cuda")
        st, cnt = ag.join_into(R, S, ws, buf[: 2 * cap], count, 0.5, sync=True, allow_capacity=True)
        check_buffer(buf, cap, st, cnt)

    tws = ag.alloc_ws(ag.join_table_bytes(R.n, 0.5))
    t = ag.join_build(R, tws, 0.5)
    sigS = torch.zeros(S.n, dtype=torch.int64, device="cuda")
    for cap in (4099, exact):
        buf = torch.full((2 * cap + 64,), CANARY, dtype=torch.int32, device="cuda")
        try:
            st, cnt = ag.AS_OK, ag.join_probe(t, S, buf[: 2 * cap], count, sigS_out=sigS)
        except ag.AlgsigError as e:
            st, cnt = e.status, int(count.item())
        check_buffer(buf, cap, st, cnt)
    assert np.array_equal(sigS.cpu().numpy().view(np.uint64), oracle.sig_batch(wl.S.arena, wl.S.off, nthreads=8))
    buf = torch.full((2 * exact + 64,), CANARY, dtype=torch.int32, device="cuda")   # S's signatures in a workspace
    cnt = ag.join_probe(t, S, buf[: 2 * exact], count, ws=ag.alloc_ws(ag.join_probe_ws_bytes(S.n)))
    check_buffer(buf, exact, ag.AS_OK, cnt)


def test_fused_pass_rejects_signature_collisions(cuda):
    """The fused signature-and-probe pass (from 2^19 S keys) with keys that
    share all four signature components with an R key but differ from it in
    five symbols (in the first 16 bytes, at both ends, on both sides of 512-
    and 1024-byte comparison steps; 10 bytes to 4 KB, odd lengths too, every
    start alignment), among ordinary candidates of similar length in the same
    groups: every one is rejected, exact copies join, and the pairs equal the
    oracle's."""
    from packing import interleave_gaps
    ag = cuda
    rng = random.Random(77)
    wl = workloads.generate(workloads.CONFIGS["plain"].scaled(20_000, (1 << 19) + 100))
    shapes = [(5, (0, 1, 2, 3, 4)), (40, (0, 7, 8, 30, 39)), (64, (0, 63, 8, 9, 10)), (100, (1, 50, 64, 65, 99)),
              (128, (0, 63, 64, 127, 100)), (300, (0, 255, 256, 299, 128)), (520, (0, 255, 256, 511, 519)),
              (2048, (0, 511, 512, 1500, 2047))]
    rkeys, skeys = [], []
    for _ in range(6):
        for n_sym, pos in shapes:
            a, b = five_symbol_collision(n_sym, pos, seed=rng.randrange(1 << 30))
            rkeys.append(a)
            skeys += [b, a]
            if max(pos) < n_sym - 1:                  # odd length: drop the last (equal) byte of both
                rkeys.append(a[:-1])
                skeys += [b[:-1], a[:-1]]
    r_list = [wl.R.key(i) for i in range(wl.R.n)] + interleave_gaps(rkeys, seed=rng.randrange(1 << 30))
    s_list = [wl.S.key(i) for i in range(wl.S.n)]
    ins = interleave_gaps(skeys, seed=rng.randrange(1 << 30))      # (gap, key) pairs at random rows
    for i in range(0, len(ins), 2):
        p = rng.randrange(len(s_list) + 1)
        s_list[p:p] = ins[i:i + 2]
    R = relation_garbage_tail(r_list, seed=5)
    S = relation_garbage_tail(s_list, seed=6)
    assert S.n >= 1 << 19
    want = oracle.join_grace(R, S, nthreads=8)
    dR, dS = dev(ag, R), dev(ag, S)
    ws = ag.alloc_ws(ag.join_ws_bytes(dR.n, dS.n, 0.5))
    pairs = torch.empty(2 * (len(want) + 4096), dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    _, cnt = ag.join_into(dR, dS, ws, pairs, count, 0.5, sync=True)
    assert cnt == len(want)
    got = oracle.sort_pairs(pairs[: 2 * cnt].cpu().numpy().view(np.uint32))
    assert np.array_equal(got, want)
