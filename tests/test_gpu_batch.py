"""Batches of joins (as_join_batch_prepare / as_join_batch_run through the C
ABI): every join's sorted pairs equal the oracle's on that join's rows, equal
the same join run alone, and a CUDA-graph replay gives the same result."""
import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu


def dev(ag, rel):
    return ag.DeviceRelation.from_host(rel.arena, rel.off, rel.ids)


@pytest.fixture(scope="module")
def batch():
    spec = workloads.BatchSpec().scaled(400, n_joins=24)
    return workloads.generate_batch(spec)


def test_batch_matches_oracle_and_solo(cuda, batch):
    ag = cuda
    Rd, Sd = dev(ag, batch.R), dev(ag, batch.S)
    R = ag.DeviceRelation(Rd.arena, Rd.off, None)     # no ids: join-local row numbers
    S = ag.DeviceRelation(Sd.arena, Sd.off, None)
    caps = [max(64, 2 * e + 64) for e in batch.expected]
    out = ag.join_batch(R, S, batch.ranges, caps, load_factor=0.5)
    for j in range(len(batch.ranges)):
        Rj, Sj = batch.join_relations(j)
        want = oracle.join_simple(Rj, Sj)
        got = oracle.sort_pairs(out[j].cpu().numpy().view(np.uint32))
        assert np.array_equal(got, want), j
        assert len(want) == batch.expected[j]
        solo = oracle.sort_pairs(ag.join(dev(ag, Rj), dev(ag, Sj)).cpu().numpy().view(np.uint32))
        assert np.array_equal(solo, got), j


def test_batch_graph_replay_and_ids(cuda, batch):
    ag = cuda
    R = dev(ag, batch.R)            # ids = global rows, so pairs carry global ids
    S = dev(ag, batch.S)
    caps = [max(64, 2 * e + 64) for e in batch.expected]
    descs = ag.make_descs(batch.ranges, caps)
    ws = ag.alloc_ws(ag.join_batch_ws_bytes(descs, R.n, S.n, 0.7))
    b = ag.join_batch_prepare(descs, R, S, ws, 0.7)
    pairs = torch.zeros(2 * ag.total_pair_cap(descs), dtype=torch.int32, device="cuda")
    counts = torch.zeros(len(descs), dtype=torch.int64, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ag.join_batch_run(b, R, S, pairs, counts)        # warm-up outside capture
    torch.cuda.synchronize()
    first = [oracle.sort_pairs(pairs[2 * d.pair_offset: 2 * (d.pair_offset + c)].cpu().numpy().view(np.uint32))
             for d, c in zip(descs, counts.cpu().tolist())]
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ag.join_batch_run(b, R, S, pairs, counts)
    for _ in range(2):
        pairs.zero_()
        g.replay()
        torch.cuda.synchronize()
        again = [oracle.sort_pairs(pairs[2 * d.pair_offset: 2 * (d.pair_offset + c)].cpu().numpy().view(np.uint32))
                 for d, c in zip(descs, counts.cpu().tolist())]
        for a_, b_ in zip(first, again):
            assert np.array_equal(a_, b_)
    for j, (rb, re_, sb, se) in enumerate(batch.ranges):
        Rj, Sj = batch.join_relations(j)
        want = oracle.join_simple(Rj, Sj).astype(np.int64)
        want[:, 0] += rb
        want[:, 1] += sb
        assert np.array_equal(first[j].astype(np.int64), want)


def test_batch_subset_of_pool(cuda, batch):
    """A batch that picks a few joins out of the resident pool (gaps between
    them, one join with no R rows, one with no S rows) reads only those rows."""
    ag = cuda
    Rd, Sd = dev(ag, batch.R), dev(ag, batch.S)
    R = ag.DeviceRelation(Rd.arena, Rd.off, None)
    S = ag.DeviceRelation(Sd.arena, Sd.off, None)
    pick = [1, 4, 5, 11, 17, 23]
    ranges = [batch.ranges[j] for j in pick]
    r0, r1, s0, s1 = ranges[2]
    ranges[2] = (r0, r0, s0, s1)                      # empty R side
    r0, r1, s0, s1 = ranges[4]
    ranges[4] = (r0, r1, s0, s0)                      # empty S side
    caps = [max(64, 2 * batch.expected[j] + 64) for j in pick]
    out = ag.join_batch(R, S, ranges, caps, load_factor=0.5)
    for k, (rb, re_, sb, se) in enumerate(ranges):
        Rj = workloads.relation_from_keys([batch.R.key(i) for i in range(rb, re_)])
        Sj = workloads.relation_from_keys([batch.S.key(i) for i in range(sb, se)])
        want = oracle.join_simple(Rj, Sj)
        got = oracle.sort_pairs(out[k].cpu().numpy().view(np.uint32))
        assert np.array_equal(got, want), k


def test_batch_contiguous_run_and_gapped_run(cuda, batch):
    """Joins whose rows form one run of the relations (starting mid-pool) take the
    signature kernel over that run; the same joins with one left out (a gap in
    the rows) take it over the joins' row ranges; with a gap in S's rows only,
    R takes the run and S the row ranges.  Every join gets the oracle's pairs."""
    ag = cuda
    Rd, Sd = dev(ag, batch.R), dev(ag, batch.S)
    R = ag.DeviceRelation(Rd.arena, Rd.off, None)
    S = ag.DeviceRelation(Sd.arena, Sd.off, None)
    run = list(range(3, 10))
    mixed = [batch.ranges[j] for j in run]
    r0, r1, s0, s1 = mixed[3]
    mixed[3] = (r0, r1, min(s0 + 5, s1), s1)          # R rows still one run, S rows with a gap
    cases = (([batch.ranges[j] for j in run], "both"), ([batch.ranges[j] for j in run[:3] + run[4:]], "neither"),
             (mixed, "R only"))
    for ranges, kind in cases:
        caps = [max(64, 2 * len(oracle.join_simple(
            workloads.relation_from_keys([batch.R.key(i) for i in range(rb, re_)]),
            workloads.relation_from_keys([batch.S.key(i) for i in range(sb, se)]))) + 64)
            for rb, re_, sb, se in ranges]
        descs = ag.make_descs(ranges, caps)
        ws = ag.alloc_ws(ag.join_batch_ws_bytes(descs, R.n, S.n, 0.5))
        b = ag.join_batch_prepare(descs, R, S, ws, 0.5)
        want_r = ranges[0][0] if kind in ("both", "R only") else ag.ROWS_SCATTERED
        want_s = ranges[0][2] if kind == "both" else ag.ROWS_SCATTERED
        assert (b.r_first, b.s_first) == (want_r, want_s), kind
        out = ag.join_batch(R, S, ranges, caps, load_factor=0.5)
        for k, (rb, re_, sb, se) in enumerate(ranges):
            Rj = workloads.relation_from_keys([batch.R.key(i) for i in range(rb, re_)])
            Sj = workloads.relation_from_keys([batch.S.key(i) for i in range(sb, se)])
            want = oracle.join_simple(Rj, Sj)
            got = oracle.sort_pairs(out[k].cpu().numpy().view(np.uint32))
            assert np.array_equal(got, want), (kind, k)


def test_batch_single_join_equals_join(cuda, batch):
    ag = cuda
    Rd, Sd = dev(ag, batch.R), dev(ag, batch.S)
    R = ag.DeviceRelation(Rd.arena, Rd.off, None)
    S = ag.DeviceRelation(Sd.arena, Sd.off, None)
    solo = oracle.sort_pairs(ag.join(R, S).cpu().numpy().view(np.uint32))
    got = ag.join_batch(R, S, [(0, R.n, 0, S.n)], [len(solo) + 64])[0]
    assert np.array_equal(oracle.sort_pairs(got.cpu().numpy().view(np.uint32)), solo)


def test_autotuned_graph_batch(cuda, batch):
    from paper_2411_18183_gb300 import tune
    ag = cuda
    Rd, Sd = dev(ag, batch.R), dev(ag, batch.S)
    R = ag.DeviceRelation(Rd.arena, Rd.off, None)
    S = ag.DeviceRelation(Sd.arena, Sd.off, None)
    caps = [max(64, 2 * e + 64) for e in batch.expected]
    gb, times, shape_times = tune.autotune(R, S, batch.ranges, caps, candidates=(0.4, 0.8), reps=1)
    assert set(times) == {0.4, 0.8} and gb.lf in times and gb.graph is not None
    # the batch's rows are one run per side, so the signature kernel's shapes were timed too
    assert set(shape_times) == set(range(len(ag.sig_shapes()))) and gb.shape in shape_times
    gb.counts.zero_()
    gb.replay()
    torch.cuda.synchronize()
    assert gb.counts.cpu().tolist() == list(batch.expected)
    for j in (0, len(batch.ranges) // 2, len(batch.ranges) - 1):
        Rj, Sj = batch.join_relations(j)
        got = oracle.sort_pairs(gb.result(j).cpu().numpy().view(np.uint32))
        assert np.array_equal(got, oracle.join_simple(Rj, Sj))


@pytest.mark.parametrize("shape", [1, 2])
def test_batch_at_every_signature_shape(cuda, batch, shape):
    """A batch run with each non-default signature kernel shape gives the
    generator's per-join counts and the oracle's pairs."""
    from paper_2411_18183_gb300 import tune
    ag = cuda
    assert shape < len(ag.sig_shapes())
    Rd, Sd = dev(ag, batch.R), dev(ag, batch.S)
    R = ag.DeviceRelation(Rd.arena, Rd.off, None)
    S = ag.DeviceRelation(Sd.arena, Sd.off, None)
    caps = [max(64, 2 * e + 64) for e in batch.expected]
    gb = tune.GraphBatch(R, S, batch.ranges, caps, 0.5, shape)
    assert gb.shape_matters()
    gb.run()
    torch.cuda.synchronize()
    assert gb.counts.cpu().tolist() == list(batch.expected)
    j = len(batch.ranges) // 3
    Rj, Sj = batch.join_relations(j)
    assert np.array_equal(oracle.sort_pairs(gb.result(j).cpu().numpy().view(np.uint32)), oracle.join_simple(Rj, Sj))


def test_autotune_cache_skips_timing_for_a_known_shape(cuda, batch, tmp_path):
    """With a TuneCache the first autotune times the candidates and records the
    winner under the batch's shape; the second takes it without timing, and
    its graph gives the same counts."""
    from paper_2411_18183_gb300 import tune
    ag = cuda
    Rd, Sd = dev(ag, batch.R), dev(ag, batch.S)
    R = ag.DeviceRelation(Rd.arena, Rd.off, None)
    S = ag.DeviceRelation(Sd.arena, Sd.off, None)
    caps = [max(64, 2 * e + 64) for e in batch.expected]
    cache = tune.TuneCache(str(tmp_path / "tune.json"))
    gb1, t1, _ = tune.autotune(R, S, batch.ranges, caps, candidates=(0.4, 0.8), reps=1, cache=cache)
    gb2, t2, s2 = tune.autotune(R, S, batch.ranges, caps, candidates=(0.4, 0.8), reps=1, cache=cache)
    assert set(t1) == {0.4, 0.8} and t2 == {} and s2 == {} and (gb2.lf, gb2.shape) == (gb1.lf, gb1.shape)
    assert (tune.TuneCache(str(tmp_path / "tune.json")).get(tune.batch_shape_key(R, S, batch.ranges))
            == (gb1.lf, gb1.shape))
    gb2.counts.zero_()
    gb2.replay()
    torch.cuda.synchronize()
    assert gb2.counts.cpu().tolist() == list(batch.expected)


@pytest.mark.parametrize("shape", [0, 2])
def test_gapped_batch_signatures_at_scale(cuda, shape):
    """A batch whose joins' rows have gaps, with more than 2^19 S rows (so the
    signature kernel splits the joins' rows over its warps by work) and
    runs that end inside a window: every virtual row's signature equals the
    oracle's signature of its relation row, at two kernel shapes."""
    ag = cuda
    wl = workloads.generate(workloads.CONFIGS["large"].scaled(60_000, 1_200_000))
    R = ag.DeviceRelation.from_host(wl.R.arena, wl.R.off, None)
    S = ag.DeviceRelation.from_host(wl.S.arena, wl.S.off, None)
    s_runs = [(0, 150_000), (200_000, 400_017), (400_017, 400_017), (450_003, 800_000), (800_010, 1_100_000),
              (1_150_000, 1_200_000)]
    r_runs = [(0, 9_000), (10_000, 20_000), (20_000, 20_000), (25_000, 40_001), (40_100, 55_000), (55_500, 60_000)]
    ranges = [(rb, re_, sb, se) for (rb, re_), (sb, se) in zip(r_runs, s_runs)]
    descs = ag.make_descs(ranges, [1 << 16] * len(ranges))
    ws = ag.alloc_ws(ag.join_batch_ws_bytes(descs, R.n, S.n, 0.5))
    b = ag.join_batch_prepare(descs, R, S, ws, 0.5)
    assert b.r_first == ag.ROWS_SCATTERED and b.s_first == ag.ROWS_SCATTERED and b.nS > (1 << 19)
    b.sig_shape = shape
    pairs = torch.empty(2 * (1 << 16) * len(ranges), dtype=torch.int32, device="cuda")
    counts = torch.zeros(len(ranges), dtype=torch.int64, device="cuda")
    ag.join_batch_run(b, R, S, pairs, counts)
    torch.cuda.synchronize()
    base = ws.data_ptr()
    for ptr, n, rel, runs in ((b.sigR, b.mR, wl.R, r_runs), (b.sigS, b.nS, wl.S, s_runs)):
        got = ws[ptr - base: ptr - base + 8 * n].view(torch.int64).cpu().numpy().view(np.uint64)
        want = oracle.sig_batch(rel.arena, rel.off, nthreads=8)
        want = np.concatenate([want[a:e] for a, e in runs])
        bad = np.nonzero(got != want)[0]
        assert bad.size == 0, (shape, bad.size, bad[:5].tolist())
