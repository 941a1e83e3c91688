"""The device input generator (workloads/gen_dev.cu) against the host
generator, byte for byte: the packed arenas and offsets of whole batches and
of waves of consecutive joins, for the letter alphabets and the XML-like text
of the serving workload."""
import dataclasses

import numpy as np
import pytest
import torch

import workloads
from workloads import device as gd

pytestmark = pytest.mark.gpu


def host_slice(rel, r0, r1):
    off = rel.off[r0: r1 + 1]
    return rel.arena[int(off[0]): int(off[-1])], (off - off[0]).astype(np.int64)


def check_wave(w, bw):
    (rb, _, sb, _), (_, re_, _, se) = bw.ranges[w.j0], bw.ranges[w.j1 - 1]
    for dev_arena, dev_off, rel, a, b in ((w.arenaR, w.offR, bw.R, rb, re_), (w.arenaS, w.offS, bw.S, sb, se)):
        want_bytes, want_off = host_slice(rel, a, b)
        got_off = dev_off.cpu().numpy()
        assert np.array_equal(got_off, want_off)
        got = dev_arena.cpu().numpy()
        n = want_bytes.shape[0]
        assert got.shape[0] == (n + 15) // 16 * 16 + 16
        bad = np.nonzero(got[:n] != want_bytes)[0]
        assert bad.size == 0, f"{bad.size} bytes differ, first at {bad[:5].tolist()}"
        assert not got[n:].any()
    assert w.expected == bw.expected[w.j0: w.j1]
    assert w.key_bytes == sum(int(r.off[b] - r.off[a]) for r, a, b in ((bw.R, rb, re_), (bw.S, sb, se)))


@pytest.mark.parametrize("which", ["batch", "serve"])
def test_device_generator_matches_host(cuda, which):
    spec = workloads.BatchSpec().scaled(400) if which == "batch" else \
        dataclasses.replace(workloads.SERVE_SPEC.scaled(100), n_joins=24)
    bw = workloads.generate_batch(spec)
    plan = gd.plan_batch(spec.joins())
    check_wave(gd.fill_wave(plan, 0, len(bw.ranges)), bw)
    # waves of consecutive joins under a byte cap, each against its slice of the host batch
    total = plan.key_bytes(0, len(bw.ranges))
    ws = gd.waves(plan, total // 5)
    assert len(ws) >= 5 and ws[0][0] == 0 and ws[-1][1] == len(bw.ranges)
    assert all(a < b and (b == c) for (a, b), (c, _) in zip(ws, ws[1:] + [(ws[-1][1], None)]))
    for j0, j1 in ws[:: max(1, len(ws) // 3)]:
        assert j1 - j0 == 1 or plan.key_bytes(j0, j1) <= total // 5
        check_wave(gd.fill_wave(plan, j0, j1), bw)


def test_device_generator_single_join_and_unsupported(cuda):
    sp = workloads.CONFIGS["plain"].scaled(3000, 30_000)
    wl = workloads.generate(sp)
    plan = gd.plan_batch([sp])
    w = gd.fill_wave(plan, 0, 1)
    assert np.array_equal(w.arenaR.cpu().numpy(), wl.R.arena) and np.array_equal(w.arenaS.cpu().numpy(), wl.S.arena)
    assert np.array_equal(w.offR.cpu().numpy(), wl.R.off.astype(np.int64))
    assert w.expected == [wl.expected_pairs()]
    with pytest.raises(ValueError):
        gd.plan_batch([workloads.CONFIGS["large"].scaled(100, 1000)])       # Zipf partners, duplicated R keys
    torch.cuda.synchronize()
