"""Parity at full size, in the bench's configuration: the large (1M x 10M) and
collision (100k x 1M) workloads.  Every R and S signature equals the oracle's
(all host cores), and the whole join, at each load factor the bench's tuning
picks from, equals the oracle's Grace hash join element by element (sorted
(r_id, s_id) lists) and the generator's ground-truth count."""
import os

import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["large", "collision"])
def test_full_size_parity(cuda, name):
    ag = cuda
    threads = max(1, os.cpu_count() or 1)
    wl = workloads.generate(workloads.CONFIGS[name])
    R = ag.DeviceRelation.from_host(wl.R.arena, wl.R.off, wl.R.ids)
    S = ag.DeviceRelation.from_host(wl.S.arena, wl.S.off, wl.S.ids)

    # every signature of both relations
    for dev, host in ((R, wl.R), (S, wl.S)):
        got = ag.sig_compute(dev).cpu().numpy().view(np.uint64)
        want = oracle.sig_batch(host.arena, host.off, nthreads=threads)
        bad = np.nonzero(got != want)[0]
        assert bad.size == 0, f"{bad.size} signature mismatches, first rows {bad[:5].tolist()}"

    # the whole join against the oracle's Grace join
    want = oracle.join_grace(wl.R, wl.S, nthreads=threads)
    assert len(want) == wl.expected_pairs()
    cap = len(want) + 4096
    pairs = torch.empty(2 * cap, dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    for lf in (0.5, 0.35, 0.25):
        ws = ag.alloc_ws(ag.join_ws_bytes(R.n, S.n, lf))
        _, cnt = ag.join_into(R, S, ws, pairs, count, lf, sync=True)
        assert cnt == len(want), lf
        got = oracle.sort_pairs(pairs[: 2 * cnt].cpu().numpy().view(np.uint32))
        assert np.array_equal(got, want), lf
        del ws
