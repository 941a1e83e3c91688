"""Parity at full size, in the bench's configuration: the large (1M x 10M) and
collision (100k x 1M) workloads.  Signatures of a seeded sample of S rows
equal the oracle's computed one by one; the join's pair count equals the
generator's ground truth; the pairs of the sampled S rows equal the oracle's
join of all of R with those rows."""
import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu

SAMPLE = 3000


@pytest.mark.parametrize("name", ["large", "collision"])
def test_full_size_sampled_parity(cuda, name):
    ag = cuda
    wl = workloads.generate(workloads.CONFIGS[name])
    R = ag.DeviceRelation.from_host(wl.R.arena, wl.R.off, wl.R.ids)
    S = ag.DeviceRelation.from_host(wl.S.arena, wl.S.off, wl.S.ids)
    rng = np.random.default_rng(20260)
    rows = np.sort(rng.choice(S.n, size=SAMPLE, replace=False))
    keys = [wl.S.key(int(i)) for i in rows]
    sample = workloads.relation_from_keys(keys, ids=wl.S.ids[rows])

    # signatures of every S row on the GPU; the sample against the oracle
    sigS = ag.sig_compute(S)
    got_sig = sigS[torch.from_numpy(rows).cuda()].cpu().numpy().view(np.uint64)
    want_sig = oracle.sig_batch(sample.arena, sample.off, nthreads=8)
    assert np.array_equal(got_sig, want_sig)

    # the whole join as bench.py runs it, at each load factor its tuning picks from
    want_sample = oracle.join_simple(wl.R, sample)
    cap = wl.expected_pairs() + 4096
    pairs = torch.empty(2 * cap, dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    for lf in (0.5, 0.35, 0.25):
        ws = ag.alloc_ws(ag.join_ws_bytes(R.n, S.n, lf))
        _, cnt = ag.join_into(R, S, ws, pairs, count, lf, sync=True)
        assert cnt == wl.expected_pairs(), lf
        got = pairs[: 2 * cnt].cpu().numpy().view(np.uint32).reshape(-1, 2)
        keep = np.isin(got[:, 1], wl.S.ids[rows])
        assert np.array_equal(oracle.sort_pairs(got[keep]), want_sample), lf
        del ws
