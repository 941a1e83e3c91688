"""Serving on the GPU: requests for pooled joins arrive as a Poisson process,
are admitted under a memory budget and batched onto two streams; the pairs
each request gets in the mix equal those of its join run alone and the
oracle's."""
import numpy as np
import pytest

import oracle
import workloads
from paper_2411_18183_gb300 import serve

pytestmark = pytest.mark.gpu


def test_serving_result_alone_equals_in_mix(cuda):
    ag = cuda
    bw = workloads.generate_batch(workloads.BatchSpec().scaled(800, n_joins=16))

    def dev(rel):
        return ag.DeviceRelation.from_host(rel.arena, rel.off, None)

    pool = serve.DevicePool.from_batch(bw, dev)
    ex = serve.GpuExecutor(pool, n_slots=2, max_batch=6, keep_pairs=True)
    budget = 3 * max(pool.req_bytes)
    arrivals = serve.poisson_arrivals(rate=4000.0, duration=0.03, pool_size=pool.n, seed=7)
    assert len(arrivals) > 40
    srv = serve.Server(ex, budget_bytes=budget, max_batch=6)
    reqs = srv.run(arrivals, timeout=120.0)
    assert srv.ledger.peak <= budget
    assert srv.batches > 1
    alone = {}
    for r in reqs:
        j = r.pool_index
        if j not in alone:
            Rj, Sj = bw.join_relations(j)
            want = oracle.join_simple(Rj, Sj)
            solo = oracle.sort_pairs(ag.join(dev(Rj), dev(Sj)).cpu().numpy().view(np.uint32))
            assert np.array_equal(solo, want), j
            alone[j] = want
        assert r.count == len(alone[j]), (r.rid, j)
        got = oracle.sort_pairs(r.pairs.numpy().view(np.uint32))
        assert np.array_equal(got, alone[j]), (r.rid, j)
    s = serve.summarize(reqs)
    assert s["completed"] == len(reqs)
