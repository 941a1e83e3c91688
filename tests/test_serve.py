"""Host logic of the serving loop (admission ledger, batch forming, Poisson
arrivals, the scheduling loop) with a fake executor: no GPU."""
import collections
import itertools

import pytest

from paper_2411_18183_gb300 import serve


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1e-4          # every look at the clock advances it a little
        return self.t


class FakeExecutor:
    """Finishes a batch a fixed number of polls after its launch; records what
    was launched and the ledger's use at each launch."""

    def __init__(self, n_slots, sizes, polls_to_finish=3, server=None):
        self.n_slots = n_slots
        self.sizes = sizes
        self.polls = polls_to_finish
        self.launched = []
        self.state = {}
        self.server = server
        self.used_at_launch = []

    def slots(self):
        return list(range(self.n_slots))

    def request_bytes(self, j):
        return self.sizes[j]

    def launch(self, slot, batch):
        assert slot not in self.state
        self.launched.append([r.pool_index for r in batch])
        self.state[slot] = [batch, 0]
        if self.server is not None:
            self.used_at_launch.append(self.server.ledger.used)

    def poll(self, slot):
        st = self.state[slot]
        st[1] += 1
        if st[1] < self.polls:
            return None
        del self.state[slot]
        return [(r, 10 * r.pool_index, None) for r in st[0]]


def test_ledger_bounds():
    L = serve.Ledger(100)
    assert L.try_admit(60)
    assert not L.try_admit(50)
    assert L.try_admit(40)
    assert L.peak == 100
    L.release(60)
    assert L.used == 40
    with pytest.raises(ValueError):
        L.try_admit(101)
    with pytest.raises(RuntimeError):
        L.release(41)


def test_poisson_arrivals_deterministic_and_rate():
    a = serve.poisson_arrivals(rate=2000.0, duration=2.0, pool_size=7, seed=5)
    b = serve.poisson_arrivals(rate=2000.0, duration=2.0, pool_size=7, seed=5)
    assert a == b
    assert all(0 <= p < 7 for _, p in a)
    assert all(t1 < t2 for (t1, _), (t2, _) in zip(a, a[1:]))
    assert 3600 < len(a) < 4400          # mean 4000, sd 63
    gaps = [t2 - t1 for (t1, _), (t2, _) in zip(a, a[1:])]
    mean = sum(gaps) / len(gaps)
    assert abs(mean - 1 / 2000.0) < 0.05 / 2000.0


def test_form_batch_distinct_sorted_and_order_kept():
    Req = serve.Request
    q = collections.deque(Req(i, p, 0.0) for i, p in enumerate([5, 3, 5, 1, 3, 9, 2]))
    b = serve.form_batch(q, max_joins=4)
    assert [r.pool_index for r in b] == [1, 3, 5, 9]
    assert [r.rid for r in q] == [2, 4, 6]          # deferred duplicates keep arrival order
    b2 = serve.form_batch(q, max_joins=8)
    assert [r.pool_index for r in b2] == [2, 3, 5]
    assert not q


@pytest.mark.parametrize("n_slots,max_batch", [(1, 4), (2, 8), (3, 64)])
def test_server_completes_all_within_budget(n_slots, max_batch):
    sizes = [10 + 7 * (j % 5) for j in range(12)]
    arrivals = serve.poisson_arrivals(rate=50000.0, duration=0.02, pool_size=12, seed=1)
    budget = 120
    ex = FakeExecutor(n_slots, sizes)
    srv = serve.Server(ex, budget_bytes=budget, max_batch=max_batch, clock=FakeClock(), idle_sleep=0)
    ex.server = srv
    reqs = srv.run(arrivals, timeout=1e6)
    assert len(reqs) == len(arrivals)
    assert all(r.done is not None and r.count == 10 * r.pool_index for r in reqs)
    assert all(r.arrival <= r.admitted <= r.launched <= r.done for r in reqs)
    assert srv.ledger.peak <= budget and srv.ledger.used == 0
    assert max(ex.used_at_launch) <= budget
    for b in ex.launched:
        assert b == sorted(b) and len(set(b)) == len(b) and len(b) <= max_batch
    assert srv.batches == len(ex.launched)
    # admission is in arrival order
    adm = sorted(reqs, key=lambda r: (r.admitted, r.rid))
    assert [r.rid for r in adm] == sorted(r.rid for r in reqs)
    s = serve.summarize(reqs)
    assert s["completed"] == len(reqs) and s["p50_ms"] <= s["p99_ms"]


def test_server_rejects_request_larger_than_budget():
    ex = FakeExecutor(1, [500])
    srv = serve.Server(ex, budget_bytes=100, clock=FakeClock(), idle_sleep=0)
    with pytest.raises(ValueError):
        srv.run([(0.0, 0)], timeout=1e6)


def test_server_overlaps_batches_on_slots():
    sizes = [1] * 8
    arrivals = [(1e-6 * i, i % 8) for i in range(64)]
    ex = FakeExecutor(2, sizes, polls_to_finish=50)
    srv = serve.Server(ex, budget_bytes=10 ** 6, max_batch=8, clock=FakeClock(), idle_sleep=0)
    reqs = srv.run(arrivals, timeout=1e6)
    assert all(r.done is not None for r in reqs)
    # with two slots, some request launched while another batch was still running
    spans = sorted((r.launched, r.done) for r in reqs)
    assert any(a2 < d1 and a2 > a1 for (a1, d1), (a2, _) in itertools.combinations(spans, 2))
