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


def test_cancel_before_launch_releases_memory_and_launched_requests_complete():
    """Host-side cancellation: requests cancelled while waiting or admitted
    are dropped and their admitted bytes released; a cancel that arrives after
    the request's batch was launched does not stop it."""
    sizes = [40] * 6
    arrivals = [(0.0, j) for j in range(6)]
    ex = FakeExecutor(1, sizes, polls_to_finish=200)
    srv = serve.Server(ex, budget_bytes=100, max_batch=2, clock=FakeClock(), idle_sleep=0)
    ex.server = srv
    # request 0/1 launch at once (2 x 40 <= 100); 2..5 wait on the budget or the one slot
    reqs = srv.run(arrivals, timeout=1e6, cancels=[(0.001, 3), (0.001, 4), (0.001, 0)])
    st = {r.rid: r.status for r in reqs}
    assert st[3] == st[4] == "cancelled"
    assert st[0] == "done" and st[1] == "done" and st[2] == "done" and st[5] == "done"
    assert all(r.count == 10 * r.pool_index for r in reqs if r.status == "done")
    launched = [p for b in ex.launched for p in b]
    assert 3 not in launched and 4 not in launched
    assert srv.ledger.used == 0
    s = serve.summarize(reqs)
    assert s["cancelled"] == 2 and s["completed"] == 4


def test_admission_timeout_drops_requests_that_wait_too_long():
    """A request that cannot be admitted within admit_timeout (the budget is
    held by a long batch) is dropped with status timeout; the one behind it in
    arrival order (admission is first come, first served) is admitted once
    the queue head is gone, and completes."""
    sizes = [90, 90, 5]
    arrivals = [(0.0, 0), (0.0, 1), (0.005, 2)]
    ex = FakeExecutor(2, sizes, polls_to_finish=400)
    srv = serve.Server(ex, budget_bytes=100, max_batch=1, clock=FakeClock(), idle_sleep=0, admit_timeout=0.01)
    reqs = srv.run(arrivals, timeout=1e6)
    st = {r.rid: r.status for r in reqs}
    assert st[0] == "done" and st[1] == "timeout" and st[2] == "done"
    assert srv.ledger.used == 0
    assert serve.summarize(reqs)["timed_out"] == 1


def test_injected_admission_failures_delay_but_do_not_lose_requests():
    """Allocation failures injected into the ledger (the next k admissions
    refused) leave the requests waiting; every one is admitted later, within
    the budget, and completes with its result."""
    sizes = [10 + j for j in range(10)]
    arrivals = [(1e-5 * j, j) for j in range(10)]
    ex = FakeExecutor(2, sizes)
    srv = serve.Server(ex, budget_bytes=60, max_batch=4, clock=FakeClock(), idle_sleep=0)
    srv.ledger.refuse_next(25)
    reqs = srv.run(arrivals, timeout=1e6)
    assert srv.ledger.refused == 25
    assert all(r.status == "done" and r.count == 10 * r.pool_index for r in reqs)
    assert srv.ledger.peak <= 60 and srv.ledger.used == 0


def test_tune_cache_keys_and_persistence(tmp_path):
    """The autotuner's cache: batches are keyed by device, key-length class
    and size class (floor log2 of the rows), and the table survives a reload
    from its JSON file."""
    from paper_2411_18183_gb300.tune import TuneCache
    k = TuneCache.key
    assert k("GPU", 100, 1000) == k("GPU", 128, 1023) != k("GPU", 129, 1000)
    assert k("GPU", 100, 1000) != k("GPU", 100, 1024) and k("GPU", 100, 1024) == k("GPU", 100, 2047)
    assert k("GPU", 9000, 5) != k("GPU", 8192, 5) and k("A", 1, 1) != k("B", 1, 1)
    path = str(tmp_path / "tune.json")
    c = TuneCache(path)
    assert c.get(k("GPU", 700, 10_000)) is None
    c.put(k("GPU", 700, 10_000), 0.35, 2)
    assert TuneCache(path).get(k("GPU", 700, 10_000)) == (0.35, 2)
    # a file written with bare load factors reads as shape 0
    import json
    with open(path, "w") as f:
        json.dump({k("GPU", 700, 10_000): 0.5}, f)
    assert TuneCache(path).get(k("GPU", 700, 10_000)) == (0.5, 0)
