"""Serving loop: join requests arrive over time, are admitted while a
device-memory budget allows, and are batched continuously onto several CUDA
streams.

Requests ask for joins from a pool whose relations are resident in device
memory (packed like a batch: one R and one S relation, each join a range of
rows).  Every scheduling tick the loop
  1. moves arrived requests to the waiting queue,
  2. admits waiting requests in arrival order while the memory ledger has room
     (a request holds its inputs, its share of the batch workspace and its
     output capacity until it completes),
  3. collects finished batches (CUDA events) and releases their memory,
  4. launches the admitted requests as one batch (as_join_batch_run) on a
     free stream slot, while earlier batches are still running on the others.
So requests that arrive while others are on the GPU join the next batch as
soon as a slot and memory are free, and their work overlaps on the device.

The scheduling logic (Ledger, form_batch, Server) is plain Python and runs
with any executor; GpuExecutor is the one that drives the library.
"""
from __future__ import annotations

import collections
import dataclasses
import gc
import math
import random
import time

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    pool_index: int
    arrival: float                  # seconds since the start
    nbytes: int = 0                 # device memory held while admitted
    admitted: float | None = None
    launched: float | None = None
    done: float | None = None
    count: int | None = None        # pairs found
    pairs: object = None            # (cnt, 2) uint32 pairs when results are kept
    status: str = "pending"         # done, cancelled (before launch) or timeout (never admitted in time)

    @property
    def latency(self) -> float | None:
        return None if self.done is None else self.done - self.arrival


class Ledger:
    """Admission accounting: admitted bytes never exceed the budget.
    refuse_next(k) makes the next k admissions fail as if the device memory
    were taken (a host-side injection of an allocation failure): the requests
    wait and are admitted later."""

    def __init__(self, budget: int):
        self.budget = int(budget)
        self.used = 0
        self.peak = 0
        self.refusals = 0
        self.refused = 0

    def refuse_next(self, k: int = 1) -> None:
        self.refusals += int(k)

    def try_admit(self, nbytes: int) -> bool:
        if nbytes > self.budget:
            raise ValueError(f"request of {nbytes} bytes can never fit a budget of {self.budget}")
        if self.refusals > 0:
            self.refusals -= 1
            self.refused += 1
            return False
        if self.used + nbytes > self.budget:
            return False
        self.used += nbytes
        self.peak = max(self.peak, self.used)
        return True

    def release(self, nbytes: int) -> None:
        self.used -= nbytes
        if self.used < 0:
            raise RuntimeError("ledger released more than it admitted")


def poisson_arrivals(rate: float, duration: float, pool_size: int, seed: int = 0):
    """(time, pool_index) pairs of a Poisson process of `rate` requests per second."""
    rng = random.Random(seed)
    t, out = 0.0, []
    while True:
        t += rng.expovariate(rate)
        if t >= duration:
            return out
        out.append((t, rng.randrange(pool_size)))


def form_batch(queue: collections.deque, max_joins: int):
    """Take up to max_joins admitted requests (arrival order) with distinct pool
    entries; the batch is ordered by pool entry, as the batch API requires."""
    taken, seen, keep = [], set(), collections.deque()
    while queue and len(taken) < max_joins:
        r = queue.popleft()
        if r.pool_index in seen:
            keep.append(r)
        else:
            seen.add(r.pool_index)
            taken.append(r)
    while keep:
        queue.appendleft(keep.pop())
    taken.sort(key=lambda r: r.pool_index)
    return taken


class Server:
    """The scheduling loop.  `executor` provides slots(), launch(slot, batch),
    poll(slot) -> list of (request, count, pairs) or None, and
    request_bytes(pool_index)."""

    def __init__(self, executor, budget_bytes: int, max_batch: int = 64, clock=time.perf_counter,
                 idle_sleep: float = 20e-6, admit_timeout: float | None = None):
        self.ex = executor
        self.ledger = Ledger(budget_bytes)
        self.max_batch = max_batch
        self.clock = clock
        self.idle_sleep = idle_sleep
        self.admit_timeout = admit_timeout      # seconds a request may wait for admission
        self.batches = 0

    def run(self, arrivals, timeout: float = 600.0, cancels=()):
        """Serve the (time, pool_index) arrivals.  cancels: (time, request id)
        pairs; a request cancelled before its batch is launched is dropped (its
        admitted bytes are released), one already launched completes."""
        # A collection of the cyclic garbage collector can pause the loop for tens
        # of milliseconds while requests keep arriving; collect once up front and
        # keep it off while requests are in flight.
        gc.collect()
        was_enabled = gc.isenabled()
        gc.disable()
        try:
            return self._run(arrivals, timeout, cancels)
        finally:
            if was_enabled:
                gc.enable()

    def _run(self, arrivals, timeout: float, cancels):
        reqs = [Request(i, p, t, self.ex.request_bytes(p)) for i, (t, p) in enumerate(sorted(arrivals))]
        pending = collections.deque(reqs)
        waiting, admitted = collections.deque(), collections.deque()
        cancel_q = collections.deque(sorted(cancels))
        busy = {}                                        # slot -> batch
        free = collections.deque(self.ex.slots())
        t0 = self.clock()
        finished = 0
        while finished < len(reqs):
            now = self.clock() - t0
            if now > timeout:
                raise TimeoutError(f"serving did not finish in {timeout} s ({finished}/{len(reqs)} done)")
            progressed = False
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            while cancel_q and cancel_q[0][0] <= now:     # cancellations due: drop requests not yet launched
                _, rid = cancel_q.popleft()
                r = reqs[rid]
                if r.status != "pending" or r.launched is not None:
                    continue
                if r in waiting:
                    waiting.remove(r)
                elif r in admitted:
                    admitted.remove(r)
                    self.ledger.release(r.nbytes)
                elif r in pending:
                    pending.remove(r)
                r.status, r.done = "cancelled", now
                finished += 1
                progressed = True
            if self.admit_timeout is not None:           # requests that waited too long for admission
                while waiting and now - waiting[0].arrival > self.admit_timeout:
                    r = waiting.popleft()
                    r.status, r.done = "timeout", now
                    finished += 1
                    progressed = True
            while waiting and self.ledger.try_admit(waiting[0].nbytes):
                r = waiting.popleft()
                r.admitted = now
                admitted.append(r)
                progressed = True
            for slot in list(busy):
                res = self.ex.poll(slot)
                if res is None:
                    continue
                t = self.clock() - t0
                for r, cnt, pairs in res:
                    r.done, r.count, r.pairs, r.status = t, cnt, pairs, "done"
                    self.ledger.release(r.nbytes)
                    finished += 1
                del busy[slot]
                free.append(slot)
                progressed = True
            while free and admitted:
                batch = form_batch(admitted, self.max_batch)
                if not batch:
                    break
                slot = free.popleft()
                t = self.clock() - t0
                for r in batch:
                    r.launched = t
                self.ex.launch(slot, batch)
                busy[slot] = batch
                self.batches += 1
                progressed = True
            if not progressed:
                if pending and not waiting and not admitted and not busy:
                    # nothing in the system: sleep until the next arrival
                    time.sleep(max(0.0, min(pending[0].arrival - (self.clock() - t0), 1e-3)))
                elif self.idle_sleep:
                    time.sleep(self.idle_sleep)
        return reqs


def summarize(reqs, wall: float | None = None) -> dict:
    served = [r for r in reqs if r.status == "done"]
    lat = np.array([r.latency for r in served if r.latency is not None])
    done = served
    span = wall if wall is not None else (max(r.done for r in done) - min(r.arrival for r in reqs)) if done else 0.0
    out = {
        "requests": len(reqs),
        "completed": len(done),
        "cancelled": sum(1 for r in reqs if r.status == "cancelled"),
        "timed_out": sum(1 for r in reqs if r.status == "timeout"),
        "p50_ms": float(np.percentile(lat, 50) * 1e3) if len(lat) else None,
        "p99_ms": float(np.percentile(lat, 99) * 1e3) if len(lat) else None,
        "max_ms": float(lat.max() * 1e3) if len(lat) else None,
        "mean_ms": float(lat.mean() * 1e3) if len(lat) else None,
        "span_s": span,
        "requests_per_s": len(done) / span if span > 0 else None,
    }
    if served:
        # where the slowest request spent its time, and the longest pause between launches
        w = max(served, key=lambda r: r.latency)
        out["slowest"] = {"at_s": w.arrival, "latency_ms": w.latency * 1e3,
                          "admission_wait_ms": (w.admitted - w.arrival) * 1e3,
                          "launch_wait_ms": (w.launched - w.admitted) * 1e3,
                          "run_ms": (w.done - w.launched) * 1e3}
        ls = sorted(r.launched for r in served)
        if len(ls) > 1:
            g = np.diff(ls)
            i = int(np.argmax(g))
            out["longest_launch_gap_ms"] = float(g[i] * 1e3)
            out["longest_launch_gap_at_s"] = float(ls[i])
    return out


class GpuExecutor:
    """Runs batches of pooled joins with the library, one workspace, pair buffer
    and stream per slot."""

    def __init__(self, pool, n_slots: int = 2, max_batch: int = 64, load_factor: float = 0.5,
                 keep_pairs: bool = False):
        import torch
        from . import alloc_ws, join_batch_ws_bytes, make_descs
        self.torch = torch
        self.pool = pool
        self.lf = load_factor
        self.keep = keep_pairs
        self.max_batch = max_batch
        # worst case per slot: the max_batch largest requests
        order = sorted(range(pool.n), key=lambda j: pool.ws_need[j], reverse=True)[:max_batch]
        order.sort()
        top = make_descs([pool.ranges[j] for j in order], [pool.pair_cap[j] for j in order])
        # a batch's workspace (tables and signatures of its joins' rows) is at most that of the
        # max_batch joins that need the most
        ws_bytes = join_batch_ws_bytes(top, pool.R.n, pool.S.n, load_factor) + 256 * max_batch
        pair_cap = sum(pool.pair_cap[j] for j in order)
        self.slots_ = []
        for _ in range(n_slots):
            self.slots_.append({
                "stream": torch.cuda.Stream(),
                "ws": alloc_ws(ws_bytes),
                "pairs": torch.empty(2 * max(1, pair_cap), dtype=torch.int32, device="cuda"),
                "counts": torch.zeros(max_batch, dtype=torch.int64, device="cuda"),
                "counts_host": torch.zeros(max_batch, dtype=torch.int64).pin_memory(),
                "event": None, "batch": None, "descs": None,
            })

    def slots(self):
        return list(range(len(self.slots_)))

    def request_bytes(self, j: int) -> int:
        return int(self.pool.req_bytes[j])

    def launch(self, slot: int, batch) -> None:
        from . import join_batch_prepare, join_batch_run, make_descs
        torch = self.torch
        s = self.slots_[slot]
        descs = make_descs([self.pool.ranges[r.pool_index] for r in batch],
                           [self.pool.pair_cap[r.pool_index] for r in batch])
        with torch.cuda.stream(s["stream"]):
            b = join_batch_prepare(descs, self.pool.R, self.pool.S, s["ws"], self.lf, stream=s["stream"])
            join_batch_run(b, self.pool.R, self.pool.S, s["pairs"], s["counts"], stream=s["stream"])
            s["counts_host"][: len(batch)].copy_(s["counts"][: len(batch)], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(s["stream"])
        s["event"], s["batch"], s["descs"] = ev, batch, descs

    def poll(self, slot: int):
        s = self.slots_[slot]
        if not s["event"].query():
            return None
        counts = s["counts_host"][: len(s["batch"])].tolist()
        out = []
        for r, d, c in zip(s["batch"], s["descs"], counts):
            pairs = None
            if self.keep:
                pairs = s["pairs"][2 * d.pair_offset: 2 * (d.pair_offset + min(c, d.pair_cap))].view(-1, 2).cpu()
            out.append((r, c, pairs))
        s["event"] = s["batch"] = s["descs"] = None
        return out


@dataclasses.dataclass
class DevicePool:
    """Joins resident in device memory: one packed R, one packed S, row ranges."""
    R: object
    S: object
    ranges: list
    pair_cap: list
    req_bytes: list
    ws_need: list
    expected: list

    @property
    def n(self) -> int:
        return len(self.ranges)

    @staticmethod
    def from_batch(bw, device_relation, load_factor: float = 0.5) -> "DevicePool":
        """A pool over a host batch (workloads.generate_batch), copied to the device."""
        R = device_relation(bw.R)
        S = device_relation(bw.S)
        key_bytes = [int(bw.R.off[r1] - bw.R.off[r0]) + int(bw.S.off[s1] - bw.S.off[s0])
                     for (r0, r1, s0, s1) in bw.ranges]
        return DevicePool._sized(R, S, list(bw.ranges), key_bytes, list(bw.expected), load_factor)

    @staticmethod
    def from_device(R, S, ranges, expected, load_factor: float = 0.5) -> "DevicePool":
        """A pool over relations already in device memory (for example a batch
        the device generator wrote); ranges: (r_begin, r_end, s_begin, s_end)."""
        import torch
        ranges = list(ranges)
        ir = torch.tensor([x for (r0, r1, _, _) in ranges for x in (r0, r1)], dtype=torch.int64, device=R.off.device)
        is_ = torch.tensor([x for (_, _, s0, s1) in ranges for x in (s0, s1)], dtype=torch.int64, device=S.off.device)
        br = R.off[ir].view(-1, 2).diff(dim=1).view(-1).cpu().tolist()
        bs = S.off[is_].view(-1, 2).diff(dim=1).view(-1).cpu().tolist()
        return DevicePool._sized(R, S, ranges, [a + b for a, b in zip(br, bs)], list(expected), load_factor)

    @staticmethod
    def _sized(R, S, ranges, key_bytes, expected, load_factor) -> "DevicePool":
        """Per join: pair capacity, workspace need and the bytes a request holds
        while admitted (its inputs with offsets and ids, workspace, pairs)."""
        caps, rb, need = [], [], []
        for (r0, r1, s0, s1), kb, e in zip(ranges, key_bytes, expected):
            m, n = r1 - r0, s1 - s0
            cap = max(64, int(e * 1.25) + 64)
            cap_slots = 1 << max(6, math.ceil(math.log2(max(1, m) / load_factor)))
            inputs = kb + 8 * (m + n) + 4 * (m + n)
            ws = 16 * cap_slots + 8 * (m + n) + 64
            caps.append(cap)
            need.append(ws)
            rb.append(inputs + ws + 8 * cap)
        return DevicePool(R, S, ranges, caps, rb, need, expected)
