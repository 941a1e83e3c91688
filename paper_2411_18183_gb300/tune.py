"""Batch runner: picks the hash-table load factor of a batch of joins by
timing the candidates on the device, then replays the batch's launches from a
captured CUDA graph.

The tile shape and warps per key of the kernels are compile-time constants of
the library (one shape serves every key length, since the tile walk is
byte-balanced); the load factor is the knob that trades table size (and the
cache footprint of the probe) against bucket-chain length, so it is the one
tuned per batch.
"""
from __future__ import annotations

import torch

from . import (DeviceRelation, alloc_ws, join_batch_prepare, join_batch_run, join_batch_ws_bytes, make_descs,
               total_pair_cap)

LOAD_FACTORS = (0.35, 0.5, 0.7, 0.9)


class GraphBatch:
    """One prepared batch with its own workspace, output buffers and stream;
    run() launches it directly, capture() records it into a CUDA graph and
    replay() relaunches the graph."""

    def __init__(self, R: DeviceRelation, S: DeviceRelation, ranges, pair_caps, load_factor: float):
        self.R, self.S = R, S
        self.descs = make_descs(ranges, pair_caps)
        self.lf = load_factor
        self.stream = torch.cuda.Stream()
        self.ws = alloc_ws(join_batch_ws_bytes(self.descs, R.n, S.n, load_factor))
        self.pairs = torch.empty(2 * max(1, total_pair_cap(self.descs)), dtype=torch.int32, device="cuda")
        self.counts = torch.zeros(len(self.descs), dtype=torch.int64, device="cuda")
        self.batch = join_batch_prepare(self.descs, R, S, self.ws, load_factor, stream=self.stream)
        self.graph = None

    def run(self):
        join_batch_run(self.batch, self.R, self.S, self.pairs, self.counts, stream=self.stream)

    def capture(self):
        self.run()                                  # first use of every kernel outside the capture
        self.stream.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=self.stream):
            self.run()
        self.graph = g
        return self

    def replay(self):
        with torch.cuda.stream(self.stream):
            self.graph.replay()

    def time_ms(self, reps: int = 3, graph: bool = True) -> float:
        go = self.replay if (graph and self.graph is not None) else self.run
        go()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(self.stream)
        for _ in range(reps):
            go()
        e1.record(self.stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    def result(self, j: int) -> torch.Tensor:
        d = self.descs[j]
        c = int(self.counts[j].item())
        return self.pairs[2 * d.pair_offset: 2 * (d.pair_offset + min(c, d.pair_cap))].view(-1, 2)


class TuneCache:
    """Best load factors found by autotune, keyed by (GPU name, key-length
    class, size class) so that batches of the same shape skip the timing.
    Optionally persisted as JSON."""

    LENGTH_CLASSES = (128, 1024, 8192)          # upper bounds of the key-length bands, then longer

    def __init__(self, path: str | None = None):
        self.path = path
        self.table: dict[str, float] = {}
        if path:
            import json
            import os
            if os.path.exists(path):
                with open(path) as f:
                    self.table = {k: float(v) for k, v in json.load(f).items()}

    @classmethod
    def key(cls, device_name: str, mean_key_bytes: float, rows: int) -> str:
        lc = next((i for i, b in enumerate(cls.LENGTH_CLASSES) if mean_key_bytes <= b), len(cls.LENGTH_CLASSES))
        sc = max(0, int(rows).bit_length() - 1)     # floor(log2(rows))
        return f"{device_name}|len{lc}|rows2^{sc}"

    def get(self, key: str):
        return self.table.get(key)

    def put(self, key: str, load_factor: float) -> None:
        self.table[key] = float(load_factor)
        if self.path:
            import json
            with open(self.path, "w") as f:
                json.dump(self.table, f, indent=1, sort_keys=True)


def batch_shape_key(R: DeviceRelation, S: DeviceRelation, ranges) -> str:
    """TuneCache key of a batch: the device, the mean key length of its S rows
    and its total S rows."""
    ranges = list(ranges)
    rows = sum(int(se) - int(sb) for (_, _, sb, se) in ranges)
    nbytes = 0
    if rows:
        idx = torch.tensor([int(x) for (_, _, sb, se) in ranges for x in (sb, se)], dtype=torch.int64,
                           device=S.off.device)
        ends = S.off[idx].cpu().view(-1, 2)
        nbytes = int((ends[:, 1] - ends[:, 0]).sum())
    return TuneCache.key(torch.cuda.get_device_name(S.off.device), nbytes / max(1, rows), rows)


def autotune(R: DeviceRelation, S: DeviceRelation, ranges, pair_caps, candidates=LOAD_FACTORS, reps: int = 3,
             cache: TuneCache | None = None):
    """Time every candidate load factor on this batch; return (best GraphBatch
    with its graph captured, {load_factor: ms}).  With a cache, a batch of a
    shape seen before takes the cached load factor without timing (the dict
    is then empty)."""
    key = batch_shape_key(R, S, ranges) if cache is not None else None
    if cache is not None and cache.get(key) is not None:
        return GraphBatch(R, S, ranges, pair_caps, cache.get(key)).capture(), {}
    times, best = {}, None
    for lf in candidates:
        gb = GraphBatch(R, S, ranges, pair_caps, lf)
        times[lf] = gb.time_ms(reps, graph=False)
        if best is None or times[lf] < times[best.lf]:
            best = gb
        else:
            del gb
    if cache is not None:
        cache.put(key, best.lf)
    return best.capture(), times
