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


def autotune(R: DeviceRelation, S: DeviceRelation, ranges, pair_caps, candidates=LOAD_FACTORS, reps: int = 3):
    """Time every candidate load factor on this batch; return (best GraphBatch
    with its graph captured, {load_factor: ms})."""
    times, best = {}, None
    for lf in candidates:
        gb = GraphBatch(R, S, ranges, pair_caps, lf)
        times[lf] = gb.time_ms(reps, graph=False)
        if best is None or times[lf] < times[best.lf]:
            best = gb
        else:
            del gb
    return best.capture(), times
