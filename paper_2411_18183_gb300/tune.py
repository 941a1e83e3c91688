"""Batch runner: picks the hash-table load factor of a batch of joins and the
launch shape of its signature kernel by timing the candidates on the device,
then replays the batch's launches from a captured CUDA graph.

The load factor trades table size (and the cache footprint of the probe)
against bucket-chain length; the signature kernel's shape (warps per block,
32-byte blocks of a key in flight) trades occupancy against registers, which
favours different shapes for short and long keys.  The load factor is tuned
first at the default shape, then the shapes at the best load factor.
"""
from __future__ import annotations

import torch

from . import (ROWS_SCATTERED, DeviceRelation, alloc_ws, join_batch_prepare, join_batch_run,
               join_batch_ws_bytes, make_descs, sig_shapes, total_pair_cap)

LOAD_FACTORS = (0.35, 0.5, 0.7, 0.9)


class GraphBatch:
    """One prepared batch with its own workspace, output buffers and stream;
    run() launches it directly, capture() records it into a CUDA graph and
    replay() relaunches the graph."""

    def __init__(self, R: DeviceRelation, S: DeviceRelation, ranges, pair_caps, load_factor: float,
                 sig_shape: int = 0):
        self.R, self.S = R, S
        self.descs = make_descs(ranges, pair_caps)
        self.lf = load_factor
        self.stream = torch.cuda.Stream()
        self.ws = alloc_ws(join_batch_ws_bytes(self.descs, R.n, S.n, load_factor))
        self.pairs = torch.empty(2 * max(1, total_pair_cap(self.descs)), dtype=torch.int32, device="cuda")
        self.counts = torch.zeros(len(self.descs), dtype=torch.int64, device="cuda")
        self.batch = join_batch_prepare(self.descs, R, S, self.ws, load_factor, stream=self.stream)
        self.graph = None
        self.set_shape(sig_shape)

    @property
    def shape(self) -> int:
        return int(self.batch.sig_shape)

    def set_shape(self, sig_shape: int) -> None:
        """Signature kernel shape of the next run (drops a captured graph)."""
        self.batch.sig_shape = int(sig_shape)
        self.graph = None

    def shape_matters(self) -> bool:
        """Whether either side's signatures run through the single-relation kernel."""
        return self.batch.r_first != ROWS_SCATTERED or self.batch.s_first != ROWS_SCATTERED

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
    """Best (load factor, signature kernel shape) found by autotune, keyed by
    (GPU name, key-length class, size class) so that batches of the same shape
    skip the timing.  Optionally persisted as JSON."""

    LENGTH_CLASSES = (128, 1024, 8192)          # upper bounds of the key-length bands, then longer

    def __init__(self, path: str | None = None):
        self.path = path
        self.table: dict[str, tuple] = {}
        if path:
            import json
            import os
            if os.path.exists(path):
                with open(path) as f:
                    for k, v in json.load(f).items():
                        # an entry is [load_factor, shape]; a bare number is a load factor at shape 0
                        self.table[k] = (float(v[0]), int(v[1])) if isinstance(v, list) else (float(v), 0)

    @classmethod
    def key(cls, device_name: str, mean_key_bytes: float, rows: int) -> str:
        lc = next((i for i, b in enumerate(cls.LENGTH_CLASSES) if mean_key_bytes <= b), len(cls.LENGTH_CLASSES))
        sc = max(0, int(rows).bit_length() - 1)     # floor(log2(rows))
        return f"{device_name}|len{lc}|rows2^{sc}"

    def get(self, key: str):
        """(load_factor, shape) or None."""
        return self.table.get(key)

    def put(self, key: str, load_factor: float, shape: int = 0) -> None:
        self.table[key] = (float(load_factor), int(shape))
        if self.path:
            import json
            with open(self.path, "w") as f:
                json.dump({k: list(v) for k, v in self.table.items()}, f, indent=1, sort_keys=True)


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
             cache: TuneCache | None = None, shapes=None):
    """Time every candidate load factor on this batch at the default signature
    kernel shape, then every shape at the best load factor; return (best
    GraphBatch with its graph captured, {load_factor: ms}, {shape: ms}).  With
    a cache, a batch of a shape seen before takes the cached choice without
    timing (the dicts are then empty).  `shapes`: shape indices to try
    (default all; skipped when no side runs the single-relation kernel)."""
    key = batch_shape_key(R, S, ranges) if cache is not None else None
    if cache is not None and cache.get(key) is not None:
        lf, shape = cache.get(key)
        return GraphBatch(R, S, ranges, pair_caps, lf, shape).capture(), {}, {}
    times, best = {}, None
    for lf in candidates:
        gb = GraphBatch(R, S, ranges, pair_caps, lf)
        times[lf] = gb.time_ms(reps, graph=False)
        if best is None or times[lf] < times[best.lf]:
            best = gb
        else:
            del gb
    shape_times = {}
    if best.shape_matters():
        if shapes is None:
            shapes = range(len(sig_shapes()))
        for sh in shapes:
            best.set_shape(sh)
            shape_times[sh] = best.time_ms(reps, graph=False)
        best.set_shape(min(shape_times, key=shape_times.get))
    if cache is not None:
        cache.put(key, best.lf, best.shape)
    return best.capture(), times, shape_times
